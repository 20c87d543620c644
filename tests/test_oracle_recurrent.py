"""Pins of the oracle's recurrent controller (Eq. g: u^t = g(s(x^t), h^t | W), h^{t+1} from the
same network, h^0 = 0) against facts that do not come from the oracle's own formulas: a scalar
recursion written out here, the reduction to the feed-forward controller when the recurrent
weights are zero, and central differences of the oracle's forward pass (no GPU)."""
import math

import numpy as np

import oracle as O
from paper_1611_01652_gb300 import workloads as WL

from test_oracle_pins import _same_activity


def _layers(widths):
    """Offsets of (W[out][in], b[out]) of every layer in the flat parameter vector."""
    out, off = [], 0
    for l in range(len(widths) - 1):
        ni, no = widths[l], widths[l + 1]
        out.append((off, off + ni * no, ni, no))
        off += ni * no + no
    return out


def test_recurrent_state_follows_scalar_recursion():
    """One recurrent unit wired as h' = tanh(w (h + 1) + b) through the two ReLU layers (h + 1 > 0
    since |h| < 1), motor outputs zero: the oracle's h sequence is that recursion from h^0 = 0."""
    H, w, b = 1, 0.7, -0.3
    m = WL.quadruped(B=1, horizon=12, n_recurrent=H)
    m.exact_mlp = 1
    assert m.widths == [25, 128, 128, 9]
    W = np.zeros(O.param_count(m.widths))
    (w1, b1, ni1, _), (w2, b2, ni2, _), (w3, b3, ni3, _) = _layers(m.widths)
    W[w1 + 0 * ni1 + 24] = 1.0  # hidden-1 unit 0 reads the recurrent input (the last input)
    W[b1 + 0] = 1.0
    W[w2 + 0 * ni2 + 0] = 1.0  # hidden-2 unit 0 copies it
    W[w3 + 8 * ni3 + 0] = w  # the recurrent output (the last output)
    W[b3 + 8] = b
    _, _, hs = O.rollout_rec(m, 0, W=W)
    h, ref = 0.0, [0.0]
    for _ in range(12):
        h = math.tanh(w * (h + 1.0) + b)
        ref.append(h)
    np.testing.assert_allclose(hs[:, 0], ref, rtol=0, atol=1e-14)


def test_recurrent_controller_with_zero_recurrent_weights_is_the_feed_forward_one():
    """Recurrent inputs with zero weights and arbitrary recurrent outputs: states and loss are those
    of the feed-forward controller with the remaining weights, bit for bit (the extra products are
    exact zeros added last), with bfloat16 storage points on."""
    ff = WL.quadruped(B=2, horizon=40, w_seed=5)
    rec = WL.quadruped(B=2, horizon=40, w_seed=5, n_recurrent=2)
    rng = np.random.default_rng(0)
    Wr = np.zeros(O.param_count(rec.widths))
    for (fw, fb, fni, fno), (rw, rb, rni, rno) in zip(_layers(ff.widths), _layers(rec.widths)):
        Wf = ff.W[fw:fw + fni * fno].reshape(fno, fni)
        blk = np.zeros((rno, rni))
        blk[:fno, :fni] = Wf
        if rno > fno:  # recurrent output rows: arbitrary
            blk[fno:, :] = rng.uniform(-0.5, 0.5, size=(rno - fno, rni))
        Wr[rw:rw + rni * rno] = blk.reshape(-1)
        Wr[rb:rb + fno] = ff.W[fb:fb + fno]
        if rno > fno:
            Wr[rb + fno:rb + rno] = rng.uniform(-0.5, 0.5, size=rno - fno)
    for i in range(2):
        sf, lf, _, _ = O.rollout(ff, i)
        sr, lr, hs = O.rollout_rec(rec, i, W=Wr)
        assert np.array_equal(sf, sr)
        assert lf == lr
        assert np.abs(hs[1:]).max() > 0.0  # the recurrent state does evolve


def test_recurrent_gradient_matches_central_differences():
    """Quadruped with a 2-unit recurrent state, 8 steps: the reverse-mode gradient (back-propagation
    through time of both the physical state and h^t) w.r.t. the recurrent weights, the other
    controller weights and the initial state equals central differences of the loss (controller
    unrounded, as for the feed-forward pin)."""
    m = WL.quadruped(B=1, horizon=8, n_recurrent=2)
    m.exact_mlp = 1
    rng = np.random.default_rng(3)
    W = m.W.astype(np.float64).copy()
    (w1, b1, ni1, no1), _, (w3, b3, ni3, no3) = _layers(m.widths)
    for o in range(no1):  # recurrent input columns of layer 1
        W[w1 + o * ni1 + 24:w1 + o * ni1 + 26] = rng.uniform(-0.4, 0.4, size=2)
    W[w3 + 8 * ni3:w3 + 10 * ni3] = rng.uniform(-0.3, 0.3, size=2 * ni3)  # recurrent output rows
    W[b3 + 8:b3 + 10] = [0.2, -0.1]
    L, g = O.rollout_grad(m, 0, W=W)
    _, _, hs = O.rollout_rec(m, 0, W=W)
    assert np.abs(hs).max() > 0.05
    idx = [w1 + 3 * ni1 + 24, w1 + 40 * ni1 + 25, w1 + 100 * ni1 + 24, w3 + 8 * ni3 + 7, w3 + 9 * ni3 + 60,
           b3 + 8, b3 + 9, w1 + 5 * ni1 + 2, w3 + 2 * ni3 + 11]
    checked = 0
    for k in idx:
        eps = 1e-6
        Wp = W.copy(); Wp[k] += eps
        Wm = W.copy(); Wm[k] -= eps
        if not _same_activity(m, 0, m.horizon, None, None, Wp, Wm):
            continue
        fd = (O.rollout(m, 0, W=Wp)[1] - O.rollout(m, 0, W=Wm)[1]) / (2 * eps)
        assert abs(fd - g["W"][k]) <= 1e-4 * (abs(fd) + 1e-4), (k, fd, g["W"][k])
        checked += 1
    base = m.state0[0].astype(np.float64)
    for k in rng.choice(base.size, 6, replace=False):
        eps = 1e-7
        xp = base.copy(); xp.flat[k] += eps
        xm = base.copy(); xm.flat[k] -= eps
        if not _same_activity(m, 0, m.horizon, {"state0": xp}, {"state0": xm}, W, W):
            continue
        fd = (O.rollout(m, 0, W=W, overrides={"state0": xp})[1] - O.rollout(m, 0, W=W, overrides={"state0": xm})[1]) / (2 * eps)
        assert abs(fd - g["state0"].flat[k]) <= 1e-4 * (abs(fd) + 1e-3), (k, fd, g["state0"].flat[k])
        checked += 1
    assert checked >= 10
    # the recurrent weights do carry gradient
    assert np.abs(g["W"][[w1 + o * ni1 + 24 for o in range(no1)]]).max() > 0.0


def test_gradient_decay_also_cuts_the_recurrent_adjoint():
    """With the decay alpha -> 0 nothing reaches step T-1 from later steps, through the state or
    through h: with the final-state loss, dL/dW is then the derivative of the last step alone,
    taken from the stored x_{T-1} and h_{T-1} (central differences of one oracle step); an
    undecayed recurrent adjoint would add the earlier steps' share through h."""
    m = WL.quadruped(B=1, horizon=6, n_recurrent=2)
    m.exact_mlp = 1
    rng = np.random.default_rng(11)
    W = m.W.astype(np.float64).copy()
    (w1, b1, ni1, no1), _, (w3, b3, ni3, no3) = _layers(m.widths)
    for o in range(no1):
        W[w1 + o * ni1 + 24:w1 + o * ni1 + 26] = rng.uniform(-0.4, 0.4, size=2)
    W[w3 + 8 * ni3:w3 + 10 * ni3] = rng.uniform(-0.3, 0.3, size=2 * ni3)
    st, _, hs = O.rollout_rec(m, 0, W=W)
    m.grad_decay = 1e-12
    _, g = O.rollout_grad(m, 0, W=W)
    T = m.horizon
    a = np.asarray(m.loss_target[0], np.float64)
    c = np.asarray(m.loss_point[0], np.float64)

    def last_step_loss(Wv):
        xn = O.step_log(m, 0, st[T - 1], t=T - 1, W=Wv, h_prev=hs[T - 1])["xn"]
        return a @ (xn[0, 0:3] + xn[0, 3:12].reshape(3, 3) @ c)  # x_T's term a.q of the displacement loss

    idx = [w1 + 7 * ni1 + 24, w1 + 90 * ni1 + 25, w1 + 3 * ni1 + 5, w3 + 2 * ni3 + 9]
    for k in idx:
        eps = 1e-6
        Wp, Wm = W.copy(), W.copy()
        Wp[k] += eps
        Wm[k] -= eps
        fd = (last_step_loss(Wp) - last_step_loss(Wm)) / (2 * eps)
        assert abs(fd - g["W"][k]) <= 1e-5 * (abs(fd) + 1e-5), (k, fd, g["W"][k])
    # the recurrent-input columns still get the last step's share (h_{T-1} != 0)
    assert any(abs(g["W"][k]) > 0 for k in idx[:2])
