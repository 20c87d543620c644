"""Pins of the oracle's learned warm start, solve residual and warm-start training gradient
(no GPU).

What each test pins:
* the 16 features of every row group (joint, hinge + motor, contact), against closed forms of
  the quadruped's first step (robot at rest vertically, joints closed, feet directly below the
  lower-link centres, gravity impulse only);
* the residual, by the facts that it vanishes at a converged solve for every row kind (a
  sliding sphere is solved exactly in one sweep; the quadruped after many sweeps) and shrinks
  with the number of sweeps;
* the warm-start network, against the textbook dense-layer definition in numpy (exact mode)
  and with torch's bfloat16 conversion at the storage points;
* the application of the warm start: with no weight on the previous impulses a zero network is
  the cold start bit for bit; with a weight it is the damped previous-impulse start projected on
  every row kind's bounds; the network's output is scaled by the rows' effective masses;
  starting from converged impulses (previous ones, or a network's output) leaves nothing for the
  sweeps;
* the training gradient, by central differences, the closed form of the output-bias gradient
  and its vanishing at a perfect fit;
* reverse mode with a state-independent warm start, by central differences.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1611_01652_gb300 import workloads as WL

G = 9.81


def ws_params(rng, scale=0.3):
    return rng.normal(0.0, scale, O.WS_PARAMS)


def split_ws(W):
    I, H, Oo = O.WS_IN, O.WS_H, O.WS_OUT
    k = 0
    out = []
    for n in (I * H, H, H * H, H, H * Oo, Oo):
        out.append(W[k:k + n])
        k += n
    W1, b1, W2, b2, W3, b3 = out
    return W1.reshape(H, I), b1, W2.reshape(H, H), b2, W3.reshape(Oo, H), b3


def const_ws(b3):
    """A network whose output is the constant b3 (every weight zero)."""
    W = np.zeros(O.WS_PARAMS)
    W[-3:] = b3
    return W


# ----------------------------------------------------------------------------- features
def test_group_features_closed_form_first_step():
    """First step of the quadruped at rest vertically (yaw 0): every body has the same velocity
    and no spin, the joints are closed, the feet sit 1 mm inside the ground straight below the
    lower-link centres, and the only impulse before the solve is gravity's."""
    m = WL.quadruped(B=3, horizon=1, yaw=0.0)  # body axes along the world axes
    groups = O.ws_groups(m)
    types = [g[0] for g in groups]
    assert types == [O.WS_JOINT, O.WS_HINGE] * 8 + [O.WS_GROUND] * 8
    for i in range(m.B):
        d = O.step_log(m, i, m.state0[i], t=0)
        f = d["feats"]
        h = m.dt
        x0 = m.state0[i]
        vx, vy = x0[0, 12], x0[0, 13]
        mass = m.mass[i]
        M = mass.sum()
        pc = (mass[:, None] * x0[:, :3]).sum(0) / M
        tau_h = m.motor[i, 0, 1] * h
        for j in range(8):  # joints: closed, no relative motion
            lin, hin = f[2 * j], f[2 * j + 1]
            child = m.joint_body[j, 1]
            q = x0[child, :3] + m.anchor[i, j, 1]
            for g, code, bound in ((lin, O.WS_JOINT, 0.0), (hin, O.WS_HINGE, tau_h)):
                np.testing.assert_allclose(g[0:3], 0.0, atol=1e-12)
                np.testing.assert_allclose(g[9], bound, rtol=1e-12)
                np.testing.assert_allclose(g[10:12], (q - pc)[:2], atol=1e-12)
                assert g[12] == 4.0
                np.testing.assert_allclose(g[13], M * G * h / 4.0, rtol=1e-12)
                np.testing.assert_allclose(g[14], q[2] - m.ground_z, atol=1e-12)
                assert g[15] == code
            np.testing.assert_allclose(lin[3:6], 0.0, atol=1e-6)  # closed joint (to the inputs' float32 grid)
            np.testing.assert_allclose(hin[3:5], 0.0, atol=1e-6)  # aligned hinge axes
            assert abs(hin[5]) <= m.motor[i, j, 2] + 1e-12  # servo rate within +-vmax
            assert (lin[6:9] > 0).all() and (hin[6:9] > 0).all()
        for c in range(4):  # feet
            g = f[16 + c]
            body = m.sphere_body[c]
            Ix = float(m.inertia[i, body, 0])  # capsule moment about a horizontal axis
            ell = -float(m.sph_off[i, c, 2]) + float(m.sph_rad[i, c])  # contact point below the centre
            q = x0[body, :3] + np.array([0.0, 0.0, -ell])
            np.testing.assert_allclose(g[0], -G * h, rtol=1e-12)
            np.testing.assert_allclose(g[1:3], [vx, vy], atol=1e-12)
            assert (g[3:6] == 0.0).all()  # inside the slop, e = 0, friction rows unbiased
            np.testing.assert_allclose(g[6], mass[body], rtol=1e-12)
            np.testing.assert_allclose(g[7:9], 1.0 / (1.0 / mass[body] + ell * ell / Ix), rtol=1e-12)
            np.testing.assert_allclose(g[9], 0.8)
            np.testing.assert_allclose(g[10:12], (q - pc)[:2], atol=1e-12)
            assert g[12] == 4.0
            np.testing.assert_allclose(g[13], M * G * h / 4.0, rtol=1e-12)
            np.testing.assert_allclose(g[14], q[2] - m.ground_z, atol=1e-12)
            assert g[15] == O.WS_GROUND
        for c in range(4, 8):  # torso spheres: inactive contacts contribute zero rows
            g = f[16 + c]
            assert (g[0:9] == 0.0).all()
        # the previous step's impulses do not enter the features
        lp = np.arange(1, len(d["lam"]) + 1) / 100.0
        np.testing.assert_array_equal(O.step_log(m, i, m.state0[i], t=0, lam_prev=lp)["feats"], f)
        assert (d["active"][-24:].reshape(8, 3)[:4] == 1).all()
        assert (d["active"][-24:].reshape(8, 3)[4:] == 0).all()


def test_pair_contact_feature_flag():
    m = WL.two_spheres(B=1)
    d = O.step_log(m, 0, m.state0[0], t=0)
    assert d["feats"].shape == (m.ns + m.np_, 16)
    assert (d["feats"][:m.ns, 15] == O.WS_GROUND).all() and (d["feats"][m.ns:, 15] == O.WS_PAIR).all()


# ----------------------------------------------------------------------------- residual
def sliding_ball(horizon=5):
    m = WL.ball(B=1, horizon=horizon)
    r = float(m.sph_rad[0, 0])
    m.state0[0, 0, 2] = r - m.slop
    m.state0[0, 0, 12:15] = [3.0, -1.0, 0.0]
    m.state0[0, 0, 15:18] = 0.0
    return m


def test_residual_vanishes_for_an_exactly_solved_contact():
    """Sliding sphere: normal and both friction rows act on decoupled directions of a sphere,
    so one sweep solves them exactly (normal bilateral-at-rest, friction saturated)."""
    m = sliding_ball()
    _, _, res = O.rollout_resid(m, 0, 5, iters=1)
    assert res.max() < 1e-12
    _, _, res20 = O.rollout_resid(m, 0, 5, iters=20)
    assert res20.max() < 1e-12


def test_residual_vanishes_at_convergence_for_every_row_kind():
    """The quadruped's solve holds joint, limit, motor, contact and friction rows; as the sweeps
    converge the residual of each kind goes to zero, and it shrinks with the sweep count."""
    m = WL.quadruped(B=2, horizon=40)
    st, _, _ = O.rollout_resid(m, 0, 40)
    kinds_seen = set()
    for t in (5, 20, 39):
        r = [O.step_log(m, 0, st[t], t=t, iters=n)["resid"] for n in (2, 20, 400, 4000)]
        assert r[0] > r[1] > r[2] > r[3], r
        assert r[3] < 1e-6 * max(1.0, r[0]), r
        d = O.step_log(m, 0, st[t], t=t)
        kinds_seen |= set(O.schedule(m)["kind"][d["active"] == 1].tolist())
    assert {0, 1, 3, 4, 5} <= kinds_seen


def test_residual_is_zero_without_active_rows():
    m = WL.ball(B=1, horizon=5)
    _, _, res = O.rollout_resid(m, 0, 5)  # in flight
    assert (res == 0.0).all()


# ----------------------------------------------------------------------------- network
def test_ws_network_matches_textbook_dense_layers():
    rng = np.random.default_rng(5)
    W = ws_params(rng)
    X = rng.normal(0, 1, (50, 16))
    W1, b1, W2, b2, W3, b3 = split_ws(W)
    h1 = np.maximum(X @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    np.testing.assert_allclose(O.ws_forward(W, X, exact=True), h2 @ W3.T + b3, rtol=1e-12, atol=1e-12)


def test_ws_network_bfloat16_storage_points():
    torch = pytest.importorskip("torch")

    def q(a):
        return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()

    rng = np.random.default_rng(6)
    W = ws_params(rng).astype(np.float32).astype(np.float64)
    X = rng.normal(0, 1, (50, 16))
    W1, b1, W2, b2, W3, b3 = split_ws(W)
    h1 = q(np.maximum(q(X) @ q(W1).T + b1, 0))
    h2 = q(np.maximum(h1 @ q(W2).T + b2, 0))
    np.testing.assert_allclose(O.ws_forward(W, X), h2 @ q(W3).T + b3, rtol=1e-9, atol=1e-12)


# ----------------------------------------------------------------------------- application
def test_zero_network_is_the_cold_start():
    m = WL.quadruped(B=2, horizon=30)
    st, L, _ = O.rollout_resid(m, 1, 30)
    m.warmstart, m.ws_W, m.ws_alpha = 1, np.zeros(O.WS_PARAMS), 0.0
    st2, L2, _ = O.rollout_resid(m, 1, 30)
    assert np.array_equal(st, st2) and L == L2


def test_zero_network_is_the_damped_previous_impulse_start():
    """With a zero network the start is alpha lambda_prev projected on the bounds: joint rows
    unchanged, normals clipped at 0, friction boxed by mu times the normal, motors by tau_max h."""
    m = WL.quadruped(B=1, horizon=40)
    st, _, _ = O.rollout_resid(m, 0, 40)
    sch = O.schedule(m)
    kind = sch["kind"]
    m.warmstart, m.ws_W, m.ws_alpha = 1, np.zeros(O.WS_PARAMS), 0.7
    rng = np.random.default_rng(3)
    lp = rng.normal(0, 0.2, len(kind))
    d = O.step_log(m, 0, st[20], t=20, lam_prev=lp)
    l0, act = d["lam0"], d["active"]
    tau_h = m.motor[0, 0, 1] * m.dt
    for s, k in enumerate(kind):
        z = 0.7 * lp[s]
        if k in (0, 1):
            assert l0[s] == z
        elif k == 3:
            assert l0[s] == min(max(z, -tau_h), tau_h)
        elif k == 2:
            assert l0[s] == 0.0  # limits start cold
        elif k == 4:
            assert l0[s] == (max(z, 0.0) if act[s] else 0.0)
        elif k == 5:
            n = s - 1 if kind[s - 1] == 4 else s - 2
            hi = float(m.sph_mu[0, sch["idx"][s]]) * l0[n]
            assert l0[s] == (min(max(z, -hi), hi) if act[s] else 0.0)


def test_converged_previous_impulses_need_no_sweeps():
    """Starting from the converged impulses of the same step (alpha = 1, zero network) leaves
    nothing for the sweeps: zero sweeps give the converged residual and state."""
    m = WL.quadruped(B=1, horizon=40)
    st, _, _ = O.rollout_resid(m, 0, 40)
    ref = O.step_log(m, 0, st[25], t=25, iters=3000)
    m.warmstart, m.ws_W, m.ws_alpha = 1, np.zeros(O.WS_PARAMS), 1.0
    d = O.step_log(m, 0, st[25], t=25, iters=0, lam_prev=ref["lam"])
    assert d["resid"] <= ref["resid"] + 1e-12
    np.testing.assert_allclose(d["xn"], ref["xn"], rtol=0, atol=1e-12)


def test_warm_start_projection_on_the_bounds():
    """The network's output is a velocity-scale correction: the start is m_eff y per row, then
    projected (normal >= 0, |friction| <= mu normal)."""
    m = sliding_ball()
    mu = float(m.sph_mu[0, 0])
    me = O.step_log(m, 0, m.state0[0], t=0)["feats"][0, 6:9]
    for y, lam in (([-1.0, 5.0, -5.0], [0.0, 0.0, 0.0]), ([2.0, 5.0, -0.5], None), ([0.5, -50.0, 50.0], None)):
        m.warmstart, m.ws_W, m.ws_alpha = 1, const_ws(y), 0.7
        d = O.step_log(m, 0, m.state0[0], t=0)
        z = me * np.array(y)
        n = max(z[0], 0.0)
        expect = [n, min(max(z[1], -mu * n), mu * n), min(max(z[2], -mu * n), mu * n)]
        np.testing.assert_allclose(d["lam0"], expect if lam is None else lam, rtol=1e-15)


def test_converged_warm_start_needs_no_sweeps():
    """A network that outputs the converged impulses of the sliding sphere (m g h normal,
    -mu m g h along each slip component), divided by the rows' effective masses, gives with zero
    sweeps the converged step."""
    m = sliding_ball()
    ref = O.step_log(m, 0, m.state0[0], t=0, iters=20)
    mass, mu, h = float(m.mass[0, 0]), float(m.sph_mu[0, 0]), m.dt
    v = m.state0[0, 0, 12:14]
    lam = mass * G * h
    # friction rows t1 = x, t2 = y; each row saturates at -mu lam sign(v) (both slip components
    # are nonzero)
    np.testing.assert_allclose(ref["lam"][1:], -mu * lam * np.sign(v), rtol=1e-9)
    np.testing.assert_allclose(ref["lam"][0], lam, rtol=1e-9)
    me = ref["feats"][0, 6:9]
    m.warmstart, m.ws_W, m.ws_alpha = 1, const_ws(ref["lam"] / me), 0.7
    ws = O.step_log(m, 0, m.state0[0], t=0, iters=0)
    np.testing.assert_allclose(ws["xn"], ref["xn"], rtol=0, atol=1e-12)
    assert ws["resid"] < 1e-12


# ----------------------------------------------------------------------------- training gradient
def harvested_like_rows(rng, n):
    X = rng.normal(0, 1, (n, 16))
    Y = rng.normal(0, 0.3, (n, 3))
    return np.concatenate([X, Y], axis=1)


def test_ws_training_gradient_central_differences():
    rng = np.random.default_rng(7)
    W = ws_params(rng)
    rows = harvested_like_rows(rng, 6)
    L, g = O.ws_loss_grad(W, rows, exact=True)
    idx = rng.choice(O.WS_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, np.arange(O.WS_PARAMS - 3, O.WS_PARAMS)])
    eps = 1e-6
    for k in idx:
        Wp, Wm = W.copy(), W.copy()
        Wp[k] += eps
        Wm[k] -= eps
        fd = (O.ws_loss_grad(Wp, rows, exact=True)[0] - O.ws_loss_grad(Wm, rows, exact=True)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_ws_training_gradient_output_bias_closed_form_and_perfect_fit():
    rng = np.random.default_rng(8)
    W = ws_params(rng)
    rows = harvested_like_rows(rng, 40)
    for exact in (True, False):
        y = O.ws_forward(W, rows[:, :16], exact=exact)
        L, g = O.ws_loss_grad(W, rows, exact=exact)
        np.testing.assert_allclose(L, ((y - rows[:, 16:]) ** 2).sum(1).mean(), rtol=1e-12)
        np.testing.assert_allclose(g[-3:], 2.0 * (y - rows[:, 16:]).mean(0), rtol=1e-10)
        fit = rows.copy()
        fit[:, 16:] = y
        L0, g0 = O.ws_loss_grad(W, fit, exact=exact)
        assert L0 == 0.0 and not g0.any()


# ----------------------------------------------------------------------------- reverse mode
def test_gradient_with_state_independent_warm_start_central_differences():
    """With a constant-output network the warm start does not depend on the state, so the
    stop-gradient reverse mode is the exact derivative: check it by central differences."""
    m = WL.quadruped(B=1, horizon=8)
    m.exact_mlp = 1
    m.warmstart, m.ws_W, m.ws_alpha = 1, const_ws([0.25, 0.01, -0.02]), 0.0
    L, g = O.rollout_grad(m, 0)
    eps = 1e-6
    for (b, f) in ((0, 12), (0, 2), (3, 16), (2, 0)):
        def loss_at(dx):
            x = m.state0[0].astype(np.float64).copy()
            x[b, f] += dx
            keep = m.state0[0].copy()
            m.state0[0] = x
            try:
                return O.rollout(m, 0)[1]
            finally:
                m.state0[0] = keep
        fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
        assert abs(fd - g["state0"][b, f]) <= 1e-5 * max(1.0, abs(fd)), (b, f, fd, g["state0"][b, f])
