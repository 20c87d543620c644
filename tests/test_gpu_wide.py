"""Wide controllers (hidden layers beyond 256, e.g. 64-1024-1024-8 with 1,124,360 parameters) run
as batched tensor-core products between step launches. Through the C ABI: the wide path against
the in-step tensor-core controller on the same 24-128-128-8 network, and the 64-1024-1024-8
network against the FP64 oracle (bfloat16 storage points; steps whose roundings came within 1e-6
of a tie are skipped, since the two sides accumulate in different precisions)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import World  # noqa: E402

from test_gpu_parity import elem_err, gpu_grads, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

WIDE = [64, 1024, 1024, 8]


def rollout(m, horizon, traj=True):
    w = World(m, horizon=horizon)
    T = w.horizon
    tr = torch.zeros(T + 1, m.B, m.nb, 18, device="cuda") if traj else None
    act = torch.zeros(T, m.B, w.n_slots, dtype=torch.uint8, device="cuda")
    loss = torch.zeros(m.B, device="cuda")
    w.rollout(torch.tensor(m.W, device="cuda"), loss, tr, act)
    w.sync()
    return tr.cpu().double().numpy() if traj else None, loss.cpu().double().numpy(), act.cpu().numpy()


def test_wide_path_matches_in_step_controller(monkeypatch):
    """Same 24-128-128-8 network on both paths: identical activation sets, states within 1e-4
    over 20 steps, losses and gradients (initial state, parameters, every weight) within 1e-3."""
    m = WL.quadruped(B=64, horizon=20)
    ta, la, aa = rollout(m, 20)
    ga = gpu_grads(m, 20)
    monkeypatch.setenv("DP_FORCE_WIDE_CONTROLLER", "1")
    tb, lb, ab = rollout(m, 20)
    gb = gpu_grads(m, 20)
    assert np.array_equal(aa, ab)
    err = np.abs(ta - tb) / np.maximum(1.0, np.abs(ta))
    assert err.max() <= 1e-4, err.max()
    np.testing.assert_allclose(lb, la, rtol=1e-3, atol=1e-6)
    for k in ("state0", "mass", "motor", "W"):
        assert rel_err(gb[k], ga[k]) <= 1e-3, (k, rel_err(gb[k], ga[k]))


def test_wide_controller_steps_match_oracle():
    """64-1024-1024-8 controller (1.1 M parameters): teacher-forced single steps from oracle
    states, next state within 1e-4 and activation sets bit-exact away from ties."""
    m = WL.quadruped(B=16, horizon=40, widths=WIDE)
    assert O.param_count(WIDE) == 1124360
    states = [O.rollout(m, i, horizon=40)[0] for i in range(m.B)]
    w = World(m, horizon=40)
    W = torch.tensor(m.W, device="cuda")
    checked = total = 0
    for t in range(0, 40, 6):
        x = np.stack([s[t] for s in states]).astype(np.float32)
        w.set_state(torch.tensor(x, device="cuda"), t)
        act = torch.zeros(1, m.B, w.n_slots, dtype=torch.uint8, device="cuda")
        w.step(1, W, act)
        out = torch.zeros(m.B, m.nb, 18, device="cuda")
        w.get_state(out)
        w.sync()
        out, act = out.cpu().double().numpy(), act.cpu().numpy()[0]
        for i in range(m.B):
            xn, a_o, gap, _, marg = O.step(m, i, x[i].astype(np.float64), t=t, margins=True)
            ok = gap >= 1e-5
            assert np.array_equal(act[i][ok], a_o[ok]), (t, i)
            total += 1
            if ok.all() and marg > 1e-6:
                err = np.abs(out[i] - xn) / np.maximum(1.0, np.abs(xn))
                assert err.max() <= 1e-4, (t, i, err.max())
                checked += 1
    assert checked >= 0.1 * total, (checked, total)


def test_wide_controller_gradients_match_oracle():
    """Reverse mode through the wide path (per-step launches, products of the deltas, split-K
    weight gradient) against the oracle over 3 steps. With 2,100 bfloat16 roundings per step some
    come within fp32 accumulation error of a tie on every instance; a rounding that goes the other
    way moves one hidden activation by one bfloat16 step, which moves the gradients far less than
    the 1e-3 tolerance (the wide-vs-in-step test above, whose accumulation orders differ, shows
    the same)."""
    m = WL.quadruped(B=4, horizon=3, widths=WIDE)
    g = gpu_grads(m, 3)
    Wsum = None
    for i in range(m.B):
        L, go = O.rollout_grad(m, i, horizon=3)
        assert abs(g["loss"][i] - L) <= 1e-4 * max(1.0, abs(L))
        Wsum = go["W"] if Wsum is None else Wsum + go["W"]
        for k in ("state0", "mass", "motor"):
            e = elem_err(g[k][i], go[k])
            assert e <= 1e-3, (i, k, e)
    assert elem_err(g["W"], Wsum) <= 1e-3, elem_err(g["W"], Wsum)


@pytest.mark.parametrize("warm", [False, True])
def test_wide_path_four_warp_kernels_match_single_warp(monkeypatch, warm):
    """The wide path's per-step launches of the compiled topology run on four warps per group of
    32 instances; the one-warp kernels (forced here) must give the same trajectory, activity log
    and losses bit for bit (the forward kernels share every sum's order), and the same gradients
    up to the order of the reverse pass's sums (64-1024-1024-8 controller; cold and damped
    start)."""
    from paper_1611_01652_gb300.binding import CTRL_WIDE, WS_PARAMS

    m = WL.quadruped(B=40, horizon=12, widths=WIDE)
    outs = []
    for single in (False, True):
        if single:
            monkeypatch.setenv("DP_SINGLE_WARP_FORWARD", "1")
            monkeypatch.setenv("DP_SINGLE_WARP_BACKWARD", "1")
        w = World(m, horizon=12, iters=10 if warm else 20, warmstart=warm)
        assert w.controller_kind == CTRL_WIDE
        if warm:
            w.set_warmstart(torch.zeros(WS_PARAMS, device="cuda"), 0.7)
        tr = torch.zeros(13, m.B, m.nb, 18, device="cuda")
        act = torch.zeros(12, m.B, w.n_slots, dtype=torch.uint8, device="cuda")
        loss = torch.zeros(m.B, device="cuda")
        w.rollout(torch.tensor(m.W, device="cuda"), loss, tr, act)
        dW = torch.zeros(w.n_params, device="cuda")
        ds = torch.zeros(m.B, m.nb, 18, device="cuda")
        w.backward(torch.ones(m.B, device="cuda"), dW, ds)
        w.sync()
        outs.append([x.cpu().numpy() for x in (tr, act, loss, dW, ds)])
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0][3:], outs[1][3:]):
        assert rel_err(a, b) <= 1e-4, rel_err(a, b)
