"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same seeded
inputs. States within 1e-4 relative (scale floor 1) over 100 steps, constraint activation
sets and slot indexing bit-exact away from near-ties (|gap| < 1e-5 m or rad), gradients within
1e-3 relative where the oracle's own finite differences agree.

A near-tie that resolves differently in FP32 and FP64 (a contact or limit decision, or the sign
choice of a pair contact's friction basis) makes the two trajectories legitimately different
from that step on, so free-running states are compared up to such a step. bfloat16 rounding of
the controller is a quantisation whose decisions FP32 and FP64 cannot share; free-running
comparisons of controlled robots therefore use the fp32 controller mode, and the bfloat16 mode
is checked one step at a time from oracle states, away from rounding ties."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import CTRL_SIMT, CTRL_TENSOR, WS_PARAMS, World  # noqa: E402

pytestmark = pytest.mark.gpu

STATE_RTOL = 1e-4
GRAD_RTOL = 1e-3
TIE = 1e-5


def gpu_rollout(m, horizon=None):
    w = World(m, horizon=horizon)
    T = w.horizon
    traj = torch.zeros(T + 1, m.B, m.nb, 18, device="cuda")
    active = torch.zeros(T, m.B, max(w.n_slots, 1), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(m.B, device="cuda")
    W = torch.tensor(m.W, device="cuda") if m.W is not None and len(m.W) else None
    w.rollout(W, loss, traj, active if w.n_slots else None)
    w.sync()
    return w, traj.cpu().double().numpy(), loss.cpu().double().numpy(), active.cpu().numpy()[:, :, :w.n_slots]


def divergence_step(act_g, act_o, gap, kinds):
    """First step at which a near-tie decision may legitimately differ between FP32 and FP64:
    an activation mismatch at a near-tie slot, or an active pair-friction row whose basis sign
    was near a tie. Mismatches away from near-ties are failures."""
    T = act_o.shape[0]
    if act_o.size == 0:
        return T
    mism = act_g != act_o
    tie = gap < TIE
    bad = mism & ~tie
    assert not bad.any(), ("activation mismatch away from a near-tie", np.argwhere(bad)[:5])
    pt = (kinds == 7)[None, :] & (act_o == 1) & tie
    t = np.flatnonzero((mism & tie).any(axis=1) | pt.any(axis=1))
    return int(t[0]) if len(t) else T


def compare_rollout(m, horizon, instances, min_clean=0.5, rtol=STATE_RTOL, rtol_window=None):
    """Free-running rollout of every instance, compared with the oracle. States match within
    ``rtol`` up to the first legitimate divergence step; with ``rtol_window = (n, tol)`` the first
    n steps use ``tol`` (the BJ bound) and the rest ``rtol``."""
    w, traj, loss, act = gpu_rollout(m, horizon)
    kinds = O.schedule(m)["kind"] if w.n_slots else np.zeros(0, np.int32)
    clean = 0
    for i in instances:
        st, L, a_o, gap = O.rollout(m, i, horizon=horizon, log=True)
        te = divergence_step(act[:, i], a_o, gap, kinds)
        n = te + 1
        err = np.abs(traj[:n, i] - st[:n]) / np.maximum(1.0, np.abs(st[:n]))
        per_step = err.max(axis=(1, 2))
        if rtol_window:
            k, tol = rtol_window
            assert per_step[: k + 1].max() <= tol, (i, per_step[: k + 1].max())
        assert per_step.max() <= rtol, (i, te, per_step.max(), int(per_step.argmax()))
        if te == horizon:
            clean += 1
            assert abs(loss[i] - L) <= rtol * max(1.0, abs(L)), (i, loss[i], L)
    assert clean >= min_clean * len(instances), (clean, len(instances))
    return w


def test_schedule_matches_oracle():
    for m in (WL.quadruped(B=2, horizon=3), WL.two_spheres(B=2), WL.pendulum3(B=2, horizon=3), WL.ball(B=1)):
        w = World(m, horizon=3)
        g, o = w.schedule(), O.schedule(m)
        for k in o:
            assert np.array_equal(g[k], o[k]), (m.name, k)


def test_ball_forward_matches_oracle():
    m = WL.ball(B=48)
    compare_rollout(m, 300, range(0, 48, 3))


def test_two_spheres_forward_matches_oracle():
    m = WL.two_spheres(B=8, e=0.3, mu=0.4)
    compare_rollout(m, 60, range(8))


def test_pendulum_forward_matches_oracle():
    """3-link chains, h = 1 ms: 1e-4 over the first 100 steps, 1e-3 over all 1000."""
    m = WL.pendulum3(B=40, horizon=1000)
    compare_rollout(m, 1000, range(0, 40, 5), rtol=1e-3, rtol_window=(100, STATE_RTOL))


def test_quadruped_forward_matches_oracle_100_steps():
    """Quadruped with its controller (fp32 controller mode), contacts, limits and servos."""
    m = WL.quadruped(B=40, horizon=100)
    m.ctrl_fp32 = 1
    compare_rollout(m, 100, range(0, 40, 4), min_clean=0.5)


def teacher_forced(m, horizon, stride=7, min_frac=0.3):
    """One GPU step from oracle states at many times: next state and active set (bfloat16
    controller: steps whose rounding decisions came within 1e-5 of a tie are skipped; at least
    ``min_frac`` of the steps must be checked)."""
    w = World(m, horizon=horizon)
    W = torch.tensor(m.W, device="cuda")
    states = [O.rollout(m, i, horizon=horizon)[0] for i in range(m.B)]
    checked = 0
    for t in range(0, horizon, stride):
        x = np.stack([s[t] for s in states]).astype(np.float32)
        w.set_state(torch.tensor(x, device="cuda"), t)
        act = torch.zeros(1, m.B, w.n_slots, dtype=torch.uint8, device="cuda")
        w.step(1, W, act)
        out = torch.zeros(m.B, m.nb, 18, device="cuda")
        w.get_state(out)
        w.sync()
        out = out.cpu().double().numpy()
        act = act.cpu().numpy()[0]
        for i in range(m.B):
            xn, a_o, gap, _, marg = O.step(m, i, x[i].astype(np.float64), t=t, margins=True)
            ok = gap >= TIE
            assert np.array_equal(act[i][ok], a_o[ok]), (t, i)
            if ok.all() and (m.ctrl_fp32 or marg > TIE):
                err = np.abs(out[i] - xn) / np.maximum(1.0, np.abs(xn))
                assert err.max() <= STATE_RTOL, (t, i, err.max())
                checked += 1
    assert checked >= min_frac * m.B * len(range(0, horizon, stride))
    return w


@pytest.mark.parametrize("fp32", [0, 1])
def test_quadruped_teacher_forced_steps(fp32):
    """One GPU step from oracle states at many times: next state and active set (bfloat16
    controller: steps whose rounding decisions came within 1e-5 of a tie are skipped)."""
    m = WL.quadruped(B=8, horizon=200)
    m.ctrl_fp32 = fp32
    teacher_forced(m, 200)


@pytest.mark.parametrize("widths", [[24, 64, 64, 8], [32, 256, 256, 8]])
def test_tensor_core_widths_teacher_forced_steps(monkeypatch, widths):
    """The 64- and 256-wide bfloat16 controllers on the tensor cores (run-time topology; the 256-wide
    one with 8 zero-padded inputs) against the oracle, one step at a time from its states. A step
    is skipped when one of its bfloat16 roundings came within 1e-5 (relative) of a tie, about
    2.6e-3 per rounding: with 2 x 256 hidden roundings per step about three steps in four, so the
    wide network samples every third step and needs a sixth of them checked."""
    monkeypatch.setenv("DP_FORCE_RUNTIME_TOPOLOGY", "1")
    m = WL.quadruped(B=8, horizon=100, widths=widths)
    w = teacher_forced(m, 100, stride=3 if widths[1] == 256 else 7, min_frac=0.15 if widths[1] == 256 else 0.3)
    assert w.controller_kind == CTRL_TENSOR


@pytest.mark.parametrize("case", ["bf16 damped start", "learned start", "bf16 cold", "fp32 controller", "recurrent"])
def test_four_warp_rollout_matches_single_warp(monkeypatch, case):
    """The compiled topology's recorded rollouts run on four warps per group of 32 instances; the
    one-warp kernel (forced here) must give the same trajectory, activity log, losses, solver tape
    (through the gradients of the reverse pass that reads it) and final state, bit for bit. With a
    learned warm-start network (a seeded random one) the four-warp kernel runs the one-warp warm
    start on its first warp."""
    m = WL.quadruped(B=40, horizon=30, n_recurrent=4 if case == "recurrent" else 0)
    if case == "fp32 controller":
        m.ctrl_fp32 = 1
    warm = case in ("bf16 damped start", "learned start")
    net = torch.zeros(WS_PARAMS, device="cuda")
    if case == "learned start":
        net = 0.05 * torch.randn(WS_PARAMS, generator=torch.Generator().manual_seed(5)).cuda()
    outs = []
    for single in (False, True):
        if single:
            monkeypatch.setenv("DP_SINGLE_WARP_FORWARD", "1")
        w = World(m, horizon=30, iters=10 if warm else 20, warmstart=warm)
        if warm:
            w.set_warmstart(net, 0.7)
        W = torch.tensor(m.W, device="cuda")
        traj = torch.zeros(31, m.B, m.nb, 18, device="cuda")
        act = torch.zeros(30, m.B, w.n_slots, dtype=torch.uint8, device="cuda")
        loss = torch.zeros(m.B, device="cuda")
        w.rollout(W, loss, traj, act)
        dW = torch.zeros(w.n_params, device="cuda")
        ds = torch.zeros(m.B, m.nb, 18, device="cuda")
        w.backward(torch.ones(m.B, device="cuda"), dW, ds)
        w.sync()
        outs.append([x.cpu().numpy() for x in (traj, act, loss, dW, ds)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_determinism_bitwise():
    m = WL.quadruped(B=64, horizon=50)
    _, t1, l1, a1 = gpu_rollout(m)
    _, t2, l2, a2 = gpu_rollout(m)
    assert np.array_equal(t1, t2) and np.array_equal(l1, l2) and np.array_equal(a1, a2)


@pytest.mark.parametrize("B", [1, 5, 33])
def test_ragged_batches(B):
    """Batches that leave a partial warp: padded lanes must not disturb real instances."""
    m = WL.quadruped(B=B, horizon=20)
    m.ctrl_fp32 = 1
    compare_rollout(m, 20, range(B), min_clean=0.0)


def test_single_step_horizon():
    m = WL.ball(B=3, horizon=1)
    compare_rollout(m, 1, range(3), min_clean=0.0)


# ------------------------------------------------------------------------------ gradients
# Gradients are compared element by element: |g_k - o_k| <= GRAD_RTOL * max(|o_k|, floor) with
# floor = ELEM_FLOOR * max_k |o_k| over the parameter group: an entry of at least a twentieth of
# the group's largest is held to 1e-3 of itself, smaller entries to 5e-5 of the largest. Small
# entries are sums of larger per-step terms that cancel (a servo gain's gradient sums
# (u - theta) w*_bar over the steps, with u and theta close), so their fp32 rounding is set by
# the terms, not by the sum; at 1e-2 the worst such entry (quadruped, 40 steps) misses by 10 %.
ELEM_FLOOR = 5e-2


def rel_err(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-12)


def elem_err(a, b, floor=ELEM_FLOOR):
    """Largest per-element error, each relative to max(|b_k|, floor * max |b|)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    top = float(np.abs(b).max()) if b.size else 0.0
    scale = np.maximum(np.abs(b), max(floor * top, 1e-30))
    return float((np.abs(a - b) / scale).max()) if b.size else 0.0


def gpu_grads(m, horizon, ckpt_every=None, rows_global=False):
    w = World(m, horizon=horizon, ckpt_every=ckpt_every, rows_global=rows_global)
    loss = torch.zeros(m.B, device="cuda")
    W = torch.tensor(m.W, device="cuda") if m.W is not None and len(m.W) else None
    w.rollout(W, loss)
    dloss = torch.ones(m.B, device="cuda")
    dW = torch.zeros(w.n_params, device="cuda") if w.n_params else None
    ds = torch.zeros(m.B, m.nb, 18, device="cuda")
    dp = {k: torch.zeros(getattr(m, k).shape, device="cuda") for k in
          ("mass", "inertia", "anchor", "limit", "motor", "sph_off", "sph_rad", "sph_mu", "sph_e", "loss_point", "loss_target")}
    w.backward(dloss, dW, ds, dp)
    w.sync()
    out = {k: v.cpu().double().numpy() for k, v in dp.items()}
    out["state0"] = ds.cpu().double().numpy()
    out["W"] = dW.cpu().double().numpy() if dW is not None else None
    out["loss"] = loss.cpu().double().numpy()
    return out


def check_grads(m, horizon, keys, instances, ckpt_every=None, with_W=False, rows_global=False):
    g = gpu_grads(m, horizon, ckpt_every, rows_global)
    Wsum = None
    for i in instances:
        L, go = O.rollout_grad(m, i, horizon=horizon)
        assert abs(g["loss"][i] - L) <= 1e-4 * max(1.0, abs(L))
        for k in keys:
            e = elem_err(g[k][i], go[k])
            assert e <= GRAD_RTOL, (m.name, i, k, e, g[k][i].ravel()[:6], go[k].ravel()[:6])
        if with_W:
            Wsum = go["W"] if Wsum is None else Wsum + go["W"]
    return g, Wsum


def test_ball_gradients_through_contact():
    m = WL.ball(B=4, horizon=60)
    for i in range(m.B):
        m.state0[i, 0, 2] = 0.6
        m.state0[i, 0, 15:18] = [1.0, -2.0, 0.5]
    check_grads(m, 60, ("state0", "sph_rad", "sph_mu", "mass", "inertia", "loss_target"), range(4))


def test_pendulum_gradients():
    m = WL.pendulum3(B=4, horizon=100)
    check_grads(m, 100, ("state0", "anchor", "inertia", "mass", "loss_point"), range(4))


def test_pendulum_gradients_with_checkpoint_segments():
    m = WL.pendulum3(B=4, horizon=100)
    check_grads(m, 100, ("state0", "anchor", "inertia", "mass"), range(4), ckpt_every=32)


def test_two_spheres_gradients():
    m = WL.two_spheres(B=4, e=0.3, mu=0.4)
    check_grads(m, 60, ("state0", "sph_rad", "sph_off", "mass", "inertia", "sph_mu", "sph_e"), range(4))


@pytest.mark.parametrize("fp32,T,ckpt", [(1, 40, None), (0, 10, None), (1, 40, 8)])
def test_quadruped_gradients_controller(fp32, T, ckpt):
    """Gradient w.r.t. every controller weight, the initial state and the model parameters
    (fp32 controller over 40 steps; bfloat16 controller over 10 steps, before rounding flips);
    full solver tape recorded by the rollout, or 8-step checkpoint segments recomputed."""
    m = WL.quadruped(B=4, horizon=T)
    m.ctrl_fp32 = fp32
    g, Wsum = check_grads(m, T, ("state0", "mass", "inertia", "anchor", "motor", "sph_off", "sph_rad"), range(4),
                          ckpt_every=ckpt, with_W=True)
    assert elem_err(g["W"], Wsum) <= GRAD_RTOL


def test_quadruped_runtime_topology_path(monkeypatch):
    """The quadruped normally runs the compiled-topology sweeps; the run-time topology loops
    must give the same answers (forced here)."""
    monkeypatch.setenv("DP_FORCE_RUNTIME_TOPOLOGY", "1")
    m = WL.quadruped(B=8, horizon=60)
    m.ctrl_fp32 = 1
    compare_rollout(m, 60, range(8), min_clean=0.5)
    m = WL.quadruped(B=2, horizon=20)
    m.ctrl_fp32 = 1  # 20 steps: beyond the horizon where bfloat16 rounding decisions are shared
    check_grads(m, 20, ("state0", "anchor", "motor"), range(2))


def _tc_case(name):
    """Workloads whose bfloat16 controllers run on the tensor cores inside the step: the quadruped's
    24-128-128-8 and its recurrent 32-128-128-16 (compiled topology), 24-64-64-8 and the uneven
    arm batch's 32-256-256-7 on the quadruped (run-time topology: the other hidden widths), and the
    4-DoF arm's 11-64-64-4 with a non-zero output layer."""
    if name == "arm4dof":
        m = WL.arm4dof(B=32, horizon=10)
        rng = np.random.default_rng(5)
        W = np.asarray(m.W, np.float32).copy()
        n3 = m.widths[2] * m.widths[3] + m.widths[3]
        W[-n3:] = rng.uniform(-0.5, 0.5, size=n3).astype(np.float32)
        m.W = W
        return m, False
    widths = {"24-128-128-8": None, "24-64-64-8": [24, 64, 64, 8], "32-256-256-7": [32, 256, 256, 7]}
    if name == "32-128-128-16 recurrent":
        return WL.quadruped(B=64, horizon=10, n_recurrent=8), False
    return WL.quadruped(B=64, horizon=10, widths=widths[name]), name != "24-128-128-8"


@pytest.mark.parametrize("name", ["24-128-128-8", "32-128-128-16 recurrent", "24-64-64-8", "32-256-256-7",
                                  "arm4dof"])
def test_tensor_core_controller_matches_simt(monkeypatch, name):
    """Every bfloat16 K0-H-H-NO controller with K0 <= 32, NO <= 16 and H in {64, 128, 256} runs on the
    tensor cores inside the step (hidden layers in 64-column chunks); the SIMT path (forced here)
    computes the same network with another summation order. Both must give the same step and the
    same gradients up to fp32 rounding (and the hi/lo bfloat16 split of the deltas), except where
    the other summation order rounds a hidden activation that lies within an fp32 rounding of a
    bfloat16 tie the other way: such an instance's trajectory then differs by a bfloat16 step, so
    the initial-state gradients are compared instance by instance and 90 % must agree (an error in
    the products would touch every instance)."""
    m, runtime = _tc_case(name)
    if runtime:
        monkeypatch.setenv("DP_FORCE_RUNTIME_TOPOLOGY", "1")
    out = []
    for force in (False, True):
        if force:
            monkeypatch.setenv("DP_FORCE_SIMT_CONTROLLER", "1")
        assert World(m, horizon=10).controller_kind == (CTRL_SIMT if force else CTRL_TENSOR)
        g = gpu_grads(m, 10)
        _, traj, loss, _ = gpu_rollout(m, 10)
        out.append((traj, g))
    (ta, ga), (tb, gb) = out
    assert np.abs(ta[1] - tb[1]).max() <= 1e-5
    errs = np.array([rel_err(ga["state0"][i], gb["state0"][i]) for i in range(m.B)])
    assert (errs <= 1e-3).mean() >= 0.9, np.sort(errs)[-8:]
    assert rel_err(ga["W"], gb["W"]) <= 1e-3
    assert np.abs(ga["W"]).max() > 0


@pytest.mark.parametrize("ckpt", [None, 8])
def test_gradients_with_rows_in_global_memory(ckpt):
    """The launch configuration that keeps the constraint rows in global memory (chosen for
    robots whose rows do not fit on chip, or by the autotuner) records them in the solver tape
    too: gradients of the whole tape and of recomputed segments match the oracle."""
    m = WL.quadruped(B=4, horizon=20)
    m.ctrl_fp32 = 1
    g, Wsum = check_grads(m, 20, ("state0", "mass", "anchor", "motor", "sph_rad"), range(4), ckpt_every=ckpt,
                          with_W=True, rows_global=True)
    assert elem_err(g["W"], Wsum) <= GRAD_RTOL
    check_grads(WL.pendulum3(B=4, horizon=60), 60, ("state0", "anchor", "mass"), range(4), ckpt_every=ckpt,
                rows_global=True)


def test_gradient_decay_quadruped():
    """Section 3.2's decay of the gradient per time step, on the quadruped (fp32 controller,
    whole tape and 8-step segments)."""
    for ckpt in (None, 8):
        m = WL.quadruped(B=4, horizon=30)
        m.ctrl_fp32 = 1
        m.grad_decay = 0.9
        g, Wsum = check_grads(m, 30, ("state0", "mass", "motor"), range(4), ckpt_every=ckpt, with_W=True)
        assert elem_err(g["W"], Wsum) <= GRAD_RTOL
