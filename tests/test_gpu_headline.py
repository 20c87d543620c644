"""The configuration bench.py times, at its full batch and in its launch configuration, against the
FP64 oracle on sampled instances: the quadruped at B = 4096 in one launch of each kernel (128
groups of 32 instances; the four-warp reverse kernel), the bfloat16 24-128-128-8 controller on the
tensor cores, the damped previous-impulse warm start (alpha = 0.7, zero network) at 10 sweeps, and
the whole solver tape recorded by the rollout.

Over the first 10 steps (the horizon over which bfloat16 rounding decisions of the controller are
shared by an fp32 and an fp64 computation; an instance that differs is set aside only if one of
its roundings came within 1e-6 of a tie, from the oracle's margin log, and at least half of the
sample must match): activation sets bit-exact away from near-ties, states
within 1e-4 relative (scale floor 1), losses within 1e-4, and, for a weighted loss over the sample
(the other instances' adjoints zero), the initial-state adjoint of every sampled instance and the
controller-weight gradient element by element within 1e-3 (floor as in the parity module)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import WS_PARAMS, World  # noqa: E402

from test_gpu_parity import GRAD_RTOL, STATE_RTOL, divergence_step, elem_err  # noqa: E402

pytestmark = pytest.mark.gpu

B, T, ITERS, ALPHA = 4096, 10, 10, 0.7
SAMPLE = [0, 1, 31, 32, 500, 777, 1024, 2048, 2500, 3001, 3500, 4095]


def test_headline_configuration_matches_oracle_on_sampled_instances():
    m = WL.quadruped(B=B, horizon=T)
    m.warmstart, m.ws_W, m.ws_alpha = 1, np.zeros(WS_PARAMS), ALPHA
    w = World(m, horizon=T, iters=ITERS, warmstart=True)
    w.set_warmstart(torch.zeros(WS_PARAMS, device="cuda"), ALPHA)
    assert w.ckpt_every == 1  # the whole tape, as in the benchmark
    W = torch.tensor(m.W, device="cuda")
    loss = torch.zeros(B, device="cuda")
    traj = torch.zeros(T + 1, B, m.nb, 18, device="cuda")
    act = torch.zeros(T, B, w.n_slots, dtype=torch.uint8, device="cuda")
    w.rollout(W, loss, traj, act)
    c = np.linspace(0.5, 2.0, len(SAMPLE))
    dl = torch.zeros(B, device="cuda")
    dl[SAMPLE] = torch.tensor(c, dtype=torch.float32, device="cuda")
    dW = torch.zeros(w.n_params, device="cuda")
    ds = torch.zeros(B, m.nb, 18, device="cuda")
    w.backward(dl, dW, ds)
    w.sync()
    loss, traj, act = loss.cpu().double().numpy(), traj.cpu().double().numpy(), act.cpu().numpy()
    dW, ds = dW.cpu().double().numpy(), ds.cpu().double().numpy()
    kinds = O.schedule(m)["kind"]
    passed, excused = [], []
    for k, i in enumerate(SAMPLE):
        st, L, a_o, gap, marg = O.rollout(m, i, horizon=T, iters=ITERS, log=True, margins=True)
        L2, go = O.rollout_grad(m, i, horizon=T, iters=ITERS)
        assert abs(L - L2) <= 1e-12 * max(1.0, abs(L))
        err = np.abs(traj[:, i] - st) / np.maximum(1.0, np.abs(st))
        ok = (divergence_step(act[:, i], a_o, gap, kinds) == T and err.max() <= STATE_RTOL and
              abs(loss[i] - L) <= STATE_RTOL * max(1.0, abs(L)) and
              elem_err(ds[i], c[k] * go["state0"]) <= GRAD_RTOL)
        if ok:
            passed.append((i, c[k], go["W"]))
        else:
            # only a bfloat16 rounding that came near a tie may make the two sides differ
            assert marg.min() <= 1e-6, (i, err.max(), elem_err(ds[i], c[k] * go["state0"]), marg.min())
            excused.append(i)
    assert len(passed) >= len(SAMPLE) // 2, ([p[0] for p in passed], excused)
    # the controller-weight gradient of the instances that passed, alone in the loss
    dl = torch.zeros(B, device="cuda")
    dl[[p[0] for p in passed]] = torch.tensor([p[1] for p in passed], dtype=torch.float32, device="cuda")
    dW = torch.zeros(w.n_params, device="cuda")
    w.backward(dl, dW)
    w.sync()
    dW = dW.cpu().double().numpy()
    Wsum = sum(p[1] * p[2] for p in passed)
    assert elem_err(dW, Wsum) <= GRAD_RTOL
    assert np.abs(dW).max() > 0
