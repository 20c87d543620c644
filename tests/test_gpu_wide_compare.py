"""The 1.1 M-parameter controller's solver comparison against the FP64 oracle: the quadruped
with the 64-1024-1024-8 controller (bfloat16, batched tensor-core products), the plain
cold-start solver at 5, 10 and 20 sweeps and the damped previous-impulse start at 10 and 14
sweeps, each against the oracle's converged solve (200 sweeps) of the same robots: the state
error over the first 6 steps (relative, scale floor 1), the gradient error of the initial
state and of the controller weights (relative norms over a sample of 4 robots), and the mean
solve residual. The plain solver's errors must not grow with its sweeps, and every variant must
stay finite; the table is printed for the record (bench.py times the same variants)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import WS_PARAMS, World  # noqa: E402

from test_gpu_parity import rel_err  # noqa: E402

pytestmark = pytest.mark.gpu

B, T, REF_ITERS = 4, 6, 200
VARIANTS = [("plain_5", 5, False), ("plain_10", 10, False), ("plain_20", 20, False), ("damped_10", 10, True),
            ("damped_14", 14, True)]


def test_wide_controller_solver_comparison_against_oracle():
    m = WL.quadruped(B=B, horizon=T, widths=[64, 1024, 1024, 8])
    ref_states, ref_W, ref_s0 = [], 0.0, []
    for i in range(B):
        st, _, _, _ = O.rollout(m, i, horizon=T, iters=REF_ITERS, log=True)
        _, go = O.rollout_grad(m, i, horizon=T, iters=REF_ITERS)
        ref_states.append(st)
        ref_W = ref_W + go["W"]
        ref_s0.append(go["state0"])
    W = torch.tensor(m.W, device="cuda")
    table = {}
    for name, iters, warm in VARIANTS:
        w = World(m, horizon=T, iters=iters, warmstart=warm)
        if warm:
            w.set_warmstart(torch.zeros(WS_PARAMS, device="cuda"), 0.7)
        w.set_residual(True)
        loss = torch.zeros(B, device="cuda")
        traj = torch.zeros(T + 1, B, m.nb, 18, device="cuda")
        w.rollout(W, loss, traj)
        res = torch.zeros(B, device="cuda")
        w.get_residual(res)
        dW = torch.zeros(w.n_params, device="cuda")
        ds = torch.zeros(B, m.nb, 18, device="cuda")
        w.backward(torch.ones(B, device="cuda"), dW, ds)
        w.sync()
        traj = traj.cpu().double().numpy()
        ds = ds.cpu().double().numpy()
        serr = max(float((np.abs(traj[:, i] - ref_states[i]) / np.maximum(1.0, np.abs(ref_states[i]))).max())
                   for i in range(B))
        gs = max(rel_err(ds[i], ref_s0[i]) for i in range(B))
        gw = rel_err(dW.cpu().double().numpy(), ref_W)
        table[name] = {"iters": iters, "resid": float(res.mean().item()), "state_err": serr, "grad_state0_err": gs,
                       "grad_W_err": gw}
        assert np.isfinite([serr, gs, gw, table[name]["resid"]]).all(), (name, table[name])
        del w
    print("1.1M-parameter controller, errors against the FP64 oracle at %d sweeps:" % REF_ITERS)
    for k, v in table.items():
        print("  %-10s %s" % (k, v))
    p5, p10, p20 = table["plain_5"], table["plain_10"], table["plain_20"]
    for key in ("resid", "state_err", "grad_W_err"):
        assert p20[key] <= 1.1 * p10[key] + 1e-6 and p10[key] <= 1.1 * p5[key] + 1e-6, (key, p5, p10, p20)
