"""The torch.autograd.Function over the library (binding.make_rollout_function): its gradients,
through torch.autograd.grad of a weighted sum of the per-instance losses, equal World.backward
with the same loss adjoint bit for bit, and match the FP64 oracle's gradients element by element
(quadruped with the fp32 controller, 10 steps, so that no bfloat16 rounding decision can differ)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1611_01652_gb300 import binding  # noqa: E402
from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import World  # noqa: E402

from test_gpu_parity import GRAD_RTOL, elem_err  # noqa: E402

pytestmark = pytest.mark.gpu

B, T = 4, 10


def test_autograd_function_matches_world_backward_and_oracle():
    m = WL.quadruped(B=B, horizon=T)
    m.ctrl_fp32 = 1
    c = torch.tensor([1.0, -0.5, 2.0, 0.25], device="cuda")  # loss weights: the adjoint of each loss
    Rollout = binding.make_rollout_function()
    W = torch.tensor(m.W, device="cuda", requires_grad=True)
    s0 = torch.tensor(m.state0, device="cuda", dtype=torch.float64, requires_grad=True)  # converted by the function
    loss = Rollout.apply(W, s0, World(m, horizon=T))
    gW, gs = torch.autograd.grad((loss * c).sum(), (W, s0))

    w = World(m, horizon=T)
    l2 = torch.zeros(B, device="cuda")
    w.rollout(W.detach(), l2)
    dW = torch.zeros(w.n_params, device="cuda")
    ds = torch.zeros(B, m.nb, 18, device="cuda")
    w.backward(c, dW, ds)
    w.sync()
    assert torch.equal(loss.detach(), l2)
    assert gs.dtype == torch.float64
    assert torch.equal(gW, dW) and torch.equal(gs.float(), ds)

    gW, gs, cc = gW.cpu().double().numpy(), gs.cpu().double().numpy(), c.cpu().double().numpy()
    Wsum = 0.0
    for i in range(B):
        L, go = O.rollout_grad(m, i, horizon=T)
        assert abs(loss[i].item() - L) <= 1e-4 * max(1.0, abs(L))
        assert elem_err(gs[i], cc[i] * go["state0"]) <= GRAD_RTOL, i
        Wsum = Wsum + cc[i] * go["W"]
    assert elem_err(gW, Wsum) <= GRAD_RTOL
    assert np.abs(gW).max() > 0
