"""dp_backward_noalloc: the controller gradient for callers that cannot allocate device memory
while they run (a training loop replayed from a captured CUDA graph, an application whose
device memory is fixed up front). Its scratch is a static device array instead of a buffer
allocated for the world; its result must equal dp_backward's, call after call.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import World  # noqa: E402

GRAD_RTOL = 1e-3


@pytest.mark.gpu
def test_backward_noalloc_matches_backward_on_two_calls():
    m = WL.quadruped(B=64, horizon=40)
    w = World(m)
    W = torch.tensor(m.W, device="cuda")
    loss = torch.zeros(m.B, device="cuda")
    w.rollout(W, loss)
    dloss = torch.linspace(0.5, 1.5, m.B, device="cuda")
    ref = torch.zeros(w.n_params, device="cuda")
    w.backward(dloss, ref)
    w.sync()
    ref = ref.cpu().double().numpy()
    assert np.isfinite(ref).all() and np.linalg.norm(ref) > 0
    for _ in range(2):
        dW = torch.full((w.n_params,), float("nan"), device="cuda")
        w.backward_noalloc(dloss, dW)
        w.sync()
        got = dW.cpu().double().numpy()
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) <= GRAD_RTOL * np.linalg.norm(ref)
    w.free()
