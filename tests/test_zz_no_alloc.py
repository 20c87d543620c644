"""dp_backward_noalloc: the controller gradient for callers that cannot allocate device memory
while they run (an application that reserves its device memory up front, or runs where an
allocation could block or fail). Its scratch is a static device array instead of a buffer
allocated for the world; its result must equal dp_backward's, call after call.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import World  # noqa: E402

GRAD_RTOL = 1e-3


def _world(B, T, dloss_lo, dloss_hi, dw_splits=0):
    m = WL.quadruped(B=B, horizon=T)
    w = World(m, dw_splits=dw_splits)
    loss = torch.zeros(m.B, device="cuda")
    w.rollout(torch.tensor(m.W, device="cuda"), loss)
    dloss = torch.linspace(dloss_lo, dloss_hi, m.B, device="cuda")
    ref = torch.zeros(w.n_params, device="cuda")
    w.backward(dloss, ref)
    w.sync()
    ref = ref.cpu().double().numpy()
    assert np.isfinite(ref).all() and np.linalg.norm(ref) > 0
    return w, dloss, ref


def _noalloc(w, dloss):
    dW = torch.full((w.n_params,), float("nan"), device="cuda")
    w.backward_noalloc(dloss, dW)
    w.sync()
    got = dW.cpu().double().numpy()
    assert np.isfinite(got).all()
    return got


def _close(got, ref):
    return np.linalg.norm(got - ref) <= GRAD_RTOL * np.linalg.norm(ref)


@pytest.mark.gpu
def test_backward_noalloc_matches_backward_on_two_calls():
    w, dloss, ref = _world(64, 40, 0.5, 1.5)
    for _ in range(2):
        assert _close(_noalloc(w, dloss), ref)
    w.free()


@pytest.mark.gpu
def test_backward_noalloc_with_clamped_splits_and_no_stale_scratch():
    """128 split-K slices ask for 128 x 128 x 128 partial sums of the hidden layer, more than the
    static array holds: the call lowers the split count for that layer. Between two calls on one
    world, a call on another world (other loss adjoints, other splits) leaves different partial
    sums in the shared array; the first world's result must not change. The call takes no device
    memory."""
    a, da, ra = _world(64, 40, 0.5, 1.5, dw_splits=128)
    b, db, rb = _world(32, 30, -1.0, 2.0, dw_splits=16)
    assert _close(_noalloc(a, da), ra)
    assert _close(_noalloc(b, db), rb)
    dW = torch.full((a.n_params,), float("nan"), device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    a.backward_noalloc(da, dW)
    a.sync()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert _close(dW.cpu().double().numpy(), ra)
    a.free()
    b.free()
