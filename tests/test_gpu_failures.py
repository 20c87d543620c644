"""Failure detection through the C ABI, with every failure made on the host (no GPU fault):

* a non-finite initial state of one instance: dp_sync reports DP_ENAN naming it, its status word
  carries DP_INST_NAN_STATE, the other instances' losses are bit-identical to a clean batch;
* a non-finite loss adjoint of one instance: DP_INST_NAN_GRAD on that instance only, cleared by the
  next clean reverse pass;
* an allocation larger than the device: DP_ENOMEM from dp_create_world, the device memory it took
  returned, and the next world created and rolled out normally;
* a reverse pass without a rollout: DP_ESTATE, nothing enqueued.
"""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1611_01652_gb300 import workloads as WL  # noqa: E402
from paper_1611_01652_gb300.binding import (DP_ENAN, DP_ENOMEM, DP_ESTATE, INST_NAN_GRAD, INST_NAN_STATE,  # noqa: E402
                                            DPError, World)

pytestmark = pytest.mark.gpu

B, T = 8, 20


def rollout(m):
    w = World(m, horizon=T)
    loss = torch.zeros(m.B, device="cuda")
    w.rollout(torch.tensor(m.W, device="cuda"), loss)
    return w, loss


def status(w):
    st = torch.full((w.B,), -1, dtype=torch.int32, device="cuda")
    w.instance_status(st)
    torch.cuda.synchronize()
    return st.cpu().numpy()


def test_nan_initial_state_flags_that_instance_only():
    m = WL.quadruped(B=B, horizon=T)
    w0, clean = rollout(m)
    w0.sync()
    bad = m.subset(range(B))
    bad.state0[3, 0, 12] = np.nan  # torso velocity of instance 3
    w, loss = rollout(bad)
    with pytest.raises(DPError) as e:
        w.sync()
    assert e.value.status == DP_ENAN and "instance 3 " in str(e.value)
    st = status(w)
    assert st[3] & INST_NAN_STATE and not (np.delete(st, 3)).any(), st
    code, detail = w.error_detail()
    assert code == DP_ENAN and "1 of 8 instances (3)" in detail, detail
    l, c = loss.cpu().numpy(), clean.cpu().numpy()
    assert not np.isfinite(l[3])
    assert np.array_equal(np.delete(l, 3), np.delete(c, 3))  # the batch is unaffected


def test_nan_loss_adjoint_flags_that_gradient_only():
    m = WL.quadruped(B=B, horizon=T)
    w, _ = rollout(m)
    dl = torch.ones(B, device="cuda")
    dl[5] = float("nan")
    dW = torch.zeros(w.n_params, device="cuda")
    ds = torch.zeros(B, m.nb, 18, device="cuda")
    w.backward(dl, dW, ds)
    with pytest.raises(DPError) as e:
        w.sync()
    assert e.value.status == DP_ENAN and "instance 5 produced a non-finite gradient" in str(e.value)
    st = status(w)
    assert st[5] == INST_NAN_GRAD and not (np.delete(st, 5)).any(), st
    assert np.isfinite(np.delete(ds.cpu().numpy(), 5, axis=0)).all()
    w.backward(torch.ones(B, device="cuda"), dW, ds)  # a clean pass clears the flag
    w.sync()
    assert not status(w).any()


def test_allocation_failure_is_enomem_and_releases_everything():
    # worlds of earlier tests that are still unreferenced would otherwise be collected (and
    # their device memory freed) while the failing creation runs
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # a state checkpoint every step of a 2,000,000-step horizon: 330 GB of checkpoints alone
    m = WL.quadruped(B=256, horizon=2_000_000)
    with pytest.raises(DPError) as e:
        World(m, horizon=2_000_000, ckpt_every=1)
    assert e.value.status == DP_ENOMEM, e.value
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (8 << 20), (free0, free1)  # nothing the failed creation took is kept
    w, loss = rollout(WL.quadruped(B=B, horizon=T))
    w.sync()
    assert torch.isfinite(loss).all()


def test_backward_before_rollout_is_estate():
    m = WL.quadruped(B=B, horizon=T)
    w = World(m, horizon=T)
    with pytest.raises(DPError) as e:
        w.backward(torch.ones(B, device="cuda"), torch.zeros(w.n_params, device="cuda"))
    assert e.value.status == DP_ESTATE
    w.sync()
