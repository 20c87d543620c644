"""Multi-GPU replicas (one process per GPU, independent batches, no exchange on the data path):
the host-side rules the benchmark applies under torchrun, run as world-size-2 gloo process
groups on the CPU: distinct per-rank batches, the job's time as the maximum over ranks (with
the barrier), and the whole-job throughput (no GPU)."""
import os

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as tmp

from paper_1611_01652_gb300 import workloads as WL
from paper_1611_01652_gb300.replicas import max_over_ranks, replica_seed, whole_job_rate


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = WL.quadruped(B=4, horizon=2, seed=replica_seed(1002, rank))
        own = [10.0 + rank, 3.0 - rank, 7.0 * (rank + 1)]  # this rank's (total, fwd, bwd) ms
        dist.barrier()
        job = max_over_ranks(own, dist, "cpu")
        out[rank] = (m.state0.copy(), job, whole_job_rate(4 * 2, world, job[0]))
    finally:
        dist.destroy_process_group()


def test_replicas_world_size_2():
    port = 29500 + (os.getpid() % 1000)
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert not np.allclose(r0[0], r1[0])  # each rank simulates its own batch
    assert r0[1] == r1[1] == [11.0, 3.0, 14.0]  # element-wise max over the ranks
    assert r0[2] == r1[2] == 4 * 2 * 2 / (11.0 / 1e3)  # all ranks' units over the slowest time


def test_single_process_rules():
    assert max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    assert replica_seed(1002, 0) == 1002 and replica_seed(1002, 3) != replica_seed(1002, 2)
    assert whole_job_rate(4096 * 1000, 1, 1000.0) == 4096 * 1000
