"""Multi-GPU replicas: instances are independent, so N GPUs run N independent batches (one
process per GPU) with no exchange on the data path. These helpers hold the host-side rules of
that mode: each rank's batch seed, the job's time as the maximum over ranks, and the whole-job
throughput."""
from __future__ import annotations


def replica_seed(base, rank):
    """Seed of rank ``rank``'s batch (distinct batches on every rank)."""
    return int(base) + 17 * int(rank)


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (the slowest rank's times); the
    values themselves without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(units_per_rank, world_size, ms):
    """Units processed by all ranks per second, given the job's time in milliseconds."""
    return float(units_per_rank) * int(world_size) / (float(ms) / 1e3)
