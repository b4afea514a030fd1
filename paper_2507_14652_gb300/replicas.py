"""Replica bookkeeping for runs on several GPUs.

Chains are independent units, so N GPUs run N replicas with no exchange on the
data path: each rank samples its own chains from its own Philox seed, and only the
timing is reduced across ranks (the job takes as long as its slowest rank).
"""


def replica_seed(rank, base=1000):
    """Philox seed of a rank's chains: distinct per rank, fixed across runs."""
    return int(base) + int(rank)


def reduce_max(x, dist=None, device="cpu"):
    """Maximum of a host scalar over all ranks (the scalar itself without a process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size, units_per_rank, seconds):
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    if seconds <= 0:
        raise ValueError("elapsed time must be positive")
    return int(world_size) * float(units_per_rank) / float(seconds)
