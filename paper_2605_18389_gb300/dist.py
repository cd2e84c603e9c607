"""Multi-GPU plumbing for replicas: the path shards by independent measure pairs.

Every rank solves its own batch of pairs on its own GPU; no data-path collective exists.
Only the timing needs the other ranks: a barrier on both sides of the timed region and
the maximum of the per-rank times (the job is as fast as its slowest rank).
"""
import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def pair_seed(base, rank):
    """Seed of rank's batch: every rank draws different pairs."""
    return base + 1000 * rank


def max_over_ranks(value, device=None):
    """max of a per-rank float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps, seconds_max, world):
    """Whole-job rate: every rank ran `steps` iterations of its own batch."""
    return world * steps / seconds_max
