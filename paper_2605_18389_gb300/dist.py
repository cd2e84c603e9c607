"""Multi-GPU plumbing: the path shards by independent measure pairs.

Every rank solves its own share of the pairs on its own GPU; no data-path collective
exists (Alg. 1 runs per pair, and the three problems of a Sinkhorn divergence share
nothing with another pair's).  Two ways to use more GPUs:

* replicas (weak scaling): each rank draws and solves its own batch (`pair_seed`);
* sharding a given problem set (strong scaling): the pairs are split across ranks by a
  static cost model, cost = 3 problems x nlat^3 x iterations (the per-order Legendre
  contractions, O(L^3) per transform, dominate; App. C.1's semi-naive transform), with
  the longest-processing-time rule, and the per-pair S and status are gathered on the
  host at the end (`gather_by_index`).

The timing needs the other ranks: a barrier on both sides of the timed region and the
maximum of the per-rank times (the job is as fast as its slowest rank).
"""
import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def pair_seed(base, rank):
    """Seed of rank's batch: every rank draws different pairs."""
    return base + 1000 * rank


def pair_cost(nlat, iterations):
    """Static cost of one measure pair: its three problems' heat convolutions,
    3 x nlat^3 x iterations (up to a constant common to all pairs)."""
    return 3.0 * float(nlat) ** 3 * float(iterations)


def partition_by_cost(costs, world):
    """Split items 0..n-1 with the given costs over `world` ranks: longest processing time
    first (items by decreasing cost, ties by index; each goes to the rank with the least
    load so far, ties to the lower rank).  Returns one ascending index list per rank; every
    item lands on exactly one rank.  Deterministic, so every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def loads(costs, parts):
    """Total cost per rank of a partition."""
    return [sum(float(costs[i]) for i in p) for p in parts]


def gather_by_index(local, n, group=None):
    """Every rank passes {item index: result} for its own items; returns the list of all n
    results in index order on every rank (one all_gather of Python objects over the
    process group; the identity without one).  Raises if an item is missing or doubled."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, dict(local), group=group)
    else:
        parts = [dict(local)]
    out = [None] * n
    seen = [False] * n
    for p in parts:
        for i, v in p.items():
            if not 0 <= i < n or seen[i]:
                raise ValueError(f"item {i} out of range or gathered twice")
            seen[i] = True
            out[i] = v
    if not all(seen):
        raise ValueError(f"items missing from the gather: {[i for i in range(n) if not seen[i]]}")
    return out


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
