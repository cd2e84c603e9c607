"""World-size-2 gloo ranks on CPU: the replica timing aggregation of bench.py."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2605_18389_gb300 import dist as sd
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = sd.env()
        assert (w, r, lr) == (world, rank, rank)
        my_time = 1.0 + rank            # rank 1 is the slow one
        dist.barrier()
        t = sd.max_over_ranks(my_time)
        out[rank] = (t, sd.job_throughput(100, t, w), sd.pair_seed(5000, rank))
    finally:
        dist.destroy_process_group()


def test_replica_timing_uses_slowest_rank():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.0          # max of 1.0 and 2.0 on both ranks
    assert out[0][1] == out[1][1] == 100.0        # 2 ranks x 100 steps / 2 s
    assert out[0][2] != out[1][2]                 # different pairs per rank


def test_single_process_defaults():
    from paper_2605_18389_gb300 import dist as sd
    assert sd.max_over_ranks(3.5) == 3.5
    assert sd.job_throughput(10, 2.0, 1) == 5.0


def _config3_costs():
    """The multi-grid workload's 96 pairs: grids 64/96/128/180 x tau {0.1, 1, 10} x 8 pairs, T = 200."""
    from paper_2605_18389_gb300 import dist as sd
    return [sd.pair_cost(nlat, 200) for nlat in (64, 96, 128, 180) for _ in range(3) for _ in range(8)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_cost_partition_covers_every_pair_once_and_balances(world):
    from paper_2605_18389_gb300 import dist as sd
    costs = _config3_costs()
    parts = sd.partition_by_cost(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    ld = sd.loads(costs, parts)
    # LPT bound: the heaviest rank exceeds the mean by at most the largest single item
    assert max(ld) <= sum(costs) / world + max(costs) + 1e-6
    # with 24 pairs of the largest grid the split is tight for these worlds
    assert max(ld) / (sum(costs) / world) < 1.10
    assert sd.partition_by_cost(costs, world) == parts          # deterministic


def test_cost_partition_small_cases():
    from paper_2605_18389_gb300 import dist as sd
    # 4 items [8, 7, 6, 5] on 2 ranks: 8 -> r0, 7 -> r1, 6 -> r1 (7 < 8), 5 -> r0: loads 13, 13
    parts = sd.partition_by_cost([8, 7, 6, 5], 2)
    assert parts == [[0, 3], [1, 2]]
    # more ranks than items: the extra ranks get nothing
    assert sd.partition_by_cost([1.0, 2.0], 4) == [[1], [0], [], []]
    with pytest.raises(ValueError):
        sd.partition_by_cost([1.0], 0)


def _gather_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2605_18389_gb300 import dist as sd
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = _config3_costs()
        parts = sd.partition_by_cost(costs, world)
        # each rank 'solves' its own pairs: S = 1.5 * index, status = index % 3 - 1
        local = {i: (1.5 * i, i % 3 - 1) for i in parts[rank]}
        allr = sd.gather_by_index(local, len(costs))
        out[rank] = (parts[rank], allr)
    finally:
        dist.destroy_process_group()


def test_sharded_gather_returns_every_pair_in_order():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_gather_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    n = len(_config3_costs())
    expect = [(1.5 * i, i % 3 - 1) for i in range(n)]
    assert list(out[0][1]) == expect and list(out[1][1]) == expect
    assert set(out[0][0]).isdisjoint(out[1][0]) and len(out[0][0]) + len(out[1][0]) == n


def test_gather_rejects_missing_or_doubled_items():
    from paper_2605_18389_gb300 import dist as sd
    assert sd.gather_by_index({1: "b", 0: "a"}, 2) == ["a", "b"]
    with pytest.raises(ValueError):
        sd.gather_by_index({0: "a"}, 2)
    with pytest.raises(ValueError):
        sd.gather_by_index({0: "a", 5: "x"}, 2)
