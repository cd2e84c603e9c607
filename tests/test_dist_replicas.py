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
