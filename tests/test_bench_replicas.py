"""Multi-GPU path of bench.py on CPU: independent replicas, one per rank (the
solves do not shard), whole-job throughput from the slowest rank's time, reduced
with a real process group (gloo, world size 2)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank            # rank 1 is the slow replica
    total = bench.max_over_ranks(local_ms, dist, torch, "cpu")
    out[rank] = (total, bench.replica_throughput(8 * 3, world, total))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    total, value = res[0]
    assert total == 150.0
    assert abs(value - 2 * 24 / 0.150) < 1e-9


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, None, None, "cpu") == 42.0
    assert bench.replica_throughput(10, 1, 1000.0) == 10.0
