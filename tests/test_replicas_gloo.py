"""Multi-GPU runs are independent replicas (one cavity per rank, no
collective on the data path): bench.py takes the slowest rank's time and
reports all ranks' cell-steps over it.  This checks that host logic with two
gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    slowest = bench.max_over_ranks(times[rank], dist, "cpu")
    rate = bench.job_rate(world, 1000, slowest)
    out[rank] = (slowest, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    times = [0.8, 1.25]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    for r in range(world):
        slowest, rate = out[r]
        assert slowest == 1.25
        assert rate == pytest.approx(world * 1000 / 1.25)


def test_without_a_process_group():
    import bench

    assert bench.max_over_ranks(0.5, None, "cpu") == 0.5
    assert bench.job_rate(1, 100, 2.0) == 50.0
