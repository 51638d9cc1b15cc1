"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): every rank
runs an independent replica; the job's throughput divides the atoms of all
ranks by the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [40.0, 55.0][rank]
    value, total = bench.job_throughput(torch, local_ms, 1000, 10, world, torch.device("cpu"))
    bench.barrier(world)
    results[rank] = (value, total)
    dist.destroy_process_group()


def test_job_throughput_uses_slowest_rank():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    # the manager's server process is spawned too: no fork of a threaded process
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    for r in range(world):
        value, total = results[r]
        assert total == pytest.approx(55.0)
        assert value == pytest.approx(2 * 1000 * 10 / 0.055)


def test_single_rank_throughput():
    import torch

    import bench

    v, t = bench.job_throughput(torch, 20.0, 500, 4, 1, torch.device("cpu"))
    assert t == 20.0 and v == pytest.approx(500 * 4 / 0.02)
