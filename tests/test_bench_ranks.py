"""Rank arithmetic of bench.py under torch.distributed (world size 2, gloo, CPU):
the slowest rank's time is taken on every rank and the job rate counts the
units of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.dist_barrier()
        ms = bench.dist_max(1.0 + 2.0 * rank)       # rank 0: 1 ms, rank 1: 3 ms
        out[rank] = (ms, bench.aggregate_rate(1000.0, ms, world))
        bench.dist_barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_rate():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        ms, rate = res[r]
        assert ms == 3.0                         # max over ranks
        assert rate == pytest.approx(2 * 1000.0 / 3e-3)   # both ranks' units over the slowest time


def test_single_process_is_identity():
    import bench
    assert bench.dist_max(2.5) == 2.5
    bench.dist_barrier()
    assert bench.aggregate_rate(10.0, 2.0, 1) == pytest.approx(5000.0)
