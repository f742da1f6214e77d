"""The whole-job rate of bench.py over replica ranks (the N > 1 path: one
independent population per rank, no data-path collective), checked with two
gloo ranks on the CPU: the job rate is world x units over the slowest rank's
time, the same on every rank."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, slowest = bench.job_rate(times[rank], 500, world,
                                       lambda x: dist.all_reduce(x, op=dist.ReduceOp.MAX))
        out[rank] = (rate, slowest)
    finally:
        dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    world, times = 2, [0.5, 2.0]
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rate, slowest = res[r]
        assert slowest == pytest.approx(2.0)
        assert rate == pytest.approx(world * 500 / 2.0)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    rate, slowest = bench.job_rate(0.25, 100, 1)
    assert slowest == pytest.approx(0.25) and rate == pytest.approx(400.0)
