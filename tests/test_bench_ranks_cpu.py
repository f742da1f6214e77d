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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the CPU oracle, no GPU needed) prints one
    JSON line with the same metric, unit and workload as the GPU arm."""
    import json
    import subprocess
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "generations/s"
    assert d["config"]["workload"] == bench.WORKLOAD and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_headline_bytes_follow_the_algorithmic_count():
    """The headline roofline's numerator is the method's traffic per
    generation: read 2N parents and write 2N offspring (P*S bytes, S = 80 B
    per bit-packed order-20 matrix) plus 16 bytes per individual; the
    implementation's own extra parent placement is reported apart."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.bytes_per_generation(20, 10_000) == 40_000 * 80 + 16 * 40_000
    assert bench.bytes_per_generation(100, 5_000) == 20_000 * 1_600 + 16 * 20_000
    assert bench.impl_bytes_per_generation(20, 10_000) > bench.bytes_per_generation(20, 10_000)


def test_gram_algorithmic_work():
    """D = (m-1)(m-2)/2 dot products per matrix: D*m multiply-adds, or
    D*ceil(m/32) population counts on bit storage."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.gram_algorithmic_work(20) == (3_420, 171)
    assert bench.gram_algorithmic_work(32) == (14_880, 465)
    assert bench.gram_algorithmic_work(100) == (485_100, 19_404)
    assert bench.gram_algorithmic_work(256) == (8_290_560, 259_080)


def test_traffic_guard_tracks_the_kernel_sources():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.fused_sources_sha256()
    assert len(h) == 64 and h == bench.fused_sources_sha256()
