"""CPU checks of bench.py's multi-rank logic: N > 1 runs independent replicas (no collective
on the data path); the job's step time is the slowest rank's, and the value is the work of
all ranks over that time. Two gloo ranks on 127.0.0.1 stand in for two GPUs; the reference
arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 20.0][rank]  # rank 1 is the slow one
        m = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (m, bench.job_gbs(world, 1e9, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    m, gbs = res[0]
    assert m == 20.0
    assert gbs == pytest.approx(2 * 1e9 / 0.020 / 1e9)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_gbs(1, 2e9, 1.0) == pytest.approx(2000.0)


@pytest.mark.parametrize("rank", [1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0
    assert p.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_batch_roofline_takes_the_slower_bound():
    b = bench
    peak, _ = b.measured_peaks()
    r = b.batch_roofline(peak * 1e9 * 1e-3, 0.0, 2.0)  # 1 ms of bytes, measured 2 ms
    assert r["bound"] == "hbm" and abs(r["frac"] - 0.5) < 1e-12 and abs(r["bound_ms"] - 1.0) < 1e-12
    r = b.batch_roofline(0.0, b.FFMA_PEAK_TFLOPS * 1e12 * 4e-3, 8.0)  # 4 ms of flops, measured 8 ms
    assert r["bound"] == "alu" and abs(r["frac"] - 0.5) < 1e-12


def test_stream_roofline_takes_the_slower_bound():
    b = bench
    # 1 GB at 1000 GB/s = 1 ms; 1 Tflop at 2 Tflop/s = 500 ms: arithmetic-bound, measured 1000 ms
    r = b.stream_roofline("k", 1e9, 1e12, 1000.0, 2.0, "measured", 1000.0, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 1.0) < 1e-12 and abs(r["frac"] - 0.5) < 1e-12 and abs(r["bound_ms"] - 500.0) < 1e-9
    # the same bytes with few flops: HBM-bound
    r = b.stream_roofline("k", 1e9, 1e6, 2.0, 2.0, "measured", 1000.0, "measured", traffic=123)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and abs(r["frac"] - 0.5) < 1e-12 and r["traffic"] == 123


def test_bottom_stream_entries_counts_the_lowest_levels():
    class Info:
        depth = 6
        rank = 4
        dense_entries = 77
        coupling_per_level = [0, 0, 1, 2, 3, 4, 5] + [0] * 25
    cpl, dns = bench.bottom_stream_entries(Info())
    assert cpl == (1 + 2 + 3 + 4 + 5) * 16 and dns == 77  # levels 2..6 (the lowest min(6, 4) + 1)
