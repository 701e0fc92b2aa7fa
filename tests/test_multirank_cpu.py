"""Multi-rank host logic of bench.py on CPU.

The method runs on one GPU; bench.py runs one independent replica per rank
(torchrun, one process per GPU) and reports the whole job: the units of all
ranks over the slowest rank's time.  These tests run that reduction with the
gloo backend at world size 2 on 127.0.0.1, and check that the reference arm
does its work on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r took 10 + 5 r ms: the job's step time is the slowest rank's
        got = bench.max_over_ranks(dist, "cpu", 10.0 + 5.0 * rank)
        assert got == 10.0 + 5.0 * (world - 1), got
        value = bench.job_throughput(world, 1000, 4, got / 1e3)
        assert abs(value - world * 1000 * 4 / (got / 1e3)) <= 1e-9 * value
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed not available")
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)


def test_single_process_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, "cpu", 12.5) == 12.5
    assert bench.job_throughput(1, 2 ** 20, 16, 0.5) == 2 ** 20 * 16 * 2


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_oracle_baseline_uses_one_leaf_per_core():
    """The CPU baseline runs one target leaf per worker, all stepping
    together, and reports the cores it used."""
    sys.path.insert(0, ROOT)
    import bench
    res = bench.oracle_sample("small", steps=1, warmup=0, workers=2)
    assert res["cores"] == 2 and res["leaves"] == 2
    assert res["rows"] == 2 * 64 and res["units_per_step"] == 2 * 64
    assert res["s_per_step"] > 0 and res["nproc"] >= 1 and res["cpu_model"]


def test_traffic_is_reported_only_for_the_captured_kernel_source():
    sys.path.insert(0, ROOT)
    import bench
    for b, src, sha, wl, fn in bench._traffic_records():
        assert b > 0 and src.endswith(".cu") and len(sha) == 16
    assert bench.recorded_traffic("p2p_tc.cu", "no-such-workload") is None


def test_reference_arm_prints_its_line_on_rank_zero():
    """Rank 0 runs the oracle sample in a child process with one BLAS thread
    (forking the per-core workers from a process with a running BLAS thread
    pool could hang them) and prints one JSON line."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
