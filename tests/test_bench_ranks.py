"""Host logic of bench.py's multi-GPU form, on the CPU: each rank solves its
own replica (the path does not shard), the job time is the largest over the
ranks (all-reduce MAX over gloo here, NCCL on GPUs), and the reference arm
runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 * (rank + 1), torch.device("cpu"))
        q.put((rank, slowest, bench.job_throughput(world, 5, slowest)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's 20 ms; 2 ranks x 5 solves in 20 ms
    assert out == [(0, 20.0, 500.0), (1, 20.0, 500.0)]


def test_single_process_needs_no_group():
    torch = pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.job_throughput(1, 10, 250.0) == 40.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_kernel_roof_picks_the_larger_time_floor():
    """The FP64 SpMV of the 200x200x100 grid as measured (27.84M blocks: 3.68
    GB and 0.891 GFLOP in 0.776 ms) against 6,672 GB/s and 1.255 TFLOP/s: its
    FP64 floor (0.710 ms) is above its HBM floor (0.551 ms), so FP64 is the
    roof, at 0.915; an FP32 kernel of the same bytes and flops is HBM-bound."""
    import bench
    fma = {"fp64_tflops": 1.255, "fp32_tflops": 73.4}
    nbytes, fl = 132.0 * 27.84e6 + 4.0 * 4e6 + 64.0 * 4e6, 32.0 * 27.84e6
    r = bench.kernel_roof(0.776, nbytes, fl, True, 6672.0, fma)
    assert r["roof"] == "fp64" and r["fp"] == "fp64"
    assert abs(r["fma_frac"] - fl / 0.776e-3 / 1.255e12) < 1e-12
    assert abs(r["roof_frac"] - r["fma_frac"]) < 1e-12 and abs(r["roof_frac"] - 0.9148) < 1e-3
    assert abs(r["frac"] - nbytes / 0.776e-3 / 6672e9) < 1e-12
    r32 = bench.kernel_roof(0.776, nbytes, fl, False, 6672.0, fma)
    assert r32["roof"] == "hbm" and r32["roof_frac"] == r32["frac"]
    # no measured FMA rate: HBM is the roof and the compute fractions are zero
    r0 = bench.kernel_roof(0.776, nbytes, fl, True, 6672.0, {"error": "no device"})
    assert r0["roof"] == "hbm" and r0["fma_frac"] == 0.0
