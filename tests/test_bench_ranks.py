"""The multi-rank path of bench.py on CPU, and its host-side helpers: two gloo ranks (world size 2) run
the barrier, the max-over-ranks timing and the whole-job throughput the GPU
bench uses under torchrun, and ranks other than 0 of the reference arm exit
without work.  No GPU: the ranks are host processes."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        bench.rank_barrier(world)
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")  # rank 1 is the slow one
        v = bench.job_throughput(world, 1000, 4, t)
        bench.rank_barrier(world)
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_job_by_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, v in res:
        assert t == 15.0
        assert v == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.rank_barrier(1)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1, 10, 2, 4.0) == pytest.approx(5000.0)


def test_reference_arm_ranks_other_than_zero_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=120, env=env)
    assert res.returncode == 0 and res.stdout.strip() == ""


def test_reference_arm_times_complete_oracle_solves():
    # the reference arm (the CPU oracle standing in for a reference implementation)
    # times whole oracle solves of the workload's grid, with the headline metric
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "1d-63-m64", "--steps", "2", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    line = json.loads(res.stdout.strip().splitlines()[-1])
    base = json.load(open(os.path.join(ROOT, "BASELINE.json")))
    assert line["impl"] == "reference" and line["metric"] == base["metric"]
    assert line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["sample"].startswith("full solve")
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_device_error_helper_matches_numpy():
    # bench's blockwise error against the separable solution, run on CPU tensors
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    B, N, M = 3, 5000, 8
    phi = rng.uniform(0.1, 1.0, N)
    W = rng.uniform(-1.0, 1.0, (B, M))
    u = phi[None, :, None] * W[:, None, :] + rng.uniform(-1e-6, 1e-6, (B, N, M)) * np.arange(1, B + 1)[:, None, None]
    want = max(np.abs(u[b] - np.outer(phi, W[b])).max() / (np.abs(phi).max() * np.abs(W[b]).max())
               for b in range(B))
    got = bench.rel_err_device(torch, torch.from_numpy(u), torch.from_numpy(phi), W)
    assert got == pytest.approx(want, rel=1e-12)


def test_bench_helpers_parse_cpu_lists_and_splits():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1608_05400_gb300 import mgwr
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    got = bench.parse_splits("sweep32=33,defect64=2", mgwr.KERNEL_CLASSES)
    assert got == {mgwr.KERNEL_CLASSES.index("sweep32"): 33, mgwr.KERNEL_CLASSES.index("defect64"): 2}
    with pytest.raises(ValueError):
        bench.parse_splits("nosuchclass=1", mgwr.KERNEL_CLASSES)
    # no GPU here: the placement helper finds nothing and changes nothing
    before = os.sched_getaffinity(0)
    with bench.GpuLocalHost(0) as host:
        pass
    assert os.sched_getaffinity(0) == before


def test_bench_nonlinear_helpers():
    sys.path.insert(0, ROOT)
    import bench
    # history sums M(M-1)/2 multiply-adds plus four Newton iterations of 30 flops per level
    assert bench.fas_line_flops(256) == 256 * 255 + 120 * 256
    u, base = bench.nonlinear_oracle_sample(0.4, 15, 16)
    assert u.shape == (15, 16) and np.isfinite(u).all()
    assert base["kind"] == "oracle" and base["value"] > 0 and base["cores"] >= 1
    assert "nonlinear-1d-255-m256" in bench.WORKLOADS
