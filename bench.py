"""Benchmark: space-time unknowns per second of MGWR solves on GB300.

Default workload (one "step" = one complete solve): 2-D MGWR, 511 x 511
interior grid, M = 4096 time steps on (0, 1], alpha = 0.5, exact solution
u = t^alpha sin(pi x) sin(pi y) (f from D^a t^a = Gamma(1+a)), 5-point
Laplacian, V(1,1) red-black cycles from u = 0 until the relative
infinity-norm defect is below 1e-8.  1.07e9 space-time unknowns; each FP64
field is 8.56 GB, far larger than the 129 MB L2, so no flush is needed between
steps.  `value` is the mixed form with FP32 cycles and an FP64 outer defect and
update (MGWR_MIXED); the same line carries the plain FP64 solve and the mixed
form with a double-float outer defect (MGWR_MIXED_DD) on the same workload
(--arms), each with its error against the oracle's exact discrete solution and
the IEEE-double defect of its result.  Other workloads (--workload):
2d-255-m1024 (2-D 255 x 255, M = 1024, u = t^2 sin sin, FP64 to 1e-10),
1d-63-m64 (1-D 63 points, M = 64), batch4096-2d-63-m256 (4096 independent 2-D
63 x 63, M = 256 solves with alpha ~ U[0.1, 0.9] in one batched handle, mixed
to 1e-8), 1d-4095-m65536 (1-D 4095 points, M = 65536, alpha = 0.2,
u = t^alpha sin, to 1e-8 with double-float inner cycles, as FP32 inner cycles
stall on h = 1/4096; --precision fp64 for the FP64 form) and served (the served
request stream; each request's precision chosen by MGWR_AUTO).

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--precision fp64|mixed|mixed_dd|dd|auto] [--arms P,P]
                  [--workload 2d-511-m4096|2d-255-m1024|1d-63-m64|
                              batch4096-2d-63-m256|1d-4095-m65536|served]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

Prints one JSON line.  Multi-GPU runs (torchrun, one rank per GPU) are
independent replicas of the same solve (weak scaling, no collective on the data
path); value = all ranks' unknowns / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

T, ALPHA = 1.0, 0.5
NU1, NU2, CYCLE = 1, 1, 1
METRIC = "space-time unknowns/s to rel-res 1e-8 (FP64 vs mixed); served p50/p99 latency"
DEFAULT_WORKLOAD = "2d-511-m4096"
# workload name -> (d, n, M, batch, exact solution, tolerance, default precision, description)
WORKLOADS = {
    "2d-255-m1024": (2, 255, 1024, 1, "t2", 1e-10, "fp64",
           "2-D plain MGWR 255x255 interior, M=1024 on (0,1], u=t^2 sin(pi x) sin(pi y)"),
    "1d-63-m64": (1, 63, 64, 1, "t2", 1e-10, "fp64", "1-D plain MGWR 63 interior points, M=64, u=t^2 sin(pi x)"),
    "2d-511-m4096": (2, 511, 4096, 1, "talpha", 1e-8, "mixed",
           "2-D MGWR 511x511 interior, M=4096, u=t^alpha sin(pi x) sin(pi y)"),
    "batch4096-2d-63-m256": (2, 63, 256, 4096, "t2", 1e-8, "mixed",
            "4096 independent 2-D 63x63, M=256 solves, alpha~U[0.1,0.9] (seed 1608), one batched handle"),
    "1d-4095-m65536": (1, 4095, 65536, 1, "talpha", 1e-8, "dd",
            "1-D MGWR 4095 interior points, M=65536 (long memory), u=t^alpha sin(pi x)"),
    "served": (0, 0, 0, 0, "", 1e-8, "auto", "served stream"),
    "nonlinear-1d-255-m256": (1, 255, 256, 1, "", 1e-10, "fp64",
            "1-D nonlinear problem of Sec. 7 (Table table_nonlinear, 256x256): D(u)=1+u^2, c=1, "
            "f=1 on (0,1)x(0,1], waveform relaxation FAS V(0,1) from u=0"),
}
# alpha of a workload when --alpha is not given
WORKLOAD_ALPHA = {"1d-4095-m65536": 0.2}
# FP32 cycles per outer defect of a mixed workload when --inner is not given
WORKLOAD_INNER = {"batch4096-2d-63-m256": 3}
# extra precisions timed beside the value on the same workload, and their steps
WORKLOAD_ARMS = {"2d-511-m4096": ("fp64", "mixed_dd")}
# CPU-baseline sample: a complete oracle solve (every time level) of the workload's
# spatial grid with this many time steps on the same (0, T] (a few seconds of host
# work); the --impl reference arm times the same sample
ORACLE_SAMPLE_M = {"2d-511-m4096": 32, "2d-255-m1024": 128, "1d-63-m64": 64,
                   "batch4096-2d-63-m256": 256, "1d-4095-m65536": 512}
UNIT = "unknowns/s"
# --precision names and the library's codes (MGWR_FP64 .. MGWR_AUTO)
PREC_CODES = {"fp64": 0, "mixed": 1, "mixed_dd": 2, "dd": 3, "auto": 4}
PREC_NAMES = {v: k for k, v in PREC_CODES.items()}
DTYPES = {"fp64": "f64", "mixed": "f32 cycles + f64 iterate/update/stencil, outer-defect time "
                                  "convolution in f32x2 (double-float; f64 below tol 1e-10)",
          "mixed_dd": "f32 cycles + f32x2 (double-float) defect/update",
          "dd": "f32x2 (double-float) cycles, defect and update",
          "auto": "f32 cycles + f32x2 (double-float) defect/update, f32x2 cycles on grids "
                  "with h <= 1/4096"}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 issue rate of a GB300 SM by unit count: 2 FP64 FMA per clock, peak at the
# maximum clock (FMA chains sustain 1.68 per clock: `--probe-peaks`, mgwr_peak_probe,
# 1.06 TFLOP/s at 2070 MHz on 152 SMs).
FP64_FMA_PER_CLK_PER_SM = 2
SMS = 152
# FP32 lanes of a GB300 SM (4 partitions x 32)
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per smoothed line of k_sweep<double> from an ncu
# capture of the finest-level half-sweep of the default workload (772.5 MB for
# 32,513 lines of 1024 doubles; profiles/k_sweep_fp64_2d_255x255_M1024.md).
SWEEP64_DRAM_BYTES_PER_LINE_M1024 = 23758.0
# DRAM bytes per line of further kernels from single-kernel ncu captures (see
# profiles/), by kernel class and M
# (k_defect<double, float>: 1059.1 MB read + 254.9 MB written for 16,129 lines of 4096,
# profiles/k_defect_fp64_outer_2d_127x127_M4096.md; k_sweep_rp_res, the resident paired
# sweep: 264.5 + 102.2 MB for 8065 red lines, 396.6 + 218.7 MB for 8064 black lines that
# record their changes, weighted as a V(1,1) cycle runs them per level (two red, one
# recording black, one plain black), profiles/k_sweep_rp_res_fp32_2d_127x127_M4096.md;
# k_defect_update_rp: 793.7 + 737.1 MB for 16,129 lines of 4096,
# profiles/k_defect_outer_forms_2d_127x127_M4096.md)
NCU_DRAM_BYTES_PER_LINE: dict = {"defect64": {4096: 81468.0}, "sweep32": {4096: 53174.0},
                                 "defect32": {4096: 94908.0}}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default=None, choices=["fp64", "mixed", "mixed_dd", "dd", "auto"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--arms", default=None,
                   help="comma-separated precisions timed beside the value on the same "
                        "workload (default: the workload's list; 'none' for none)")
    p.add_argument("--arm-steps", type=int, default=None,
                   help="timed steps of each extra arm (default: fewer for slow arms)")
    p.add_argument("--e2e-steps", type=int, default=None,
                   help="timed steps of the end-to-end measurement (default min(steps, 5))")
    p.add_argument("--requests", type=int, default=2000, help="served: first R requests of the stream")
    p.add_argument("--slots", type=int, default=8, help="served: server slots")
    p.add_argument("--rate", type=float, default=None,
                   help="served: Poisson arrival rate, requests/s (default 0.7 x the sustained rate)")
    p.add_argument("--submit", default="buffer", choices=["buffer", "copy"],
                   help="served: right-hand sides into server-lent page-locked buffers, or copied")
    p.add_argument("--policy", default="fifo", choices=["fifo", "smallest"],
                   help="served: server admission order")
    p.add_argument("--inner", type=int, default=None, help="mixed modes: FP32 cycles per outer defect")
    p.add_argument("--outer-switch", type=float, default=None,
                   help="mixed modes: fraction of the last full outer defect down to which an "
                        "outer step carries its defect by the correction (mgwr_set_outer_switch)")
    p.add_argument("--alpha", type=float, default=None)
    p.add_argument("--no-autotune", action="store_true", help="keep the default engine launch shapes")
    p.add_argument("--split", default=None,
                   help="CLASS=E[,CLASS=E]: engine launch shape of a kernel class on every level, "
                        "set after the tuner (e.g. sweep32=33: the tensor-core sweep; profiling)")
    p.add_argument("--shape", default=None,
                   help="d,n,M replacing the workload's grid (small cases for profiling)")
    p.add_argument("--batch", type=int, default=None, help="instances replacing the workload's batch")
    p.add_argument("--probe-peaks", action="store_true",
                   help="print the FP64 / FP32 FMA-chain peaks (mgwr_peak_probe) with the SM "
                        "clocks sampled meanwhile, and exit")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_barrier(world: int) -> None:
    """Barrier over the job's ranks (nothing to wait for with one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest of the ranks' values of x: the job's time is its slowest rank's."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, unknowns_per_rank: int, steps: int, t_max_ms: float) -> float:
    """Whole-job unknowns per second: every rank solves its own replica."""
    return world * unknowns_per_rank * steps / (t_max_ms * 1e-3)


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh)
    except OSError:
        return {}


def parse_cpulist(text: str) -> set:
    """CPUs of a sysfs cpulist such as "0-15,32,40-41"."""
    cpus = set()
    for part in text.strip().split(","):
        if part:
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def parse_splits(text: str, classes) -> dict:
    """{class index: split} from "CLASS=E[,CLASS=E]" (names from `classes`)."""
    out = {}
    for item in text.split(","):
        name, val = item.split("=")
        out[list(classes).index(name.strip())] = int(val)
    return out


def gpu_local_cpus(index: int):
    """The CPUs of the NUMA node the GPU is attached to (from its PCI device in
    sysfs), or None when that cannot be read."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=30).stdout.strip()
        dom, rest = out.split(":", 1)
        path = f"/sys/bus/pci/devices/{dom[-4:].lower()}:{rest.lower()}/local_cpulist"
        with open(path) as fh:
            cpus = parse_cpulist(fh.read())
        return cpus & set(os.sched_getaffinity(0)) or None
    except (OSError, ValueError, subprocess.SubprocessError):
        return None


class GpuLocalHost:
    """Runs a block on the GPU's local CPUs, so that host buffers first touched
    there (pinned copies of the inputs and outputs) sit in the memory next to the
    GPU; restores the process's affinity afterwards (a setting of this process)."""

    def __init__(self, index: int):
        self.cpus = gpu_local_cpus(index)
        self.saved = None

    def __enter__(self):
        if self.cpus:
            self.saved = os.sched_getaffinity(0)
            os.sched_setaffinity(0, self.cpus)
        return self

    def __exit__(self, *exc):
        if self.saved is not None:
            os.sched_setaffinity(0, self.saved)


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.path = None
        self.proc = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def conv_flops_per_line(Mv: int) -> float:
    """Algorithmic flops of one line's causal FFT convolution: half of a line
    pair's complex work.  Up to M = 4096 one transform pair of length L = 2M
    (5 L log2 L each) and the spectrum product (6 L); beyond, P = M/4096 blocks
    with transforms of length 8192 and P(P+1)/2 block products accumulated
    (8 flops per value)."""
    if Mv <= 4096:
        L = 2 * Mv
        return 0.5 * (2 * 5 * L * math.log2(L) + 6 * L)
    Lb, P = 8192, Mv // 4096
    return 0.5 * (2 * P * 5 * Lb * math.log2(Lb) + 8 * Lb * P * (P + 1) / 2)


def sweep_flops_per_line(d: int, Mv: int) -> float:
    """Convolution plus the stencil gather (2d adds, one multiply, one add per
    time value) of one smoothed time line."""
    return conv_flops_per_line(Mv) + (2 * d + 2) * Mv


def defect_flops_per_line(d: int, Mv: int) -> float:
    return conv_flops_per_line(Mv) + (2 * d + 4) * Mv


def fp64_peak_tflops(pk: dict) -> float:
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    return SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12


def fp32_peak_tflops(pk: dict) -> float:
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    return SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12


# kernel class -> (kernel name, word bytes of its fields, sweep or defect)
CLASS_KERNELS = {
    "sweep64": ("k_sweep<double>", 8, "sweep"), "sweep32": ("k_sweep<float>", 4, "sweep"),
    "sweep_dd": ("k_sweep<dd>", 8, "sweep"), "defect64": ("k_defect<double>", 8, "defect"),
    "defect32": ("k_defect_update_rp<dd> (carried outer defect) / k_defect<float>", 4, "defect"),
    "defect_dd": ("k_defect_anchor (MGWR_MIXED) / k_defect<dd> (MGWR_MIXED_DD)", 8, "defect"),
}


def kernel_roofline(cls: str, p: dict, d: int, M: int, pk: dict) -> dict:
    """Roofline of one kernel class from its summed event-timed launches: the
    FP64 kernels against the FP64 ALU peak (GB300 runs FP64 at 1/64 of FP32),
    the FP32 and line kernels against HBM with the FP32-issue view beside."""
    secs = p["ms"] * 1e-3
    name, word, kind = CLASS_KERNELS.get(cls, (cls, 8, "line"))
    long = M > 4096
    if long and kind != "line":
        name = f"k_long_forward+k_long_inverse ({name})"
    per_line = (sweep_flops_per_line(d, M) if kind == "sweep" else defect_flops_per_line(d, M)) \
        if kind != "line" else 0.0
    flops = p["lines"] * per_line
    # algorithmic bytes: a sweep reads f and one line of the other colour and writes
    # its line; a defect reads u and f and writes r (the FP64 outer defect of the
    # mixed form writes FP32); the carried outer defect reads the FP32 correction and
    # the double-float defect and writes it back and rounded (24 bytes per value);
    # line kernels: three words per line value
    if cls == "defect32":
        bytes_per_line = 24 * M
    elif kind == "defect":
        bytes_per_line = (2 * word + (4 if cls == "defect64" else word)) * M
    else:
        bytes_per_line = 3 * word * M
    bytes_alg = p["lines"] * bytes_per_line
    hbm = bytes_alg / secs / 1e9
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    out = {"kernel": name, "class": cls, "launches": p["launches"],
           "avg_launch_ms": p["ms"] / max(p["launches"], 1),
           "lines_per_launch": p["lines"] / max(p["launches"], 1),
           "bytes_per_line": bytes_per_line, "flops_per_line": per_line}
    if cls in ("sweep64", "defect64"):
        peak = fp64_peak_tflops(pk)
        achieved = flops / secs / 1e12
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock "
                                   "(FMA-chain probe mgwr_peak_probe: 1.06 TFLOP/s at 2070 MHz)",
                    "hbm_view": {"achieved_gbs": hbm, "peak_gbs": hbm_peak, "frac": hbm / hbm_peak}})
    else:
        out.update({"bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm / hbm_peak, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"})
        if per_line:
            fl = flops / secs / 1e12
            out["fp32_issue_view"] = {"achieved_tflops": fl, "peak_tflops": fp32_peak_tflops(pk),
                                      "frac": fl / fp32_peak_tflops(pk),
                                      "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop "
                                                     "x max SM clock"}
    out["traffic"] = None
    if cls == "sweep64" and M == 1024:
        out["traffic"] = SWEEP64_DRAM_BYTES_PER_LINE_M1024 * out["lines_per_launch"]
        out["traffic_note"] = "ncu dram bytes per line x lines per launch"
    elif cls in NCU_DRAM_BYTES_PER_LINE and M in NCU_DRAM_BYTES_PER_LINE[cls]:
        out["traffic"] = NCU_DRAM_BYTES_PER_LINE[cls][M] * out["lines_per_launch"]
        out["traffic_note"] = "ncu dram bytes per line (small-case capture) x lines per launch"
    return out


def roofline_from_profile(prof: dict, d: int, M: int, pk: dict) -> dict:
    dom = max(prof, key=lambda k: prof[k]["ms"])
    return kernel_roofline(dom, prof[dom], d, M, pk)


def oracle_threads() -> int:
    """Threads the oracle's library calls may use (its BLAS pool), else the host's CPUs."""
    try:
        from threadpoolctl import threadpool_info
        return max(int(x.get("num_threads", 1)) for x in threadpool_info()) or os.cpu_count()
    except Exception:  # noqa: BLE001 - optional helper, absent on some hosts
        return os.cpu_count()


def cpu_oracle_sample(d: int, n: int, Ms: int, alpha: float, kind: str):
    """One complete CPU-oracle solve (direct L1 time stepping over every time
    level) of the workload's spatial grid with Ms time steps on the same (0, T]."""
    from oracle import direct
    from paper_1608_05400_gb300 import inputs

    prob = inputs.Problem(d, n, Ms, T, alpha, kind)
    f = prob.rhs()
    t0 = time.perf_counter()
    direct.time_stepping(d, n, Ms, T, alpha, f)
    dt = time.perf_counter() - t0
    grid = f"{n}x{n}" if d == 2 else f"{n}-point"
    return {"value": prob.unknowns / dt, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
            "sample": f"full solve: direct L1 time stepping (sparse LU of r_1 I + A_h once, then "
                      f"every one of the {Ms} time levels with its history sum) of the "
                      f"{grid} grid, M={Ms} on (0,{T:g}], alpha={alpha}, {kind} source, "
                      f"{prob.unknowns} unknowns in {dt:.2f} s"}


def oracle_time_factors(d: int, n: int, Mv: int, alphas, kind: str) -> np.ndarray:
    """The oracle's exact discrete solution of each instance's separable source:
    u_b = w_b(t) phi(x) with (T_M + lambda_h I) w_b = F_b (one triangular solve)."""
    from oracle import separable
    from paper_1608_05400_gb300 import inputs

    return np.stack([separable.time_factor(d, n, Mv, T, float(a),
                                           inputs.Problem(d, n, Mv, T, float(a), kind).rhs_profile())
                     for a in alphas])


def rel_err_device(torch, u, phi, W) -> float:
    """max over instances of max |u_b - phi w_b| / max |phi w_b|, on the device in
    blocks (u: (B, N, M) or (N, M) device tensor; W: (B, M) host array)."""
    Wd = torch.from_numpy(W).to(u.device)
    ub = u.reshape(Wd.shape[0], -1, Wd.shape[1])
    worst = 0.0
    rows = max(1, (1 << 27) // (ub.shape[1] * ub.shape[2]))
    for b0 in range(0, ub.shape[0], rows):
        ref_scale = phi.abs().max() * Wd[b0:b0 + rows].abs().amax(dim=1)
        err = torch.zeros_like(ref_scale)
        for a in range(0, ub.shape[1], 4096):
            ref = phi[None, a:a + 4096, None] * Wd[b0:b0 + rows, None, :]
            err = torch.maximum(err, (ub[b0:b0 + rows, a:a + 4096] - ref).abs().amax(dim=(1, 2)))
        worst = max(worst, float((err / ref_scale).max()))
    return worst


def fas_line_flops(Mv: int) -> float:
    """Algorithmic flops of one nonlinear line solve: the history sums of the L1
    matrix (M(M-1)/2 multiply-adds) and four Newton iterations of about 30 flops
    per time level."""
    return Mv * (Mv - 1) + 4 * 30 * Mv


def nonlinear_oracle_sample(delta: float, n: int, Mv: int):
    """The CPU oracle's FAS solve of the nonlinear workload (the whole solve)."""
    from oracle import fas

    f = np.ones((n, Mv))
    try:  # the oracle's small products run fastest on one BLAS thread
        from threadpoolctl import threadpool_limits
        limit, cores = threadpool_limits(1), 1
    except ImportError:
        limit, cores = None, os.cpu_count()
    t0 = time.perf_counter()
    W = fas.WRFAS(n, Mv, 1.0, delta, c=1.0, order="table")
    u, hist = W.solve(f, 0, 1, tol=1e-10, max_cycles=30)
    dt = time.perf_counter() - t0
    if limit is not None:
        limit.restore_original_limits()
    return u, {"value": n * Mv / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"oracle WRFAS V(0,1) solve of the whole {n}x{Mv} workload to 1e-10 "
                         f"({len(hist) - 1} cycles, {dt:.1f} s)"}


def run_nonlinear(args):
    """The nonlinear workload of Sec. 7 through mgwr_fas_*: one step is one FAS
    V(0,1) solve from u = 0 to a 1e-10 defect reduction (Table table_nonlinear)."""
    import torch

    from paper_1608_05400_gb300 import mgwr

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    _, n, Mw, _, _, tol, _, desc = WORKLOADS[args.workload]
    delta = args.alpha if args.alpha is not None else 0.4
    unknowns = n * Mw
    f = np.ones((n, Mw))
    g = mgwr.FAS(n, Mw, 1.0, delta, 1.0)
    g.set_order(mgwr.MGWR_ORDER_TABLE)
    stream = torch.cuda.Stream()
    g.set_stream(stream.cuda_stream)
    g.set_rhs(f)

    def step():
        g.reset()
        return g.solve(1, 0, 1, tol, 30)

    for _ in range(max(args.warmup, 3)):
        step()
    l0 = mgwr.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        rank_barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        stats = [step() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier(world)
    launches = mgwr.launch_count() - l0
    t_max = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    value = job_throughput(world, unknowns, args.steps, t_max)
    u = g.solution()

    # the dominant kernel, the finest level's smoother: red half-sweeps of the
    # iterate after a cycle, timed with events on the launching stream (each call
    # also reads back 16 bytes of status); the whole-line fixed point (M a power of
    # two from 128) counts its iterations, each one FFT convolution per line
    L = g.num_levels() - 1
    reps = 20
    g.reset()
    g.cycle(1, 0, 1)
    it0 = g.line_iterations()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        g.smooth(L, mgwr.MGWR_RED)
    k1.record(stream)
    torch.cuda.synchronize()
    line_ms = k0.elapsed_time(k1) / reps
    line_iters = (g.line_iterations() - it0) / reps
    lines = (n + 1) // 2
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak = SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12
    fixed = line_iters > 0
    flops = (line_iters * (conv_flops_per_line(Mw) + 20 * Mw) if fixed
             else lines * fas_line_flops(Mw))
    achieved = flops / (line_ms * 1e-3) / 1e12

    e2e = None
    if not args.no_e2e:
        pin_f = torch.from_numpy(f).pin_memory()
        pin_u = torch.empty_like(pin_f).pin_memory()
        fp, up = pin_f.numpy(), pin_u.numpy()

        def e2e_step():
            g.set_rhs(fp)
            st = g.solve(1, 0, 1, tol, 30)
            g.lib.mgwr_fas_get_solution(g.h, up.ctypes.data_as(mgwr._dp))
            return st

        for _ in range(max(args.warmup, 1)):
            e2e_step()
        rank_barrier(world)
        torch.cuda.synchronize()
        ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ee0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        ee1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(ee0.elapsed_time(ee1), world, "cuda")
        e2e = {"value": job_throughput(world, unknowns, args.steps, ems), "unit": UNIT,
               "h2d_bytes_per_step": unknowns * 8, "d2h_bytes_per_step": unknowns * 8,
               "host_buffers": "pinned"}
    g.close()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    out = {
        "metric": "space-time unknowns/s to rel-res 1e-10 (nonlinear FAS, FP64)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{desc}, delta={delta}, rel-res {tol}", "name": args.workload,
                   "precision": "fp64", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs smaller than L2 (0.5 MB per field): a latency-bound "
                         "sequential time march, not a bandwidth measurement"},
        "solve": {"cycles": stats[-1].cycles, "relres": stats[-1].relres,
                  "factor": stats[-1].factor},
        "gpu_launches": launches,
        "roofline": {"kernel": "k_fas_fixed" if fixed else "k_fas_line", "bound": "alu",
                     "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock",
                     "avg_launch_ms": line_ms, "lines_per_launch": lines,
                     "fixed_point_iterations_per_line": line_iters / lines if fixed else None,
                     "note": ("whole-line fixed point: one FP64 FFT convolution per line and "
                              "iteration, a few hundred lines per launch (latency-bound)") if fixed
                     else "latency-bound: one warp per line marches M dependent Newton solves"},
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if not args.no_cpu and world == 1:
        uo, out["cpu_baseline"] = nonlinear_oracle_sample(delta, n, Mw)
        out["solve"]["rel_diff_vs_oracle"] = float(np.abs(u - uo).max() / np.abs(uo).max())
    print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def workload_config(name: str, d: int, n: int, Mw: int, batch: int, tol: float, desc: str,
                    alpha, precision: str, world: int) -> dict:
    return {"workload": f"{desc}, " + (f"alpha={alpha}, " if batch == 1 else "")
                        + f"V({NU1},{NU2}) red-black, rel-res {tol}",
            "name": name, "precision": precision,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": f"inputs larger than L2 ({batch * n ** d * Mw * 8 / 1e6:.0f} MB per FP64 field)"}


def run_reference(args):
    """The reference arm: there is no reference implementation of this method, so
    the CPU oracle stands in for it, timed as it is on the host cores.  Each step
    is one complete oracle solve of the workload's grid at the CPU-baseline
    sample's number of time steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    d, n, Mw, batch, kind, tol, prec, desc = WORKLOADS[args.workload]
    if args.workload not in ORACLE_SAMPLE_M:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle sample for {args.workload}"}))
        return 0
    alpha = args.alpha if args.alpha is not None else WORKLOAD_ALPHA.get(args.workload, ALPHA)
    Ms = ORACLE_SAMPLE_M[args.workload]
    for _ in range(args.warmup):
        cpu_oracle_sample(d, n, Ms, alpha, kind)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(d, n, Ms, alpha, kind))
    dt = time.perf_counter() - t0
    unknowns = n ** d * Ms
    v = args.steps * unknowns / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": workload_config(args.workload, d, n, Mw, batch, tol, desc, alpha,
                                     args.precision or prec, args.gpus),
           "cpu_baseline": dict(vals[0], value=v),
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_served(args):
    """The served workload: a stream of mixed-shape requests through mgwr_submit / mgwr_poll.

    Pass 1 submits the whole list as fast as the server takes it and measures
    the sustained rate; pass 2 replays it with Poisson arrivals at 0.7 x that
    rate and records the latency of every request (scheduled arrival -> result
    ready).  Both passes keep at most 24 GB of submitted right-hand sides in
    host memory (the server holds a copy of each until its request is done);
    time a request waits for that window counts in its latency."""
    import threading

    import torch

    from paper_1608_05400_gb300 import inputs, mgwr

    torch.cuda.set_device(0)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    reqs = inputs.request_stream(count=2000, seed=1608, rate=1.0)[: args.requests]
    tol = WORKLOADS["served"][5]
    precision = args.precision or WORKLOADS["served"][6]
    prec = PREC_CODES[precision]

    zero_copy = args.submit == "buffer"

    def rhs(rq, srv):
        prob = inputs.Problem(rq["d"], rq["n"], rq["M"], 1.0, rq["alpha"], rq["kind"])
        if not zero_copy:
            return prob.rhs()
        # straight into a page-locked buffer lent by the server (no copy at submit)
        return prob.rhs(out=srv.buffer(rq["n"] ** rq["d"], rq["M"]))

    def unknowns(rq):
        return rq["n"] ** rq["d"] * rq["M"]

    # host bytes of right-hand sides submitted and not yet completed: the server
    # copies each f until its request finishes, so bound what is outstanding
    host_cap = 24 << 30

    def run(arrivals):
        lat, results = [None] * len(reqs), [None] * len(reqs)
        delay = [0.0] * len(reqs)
        outstanding = [0]
        lock = threading.Condition()
        with mgwr.Server(hbm_budget=budget, slots=args.slots) as srv:
            srv.set_policy(mgwr.MGWR_POLICY_SMALLEST if args.policy == "smallest"
                           else mgwr.MGWR_POLICY_FIFO)
            tickets = [None] * len(reqs)
            t0 = time.perf_counter()

            def submitter():
                # right-hand sides are generated ahead of their arrival by a pool of
                # host threads (numpy releases the GIL), within the host window
                import concurrent.futures as cf
                pending = {}
                nxt = [0]

                def fill(pool):
                    while nxt[0] < len(reqs):
                        nbytes = 8 * unknowns(reqs[nxt[0]])
                        with lock:
                            if outstanding[0] and outstanding[0] + nbytes > host_cap:
                                return
                            outstanding[0] += nbytes
                        pending[nxt[0]] = pool.submit(rhs, reqs[nxt[0]], srv)
                        nxt[0] += 1

                with cf.ThreadPoolExecutor(8) as pool:
                    for i, rq in enumerate(reqs):
                        fill(pool)
                        while i not in pending:  # the window is full: wait for completions
                            with lock:
                                lock.wait(0.01)
                            fill(pool)
                        f = pending.pop(i).result()
                        wait = t0 + arrivals[i] - time.perf_counter()
                        if wait > 0:
                            time.sleep(wait)
                        # time a request waited for its data counts in its latency
                        delay[i] = max(0.0, time.perf_counter() - (t0 + arrivals[i]))
                        if zero_copy:
                            tickets[i] = srv.submit_buffer(rq["d"], rq["n"], rq["M"], 1.0,
                                                           rq["alpha"], f, precision=prec, tol=tol)
                        else:
                            tickets[i] = srv.submit(rq["d"], rq["n"], rq["M"], 1.0, rq["alpha"], f,
                                                    precision=prec, tol=tol)
                        del f

            th = threading.Thread(target=submitter)
            th.start()
            done = 0
            while done < len(reqs):
                for i in range(len(reqs)):
                    if results[i] is None and tickets[i] is not None:
                        r = srv.poll(tickets[i], timeout_us=0, copy_solution=False)
                        if r is not None:
                            results[i] = r
                            lat[i] = r.latency_s + delay[i]
                            done += 1
                            with lock:
                                outstanding[0] -= 8 * unknowns(reqs[i])
                                lock.notify_all()
                time.sleep(0.002)
            th.join()
            makespan = time.perf_counter() - t0
            info = srv.info()
        return makespan, lat, results, info

    total = sum(unknowns(r) for r in reqs)
    # the server's pinned buffers are first touched by these threads: keep them on
    # the GPU-local CPUs so that the buffers sit next to the GPU
    with GpuLocalHost(0) as host:
        span1, _, res1, _ = run([0.0] * len(reqs))
        rate = len(reqs) / span1
        offered = args.rate if args.rate else 0.7 * rate
        rng = np.random.default_rng(1608)
        arr = np.cumsum(rng.exponential(1.0 / offered, size=len(reqs)))
        span2, lat, res2, info = run(list(arr))
    ok = sum(1 for r in res2 if r.status == mgwr.MGWR_OK)
    lat_ms = np.array(lat) * 1e3
    out = {
        "metric": "served p50/p99 latency and space-time unknowns/s (mixed, rel-res 1e-8)",
        "precision": precision,
        "value": total / span2, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[precision], "data": "synthetic",
        "config": {"workload": f"served stream: {len(reqs)} of 2000 requests (seed 1608), "
                               "1-D n=2^k-1 k~U{5..12} or 2-D k~U{5..9}, M=2^j j~U{7..12}, "
                               "alpha~U[0.1,0.9], u=t^2 or t^alpha sin, Poisson arrivals at 0.7x "
                               "the sustained rate", "name": "served", "slots": args.slots,
                   "admission": args.policy,
                   "host_buffers": (f"pinned, on the {len(host.cpus)} GPU-local CPUs"
                                    if host.cpus else "pinned"),
                   "hbm_budget_bytes": budget, "host_window_bytes": host_cap},
        "served": {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                   "sustained_requests_per_s": rate, "offered_requests_per_s": offered,
                   "back_to_back_unknowns_per_s": total / span1, "completed_ok": ok,
                   "requests": len(reqs), "total_unknowns": total, "peak_bytes": info["peak_bytes"],
                   "submit": ("zero-copy: f generated into page-locked buffers lent by the server "
                              "(mgwr_server_buffer / mgwr_submit_buffer)" if zero_copy else
                              "mgwr_submit (f copied into the server's page-locked pool)"),
                   "host_seconds_pass2": {k: info[k] for k in ("submit_copy_s", "prepare_s",
                                                               "finish_s", "pin_s")},
                   "pinned_buffers_pass2": info["pinned_buffers"],
                   "reused_handles_pass2": info["reused_handles"]},
    }
    print(json.dumps(out))
    return 0


def measure_arm(args, torch, mgwr, wl: dict, precision: str, steps: int, warmup: int,
                e2e_steps: int, stream, world: int, local: int, W=None, main_arm=False) -> dict:
    """Times `steps` complete solves of the workload in one precision: inputs
    resident on the device, CUDA events on the handle's stream, launch shapes
    tuned first.  The main arm also samples clocks, profiles one extra solve per
    kernel class and runs the end-to-end loop through host buffers."""
    d, n, Mw, batch, tol = wl["d"], wl["n"], wl["M"], wl["batch"], wl["tol"]
    s = mgwr.Solver(d, n, Mw, T, wl["alpha"])
    s.set_stream(stream.cuda_stream)
    if precision != "fp64":
        s.set_precision(PREC_CODES[precision])
        precision = PREC_NAMES[s.precision()]  # MGWR_AUTO resolves on this grid
    mixed = precision in ("mixed", "mixed_dd")
    inner = args.inner or WORKLOAD_INNER.get(args.workload)
    if mixed and inner:
        s.set_inner_cycles(inner)
    if mixed and args.outer_switch is not None:
        s.set_outer_switch(args.outer_switch)
    # launch shapes of the FFT-engine kernels, timed on this handle's data (setup,
    # outside the timed region)
    splits = None if args.no_autotune else s.autotune()
    if args.split:
        for cls, val in parse_splits(args.split, mgwr.KERNEL_CLASSES).items():
            s.set_engine_split(cls, val)
        splits = dict(splits or {}, forced=args.split)
    f_dev = wl["f_dev"]

    def step():
        s.set_rhs_dev(f_dev.data_ptr())
        return s.solve(CYCLE, NU1, NU2, tol, 100)

    for _ in range(warmup):
        step()
    l0 = mgwr.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local) if main_arm else None
    if clk is not None:
        clk.__enter__()
    try:
        rank_barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        stats = [step() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier(world)
    finally:
        if clk is not None:
            clk.__exit__(None, None, None)
    launches = mgwr.launch_count() - l0
    t_max = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    out = {"precision": precision, "dtype": DTYPES[precision],
           "value": job_throughput(world, wl["unknowns"], steps, t_max), "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": t_max / steps,
           "solve": {"cycles": stats[-1].cycles, "outer": stats[-1].outer,
                     "relres": stats[-1].relres, "factor": stats[-1].factor},
           "gpu_launches": launches, "engine_splits": splits,
           "inner_cycles": (inner or 2) if mixed else None}
    if clk is not None:
        out["clocks"] = clk.summary()
    field_bytes = wl["unknowns"] * 8
    if W is not None:
        u = torch.empty((batch, n ** d, Mw), dtype=torch.float64, device="cuda")
        s.solution_dev(u.data_ptr())
        torch.cuda.synchronize()
        out["solve"]["rel_err_vs_oracle"] = rel_err_device(torch, u, wl["phi_dev"], W)
        del u
        torch.cuda.empty_cache()
    # the IEEE-double defect of the result, recomputed in FP64 whatever the precision
    # (it needs one more FP64 field on the device)
    if precision == "fp64" or torch.cuda.mem_get_info()[0] > field_bytes + (2 << 30):
        out["solve"]["relres_fp64"] = s.residual()
    else:
        out["solve"]["relres_fp64"] = None
        out["solve"]["relres_fp64_note"] = "skipped: no room for one more FP64 field"
    if main_arm:
        # per-kernel-class times from one profiled solve (outside the timed region)
        s.profile(True)
        step()
        out["kernel_classes"] = {k: v for k, v in s.profile_read().items() if v["launches"]}
        s.profile(False)
    if e2e_steps > 0 and wl.get("f_host") is not None:
        with GpuLocalHost(local) as host:
            pin_f = torch.from_numpy(wl["f_host"]).pin_memory()
            pin_u = torch.empty_like(pin_f).pin_memory()
            fp, up = pin_f.numpy(), pin_u.numpy()
            ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

            def e2e_step():  # synchronous calls: copy in, solve, copy out
                s.set_rhs(fp)
                s.solve(CYCLE, NU1, NU2, tol, 100)
                s.lib.mgwr_get_solution(s.h, up.ctypes.data_as(mgwr._dp))

            def e2e_pipelined(k):
                # each step's right-hand side is staged while the previous solve
                # runs and its solution returned while the next one runs
                s.stage_rhs(fp)
                for i in range(k):
                    s.take_rhs()
                    if i + 1 < k:
                        s.stage_rhs(fp)
                    s.solve(CYCLE, NU1, NU2, tol, 100)
                    s.stage_solution(up)
                s.wait_staged()

            def timed(run):
                rank_barrier(world)
                torch.cuda.synchronize()
                ee0.record(stream)
                run()
                ee1.record(stream)
                torch.cuda.synchronize()
                return max_over_ranks(ee0.elapsed_time(ee1), world, "cuda")

            # untimed warm-up through the same paths: the profiled solve above ran
            # without graphs, so the first steps after it capture them again
            for _ in range(max(min(warmup, 2), 1)):
                e2e_step()
            e2e_pipelined(2)
            ems = timed(lambda: e2e_pipelined(e2e_steps))
            serial_steps = max(1, min(e2e_steps, 3))

            def serial():
                for _ in range(serial_steps):
                    e2e_step()

            sms = timed(serial)
            nbytes = wl["unknowns"] * 8
            out["e2e"] = {"value": job_throughput(world, wl["unknowns"], e2e_steps, ems),
                          "unit": UNIT, "steps": e2e_steps,
                          "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                          "host_buffers": (f"pinned, first touched on the {len(host.cpus)} "
                                           f"GPU-local CPUs" if host.cpus else "pinned"),
                          "transfers": "pipelined (mgwr_stage_rhs / mgwr_take_rhs / "
                                       "mgwr_stage_solution): each step's right-hand side in and "
                                       "solution out on copy streams during the neighbouring solves",
                          "serial_value": job_throughput(world, wl["unknowns"], serial_steps, sms),
                          "serial_steps": serial_steps,
                          "serial_transfers": "mgwr_set_rhs, mgwr_solve, mgwr_get_solution in turn"}
            del pin_f, pin_u
    s.close()
    return out


def run_probe_peaks(args) -> None:
    """The arithmetic denominators of the FP64 and FP32 rooflines, measured on this
    GPU (dependent FMA chains, mgwr_peak_probe), with the clocks seen meanwhile and
    the per-clock rates they imply (152 SMs)."""
    import torch
    from paper_1608_05400_gb300 import mgwr
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    mgwr.load()
    mgwr.peak_probe()  # warm-up: module load, clocks up
    with ClockSampler(local) as clk:
        res = mgwr.peak_probe()
    c = clk.summary()
    mhz = c.get("sm_mhz") or float("nan")
    res.update({"clocks": c,
                "fp64_fma_per_clk_per_sm": res["fp64_tflops"] * 1e12 / 2 / (SMS * mhz * 1e6),
                "fp32_fma_per_clk_per_sm": res["fp32_tflops"] * 1e12 / 2 / (SMS * mhz * 1e6)})
    print(json.dumps(res))


def main():
    args = parse()
    if args.probe_peaks:
        return run_probe_peaks(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload.startswith("nonlinear"):
        return run_nonlinear(args)
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    from paper_1608_05400_gb300 import inputs, mgwr

    d, n, Mw, batch, kind, tol, prec_default, desc = WORKLOADS[args.workload]
    profiling_case = bool(args.shape or args.batch)
    if profiling_case:
        if args.shape:
            d, n, Mw = (int(x) for x in args.shape.split(","))
        batch = args.batch or batch
        desc = f"{args.workload} settings on {d}-D n={n}, M={Mw}, batch {batch} (profiling case)"
        args.no_cpu = True
    precision = args.precision or prec_default
    alpha = args.alpha if args.alpha is not None else WORKLOAD_ALPHA.get(args.workload, ALPHA)
    ph = torch.from_numpy(inputs.phi(d, n)).cuda()
    if batch == 1:
        alphas = np.array([alpha])
        F = inputs.Problem(d, n, Mw, T, alpha, kind).rhs_profile()[None, :]
    else:
        alphas = inputs.random_alphas(batch, seed=1608)
        F = np.stack([inputs.Problem(d, n, Mw, T, float(a), kind).rhs_profile() for a in alphas])
    # f_b = F_b(t) phi(x), built on the device (and on the host for the e2e loop)
    f_dev = (ph[None, :, None] * torch.from_numpy(F).cuda()[:, None, :]).reshape(-1, Mw)
    unknowns = batch * n ** d * Mw
    wl = {"d": d, "n": n, "M": Mw, "batch": batch, "tol": tol, "unknowns": unknowns,
          "alpha": alpha if batch == 1 else alphas, "f_dev": f_dev, "phi_dev": ph}
    # the pipelined loop exposes only the first upload and the last download: over
    # ten steps they are a tenth of a step each
    e2e_steps = 0 if args.no_e2e else (args.e2e_steps or min(args.steps, 10))
    if e2e_steps and batch == 1:
        wl["f_host"] = f_dev.cpu().numpy()
    cpu_leg = not args.no_cpu and world == 1
    W = oracle_time_factors(d, n, Mw, alphas, kind) if cpu_leg else None
    stream = torch.cuda.Stream()
    warmup = max(args.warmup, 3) if args.warmup >= 3 else args.warmup

    main_arm = measure_arm(args, torch, mgwr, wl, precision, args.steps, warmup, e2e_steps,
                           stream, world, local, W=W, main_arm=True)
    arms = []
    if args.arms is not None:
        arms = [] if args.arms == "none" else [a.strip() for a in args.arms.split(",") if a.strip()]
    elif not profiling_case and args.precision is None:
        arms = list(WORKLOAD_ARMS.get(args.workload, ()))
    arm_out = {}
    for a in arms:
        if a == main_arm["precision"]:
            continue
        # the FP64 arm of the largest workload takes seconds per solve: fewer steps
        k = args.arm_steps or (min(args.steps, 2) if a == "fp64" else min(args.steps, 5))
        w = min(warmup, 1) if a == "fp64" else min(warmup, 3)
        arm_out[a] = measure_arm(args, torch, mgwr, wl, a, k, w, 0, stream, world, local, W=W)
    del f_dev, wl["f_dev"]
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    pk = peaks()
    prof = main_arm.pop("kernel_classes")
    out = {
        "metric": METRIC, "value": main_arm["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": warmup, "ms_per_step": main_arm["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": main_arm["dtype"], "data": "synthetic",
        "config": dict(workload_config(args.workload, d, n, Mw, batch, tol, desc, alpha,
                                       main_arm["precision"], world),
                       engine_splits=main_arm["engine_splits"],
                       inner_cycles=main_arm["inner_cycles"]),
        "solve": main_arm["solve"],
        "gpu_launches": main_arm["gpu_launches"],
        "roofline": roofline_from_profile(prof, d, Mw, pk),
        "kernel_classes": prof,
        "clocks": main_arm["clocks"],
        "e2e": main_arm.get("e2e"),
    }
    if "sweep32" in prof and out["roofline"]["class"] != "sweep32":
        out["roofline_sweep32"] = kernel_roofline("sweep32", prof["sweep32"], d, Mw, pk)
    # name the FP32 sweep by the engine the tuner chose for the finest level
    sp = (main_arm["engine_splits"] or {}).get("sweep32")
    if sp:
        eng = ("k_sweep_rp_res<float> (resident register-pass engine)"
               if sp[-1] & 64 and sp[-1] & 7 == 4 else
               "k_sweep_rp<float> (register-pass engine)" if sp[-1] & 64 else
               "k_sweep_tc (tensor cores)" if sp[-1] & 32 else
               "k_sweep_staged<float>" if sp[-1] & 16 else f"k_sweep<float> (E={sp[-1]})")
        for key in ("roofline", "roofline_sweep32"):
            if key in out and out[key].get("class") == "sweep32":
                out[key]["kernel"] = eng + " [finest level; all levels' launches timed]"
    for a, res in arm_out.items():
        res.pop("engine_splits", None)
        out[f"{a}_arm"] = res
    if cpu_leg and args.workload in ORACLE_SAMPLE_M:
        out["cpu_baseline"] = cpu_oracle_sample(d, n, ORACLE_SAMPLE_M[args.workload], alpha, kind)
    print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
