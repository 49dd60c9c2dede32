#!/usr/bin/env python
"""Benchmark of the collapse-time hot path (arXiv:2510.02873, Sec. 3 / Sec. 4.1).

Workload (one step): a 256^3 grid x 25 smoothing radii, six FP64
structure-of-arrays Hessian planes per radius (20.1 GB, resident in HBM, far
larger than L2), s(R) log-spaced 0.2 -> 6.0, flat LCDM (Om = 0.3, OL = 0.7),
512-knot growth table. A step is one pass of the whole path over the grid:
reset of the two per-point maxima, then the fused launch over all radii
(eigenvalues, LPT collapse condition, inverse-growth spline, running max).

Metric: collapse evaluations (points x radii) per second on the GPU(s).
Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
(the baseline this project checks against) on bounded samples of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = 256
N_RADII = 25
S_LO, S_HI = 0.2, 6.0
SEED = 2512
COSMO = dict(omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0)
WORKLOAD = "collapse 256^3 grid x 25 radii, FP64 SoA Hessian planes (20.1 GB resident), 512-knot a(D) spline"

# FP64 floating-point operations per (point, radius) evaluation of the FP64
# kernel, from ncu thread-instruction counters (dadd + dmul + 2 dfma) divided
# by the evaluations of the captured launch (profiles/collapse_kernel_*_128cube_x4.md).
# None until a capture of the current kernel exists.
FP64_FLOPS_PER_EVAL = 70.0   # profiles/collapse_kernel_fp64_128cube_x4.md
FP64_FLOPS_PER_EVAL_MIXED = 8.1  # profiles/collapse_kernel_mixed_128cube_x30.md
# FP64-pipe warp instructions of every kind (DFMA, DMUL, DADD, compares) per
# evaluation, from the same captures: the FP64 unit issues one per lane slot
# whatever the instruction, so this count, not the flop count, sets the time.
FP64_PIPE_INST_PER_EVAL = {"fp64": 45.0, "mixed": 5.1}
FP64_LANES_PER_CLK_PER_SM = 2.0
# DRAM bytes (read + write) of one full launch of the default workload, from
# an ncu capture of that launch (profiles/collapse_kernel_fp64_256cube_x25_dram.md).
TRAFFIC_BYTES_DEFAULT = 20.83e9
# FP64 FMA rate of one GB300 SM: 1.25 TFLOP/s nominal at 2070 MHz over 152 SMs
# = 3.97 flop/clk/SM, i.e. 2 DFMA per clock per SM (confirmed by a DFMA-chain probe).
FP64_FLOP_PER_CLK_PER_SM = 4.0
def _measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine type (MEASURED_PEAKS.json at the repository root)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


HBM_GBS = _measured_hbm_gbs()


def _measured_bf16_tflops():
    """Dense BF16 GEMM rate measured on this machine type (burst; MEASURED_PEAKS.json)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return None


BF16_TFLOPS = _measured_bf16_tflops()
# the network's algorithmic work per evaluation: 2 (3 x 64 + 64 x 64 + 64 x 64 + 64 x 1) flops
MLP_FLOPS_PER_EVAL = 2.0 * (3 * 64 + 64 * 64 * 2 + 64)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-variants", action="store_true")
    # smaller problems for profiler captures only (the benchmark workload is the default)
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--radii", type=int, default=N_RADII)
    ap.add_argument("--mode", choices=["fp64", "mixed", "f32x2", "surrogate", "exact_growth", "tabulated"],
                    default="fp64")
    ap.add_argument("--surrogate-engine", choices=["mma_sync", "tcgen05"], default="tcgen05",
                    help="kernel for --mode surrogate (cc_set_surrogate_engine)")
    # --mode surrogate trains the network first (untimed) on this many points and steps
    ap.add_argument("--train-points", type=int, default=4 * 1024 * 1024)
    ap.add_argument("--train-steps", type=int, default=300)
    # run one variant alone at --grid / --radii (profiler captures)
    ap.add_argument("--variant", choices=["science", "field", "batched"], default=None)
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        """Start sampling; returns once the first sample has arrived, so that
        nvidia-smi's start-up does not fall inside the timed region."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.first = self.proc.stdout.readline()
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.first + out).strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- CPU oracle
def _cpu_times():
    """Per-core (busy, steal, total) jiffies from /proc/stat, or None where the
    host has none. busy = user + nice + system + irq + softirq."""
    try:
        with open("/proc/stat") as f:
            rows = [line.split() for line in f if re.match(r"cpu\d+ ", line)]
    except OSError:
        return None
    out = []
    for row in rows:
        v = [int(x) for x in row[1:9]]
        out.append((v[0] + v[1] + v[2] + v[5] + v[6], v[7], sum(v)))
    return out


def _cpu_share(before, after) -> dict | None:
    """What the host's cores did between two _cpu_times() snapshots: mean busy
    and steal fractions over all cores and the least busy core's fraction."""
    if not before or not after or len(before) != len(after):
        return None
    per = []
    for (b0, s0, t0), (b1, s1, t1) in zip(before, after):
        dt = max(t1 - t0, 1)
        per.append(((b1 - b0) / dt, (s1 - s0) / dt))
    return {"busy_frac": round(sum(p[0] for p in per) / len(per), 3),
            "steal_frac": round(sum(p[1] for p in per) / len(per), 3),
            "min_core_busy_frac": round(min(p[0] for p in per), 3)}


def cpu_oracle_rate(seconds: float, first_point: int = 0, points_per_chunk: int | None = None):
    """The FP64 oracle on consecutive chunks of the workload's points (all 25
    radii each), until `seconds` of CPU work. Inputs are drawn before timing.
    The oracle hands out points to its threads 256 at a time, so the default
    chunk gives every host core four such blocks per radius (a chunk of 2048
    points kept 8 of 16 cores busy)."""
    import numpy as np

    if points_per_chunk is None:
        points_per_chunk = 1024 * (os.cpu_count() or 1)

    import hessgen
    import oracle

    t = oracle.Tables(**{k: COSMO[k] for k in ("omega_m", "omega_l", "n_knots", "a_min", "a_max")})
    sig = hessgen.sigma_schedule(N_RADII, S_LO, S_HI)
    evals, elapsed, p0 = 0, 0.0, first_point
    cpu_acc = None  # per-core jiffies summed over the timed calls only
    while evals == 0 or elapsed < seconds:
        pts = np.arange(p0, p0 + points_per_chunk, dtype=np.int64)
        stack = np.stack([hessgen.hessian_points(SEED, 0, r, sig[r], pts) for r in range(N_RADII)])
        F = np.zeros(len(pts))
        idx = np.full(len(pts), -1, dtype=np.int32)
        c0 = _cpu_times()
        t0 = time.perf_counter()
        for r in range(N_RADII):
            t.collapse_scale(stack[r], F, idx, r)
        elapsed += time.perf_counter() - t0
        c1 = _cpu_times()
        if c0 and c1:
            cpu_acc = [tuple(a + (y - x) for a, x, y in zip(acc, u, w))
                       for acc, u, w in zip(cpu_acc or [(0, 0, 0)] * len(c0), c0, c1)]
        evals += len(pts) * N_RADII
        p0 += points_per_chunk
    cores = os.cpu_count()
    out = {"value": evals / elapsed, "unit": "evals/s", "cores": cores, "kind": "oracle",
           "sample": f"{p0 - first_point} points x {N_RADII} radii of the workload "
                     f"({evals} evaluations, {elapsed:.1f} s, OpenMP over {cores} threads)"}
    if cpu_acc:
        # the host's cores over the timed calls (all processes, from /proc/stat)
        out["host_cpu"] = _cpu_share([(0, 0, 0)] * len(cpu_acc), cpu_acc)
    if seconds > 0:
        # one thread on the next chunk of points
        pts = np.arange(p0, p0 + 512, dtype=np.int64)
        stack = np.stack([hessgen.hessian_points(SEED, 0, r, sig[r], pts) for r in range(N_RADII)])
        F = np.zeros(len(pts))
        idx = np.full(len(pts), -1, dtype=np.int32)
        t0 = time.perf_counter()
        for r in range(N_RADII):
            t.collapse_scale(stack[r], F, idx, r, nthreads=1)
        out["single_thread_value"] = len(pts) * N_RADII / (time.perf_counter() - t0)
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(0.0, first_point=4096 * i, points_per_chunk=4096)
        if i >= args.warmup:
            steps.append(r)
    evals = sum(4096 * N_RADII for _ in steps)
    secs = sum(4096 * N_RADII / r["value"] for r in steps)
    value = evals / secs
    line = {
        "impl": "reference", "metric": "collapse evals/s (points x radii)", "value": value,
        "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / len(steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "f32x2": "f32x2 (float-float)", "mixed": "f32+f64",
                                       "surrogate": "bf16+f32+f64", "exact_growth": "f64",
                                       "tabulated": "f64"}[args.mode],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": f"4096 points x {N_RADII} radii"},
        "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": value, "unit": "evals/s",
                         "sample": f"{args.steps} steps of 4096 points x {N_RADII} radii"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    shares = [r["host_cpu"] for r in steps if r.get("host_cpu")]
    if shares:
        line["cpu_baseline"]["host_cpu"] = {
            "busy_frac": round(statistics.mean(h["busy_frac"] for h in shares), 3),
            "steal_frac": round(statistics.mean(h["steal_frac"] for h in shares), 3),
            "min_core_busy_frac": min(h["min_core_busy_frac"] for h in shares)}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- float-float variant
def run_f32x2_variant(ctx, hess, sig, F_ref, idx_ref, stream, steps: int, mode: str = "f32x2") -> dict:
    """Another mode on the same FP64 planes as the main workload, timed the same
    way, and compared with the FP64 kernel's result point by point: the FP64
    path's steps in float-float arithmetic (CC_MODE_F32X2, held to the same
    1e-10), the exact-background growth ratios (CC_MODE_EXACT_GROWTH, a
    different collapse condition: the differences are the physics, not errors),
    or the tabulated 1/D_c (CC_MODE_TABULATED: the differences are the
    table's interpolation error)."""
    import torch

    n = F_ref.numel()
    R = hess.shape[0]
    F = torch.empty_like(F_ref)
    idx = torch.empty_like(idx_ref)
    for _ in range(2):
        ctx.reset_max(F, idx)
        ctx.collapse_multi(hess, sig, F, idx, mode=mode)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        ctx.reset_max(F, idx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.collapse_multi(hess, sig, F, idx, mode=mode)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    both = (F_ref > 0) & (F > 0)
    rel = ((F - F_ref).abs() / F_ref)[both]
    ms = statistics.mean(times)
    return {
        "workload": "the main workload's planes (256^3 x 25, FP64)",
        "evals_per_s": float(n) * R / (ms * 1e-3), "kernel_ms": ms,
        "max_rel_diff_vs_fp64_kernel": float(rel.max()), "rms_rel_diff_vs_fp64_kernel": float(rel.pow(2).mean().sqrt()),
        "collapse_decision_differs": int(((F_ref > 0) != (F > 0)).sum()),
        "argmax_differs": int((idx != idx_ref).sum()),
        "bound_tol": 1e-10 if mode == "f32x2" else None,  # exact growth / table: different arithmetic
    }


def run_streamed_variant(ctx, hess, sig, F_ref, idx_ref, stream, steps: int) -> dict:
    """The paper's own launch pattern on the same device-resident FP64 planes:
    one cc_collapse_scale launch per radius, each reading and updating
    F_max/idx in HBM (24 B/point per radius more than the fused launch), against
    the fused multi-radius launch of the main line. Results must be identical."""
    import torch

    n = F_ref.numel()
    R = hess.shape[0]
    F = torch.empty_like(F_ref)
    idx = torch.empty_like(idx_ref)

    def one_step():
        ctx.reset_max(F, idx)
        for r in range(R):
            ctx.collapse_scale(hess[r], sig[r], F, idx, r)

    for _ in range(2):
        one_step()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    return {
        "workload": "the main workload's planes (256^3 x 25, FP64), one launch per radius",
        "evals_per_s": float(n) * R / (ms * 1e-3), "step_ms": ms, "launches_per_step": R + 1,
        "results_identical_to_fused": bool(torch.equal(F, F_ref) and torch.equal(idx, idx_ref)),
    }


# ----------------------------------------------------------------------------- tabulated table
def table_axes(nd: int = 128, nxy: int = 64, d_max: float = 40.0, xy_max: float = 40.0):
    """Non-uniform axes of the tabulated mode: delta sinh-spaced (dense near 0),
    x = l1 - l2 and y = l2 - l3 quadratically spaced from 0."""
    import numpy as np
    t = np.linspace(-1.0, 1.0, nd)
    dg = d_max * np.sinh(2.5 * t) / np.sinh(2.5)
    u = np.linspace(0.0, 1.0, nxy)
    xg = xy_max * (0.3 * u + 0.7 * u ** 2)
    return dg, xg, xg.copy()


def load_table(ctx):
    """Node values 1/D_c computed on the device (cc_table_nodes_rlpt), then the table (cc_set_table)."""
    dg, xg, yg = table_axes()
    ctx.set_table(dg, xg, yg, ctx.table_nodes_rlpt(dg, xg, yg))


# ----------------------------------------------------------------------------- science proxy
SCI_RHO = 0.9
SCI_EDGES = [1.0 + 0.25 * k for k in range(41)]  # z_c bins of 0.25 from 0 to 10


def run_science_variant(ctx, dev, stream, reps: int = 10, grid: int = GRID, R: int = N_RADII) -> dict:
    """The paper's science check (collapsed points per redshift bin) on a
    256^3 x 25 FP64 field whose radii are correlated (AR(1) chain, rho = 0.9):
    FP64 collapse, then the counts per z_c bin on the GPU."""
    import torch

    import hessgen
    import hessgen.device as hdev

    n = grid ** 3
    sig = hessgen.sigma_schedule(R, S_LO, S_HI)
    hess = torch.empty((R, 6, n), dtype=torch.float64, device=dev)
    state = torch.empty((6, n), dtype=torch.float64, device=dev)
    for r in range(R):
        hdev.fill_correlated(hess[r], state, SEED + 7, 0, r, sig[r], SCI_RHO, first=(r == 0))
    del state
    F = torch.empty(n, dtype=torch.float64, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    ctx.reset_max(F, idx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.collapse_multi(hess, sig, F, idx, mode="fp64")
    e1.record(stream)
    counts = torch.empty(len(SCI_EDGES) + 1, dtype=torch.int64, device=dev)
    ctx.histogram(F, SCI_EDGES, counts)
    torch.cuda.synchronize()
    collapse_ms = e0.elapsed_time(e1)
    times = []
    for _ in range(reps):
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        ctx.histogram(F, SCI_EDGES, counts)
        h1.record(stream)
        torch.cuda.synchronize()
        times.append(h0.elapsed_time(h1))
    c = counts.cpu().tolist()
    hist_ms = statistics.median(times)
    del hess
    torch.cuda.empty_cache()
    return {
        "workload": f"{grid}^3 grid x {R} correlated radii (rho {SCI_RHO}), FP64 planes",
        "z_edges": [round(e - 1.0, 4) for e in SCI_EDGES],
        "collapsed_per_z_bin": c[1:-1], "not_collapsed_or_z_below_0": c[0], "z_above_last_edge": c[-1],
        "collapsed_fraction": float((F > 0).double().mean()),
        "collapse_kernel_ms": collapse_ms, "evals_per_s": n * R / (collapse_ms * 1e-3),
        "histogram_kernel_ms": hist_ms,
        "histogram_roofline": {"bound": "hbm", "unit": "GB/s", "achieved": 8.0 * n / (hist_ms * 1e-3) / 1e9,
                               "peak": HBM_GBS, "frac": (8.0 * n / (hist_ms * 1e-3) / 1e9 / HBM_GBS) if HBM_GBS else None,
                               "algorithmic_bytes": 8.0 * n},
    }


# ----------------------------------------------------------------------------- field -> Hessian -> collapse
FIELD_SPEC = dict(amplitude=222.0, index=-1.5, k_cut=1.2)  # box = 2 x grid cells
FIELD_RADII = (1.0, 12.0)


def run_field_variant(ctx, dev, stream, reps: int = 2, grid: int = GRID, R: int = N_RADII) -> dict:
    """One realization kept on the device from white noise to F_max: cuFFT
    smoothing into the six Hessian planes per radius, then the collapse
    launch on those planes (256^3 grid, 25 radii). FP64 planes + FP64
    collapse, and FP32 planes + mixed collapse."""
    import numpy as np
    import torch

    import hessgen.device as hdev
    import paper_2510_02873_gb300 as cc

    n = grid ** 3
    spec = dict(FIELD_SPEC, box=2.0 * grid)
    white = torch.empty(n, dtype=torch.float64, device=dev)
    hdev.white(white, SEED + 8, 0)
    field = cc.Field(ctx, white, **spec)
    del white
    radii = np.geomspace(FIELD_RADII[0], FIELD_RADII[1], R)
    sig = [field.sigma(x) for x in radii]
    out = {}
    for label, dt, mode in (("fp64", torch.float64, "fp64"), ("fp32_planes_mixed", torch.float32, "mixed")):
        planes = torch.empty((6, n), dtype=dt, device=dev)
        F = torch.empty(n, dtype=torch.float64, device=dev)
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        fft_ms, col_ms, tot_ms = [], [], []
        for rep in range(reps + 1):
            ctx.reset_max(F, idx)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * R + 1)]
            ev[0].record(stream)
            for r in range(R):
                field.hessian(radii[r], planes)
                ev[2 * r + 1].record(stream)
                ctx.collapse_scale(planes, sig[r], F, idx, r, mode=mode)
                ev[2 * r + 2].record(stream)
            torch.cuda.synchronize()
            if rep == 0:
                continue  # first pass builds the cuFFT plans
            fft_ms.append(sum(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(R)))
            col_ms.append(sum(ev[2 * r + 1].elapsed_time(ev[2 * r + 2]) for r in range(R)))
            tot_ms.append(ev[0].elapsed_time(ev[2 * R]))
        t = statistics.mean(tot_ms)
        out[label] = {"evals_per_s": n * R / (t * 1e-3), "ms_per_realization": t,
                      "hessian_fft_ms": statistics.mean(fft_ms), "collapse_ms": statistics.mean(col_ms),
                      "collapsed_fraction": float((F > 0).double().mean())}
        del planes
    field.close()
    torch.cuda.empty_cache()
    return {"workload": f"{grid}^3 white noise -> P(k) = A k^n exp(-(k/k_c)^2) ({spec}) -> "
                        f"{R} Gaussian radii {FIELD_RADII[0]}..{FIELD_RADII[1]} -> Hessian planes -> collapse, all on the device",
            "sigma_range": [float(sig[-1]), float(sig[0])], **out}


# ----------------------------------------------------------------------------- mixed variant
MIXED_GRID, MIXED_RADII = 512, 30


def run_mixed_variant(ctx, dev, stream, reps: int = 3) -> dict:
    """Mixed precision (FP32 planes, FP64 only where it sets accuracy) on a
    512^3 x 30 grid (96.6 GB of FP32 planes), timed like the main workload and
    compared with the FP64 kernel on the same planes (which agrees with the
    FP64 oracle to ~1e-13)."""
    import torch

    import hessgen
    import hessgen.device as hdev

    n, R = MIXED_GRID ** 3, MIXED_RADII
    sig = hessgen.sigma_schedule(R, S_LO, S_HI)
    hess = torch.empty((R, 6, n), dtype=torch.float32, device=dev)
    for r in range(R):
        hdev.fill(hess[r], SEED + 1, 0, r, sig[r])
    out = {}
    F = {}
    for mode in ("fp64", "mixed"):
        Fm = torch.empty(n, dtype=torch.float64, device=dev)
        im = torch.empty(n, dtype=torch.int32, device=dev)
        ctx.reset_max(Fm, im)
        ctx.collapse_multi(hess, sig, Fm, im, mode=mode)  # warm-up
        times = []
        ctx.reset_stats()
        for _ in range(reps):
            ctx.reset_max(Fm, im)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.collapse_multi(hess, sig, Fm, im, mode=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        st = ctx.stats()
        F[mode] = (Fm, im)
        out[mode] = {"kernel_ms": statistics.mean(times), "evals_per_s": n * R / (statistics.mean(times) * 1e-3),
                     "fp64_branch_fraction": st["fp64_branch"] / st["evaluations"]}
    Fr, ir = F["fp64"]
    Fx, ix = F["mixed"]
    nz = Fr > 0
    rel = torch.where(nz, (Fx - Fr).abs() / torch.where(nz, Fr, torch.ones_like(Fr)), (Fx - Fr).abs())
    edge = ((Fr > 0) & (Fr < 1.0 + 1.2e-4)) | ((Fx > 0) & (Fx < 1.0 + 1.2e-4))
    rel_ok = rel[~edge]
    del hess
    torch.cuda.empty_cache()
    return {
        "workload": f"{MIXED_GRID}^3 grid x {MIXED_RADII} radii, FP32 SoA planes (96.6 GB resident)",
        "evals_per_s": out["mixed"]["evals_per_s"], "kernel_ms": out["mixed"]["kernel_ms"],
        "fp64_kernel_same_planes_evals_per_s": out["fp64"]["evals_per_s"],
        "speedup_vs_fp64_kernel": out["fp64"]["kernel_ms"] / out["mixed"]["kernel_ms"],
        "max_rel_diff_vs_fp64": float(rel_ok.max()), "rms_rel_diff_vs_fp64": float(rel_ok.pow(2).mean().sqrt()),
        "edge_points_excluded": int(edge.sum()),
        "argmax_diff_fraction": float((ix != ir).double().mean()),
        "fp64_branch_fraction": out["mixed"]["fp64_branch_fraction"],
        "roofline": {
            "hbm": {"bytes_per_eval": 24, "achieved_gbs": 24.0 * out["mixed"]["evals_per_s"] / 1e9,
                    "peak_gbs": HBM_GBS,
                    "frac": 24.0 * out["mixed"]["evals_per_s"] / 1e9 / HBM_GBS if HBM_GBS else None},
            "fp64_pipe": {"inst_per_eval": FP64_PIPE_INST_PER_EVAL["mixed"],
                          "frac": FP64_PIPE_INST_PER_EVAL["mixed"] * out["mixed"]["evals_per_s"]
                          / (FP64_LANES_PER_CLK_PER_SM * 152 * 2070e6)},
            "note": "issue-bound (71 % of issue slots, profiles/collapse_kernel_mixed_128cube_x30.md)",
        },
        "bound_tol": 3e-5,
    }


# ----------------------------------------------------------------------------- batched variant
BATCH_SEED, BATCH_N = 2514, 48
BATCH_GRIDS = (64, 96, 128, 192, 256, 384)


def run_batch_variant(ctx, dev, stream, reps: int = 3, grids=BATCH_GRIDS, n_items: int = BATCH_N) -> dict:
    """48 realizations, grids drawn from {64..384}^3 and 8..40 radii (seeded),
    FP32 planes (240.5 GB resident), mixed precision: one persistent launch
    replayed from a CUDA graph with autotuned tiles, against one
    cc_collapse_multi launch per realization on the same data."""
    import numpy as np
    import torch

    import hessgen
    import hessgen.device as hdev
    import paper_2510_02873_gb300 as cc

    rng = np.random.default_rng(BATCH_SEED)
    grid_choice = grids
    grids = rng.choice(grid_choice, n_items)
    radii = rng.integers(8, 41, n_items)
    items = []
    for k, (g, R) in enumerate(zip(grids, radii)):
        n, R = int(g) ** 3, int(R)
        sig = hessgen.sigma_schedule(R, S_LO, S_HI)
        hess = torch.empty((R, 6, n), dtype=torch.float32, device=dev)
        for r in range(R):
            hdev.fill(hess[r], BATCH_SEED, k, r, sig[r])
        items.append((hess, sig, torch.zeros(n, dtype=torch.float64, device=dev),
                      torch.full((n,), -1, dtype=torch.int32, device=dev)))
    evals = int(sum(h.shape[0] * h.shape[2] for h, *_ in items))

    def reset():
        for _, _, F, idx in items:
            F.zero_()
            idx.fill_(-1)

    batch = cc.Batch(ctx, items, mode="mixed")
    t0 = time.perf_counter()
    batch.autotune(None, stream)
    tune_s = time.perf_counter() - t0
    blk, tiles = batch.config()
    reset()
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(side):
        batch.run_graph(side)  # capture + first replay
        side.synchronize()
        graph_ms = []
        for _ in range(reps):
            reset()
            side.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(side)
            batch.run_graph(side)
            e1.record(side)
            side.synchronize()
            graph_ms.append(e0.elapsed_time(e1))
    F_batch = [F.clone() for _, _, F, _ in items]
    # baseline: one fused launch per realization
    loop_ms = []
    for _ in range(reps):
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for hess, sig, F, idx in items:
            ctx.collapse_multi(hess, sig, F, idx, mode="mixed")
        e1.record(stream)
        torch.cuda.synchronize()
        loop_ms.append(e0.elapsed_time(e1))
    same = all(torch.equal(a, F) for a, (_, _, F, _) in zip(F_batch, items))
    batch.close()
    del items, F_batch
    torch.cuda.empty_cache()
    g, l = statistics.mean(graph_ms), statistics.mean(loop_ms)
    return {
        "workload": f"{n_items} realizations, grids {{{min(grid_choice)}..{max(grid_choice)}}}^3, 8..40 radii (seed {BATCH_SEED}), "
                    f"{evals} evaluations, FP32 planes ({evals * 24 / 1e9:.1f} GB resident), mixed precision",
        "evals_per_s": evals / (g * 1e-3), "graph_replay_ms": g,
        "per_realization_launches_ms": l, "speedup_vs_per_realization": l / g,
        "results_identical_to_per_realization": bool(same),
        "autotune_s": tune_s, "threads_per_block": blk,
        "tile_points_by_grid": {int(n): t for n, t in sorted(set((int(gg) ** 3, t) for gg, t in zip(grids, tiles)))},
    }


# ----------------------------------------------------------------------------- surrogate variant
SUR_GRID, SUR_RADII = 768, 40
SUR_TRAIN_POINTS = 40 * 1024 * 1024  # ~2e7 collapsing samples at s = 1


def run_surrogate_variant(ctx, dev, stream, steps: int = 3000) -> dict:
    """Train the MLP surrogate on the GPU (samples from the exact FP64 path on
    4.2e7 isotropic-field points at s = 1), then evaluate a 768^3 grid x 40
    radii of FP32 planes (435 GB in total, so generated one radius at a time,
    untimed) with the surrogate, the mixed path (the same pipeline with the
    closed-form cubic instead of the network) and the FP64 kernel; only the
    collapse launches are timed."""
    import torch

    import hessgen
    import hessgen.device as hdev

    h = torch.empty((6, SUR_TRAIN_POINTS), dtype=torch.float32, device=dev)
    hdev.fill(h, SEED + 5, 99, 0, 1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.surrogate_train(h, 1.0, steps=steps, batch=16384, lr=3e-3, seed=11)
    train_s = time.perf_counter() - t0
    del h
    torch.cuda.empty_cache()
    n, R = SUR_GRID ** 3, SUR_RADII
    sig = hessgen.sigma_schedule(R, S_LO, S_HI)
    planes = torch.empty((6, n), dtype=torch.float32, device=dev)
    outs = {m: (torch.zeros(n, dtype=torch.float64, device=dev), torch.full((n,), -1, dtype=torch.int32, device=dev))
            for m in ("surrogate", "surrogate_mma_sync", "mixed", "fp64")}
    ms = {m: 0.0 for m in outs}
    stats = {m: {"evaluations": 0, "fallback": 0, "fp64_branch": 0, "error_flags": 0} for m in outs}
    for r in range(R):
        hdev.fill(planes, SEED + 6, 0, r, sig[r])
        for m, (F, idx) in outs.items():
            ctx.reset_stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if m == "surrogate_mma_sync":
                ctx.set_surrogate_engine("mma_sync")
            e0.record(stream)
            ctx.collapse_scale(planes, sig[r], F, idx, r, mode=m.split("_")[0])
            e1.record(stream)
            ctx.set_surrogate_engine("tcgen05")
            torch.cuda.synchronize()
            ms[m] += e0.elapsed_time(e1)
            st = ctx.stats()
            for k in stats[m]:
                stats[m][k] += st[k]
    Fs, Fx, F64 = outs["surrogate"][0], outs["mixed"][0], outs["fp64"][0]

    def rel(a, b):
        ok = (b > 1.0 + 1.2e-4) & (a > 1.0 + 1.2e-4)
        d = ((a - b).abs() / b)[ok]
        return float(d.max()), float(d.pow(2).mean().sqrt())

    s_max, s_rms = rel(Fs, F64)
    x_max, x_rms = rel(Fx, F64)
    t_max, _ = rel(outs["surrogate_mma_sync"][0], F64)
    evals = float(n) * R
    del planes, outs
    torch.cuda.empty_cache()
    return {
        "workload": f"{SUR_GRID}^3 grid x {SUR_RADII} radii, FP32 planes streamed per radius (10.9 GB each)",
        "train": {**rep, "seconds": train_s, "steps": steps, "batch": 16384},
        "evals_per_s": evals / (ms["surrogate"] * 1e-3),
        "engine": "tcgen05",
        "error_flags": stats["surrogate"]["error_flags"],
        "tensor": {"algorithmic_flops_per_eval": MLP_FLOPS_PER_EVAL,
                   "achieved_tflops": MLP_FLOPS_PER_EVAL * evals / (ms["surrogate"] * 1e-3) / 1e12,
                   "peak_tflops": BF16_TFLOPS, "peak_basis": "measured dense BF16 GEMM (burst)",
                   "frac": (MLP_FLOPS_PER_EVAL * evals / (ms["surrogate"] * 1e-3) / 1e12 / BF16_TFLOPS)
                   if BF16_TFLOPS else None},
        "mma_sync_engine": {"evals_per_s": evals / (ms["surrogate_mma_sync"] * 1e-3),
                            "max_rel_diff_vs_fp64": t_max,
                            "fallback_fraction": stats["surrogate_mma_sync"]["fallback"]
                            / stats["surrogate_mma_sync"]["evaluations"]},
        "mixed_evals_per_s": evals / (ms["mixed"] * 1e-3),
        "fp64_evals_per_s": evals / (ms["fp64"] * 1e-3),
        "gain_over_method_without_network": ms["mixed"] / ms["surrogate"],
        "speedup_vs_fp64_kernel": ms["fp64"] / ms["surrogate"],
        "fallback_fraction": stats["surrogate"]["fallback"] / stats["surrogate"]["evaluations"],
        "max_rel_diff_vs_fp64": s_max, "rms_rel_diff_vs_fp64": s_rms,
        "mixed_max_rel_diff_vs_fp64": x_max, "mixed_rms_rel_diff_vs_fp64": x_rms,
        "bound_tol": 3e-5,
    }


def job_rate(elapsed_ms: float, evals: float, world: int, device) -> tuple:
    """Whole-job throughput over ranks: every rank's evaluations divided by the
    slowest rank's time (max over ranks)."""
    import torch
    import torch.distributed as dist

    if world <= 1:
        return evals / (elapsed_ms * 1e-3), elapsed_ms
    mx = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    sm = torch.tensor([evals], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(sm.item()) / (float(mx.item()) * 1e-3), float(mx.item())


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.variant:
        import torch

        import hessgen.device as hdev
        import paper_2510_02873_gb300 as cc
        cc.buildlib.build()
        hdev.build()
        dev = torch.device("cuda", 0)
        ctx = cc.Context(**COSMO, device=0)
        if args.variant == "batched":  # 12 realizations of grids up to --grid
            out = run_batch_variant(ctx, dev, torch.cuda.current_stream(),
                                    grids=tuple(g for g in BATCH_GRIDS if g <= args.grid), n_items=12)
        else:
            fn = {"science": run_science_variant, "field": run_field_variant}[args.variant]
            out = fn(ctx, dev, torch.cuda.current_stream(), grid=args.grid, R=args.radii)
        print(json.dumps({"variant": args.variant, **out}), flush=True)
        ctx.close()
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import hessgen
    import hessgen.device as hdev
    import paper_2510_02873_gb300 as cc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cc.buildlib.build() if hasattr(cc, "buildlib") else None
    hdev.build()

    n = args.grid ** 3
    R = args.radii
    sig = hessgen.sigma_schedule(R, S_LO, S_HI)
    ctx = cc.Context(**COSMO, device=local)
    plane_dtype = torch.float32 if args.mode in ("mixed", "surrogate") else torch.float64
    if args.mode == "surrogate":
        h = torch.empty((6, args.train_points), dtype=torch.float32, device=dev)
        hdev.fill(h, SEED + 5, 99, 0, 1.0)
        ctx.surrogate_train(h, 1.0, steps=args.train_steps, batch=16384, lr=3e-3, seed=11)
        ctx.set_surrogate_engine(args.surrogate_engine)
        del h
    if args.mode == "tabulated":
        load_table(ctx)
    hess = torch.empty((R, 6, n), dtype=plane_dtype, device=dev)
    for r in range(R):
        hdev.fill(hess[r], SEED, rank, r, sig[r])  # realization = rank: independent problem per GPU
    F = torch.empty(n, dtype=torch.float64, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        ctx.reset_max(F, idx)
        if ev is not None:
            ev[0].record(stream)
        ctx.collapse_multi(hess, sig, F, idx, mode=args.mode)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.reset_stats()
    kernel_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                     for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        step(kernel_events[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    kernel_ms = [a.elapsed_time(b) for a, b in kernel_events]
    stats = ctx.stats()
    assert stats["evaluations"] == n * R * args.steps, stats
    value, elapsed_ms = job_rate(elapsed_ms, float(n) * R * args.steps, world, dev)

    # roofline of the dominant kernel (FP64 ALU bound)
    kern_avg_s = statistics.mean(kernel_ms) * 1e-3
    evals_launch = float(n) * R
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clk.get("sm_max_mhz") or 2070.0
    peak_tflops = FP64_FLOP_PER_CLK_PER_SM * sm_count * clk_mhz * 1e6 / 1e12
    fpe = {"fp64": FP64_FLOPS_PER_EVAL, "mixed": FP64_FLOPS_PER_EVAL_MIXED}.get(args.mode)
    achieved = fpe * evals_launch / kern_avg_s / 1e12 if fpe else None
    roofline = {
        "bound": "alu", "kernel": f"collapse_kernel ({args.mode})", "unit": "TFLOP/s",
        "achieved": achieved, "peak": peak_tflops,
        "frac": (achieved / peak_tflops) if achieved else None,
        "peak_basis": f"FP64 {FP64_FLOP_PER_CLK_PER_SM:g} flop/clk/SM x {sm_count} SMs x {clk_mhz:.0f} MHz (max SM clock)",
        "flops_per_eval": fpe,
        "evals_per_s_kernel": evals_launch / kern_avg_s,
        "kernel_ms": statistics.mean(kernel_ms),
        "traffic": TRAFFIC_BYTES_DEFAULT if ((args.grid, R) == (GRID, N_RADII) and args.mode == "fp64") else None,
        "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one full launch",
        "algorithmic_bytes": 48.0 * evals_launch + 12.0 * 2 * n,
    }
    ipe = FP64_PIPE_INST_PER_EVAL.get(args.mode)
    if ipe:
        pipe_peak = FP64_LANES_PER_CLK_PER_SM * sm_count * clk_mhz * 1e6
        pipe_rate = ipe * evals_launch / kern_avg_s
        roofline["fp64_pipe"] = {
            "inst_per_eval": ipe, "achieved_inst_per_s": pipe_rate, "peak_inst_per_s": pipe_peak,
            "frac": pipe_rate / pipe_peak,
            "basis": "ncu FP64-pipe thread instructions per evaluation x live evaluations/s, against "
                     f"{FP64_LANES_PER_CLK_PER_SM:g} FP64 lanes/clk/SM x {sm_count} SMs x {clk_mhz:.0f} MHz",
        }
    if clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = (achieved / (peak_tflops * clk["sm_mhz"] / clk_mhz)) if achieved else None

    result = {
        "metric": "collapse evals/s (points x radii)", "value": value, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "f32x2": "f32x2 (float-float)", "mixed": "f32+f64",
                                       "surrogate": "bf16+f32+f64", "exact_growth": "f64",
                                       "tabulated": "f64"}[args.mode],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (args.grid, R) == (GRID, N_RADII) else f"profiling case {args.grid}^3 x {R}", "points": n, "radii": R, "mode": args.mode,
                   **({"surrogate_engine": args.surrogate_engine} if args.mode == "surrogate" else {}),
                   "per_gpu": "one independent realization per GPU",
                   "l2": f"inputs {6 * hess.element_size() * n * R / 1e9:.1f} GB per step vs 129 MB L2 (no flush needed)"},
        "roofline": roofline,
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "stats": {k: stats[k] for k in ("evaluations", "collapsed", "eds_branch", "refined", "error_flags")},
    }

    if rank == 0 and not args.no_variants and (args.grid, R) == (GRID, N_RADII) and args.mode == "fp64":
        result["variants"] = {"f32x2": run_f32x2_variant(ctx, hess, sig, F, idx, stream, args.steps)}
        result["variants"]["streamed_per_radius"] = run_streamed_variant(ctx, hess, sig, F, idx, stream, args.steps)
        result["variants"]["exact_growth"] = run_f32x2_variant(ctx, hess, sig, F, idx, stream, args.steps,
                                                               mode="exact_growth")
        load_table(ctx)
        result["variants"]["tabulated"] = run_f32x2_variant(ctx, hess, sig, F, idx, stream, args.steps,
                                                            mode="tabulated")

    # end to end through the host-buffer entry point (H2D of every radius inside the timed region)
    if not args.no_e2e and rank == 0 and args.mode == "fp64":
        host = torch.empty((R, 6, n), dtype=torch.float64, pin_memory=True)
        for r in range(R):
            host[r].copy_(hess[r], non_blocking=False)
        del hess
        torch.cuda.empty_cache()
        Fh = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ih = torch.empty(n, dtype=torch.int32, pin_memory=True)
        # each timed step of the host-buffer entry point is followed by the
        # same bytes copied alone (the step's planes host -> device, one
        # stream, no kernel): the host link's own rate at that moment
        dbuf = torch.empty_like(host[0], device=dev)
        e2e_times, link_times = [], []
        for k in range(args.warmup + args.steps):
            Fh.zero_()
            ih.fill_(-1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.collapse_multi_host(host, sig, Fh, ih)
            dt = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for r in range(R):
                dbuf.copy_(host[r], non_blocking=True)
            torch.cuda.synchronize()
            dl = time.perf_counter() - t0
            if k >= args.warmup:
                e2e_times.append(dt)
                link_times.append(dl)
        del dbuf
        h2d_bytes = int(host.numel() * 8 + n * 12)
        e2e_s = statistics.mean(e2e_times)
        link_s = statistics.mean(link_times)
        result["e2e"] = {
            "value": float(n) * R / e2e_s, "unit": "evals/s",
            "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": int(n * 12),
            "api": "cc_collapse_multi_host (pinned host planes, per-radius H2D overlapped with compute)",
            "ms_per_step": 1e3 * e2e_s,
            "step_ms": {"min": 1e3 * min(e2e_times), "median": 1e3 * statistics.median(e2e_times),
                        "max": 1e3 * max(e2e_times)},
            "link": {"bound": "host link", "achieved_h2d_gbs": h2d_bytes / e2e_s / 1e9,
                     "copies_alone_h2d_gbs": host.numel() * 8 / link_s / 1e9, "frac": link_s / e2e_s,
                     "copy_step_ms": {"min": 1e3 * min(link_times), "median": 1e3 * statistics.median(link_times),
                                      "max": 1e3 * max(link_times)},
                     "peak_basis": f"the step's planes copied host-to-device alone ({R} x "
                                   f"{host[0].numel() * 8 / 1e6:.0f} MB, one stream, no kernel) after every "
                                   "timed step; mean over the steps"},
        }
        F_check = F.cpu()
        assert torch.equal(Fh, F_check), "e2e result differs from the device-resident run"
        result["gpu_launches"] += R * args.steps
    if rank == 0 and not args.no_variants and (args.grid, R) == (GRID, N_RADII) and args.mode == "fp64":
        if "hess" in locals():
            del hess
        torch.cuda.empty_cache()
        result.setdefault("variants", {})["mixed"] = run_mixed_variant(ctx, dev, stream)
        result["variants"]["batched"] = run_batch_variant(ctx, dev, stream)
        result["variants"]["surrogate"] = run_surrogate_variant(ctx, dev, stream)
        result["variants"]["science_proxy"] = run_science_variant(ctx, dev, stream)
        result["variants"]["field_to_collapse"] = run_field_variant(ctx, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and (args.grid, R) == (GRID, N_RADII):
        result["cpu_baseline"] = cpu_oracle_rate(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
