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

from paper_2510_02873_gb300 import configs as CFG  # noqa: E402  (the workloads as data)

GRID = CFG.FP64.grid
N_RADII = CFG.FP64.radii
S_LO, S_HI = CFG.FP64.s_lo, CFG.FP64.s_hi
SEED = CFG.FP64.seed
COSMO = CFG.COSMOLOGY.kwargs()
WORKLOAD = "collapse 256^3 grid x 25 radii, FP64 SoA Hessian planes (20.1 GB resident), 512-knot a(D) spline"

# FP64 floating-point operations per (point, radius) evaluation of the FP64
# kernel: ncu thread-instruction counters (dadd + dmul + 2 dfma) of one launch
# of the 128^3 x 4 case divided by its evaluations (the FP64 and mixed kernels
# as they stand; re-taken whenever either kernel changes).
FP64_FLOPS_PER_EVAL = 67.0
FP64_FLOPS_PER_EVAL_MIXED = 7.96
# FP64-pipe thread instructions of every kind (DFMA, DMUL, DADD, DSETP) per
# evaluation, from the same captures: the FP64 unit issues one per lane slot
# whatever the instruction, so this count, not the flop count, sets the time.
# For the mixed kernel, the lane slots the pipe was busy for (its busy
# fraction x 2 lanes/clk/SM x active SM cycles / evaluations): 4.0 against
# 3.98 DFMA thread instructions, its FP64 instructions running on full warps.
FP64_PIPE_INST_PER_EVAL = {"fp64": 38.5, "mixed": 4.0}
FP64_LANES_PER_CLK_PER_SM = 2.0
# DRAM bytes (read + write) of a launch, scaled from the 128^3 x 4 ncu capture
# of the FP64 kernel (dram__bytes_read 420.716544 MB, write 23.085056 MB for
# 8,388,608 evaluations of 2,097,152 points): the planes are read once, 48 B
# per evaluation; the rest (F_max/idx read and written for collapsed points)
# scales with the points. The full 20 GB launch is not captured.
TRAFFIC_PLANE_BYTES_PER_EVAL = 48.0
TRAFFIC_OUT_BYTES_PER_POINT = (420.716544e6 - 48.0 * 8388608 + 23.085056e6) / 2097152
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
    # points of each workload's oracle leg (CPU baseline + parity): the main
    # workload's and, divided by 2.6, each variant's (1e6 is the survey's figure)
    ap.add_argument("--cpu-points", type=int, default=262144)
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
    ap.add_argument("--variant", choices=["science", "field", "batched", "toys"], default=None)
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


# ----------------------------------------------------------------------------- oracle legs
# Each GPU leg ends (outside its timed region) with an oracle leg on a seeded
# sample of its own points: the FP64 CPU oracle evaluates every radius of the
# sampled points from the same input planes (copied from the device), timed on
# all host cores and on one thread, and the GPU's running maximum at those
# points is compared with the oracle's, element by element. The same run is
# that workload's CPU baseline and its parity report.
def _rel_err(got, ref):
    import numpy as np
    err = np.abs(got - ref)
    nz = ref != 0
    err[nz] /= np.abs(ref[nz])
    return err


def parity_report(F_gpu, idx_gpu, F_all, flags_all, tol: float, reduced: bool, scale_idx0: int = 0,
                  counts: dict | None = None) -> dict:
    """GPU F_max/idx against the oracle's per-radius values F_all (R, m) with
    flags: max and RMS relative error on F, argmax mismatches outside ties,
    and the excluded points. Ambiguous points (an eigenvalue sign or D_top on
    an oracle-flagged edge) and, for the reduced-precision paths, points whose
    F lies within 4 tol of 1 (the a_max clip) are excluded and counted, as in
    the parity tests; ties are radii whose F differ by less than 1e-9 (FP64) or
    2 tol (reduced)."""
    import numpy as np
    import oracle

    R, m = F_all.shape
    F_ref = np.zeros(m)
    idx_ref = np.full(m, -1, dtype=np.int64)
    for r in range(R):
        better = F_all[r] > F_ref
        F_ref[better] = F_all[r][better]
        idx_ref[better] = scale_idx0 + r
    amb = (flags_all & oracle.FLAGS_AMBIGUOUS).any(axis=0)
    srt = np.sort(F_all, axis=0)
    tie = np.zeros(m, dtype=bool)
    if R > 1:
        tie = (srt[-1] > 0) & (srt[-1] - srt[-2] <= (2 * tol if reduced else 1e-9) * srt[-1])
    edge = np.zeros(m, dtype=bool)
    if reduced:
        edge = ((F_ref > 0) & (F_ref < 1.0 + 4 * tol)) | ((F_gpu > 0) & (F_gpu < 1.0 + 4 * tol))
    ok = ~amb & ~edge
    err = _rel_err(np.asarray(F_gpu, dtype=np.float64), F_ref)
    out = {"points": int(m), "evaluations": int(m * R), "tol": tol,
           "max_rel_err": float(err[ok].max()) if ok.any() else 0.0,
           "rms_rel_err": float(np.sqrt(np.mean(err[ok] ** 2))) if ok.any() else 0.0,
           "within_tol": bool((err[ok] <= tol).all()),
           "idx_mismatch": int((np.asarray(idx_gpu)[ok & ~tie] != idx_ref[ok & ~tie]).sum()),
           "ambiguous": int(amb.sum()), "ties": int(tie.sum()),
           "collapsed_fraction_oracle": float((F_ref > 0).mean()),
           "eds_evaluations_oracle": int(((flags_all & oracle.FLAG_EDS) != 0).sum())}
    if reduced:
        out["edge"] = int(edge.sum())
    if counts:
        out.update(counts)
    return out


def oracle_leg(planes, F_gpu, idx_gpu, tol: float, reduced: bool, kind: str = "classic", tab=None,
               scale_idx0: int = 0, counts: dict | None = None, single_points: int = 512) -> dict:
    """planes: (R, 6, m) host array (FP64, or FP32 widened exactly) of the
    sampled points; F_gpu/idx_gpu: the GPU's results at those points. kind:
    "classic" (Tables), "exact" (RatioTables, exact growth ratios) or "tab"
    (tab = oracle.Tab of the same table)."""
    import numpy as np
    import oracle

    cos = {k: COSMO[k] for k in ("omega_m", "omega_l", "n_knots", "a_min", "a_max")}
    tables = oracle.Tables(**cos)
    rt = oracle.RatioTables(**cos) if kind == "exact" else None
    R, _, m = planes.shape

    def run(h, nthreads):
        if kind == "exact":
            return rt.F_points(h, nthreads=nthreads)
        if kind == "tab":
            return tab.F_points(tables, h, nthreads=nthreads)
        return tables.F_points(h, nthreads=nthreads)

    Fs, fl = [], []
    c0 = _cpu_times()
    t0 = time.perf_counter()
    for r in range(R):
        F, f = run(planes[r], 0)
        Fs.append(F)
        fl.append(f)
    dt = time.perf_counter() - t0
    c1 = _cpu_times()
    ms = min(single_points, m)
    t1 = time.perf_counter()
    for r in range(R):
        run(np.ascontiguousarray(planes[r][:, :ms]), 1)
    dt1 = time.perf_counter() - t1
    F_all, flags_all = np.stack(Fs), np.stack(fl)
    cpu = {"value": m * R / dt, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{m} points x {R} radii ({m * R} evaluations, {dt:.1f} s, OpenMP over {os.cpu_count()} threads)",
           "single_thread_value": ms * R / dt1, "single_thread_sample": f"{ms} points x {R} radii"}
    share = _cpu_share(c0, c1)
    if share:
        cpu["host_cpu"] = share
    return {"parity": parity_report(np.asarray(F_gpu), np.asarray(idx_gpu), F_all, flags_all, tol, reduced,
                                    scale_idx0, counts), "cpu": cpu, "F_all": F_all, "flags": flags_all}


def sample_points(n: int, m: int, seed: int):
    """m distinct seeded point indices of an n-point grid, with both ends."""
    import numpy as np
    rng = np.random.default_rng(seed)
    if m >= n:
        return np.arange(n, dtype=np.int64)
    pts = np.unique(np.concatenate([rng.choice(n, m - 2, replace=False), [0, n - 1]]))
    return pts.astype(np.int64)


def gather_planes(hess, pts):
    """(R, 6, m) host copy of the sampled points of device planes hess (R, 6, n)."""
    import torch
    idx = torch.from_numpy(pts).to(hess.device)
    return hess.index_select(2, idx).cpu().numpy()


def clk_mhz_default(dev) -> float:
    """The SM clock the FP64-pipe fractions of the variants are taken at: the
    device's maximum SM clock (nvidia-smi's clocks.max.sm; 2070 MHz on GB300)."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i",
                              str(dev.index or 0)], capture_output=True, text=True, timeout=20).stdout.strip()
        return float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return 2070.0


def timing_stats(ms: list) -> dict:
    """median, min, max and relative standard deviation of per-launch times."""
    med = statistics.median(ms)
    rsd = statistics.pstdev(ms) / statistics.mean(ms) if len(ms) > 1 else 0.0
    return {"median": med, "min": min(ms), "max": max(ms), "rsd": rsd, "n": len(ms)}


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
def run_f32x2_variant(ctx, hess, sig, F_ref, idx_ref, stream, steps: int, mode: str = "f32x2",
                      oracle_in: dict | None = None) -> dict:
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
    parity = None
    if oracle_in is not None:  # the oracle on sampled points of the same planes
        import torch as _t
        pts = oracle_in["pts"]
        pi = _t.from_numpy(pts).to(F.device)
        Fg, ig = F.index_select(0, pi).cpu().numpy(), idx.index_select(0, pi).cpu().numpy()
        if mode == "f32x2":
            parity = parity_report(Fg, ig, oracle_in["F_all"], oracle_in["flags"], 1e-10, False)
        else:
            m = min(len(pts), 20000)
            kind = "exact" if mode == "exact_growth" else "tab"
            tab = None
            if kind == "tab":
                import oracle
                dg, xg, yg = table_axes()
                tab = oracle.Tab(dg, xg, yg, oracle.tab_node_values(dg, xg, yg))
            leg = oracle_leg(oracle_in["planes"][:, :, :m], Fg[:m], ig[:m], 1e-10, False, kind=kind, tab=tab)
            parity = leg["parity"]
            parity["cpu_oracle_evals_per_s"] = leg["cpu"]["value"]
    return {
        "workload": "the main workload's planes (256^3 x 25, FP64)",
        "evals_per_s": float(n) * R / (ms * 1e-3), "kernel_ms": ms, "kernel_ms_stats": timing_stats(times),
        **({"parity": parity} if parity is not None else {}),
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
HIST_CALLS_PER_GROUP = 10


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
    # groups of back-to-back calls between one pair of events, so that the
    # stream never waits on the host between calls: per call, the counts'
    # memset and the kernel
    times = []
    for _ in range(reps):
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(HIST_CALLS_PER_GROUP):
            ctx.histogram(F, SCI_EDGES, counts)
        h1.record(stream)
        torch.cuda.synchronize()
        times.append(h0.elapsed_time(h1) / HIST_CALLS_PER_GROUP)
    c = counts.cpu().tolist()
    hist_ms = statistics.median(times)
    pts = sample_points(n, 20000, SEED + 13)
    pi = torch.from_numpy(pts).to(dev)
    leg = oracle_leg(gather_planes(hess, pts), F.index_select(0, pi).cpu().numpy(),
                     idx.index_select(0, pi).cpu().numpy(), 1e-10, False)
    import oracle
    F_or = leg["F_all"].max(axis=0)
    c_or = oracle.histogram(F_or, SCI_EDGES)
    c_gpu_sample = oracle.histogram(F.index_select(0, pi).cpu().numpy(), SCI_EDGES)
    del hess
    torch.cuda.empty_cache()
    return {
        "workload": f"{grid}^3 grid x {R} correlated radii (rho {SCI_RHO}), FP64 planes",
        "z_edges": [round(e - 1.0, 4) for e in SCI_EDGES],
        "collapsed_per_z_bin": c[1:-1], "not_collapsed_or_z_below_0": c[0], "z_above_last_edge": c[-1],
        "collapsed_fraction": float((F > 0).double().mean()),
        "collapse_kernel_ms": collapse_ms, "evals_per_s": n * R / (collapse_ms * 1e-3),
        "histogram_kernel_ms": hist_ms, "histogram_kernel_ms_stats": timing_stats(times),
        "histogram_timing": f"per cc_histogram call (counts memset + kernel): mean of {HIST_CALLS_PER_GROUP} "
                            f"back-to-back calls per event pair, median over {reps} pairs; F ({8 * n / 1e6:.0f} MB) "
                            "streams through L2 between calls",
        "parity": leg["parity"],
        "sample_counts_differ_from_oracle": int(abs(c_or - c_gpu_sample).sum()),
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
    pts = sample_points(n, 20000, SEED + 14)
    pi = torch.from_numpy(pts).to(dev)
    for label, dt, mode in (("fp64", torch.float64, "fp64"), ("fp32_planes_mixed", torch.float32, "mixed")):
        sample_planes = np.empty((R, 6, len(pts)), dtype=np.float64 if dt == torch.float64 else np.float32)
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
        # untimed pass: the same planes again (deterministic), sampled for the oracle
        for r in range(R):
            field.hessian(radii[r], planes)
            sample_planes[r] = planes.index_select(1, pi).cpu().numpy()
        leg = oracle_leg(sample_planes, F.index_select(0, pi).cpu().numpy(), idx.index_select(0, pi).cpu().numpy(),
                         1e-10 if mode == "fp64" else 3e-5, mode != "fp64")
        out[label] = {"evals_per_s": n * R / (t * 1e-3), "ms_per_realization": t,
                      "ms_per_realization_stats": timing_stats(tot_ms),
                      "hessian_fft_ms": statistics.mean(fft_ms), "collapse_ms": statistics.mean(col_ms),
                      "collapsed_fraction": float((F > 0).double().mean()), "parity": leg["parity"]}
        del planes
    field.close()
    torch.cuda.empty_cache()
    return {"workload": f"{grid}^3 white noise -> P(k) = A k^n exp(-(k/k_c)^2) ({spec}) -> "
                        f"{R} Gaussian radii {FIELD_RADII[0]}..{FIELD_RADII[1]} -> Hessian planes -> collapse, all on the device",
            "sigma_range": [float(sig[-1]), float(sig[0])], **out}


# ----------------------------------------------------------------------------- interpolation toys
TOY_QUERIES = (10 ** 2, 10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7, 10 ** 8)


def run_toys_variant(ctx, dev, stream, reps: int = 10, max_queries: int = 10 ** 8) -> dict:
    """The paper's two interpolation toys (Sec. 4.3, 5.1, 5.2) on the GPU:
    y = x^2 through a natural spline on 512 random knots (cc_spline_eval), and
    z = x^2 + y^2 on a random 64 x 64 grid whose nodes carry 128-knot splines
    (cc_table_query), each at 1e2 .. 1e8 uniformly random queries. Per size:
    device time (CUDA events around the call, queries resident) and end-to-end
    time (queries copied from pinned host memory, the call, results copied
    back), over `reps` repetitions (median, min, max, RSD as in the paper's
    timing table); the mean relative residual against the analytic function
    and the largest relative difference from the CPU oracle's interpolation
    (which is also timed, on all host cores, up to 1e7 queries)."""
    import numpy as np
    import torch

    import oracle

    rng = np.random.default_rng(SEED + 20)
    xk = np.sort(rng.uniform(0.0, 1.0, 512))
    yk = xk * xk
    Mk = oracle.spline_build(xk, yk)
    dg = np.sort(rng.uniform(-1.0, 1.0, 128))
    xg = np.sort(rng.uniform(0.0, 1.0, 64))
    yg = np.sort(rng.uniform(0.0, 1.0, 64))
    val = np.repeat((xg[:, None] ** 2 + yg[None, :] ** 2)[:, :, None], 128, axis=2)
    ctx.set_table(dg, xg, yg, val)
    tab = oracle.Tab(dg, xg, yg, val)
    out = {"spline_1d": [], "bilinear_2d": []}
    for m in (q for q in TOY_QUERIES if q <= max_queries):
        for toy in ("spline_1d", "bilinear_2d"):
            if toy == "spline_1d":
                qh = [torch.from_numpy(rng.uniform(xk[0], xk[-1], m)).pin_memory()]
            else:
                qh = [torch.from_numpy(rng.uniform(lo, hi, m)).pin_memory()
                      for lo, hi in ((dg[0], dg[-1]), (xg[0], xg[-1]), (yg[0], yg[-1]))]
            qd = [a.to(dev) for a in qh]
            od = torch.empty(m, dtype=torch.float64, device=dev)
            oh = torch.empty(m, dtype=torch.float64, pin_memory=True)

            def call(qs):
                if toy == "spline_1d":
                    ctx.spline_eval(xk, yk, qs[0], od, stream)
                else:
                    ctx.table_query(*qs, od, stream)

            call(qd)
            torch.cuda.synchronize()
            dev_ms, e2e_ms = [], []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call(qd)
                e1.record(stream)
                torch.cuda.synchronize()
                dev_ms.append(e0.elapsed_time(e1))
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for a, b in zip(qd, qh):
                    a.copy_(b, non_blocking=True)
                call(qd)
                oh.copy_(od, non_blocking=True)
                torch.cuda.synchronize()
                e2e_ms.append(1e3 * (time.perf_counter() - t0))
            got = oh.numpy()
            qn = [a.numpy() for a in qh]
            exact = qn[0] ** 2 if toy == "spline_1d" else qn[1] ** 2 + qn[2] ** 2
            mc = min(m, 10 ** 7)
            t0 = time.perf_counter()
            if toy == "spline_1d":
                ref = oracle.spline_eval_many(xk, yk, Mk, qn[0][:mc])
            else:
                ref = tab.query_many(qn[0][:mc], qn[1][:mc], qn[2][:mc])
            cpu_s = time.perf_counter() - t0
            out[toy].append({
                "queries": m,
                "device_ms": timing_stats(dev_ms), "e2e_ms": timing_stats(e2e_ms),
                "device_queries_per_s": m / (statistics.median(dev_ms) * 1e-3),
                "e2e_queries_per_s": m / (statistics.median(e2e_ms) * 1e-3),
                "mean_rel_residual_vs_analytic": float(np.mean(np.abs(got - exact) / exact)),
                "max_rel_diff_vs_oracle": float(np.max(np.abs(got[:mc] - ref) / np.maximum(np.abs(ref), 1e-300))),
                "cpu_oracle_queries_per_s": mc / cpu_s, "cpu_oracle_queries": mc,
            })
            del qd, od, oh, qh
    torch.cuda.empty_cache()
    return {"workload": "y = x^2 on 512 random knots in [0, 1]; z = x^2 + y^2 on a random 64 x 64 grid in [0, 1]^2 "
                        "with 128 random knots along delta in [-1, 1]; uniformly random queries",
            "cores": os.cpu_count(), **out}


# ----------------------------------------------------------------------------- mixed variant
MIXED_GRID, MIXED_RADII = CFG.MIXED.grid, CFG.MIXED.radii


def run_mixed_variant(ctx, dev, stream, reps: int = 3, sample: int = 100000) -> dict:
    """Mixed precision (FP32 planes, FP64 only where it sets accuracy) on a
    512^3 x 30 grid (96.6 GB of FP32 planes), timed like the main workload and
    compared with the FP64 kernel on the same planes (which agrees with the
    FP64 oracle to ~1e-13)."""
    import torch

    import hessgen
    import hessgen.device as hdev

    n, R = MIXED_GRID ** 3, MIXED_RADII
    sig = hessgen.sigma_schedule(R, S_LO, S_HI)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clk_mhz_default(dev)
    hess = torch.empty((R, 6, n), dtype=torch.float32, device=dev)
    for r in range(R):
        hdev.fill(hess[r], CFG.MIXED.seed, 0, r, sig[r])
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
                     "kernel_ms_stats": timing_stats(times),
                     "fp64_branch_fraction": st["fp64_branch"] / st["evaluations"], "stats": st}
    Fr, ir = F["fp64"]
    Fx, ix = F["mixed"]
    nz = Fr > 0
    rel = torch.where(nz, (Fx - Fr).abs() / torch.where(nz, Fr, torch.ones_like(Fr)), (Fx - Fr).abs())
    edge = ((Fr > 0) & (Fr < 1.0 + 1.2e-4)) | ((Fx > 0) & (Fx < 1.0 + 1.2e-4))
    rel_ok = rel[~edge]
    # oracle leg on sampled points of the same FP32 planes (config 3's CPU baseline)
    pts = sample_points(n, sample, SEED + 11)
    planes = gather_planes(hess, pts)
    pi = torch.from_numpy(pts).to(dev)
    st = out["mixed"]["stats"]
    leg = oracle_leg(planes, Fx.index_select(0, pi).cpu().numpy(), ix.index_select(0, pi).cpu().numpy(), 3e-5, True,
                     counts={"fp64_branch_fraction_gpu": st["fp64_branch"] / st["evaluations"],
                             "eds_fraction_gpu": st["eds_branch"] / st["evaluations"],
                             "refined_fraction_gpu": st["refined"] / st["evaluations"]})
    leg64 = parity_report(Fr.index_select(0, pi).cpu().numpy(), ir.index_select(0, pi).cpu().numpy(),
                          leg["F_all"], leg["flags"], 1e-10, False)
    del hess, planes
    torch.cuda.empty_cache()
    return {
        "workload": f"{MIXED_GRID}^3 grid x {MIXED_RADII} radii, FP32 SoA planes (96.6 GB resident)",
        "evals_per_s": out["mixed"]["evals_per_s"], "kernel_ms": out["mixed"]["kernel_ms"],
        "kernel_ms_stats": out["mixed"]["kernel_ms_stats"],
        "parity": leg["parity"], "fp64_kernel_same_planes_parity": leg64, "cpu_baseline": leg["cpu"],
        "fp64_kernel_same_planes_evals_per_s": out["fp64"]["evals_per_s"],
        "speedup_vs_fp64_kernel": out["fp64"]["kernel_ms"] / out["mixed"]["kernel_ms"],
        "vs_fp64_kernel_all_points": {"max_rel_diff": float(rel_ok.max()),
                                      "rms_rel_diff": float(rel_ok.pow(2).mean().sqrt()),
                                      "edge_points_excluded": int(edge.sum())},
        "argmax_diff_fraction": float((ix != ir).double().mean()),
        "fp64_branch_fraction": out["mixed"]["fp64_branch_fraction"],
        "roofline": {
            "hbm": {"bytes_per_eval": 24, "achieved_gbs": 24.0 * out["mixed"]["evals_per_s"] / 1e9,
                    "peak_gbs": HBM_GBS,
                    "frac": 24.0 * out["mixed"]["evals_per_s"] / 1e9 / HBM_GBS if HBM_GBS else None},
            "fp64_pipe": {"inst_per_eval": FP64_PIPE_INST_PER_EVAL["mixed"],
                          "frac": FP64_PIPE_INST_PER_EVAL["mixed"] * out["mixed"]["evals_per_s"]
                          / (FP64_LANES_PER_CLK_PER_SM * sm_count * clk_mhz * 1e6),
                          "basis": f"{FP64_LANES_PER_CLK_PER_SM:g} FP64 lanes/clk/SM x {sm_count} SMs x "
                                   f"{clk_mhz:.0f} MHz"},
            "note": "issue-bound: the FP32 and integer instructions of the eigen and root stages fill the issue "
                    "slots before HBM or the FP64 unit saturate",
        },
        "bound_tol": 3e-5,
    }


# ----------------------------------------------------------------------------- batched variant
BATCH_SEED, BATCH_N = CFG.BATCHED.seed, CFG.BATCHED.realizations
BATCH_GRIDS = CFG.BATCHED.grids


def merge_parity(reports: list) -> dict:
    """One parity report from several (realizations of a batch)."""
    import math
    pts = sum(r["points"] for r in reports)
    out = {"points": pts, "evaluations": sum(r["evaluations"] for r in reports), "tol": reports[0]["tol"],
           "max_rel_err": max(r["max_rel_err"] for r in reports),
           "rms_rel_err": math.sqrt(sum(r["rms_rel_err"] ** 2 * r["points"] for r in reports) / pts),
           "within_tol": all(r["within_tol"] for r in reports)}
    for k in ("idx_mismatch", "ambiguous", "ties", "edge", "eds_evaluations_oracle"):
        if k in reports[0]:
            out[k] = sum(r[k] for r in reports)
    out["collapsed_fraction_oracle"] = sum(r["collapsed_fraction_oracle"] * r["points"] for r in reports) / pts
    return out


def run_batch_variant(ctx, dev, stream, reps: int = 3, grids=BATCH_GRIDS, n_items: int = BATCH_N,
                      sample: int = 100000) -> dict:
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
    radii = rng.integers(CFG.BATCHED.radii_range[0], CFG.BATCHED.radii_range[1] + 1, n_items)
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
    # oracle leg: a seeded sample of every realization (config 4's CPU baseline)
    reports, evals_cpu, secs_cpu, evals_1, secs_1 = [], 0, 0.0, 0, 0.0
    per = max(256, sample // n_items)
    for k, (hess, sig, F, idx) in enumerate(items):
        pts = sample_points(hess.shape[2], per, BATCH_SEED + 100 + k)
        pi = torch.from_numpy(pts).to(dev)
        leg = oracle_leg(gather_planes(hess, pts), F_batch[k].index_select(0, pi).cpu().numpy(),
                         idx.index_select(0, pi).cpu().numpy(), 3e-5, True, single_points=32)
        reports.append(leg["parity"])
        ev = leg["parity"]["evaluations"]
        evals_cpu += ev
        secs_cpu += ev / leg["cpu"]["value"]
        ev1 = 32 * hess.shape[0]
        evals_1 += ev1
        secs_1 += ev1 / leg["cpu"]["single_thread_value"]
    cpu = {"value": evals_cpu / secs_cpu, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{per} points of each of the {n_items} realizations x their radii ({evals_cpu} evaluations, "
                     f"{secs_cpu:.1f} s, OpenMP over {os.cpu_count()} threads)",
           "single_thread_value": evals_1 / secs_1, "single_thread_sample": "32 points of each realization"}
    batch.close()
    del items, F_batch
    torch.cuda.empty_cache()
    g, l = statistics.mean(graph_ms), statistics.mean(loop_ms)
    return {
        "workload": f"{n_items} realizations, grids {{{min(grid_choice)}..{max(grid_choice)}}}^3, 8..40 radii (seed {BATCH_SEED}), "
                    f"{evals} evaluations, FP32 planes ({evals * 24 / 1e9:.1f} GB resident), mixed precision",
        "evals_per_s": evals / (g * 1e-3), "graph_replay_ms": g, "graph_replay_ms_stats": timing_stats(graph_ms),
        "parity": merge_parity(reports), "cpu_baseline": cpu,
        "per_realization_launches_ms": l, "speedup_vs_per_realization": l / g,
        "results_identical_to_per_realization": bool(same),
        "autotune_s": tune_s, "threads_per_block": blk,
        "tile_points_by_grid": {int(n): t for n, t in sorted(set((int(gg) ** 3, t) for gg, t in zip(grids, tiles)))},
    }


# ----------------------------------------------------------------------------- surrogate variant
SUR_GRID, SUR_RADII = CFG.SURROGATE.grid, CFG.SURROGATE.radii
SUR_TRAIN_POINTS = CFG.SURROGATE_TRAIN_POINTS  # ~2e7 collapsing samples at s = 1


def run_surrogate_variant(ctx, dev, stream, steps: int = 3000, sample: int = 100000) -> dict:
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
    per_radius_ms = {m: [] for m in outs}
    stats = {m: {"evaluations": 0, "fallback": 0, "fp64_branch": 0, "error_flags": 0} for m in outs}
    import numpy as np
    pts = sample_points(n, sample, SEED + 12)
    pi = torch.from_numpy(pts).to(dev)
    sample_planes = np.empty((R, 6, len(pts)), dtype=np.float32)
    for r in range(R):
        hdev.fill(planes, CFG.SURROGATE.seed, 0, r, sig[r])
        sample_planes[r] = planes.index_select(1, pi).cpu().numpy()
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
            per_radius_ms[m].append(e0.elapsed_time(e1))
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
    # oracle leg on the sampled points of every radius (config 5's CPU baseline)
    sel = {m: (outs[m][0].index_select(0, pi).cpu().numpy(), outs[m][1].index_select(0, pi).cpu().numpy())
           for m in outs}
    st_s = stats["surrogate"]
    leg = oracle_leg(sample_planes, *sel["surrogate"], 3e-5, True,
                     counts={"fallback_fraction_gpu": st_s["fallback"] / st_s["evaluations"]})
    par = {m: parity_report(*sel[m], leg["F_all"], leg["flags"], 1e-10 if m == "fp64" else 3e-5, m != "fp64")
           for m in ("surrogate_mma_sync", "mixed", "fp64")}
    del planes, outs
    torch.cuda.empty_cache()
    return {
        "workload": f"{SUR_GRID}^3 grid x {SUR_RADII} radii, FP32 planes streamed per radius (10.9 GB each)",
        "train": {**rep, "seconds": train_s, "steps": steps, "batch": 16384},
        "evals_per_s": evals / (ms["surrogate"] * 1e-3),
        "per_radius_kernel_ms_stats": timing_stats(per_radius_ms["surrogate"]),
        "parity": leg["parity"], "cpu_baseline": leg["cpu"],
        "parity_same_planes": {"mma_sync_engine": par["surrogate_mma_sync"], "mixed": par["mixed"],
                               "fp64_kernel": par["fp64"]},
        "engine": "tcgen05",
        "error_flags": stats["surrogate"]["error_flags"],
        "tensor": {"algorithmic_flops_per_eval": MLP_FLOPS_PER_EVAL,
                   "achieved_tflops": MLP_FLOPS_PER_EVAL * evals / (ms["surrogate"] * 1e-3) / 1e12,
                   "peak_tflops": BF16_TFLOPS, "peak_basis": "measured dense BF16 GEMM (burst)",
                   "frac": (MLP_FLOPS_PER_EVAL * evals / (ms["surrogate"] * 1e-3) / 1e12 / BF16_TFLOPS)
                   if BF16_TFLOPS else None},
        "mma_sync_engine": {"evals_per_s": evals / (ms["surrogate_mma_sync"] * 1e-3),
                            "max_rel_diff_vs_fp64_kernel": t_max,
                            "fallback_fraction": stats["surrogate_mma_sync"]["fallback"]
                            / stats["surrogate_mma_sync"]["evaluations"]},
        "mixed_evals_per_s": evals / (ms["mixed"] * 1e-3),
        "fp64_evals_per_s": evals / (ms["fp64"] * 1e-3),
        "gain_over_method_without_network": ms["mixed"] / ms["surrogate"],
        "speedup_vs_fp64_kernel": ms["fp64"] / ms["surrogate"],
        "fallback_fraction": stats["surrogate"]["fallback"] / stats["surrogate"]["evaluations"],
        "vs_fp64_kernel_all_points": {"surrogate_max_rel_diff": s_max, "surrogate_rms_rel_diff": s_rms,
                                      "mixed_max_rel_diff": x_max, "mixed_rms_rel_diff": x_rms},
        "bound_tol": 3e-5,
    }


def run_config1_leg(ctx, dev) -> dict:
    """The small configuration in full: 32^3 points x 8 radii (s 0.3 -> 4.0,
    FP64 planes, seed 2511) on the GPU (one fused launch), and the oracle on
    every evaluation (all host cores; one thread on the first 4096 points)."""
    import torch

    import hessgen

    w = CFG.SMALL_FP64
    n, R = w.points, w.radii
    sig = hessgen.sigma_schedule(R, w.s_lo, w.s_hi)
    stack = hessgen.hessian_stack(w.seed, 0, sig, n)
    hess = torch.from_numpy(stack).to(dev)
    F = torch.empty(n, dtype=torch.float64, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    ctx.reset_max(F, idx)
    ctx.collapse_multi(hess, sig, F, idx, mode="fp64")
    torch.cuda.synchronize()
    return oracle_leg(stack, F.cpu().numpy(), idx.cpu().numpy(), 1e-10, False, single_points=4096)


# Bound on every collective of a multi-rank run: a rank that dies or stops
# answering surfaces on the others as an error at their next collective
# (barrier or all_reduce) within this time instead of a hang.
PG_TIMEOUT_S = 600.0


def init_ranks(backend: str, timeout_s: float = PG_TIMEOUT_S) -> None:
    """Join the process group (RANK, WORLD_SIZE, MASTER_ADDR/PORT from the
    environment) with a bounded collective timeout."""
    import datetime

    import torch.distributed as dist
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))


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
        elif args.variant == "toys":
            out = run_toys_variant(ctx, dev, torch.cuda.current_stream())
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
        init_ranks("nccl")
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
        if ev is not None:
            ev[2].record(stream)
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
    # per step: kernel start, kernel end, step start (the reset of F_max/idx)
    kernel_events = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
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
    kernel_ms = [a.elapsed_time(b) for a, b, _ in kernel_events]
    step_ms = [c.elapsed_time(b) for _, b, c in kernel_events]
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
        "kernel_ms_stats": timing_stats(kernel_ms),
        "traffic": (TRAFFIC_PLANE_BYTES_PER_EVAL * evals_launch + TRAFFIC_OUT_BYTES_PER_POINT * n)
        if args.mode == "fp64" else None,
        "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 128^3 x 4 launch of the same "
                         "kernel, scaled to this launch: plane reads by evaluations, F_max/idx traffic by points",
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
        "timing": {"step_ms": timing_stats(step_ms), "kernel_ms": timing_stats(kernel_ms),
                   "value_at_median_step": float(n) * R * world / (statistics.median(step_ms) * 1e-3),
                   "basis": "CUDA events on the launching stream around each timed step (reset + fused "
                            "launch) and around each fused launch; value is the whole timed region"},
        # per step: the reset kernel and the collapse kernel (mixed: also its two
        # kernels for the recorded points)
        "gpu_launches": (4 if args.mode == "mixed" else 2) * args.steps,
        "clocks": clk,
        "stats": {k: stats[k] for k in ("evaluations", "collapsed", "eds_branch", "refined", "error_flags")},
    }

    full = (args.grid, R) == (GRID, N_RADII)
    main_leg = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and full:
        # oracle leg of the main workload: sampled points of the device planes,
        # every radius; its timing is the CPU baseline, its comparison the parity
        pts = sample_points(n, args.cpu_points, SEED + 10)
        planes = gather_planes(hess, pts)
        pi = torch.from_numpy(pts).to(dev)
        tol = 1e-10 if args.mode in ("fp64", "f32x2", "exact_growth", "tabulated") else 3e-5
        main_leg = oracle_leg(planes, F.index_select(0, pi).cpu().numpy(), idx.index_select(0, pi).cpu().numpy(),
                              tol, tol > 1e-10,
                              counts={"eds_evaluations_gpu_whole_grid": stats["eds_branch"] // args.steps,
                                      "refined_evaluations_gpu_whole_grid": stats["refined"] // args.steps,
                                      "fp64_branch_evaluations_gpu_whole_grid": stats["fp64_branch"] // args.steps,
                                      "fallback_evaluations_gpu_whole_grid": stats["fallback"] // args.steps})
        result["parity"] = main_leg["parity"]
        result["cpu_baseline"] = main_leg["cpu"]
        main_leg = {"pts": pts, "planes": planes, "F_all": main_leg["F_all"], "flags": main_leg["flags"]}
    if rank == 0 and not args.no_variants and (args.grid, R) == (GRID, N_RADII) and args.mode == "fp64":
        result["variants"] = {"f32x2": run_f32x2_variant(ctx, hess, sig, F, idx, stream, args.steps,
                                                         oracle_in=main_leg)}
        result["variants"]["streamed_per_radius"] = run_streamed_variant(ctx, hess, sig, F, idx, stream, args.steps)
        result["variants"]["exact_growth"] = run_f32x2_variant(ctx, hess, sig, F, idx, stream, args.steps,
                                                               mode="exact_growth", oracle_in=main_leg)
        load_table(ctx)
        result["variants"]["tabulated"] = run_f32x2_variant(ctx, hess, sig, F, idx, stream, args.steps,
                                                            mode="tabulated", oracle_in=main_leg)

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
        result["gpu_launches"] += (3 if args.mode == "mixed" else 1) * R * args.steps
    if rank == 0 and not args.no_variants and (args.grid, R) == (GRID, N_RADII) and args.mode == "fp64":
        if "hess" in locals():
            del hess
        torch.cuda.empty_cache()
        vs = max(10000, int(args.cpu_points / 2.62144))  # 100,000 points at the default
        result.setdefault("variants", {})["mixed"] = run_mixed_variant(ctx, dev, stream, sample=vs)
        result["variants"]["batched"] = run_batch_variant(ctx, dev, stream, sample=vs)
        result["variants"]["surrogate"] = run_surrogate_variant(ctx, dev, stream, sample=vs)
        result["variants"]["science_proxy"] = run_science_variant(ctx, dev, stream)
        result["variants"]["field_to_collapse"] = run_field_variant(ctx, dev, stream)
        result["variants"]["interpolation_toys"] = run_toys_variant(ctx, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and full:
        # the oracle on all of the small configuration (32^3 x 8, FP64), and the
        # per-configuration baselines gathered from the legs above
        c1 = run_config1_leg(ctx, dev)
        result["cpu_baselines"] = {"config1_32cube_x8_fp64_full": c1["cpu"],
                                   "config2_256cube_x25_fp64_sample": result.get("cpu_baseline")}
        result["parity_config1_32cube_x8"] = c1["parity"]
        var = result.get("variants", {})
        for key, name in (("mixed", "config3_512cube_x30_mixed_sample"), ("batched", "config4_batched_sample"),
                          ("surrogate", "config5_768cube_x40_surrogate_sample")):
            if key in var and "cpu_baseline" in var[key]:
                result["cpu_baselines"][name] = var[key]["cpu_baseline"]
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
