"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on
CPU: its JSON line carries the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_cpu_baseline_keeps_every_host_core_busy():
    """The CPU baseline's sample gives every host core work: its chunks hold
    four of the oracle's 256-point blocks per core, and the cores' busy share
    over the timed calls (from /proc/stat, where the host has it) is reported
    with the rate."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.cpu_oracle_rate(0.0)
    cores = os.cpu_count() or 1
    assert r["value"] > 0 and r["cores"] == cores
    assert r["sample"].startswith(f"{1024 * cores} points")
    if os.path.exists("/proc/stat"):
        h = r["host_cpu"]
        assert 0.0 <= h["steal_frac"] <= 1.0 and 0.0 <= h["min_core_busy_frac"] <= h["busy_frac"] <= 1.0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]


@pytest.mark.gpu
def test_gpu_arm_json_line_small_case():
    """The GPU arm on a small grid: the line carries the roofline, e2e, clocks
    and launch count the contract asks for (values are not checked here)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    out = subprocess.run([sys.executable, "bench.py", "--grid", "64", "--radii", "8", "--steps", "3", "--warmup", "3",
                          "--no-variants", "--no-cpu-baseline"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    d = json.loads(lines[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in d["roofline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in d["e2e"], key
    assert d["gpu_launches"] > 0 and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0
    assert "workload" in d["config"]



def test_workloads_as_data():
    """The five workloads the bench and the tests use, from one module: the
    shapes, plane types, modes and s(R) ranges the benchmark is specified
    with, and the bench's own constants taken from them."""
    import bench
    from paper_2510_02873_gb300 import configs as cfg
    assert (cfg.SMALL_FP64.grid, cfg.SMALL_FP64.radii, cfg.SMALL_FP64.s_lo, cfg.SMALL_FP64.s_hi) == (32, 8, 0.3, 4.0)
    assert (cfg.FP64.grid, cfg.FP64.radii, cfg.FP64.planes, cfg.FP64.mode) == (256, 25, "f64", "fp64")
    assert (cfg.MIXED.grid, cfg.MIXED.radii, cfg.MIXED.planes, cfg.MIXED.mode) == (512, 30, "f32", "mixed")
    assert cfg.BATCHED.realizations == 48 and cfg.BATCHED.grids == (64, 96, 128, 192, 256, 384)
    assert cfg.BATCHED.radii_range == (8, 40)
    assert (cfg.SURROGATE.grid, cfg.SURROGATE.radii, cfg.SURROGATE.planes) == (768, 40, "f32")
    assert cfg.FP64.evaluations == 256 ** 3 * 25
    assert (bench.GRID, bench.N_RADII, bench.MIXED_GRID, bench.SUR_GRID) == (256, 25, 512, 768)
    assert bench.COSMO == dict(omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0)
    assert len(cfg.WORKLOADS) == 5
