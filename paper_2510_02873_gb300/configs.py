"""The benchmark workloads and the cosmology they share, as data.

Five workloads exercise the collapse computation (arXiv:2510.02873, Sec. 5:
the method on one accelerator at production grid sizes, and its
reduced-precision and learned variants):

1. ``SMALL_FP64``  -- the plain FP64 method on a grid the CPU oracle finishes in seconds;
2. ``FP64``        -- the plain FP64 method at the production shape (the main bench line);
3. ``MIXED``       -- FP32 planes, FP64 only where it sets the accuracy;
4. ``BATCHED``     -- many independent realizations of uneven size in one persistent launch;
5. ``SURROGATE``   -- the learned seed with its exact fallback, planes streamed per radius.

Every workload draws its Hessian planes from the isotropic-field statistics
of ``hessgen`` with s(R) log-spaced between ``s_lo`` and ``s_hi``; ``seed``
is the base seed of the input generator. ``bench.py`` takes its workload
constants from here.
"""
from __future__ import annotations

from dataclasses import asdict, dataclass


@dataclass(frozen=True)
class Cosmology:
    """Flat LCDM-like background and the a(D) spline's knots (cc_cosmology)."""
    omega_m: float = 0.3
    omega_l: float = 0.7
    n_knots: int = 512
    a_min: float = 1e-3
    a_max: float = 1.0

    def kwargs(self) -> dict:
        return asdict(self)


@dataclass(frozen=True)
class Workload:
    """One grid of points with its smoothing radii."""
    name: str
    grid: int        # points per side: grid^3 points
    radii: int       # smoothing radii per point
    planes: str      # element type of the Hessian planes: "f64" or "f32"
    mode: str        # collapse mode (cc_mode name)
    s_lo: float      # s(R), the rms of the smoothed density, log-spaced from s_lo ...
    s_hi: float      # ... to s_hi
    seed: int        # base seed of the input generator

    @property
    def points(self) -> int:
        return self.grid ** 3

    @property
    def evaluations(self) -> int:
        return self.points * self.radii


@dataclass(frozen=True)
class BatchedWorkload:
    """Independent realizations whose sides and radius counts are drawn (seeded)."""
    name: str
    realizations: int
    grids: tuple       # sides the realizations draw from
    radii_range: tuple  # (fewest, most) radii per realization
    planes: str
    mode: str
    s_lo: float
    s_hi: float
    seed: int


COSMOLOGY = Cosmology()

SMALL_FP64 = Workload("plain FP64, small", 32, 8, "f64", "fp64", 0.3, 4.0, 2511)
FP64 = Workload("plain FP64, production shape", 256, 25, "f64", "fp64", 0.2, 6.0, 2512)
MIXED = Workload("mixed precision", 512, 30, "f32", "mixed", 0.2, 6.0, 2513)
BATCHED = BatchedWorkload("batched realizations", 48, (64, 96, 128, 192, 256, 384), (8, 40), "f32", "mixed",
                          0.2, 6.0, 2514)
SURROGATE = Workload("learned surrogate", 768, 40, "f32", "surrogate", 0.2, 6.0, 2518)
SURROGATE_TRAIN_POINTS = 40 * 1024 * 1024  # training inputs at s = 1 (about 2e7 collapsing samples)

WORKLOADS = (SMALL_FP64, FP64, MIXED, BATCHED, SURROGATE)
