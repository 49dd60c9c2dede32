"""Seeded synthetic Hessian generator shared by the tests, the oracle runs and the bench.

This module holds no arithmetic of the collapse-time method. It only draws
Gaussian random numbers and mixes them into the six independent components of
a symmetric 3x3 matrix with the covariance of an isotropic Gaussian field's
potential Hessian: <d_ii^2> = s^2/5, <d_ii d_jj> = s^2/15 (i != j),
<d_ij^2> = s^2/15, so that var(tr d) = s^2. These stand in for the FFT-smoothed
Hessians of the paper's Fmax stage (Sec. 3), which need a power spectrum and
initial conditions that are not reproduced here.

Random numbers come from Philox-4x32-10 (Salmon, Moraes, Dror & Shaw 2011,
"Parallel random numbers: as easy as 1, 2, 3"), written here from its
published definition. One point draws four Philox blocks:

    counter = (lo32(4*point + k), hi32(4*point + k), radius, realization), k = 0..3
    key     = (lo32(seed), hi32(seed))

giving 16 words -> 8 uniform doubles in (0, 1) with 52 random bits each
(u = (m + 0.5) * 2^-52) -> 8 Gaussians by Box-Muller (pairs (u0,u1), (u2,u3),
...). Gaussians g[0..6] are used: g0 is the shared isotropic part,
g1..g3 the diagonal, g4..g6 the off-diagonal (xy, xz, yz).

    d_ii = s * (c2 * g_i + c1 * g0),   c2 = sqrt(2/15), c1 = sqrt(1/15)
    d_ij = s * (c1 * g_ij)

Component planes are ordered xx, yy, zz, xy, xz, yz. FP32 inputs are the FP64
draw rounded to nearest.

The device-side generator (hessgen/hessgen.cu, loaded by ``device``) follows
the same definition with no fused multiply-adds in the mixing step; it agrees
with this host version to the last few ulps (the Box-Muller transcendentals of
the two math libraries are not bit-identical).
"""
from __future__ import annotations

import math

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

C1 = math.sqrt(1.0 / 15.0)
C2 = math.sqrt(2.0 / 15.0)

COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox-4x32-10 block function.

    ctr: (4, N) uint32 counters; key: (2,) or (2, N) uint32 keys.
    Returns (4, N) uint32 output words.
    """
    c0, c1, c2, c3 = (np.asarray(ctr[i], dtype=np.uint32).copy() for i in range(4))
    key = np.asarray(key, dtype=np.uint32)
    k0 = np.broadcast_to(key[0], c0.shape).astype(np.uint32)
    k1 = np.broadcast_to(key[1], c0.shape).astype(np.uint32)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            p0 = c0.astype(np.uint64) * PHILOX_M0
            p1 = c2.astype(np.uint64) * PHILOX_M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3])


def uniforms(seed: int, realization: int, radius: int, points: np.ndarray) -> np.ndarray:
    """(8, N) uniform doubles in (0, 1) for the given point indices."""
    points = np.asarray(points, dtype=np.int64)
    n = points.shape[0]
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    words = np.empty((16, n), dtype=np.uint32)
    for k in range(4):
        c = points.astype(np.uint64) * np.uint64(4) + np.uint64(k)
        ctr = np.stack([
            (c & MASK32).astype(np.uint32),
            (c >> np.uint64(32)).astype(np.uint32),
            np.full(n, radius, dtype=np.uint32),
            np.full(n, realization, dtype=np.uint32),
        ])
        words[4 * k:4 * k + 4] = philox4x32_10(ctr, key)
    hi = words[0::2].astype(np.uint64)  # 8 x N
    lo = words[1::2].astype(np.uint64)
    m = ((hi & np.uint64(0xFFFFF)) << np.uint64(32)) | lo  # 52 random bits
    return (m.astype(np.float64) + 0.5) * (2.0 ** -52)


def gaussians(seed: int, realization: int, radius: int, points: np.ndarray) -> np.ndarray:
    """(8, N) standard normal draws (Box-Muller on consecutive uniform pairs)."""
    u = uniforms(seed, realization, radius, points)
    out = np.empty_like(u)
    for j in range(4):
        r = np.sqrt(-2.0 * np.log(u[2 * j]))
        t = (2.0 * math.pi) * u[2 * j + 1]
        out[2 * j] = r * np.cos(t)
        out[2 * j + 1] = r * np.sin(t)
    return out


def hessian_points(seed: int, realization: int, radius: int, s: float,
                   points: np.ndarray, dtype=np.float64) -> np.ndarray:
    """(6, N) Hessian components for the given point indices at rms s."""
    g = gaussians(seed, realization, radius, points)
    h = np.empty((6, g.shape[1]), dtype=np.float64)
    for i in range(3):
        h[i] = s * (C2 * g[1 + i] + C1 * g[0])
    for j in range(3):
        h[3 + j] = s * (C1 * g[4 + j])
    return h.astype(dtype)


def hessian_planes(seed: int, realization: int, radius: int, s: float, n_points: int,
                   dtype=np.float64) -> np.ndarray:
    """(6, n_points) SoA planes for points 0..n_points-1."""
    return hessian_points(seed, realization, radius, s, np.arange(n_points, dtype=np.int64), dtype)


def sigma_schedule(n_radii: int, s_lo: float, s_hi: float) -> np.ndarray:
    """s(R) log-spaced from s_lo to s_hi over n_radii smoothing radii."""
    if n_radii == 1:
        return np.array([s_lo])
    return np.exp(np.linspace(math.log(s_lo), math.log(s_hi), n_radii))


def hessian_stack(seed: int, realization: int, sigmas, n_points: int, dtype=np.float64) -> np.ndarray:
    """(R, 6, n_points) planes for every radius."""
    return np.stack([hessian_planes(seed, realization, r, float(s), n_points, dtype)
                     for r, s in enumerate(sigmas)])


def hessian_stack_correlated(seed: int, realization: int, sigmas, n_points: int, rho: float,
                             dtype=np.float64) -> np.ndarray:
    """(R, 6, n_points) planes with correlated radii: a unit-rms field
    G_0 = N_0, G_r = rho G_{r-1} + sqrt(1 - rho^2) N_r (N_r the radius-r draw at
    s = 1), planes_r = s_r G_r. Smoothing the same field at neighbouring radii
    correlates its Hessians; this AR(1) chain stands in for that."""
    points = np.arange(n_points, dtype=np.int64)
    crho = math.sqrt(1.0 - rho * rho)
    out = np.empty((len(sigmas), 6, n_points), dtype=dtype)
    G = None
    for r, s in enumerate(sigmas):
        N = hessian_points(seed, realization, r, 1.0, points)
        G = N if G is None else rho * G + crho * N
        out[r] = (float(s) * G).astype(dtype)
    return out


WHITE_SLOT = 0xFFFFFFFF  # stream slot (radius word of the counter) of the white-noise draws


def white_noise(seed: int, realization: int, n_points: int) -> np.ndarray:
    """n_points unit Gaussians: the first Box-Muller draw of each point's stream
    in the white-noise slot (input of the field -> Hessian stage)."""
    u = uniforms(seed, realization, WHITE_SLOT, np.arange(n_points, dtype=np.int64))
    return np.sqrt(-2.0 * np.log(u[0])) * np.cos((2.0 * math.pi) * u[1])

