"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
binding, run the oracle on the same inputs, compare element by element."""
from __future__ import annotations

import numpy as np

import oracle

REL_TOL_FP64 = 1e-10     # FP64 path vs oracle, relative on F
TIE_TOL = 1e-9           # two radii whose F differ by less than this (relative) are a tie


def oracle_per_radius(tables: "oracle.Tables", stack: np.ndarray):
    """(R, 6, n) planes -> per-radius F (R, n) and flags (R, n) from the oracle."""
    R = stack.shape[0]
    Fs, fl = [], []
    for r in range(R):
        h = stack[r].astype(np.float64) if stack.dtype != np.float64 else stack[r]
        F, flags = tables.F_points(h)
        Fs.append(F)
        fl.append(flags)
    return np.stack(Fs), np.stack(fl)


def running_max(F_all: np.ndarray, scale_idx0: int = 0):
    """Strict '>' running maximum over radii, F_max from 0 and idx from -1."""
    R, n = F_all.shape
    F_max = np.zeros(n)
    idx = np.full(n, -1, dtype=np.int32)
    for r in range(R):
        better = F_all[r] > F_max
        F_max[better] = F_all[r][better]
        idx[better] = scale_idx0 + r
    return F_max, idx


def rel_err(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    err = np.abs(got - ref)
    nz = ref != 0
    err[nz] /= np.abs(ref[nz])
    return err


def compare_max(F_gpu, idx_gpu, F_all, flags_all, tol=REL_TOL_FP64, scale_idx0: int = 0):
    """Element-by-element check of F_max/idx against the oracle's per-radius values.

    Points where some radius sits on a discontinuity of F (flagged by the
    oracle) are checked only for a valid value; ties between radii only for
    the F value. Returns a summary dict."""
    F_ref, idx_ref = running_max(F_all, scale_idx0)
    amb = (flags_all & oracle.FLAGS_AMBIGUOUS).any(axis=0)
    srt = np.sort(F_all, axis=0)
    tie = np.zeros_like(amb)
    if F_all.shape[0] > 1:
        top, second = srt[-1], srt[-2]
        tie = (top > 0) & (top - second <= TIE_TOL * top)
    ok = ~amb
    err = rel_err(F_gpu, F_ref)
    worst = float(err[ok].max()) if ok.any() else 0.0
    assert worst <= tol, f"max relative F error {worst:.3e} > {tol:.1e}"
    idx_ok = ok & ~tie
    mism = int((idx_gpu[idx_ok] != idx_ref[idx_ok]).sum())
    assert mism == 0, f"{mism} argmax mismatches outside ties"
    # ambiguous points (a radius on the lambda1 = 0 or D_c = D_top edge) may take
    # either side of the discontinuity; they are counted and must stay valid
    assert np.all(np.isfinite(F_gpu)) and np.all(F_gpu >= 0)
    assert np.all((F_gpu == 0) == (idx_gpu == -1))
    return {"max_rel_err": worst, "ambiguous": int(amb.sum()), "ties": int(tie.sum()),
            "rms_rel_err": float(np.sqrt(np.mean(err[ok] ** 2))) if ok.any() else 0.0}


REL_TOL_REDUCED = 3e-5   # mixed and surrogate paths vs oracle, relative on F


def compare_reduced(F, idx, F_all, flags_all, tol=REL_TOL_REDUCED):
    """compare_max for the reduced-precision paths: points whose best radius
    lies within the tolerance of the a_max edge (F ~ 1) may take either side
    of it and are only checked for a valid value, as are radii closer than the
    tolerance (ties) for the argmax."""
    F_ref, idx_ref = running_max(F_all)
    amb = (flags_all & oracle.FLAGS_AMBIGUOUS).any(axis=0)
    srt = np.sort(F_all, axis=0)
    tie = np.zeros_like(amb)
    if F_all.shape[0] > 1:
        tie = (srt[-1] > 0) & (srt[-1] - srt[-2] <= 2 * tol * srt[-1])
    edge = ((F_ref > 0) & (F_ref < 1.0 + 4 * tol)) | ((F > 0) & (F < 1.0 + 4 * tol))
    ok = ~amb & ~edge
    err = rel_err(F, F_ref)
    worst = float(err[ok].max()) if ok.any() else 0.0
    assert worst <= tol, f"max relative F error {worst:.3e} > {tol:.1e}"
    mism = int((idx[ok & ~tie] != idx_ref[ok & ~tie]).sum())
    assert mism == 0, f"{mism} argmax mismatches outside ties"
    assert np.all(np.isfinite(F)) and np.all(F >= 0)
    return {"max_rel_err": worst, "rms_rel_err": float(np.sqrt(np.mean(err[ok] ** 2))) if ok.any() else 0.0,
            "ambiguous": int(amb.sum()), "edge": int(edge.sum()), "ties": int(tie.sum())}


def near_pair_corner_planes(n: int, seed: int) -> np.ndarray:
    """(1, 6, n) planes of the spectra hardest for a single FP64 Newton step on
    l1: l1 - l2 just above the deflation threshold (1 + r between 1e-4 and
    ~3e-3), small l1 (0.03 .. 3) against a large negative l3 (gap 1 .. 32),
    where the FP32 rounding of the characteristic cubic's coefficients moves
    the FP32 root most and D_c is most sensitive to l1. Random frames."""
    rng = np.random.default_rng(seed)
    base = 10.0 ** rng.uniform(-1.5, 0.5, n)
    gap = 10.0 ** rng.uniform(0.0, 1.5, n)
    d = 10.0 ** rng.uniform(np.log10(0.012), np.log10(0.06), n) * gap / 3.0
    lam = np.stack([base + d, base, base - gap], axis=1)
    Q = np.linalg.qr(rng.normal(size=(n, 3, 3)))[0]
    M = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    return np.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]])[None]
