"""Python access to the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE. The oracle is the slow, plain statement of the
collapse-time computation of arXiv:2510.02873 (Sec. 3 and Sec. 4.1-4.2) that
the CUDA library is checked against. Only tests/, __graft_entry__.smoke() and
the CPU-baseline / reference legs of bench.py may import this package; the
product path never does. It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c")]

FLAG_COLLAPSED = 1
FLAG_EDGE = 4
FLAG_SIGN0 = 8
FLAG_EDS = 16
FLAG_AXIS23 = 32
FLAG_HULL_OUT = 64
FLAG_HULL_EDGE = 128
# flags whose points sit on a discontinuity of F (either branch is a valid answer)
FLAGS_AMBIGUOUS = FLAG_EDGE | FLAG_SIGN0 | FLAG_HULL_EDGE

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, no FMA contraction, OpenMP)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "oracle.h")])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-D_DEFAULT_SOURCE", *SOURCES, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Tables(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("a", ctypes.POINTER(ctypes.c_double)),
                ("D", ctypes.POINTER(ctypes.c_double)), ("M", ctypes.POINTER(ctypes.c_double))]


class _Tab(ctypes.Structure):
    _fields_ = [("nd", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dg", ctypes.POINTER(ctypes.c_double)), ("xg", ctypes.POINTER(ctypes.c_double)),
                ("yg", ctypes.POINTER(ctypes.c_double)), ("val", ctypes.POINTER(ctypes.c_double)),
                ("M", ctypes.POINTER(ctypes.c_double))]


class _RatioTables(ctypes.Structure):
    _fields_ = [("base", _Tables), ("r", ctypes.POINTER(ctypes.c_double) * 3),
                ("Mr", ctypes.POINTER(ctypes.c_double) * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            d, i, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            L.or_growth_table.argtypes = [d, d, i, d, d, vp, vp]
            L.or_growth_at.argtypes = [d, d, d]
            L.or_growth_at.restype = d
            L.or_spline_build.argtypes = [i, vp, vp, d, d, vp]
            L.or_spline_eval.argtypes = [i, vp, vp, vp, d]
            L.or_spline_eval.restype = d
            L.or_bilinear.argtypes = [i, vp, i, vp, vp, d, d]
            L.or_bilinear.restype = d
            L.or_eigen_jacobi.argtypes = [vp, vp]
            L.or_eigen_trig.argtypes = [vp, vp]
            L.or_axis_stretch.argtypes = [vp, i, d]
            L.or_axis_stretch.restype = d
            L.or_axis_coeffs.argtypes = [vp, i, vp]
            L.or_collapse_D.argtypes = [vp, d, ctypes.POINTER(ctypes.c_int)]
            L.or_collapse_D.restype = d
            L.or_tables_init.argtypes = [ctypes.POINTER(_Tables), d, d, i, d, d]
            L.or_tables_free.argtypes = [ctypes.POINTER(_Tables)]
            L.or_a_of_D.argtypes = [ctypes.POINTER(_Tables), d, ctypes.POINTER(ctypes.c_int)]
            L.or_a_of_D.restype = d
            L.or_F_point.argtypes = [ctypes.POINTER(_Tables), vp, ctypes.POINTER(ctypes.c_int)]
            L.or_F_point.restype = d
            L.or_collapse_scale.argtypes = [ctypes.POINTER(_Tables), vp, i64, i64, vp, vp,
                                            ctypes.c_int32, vp, i]
            L.or_collapse_scale_f32.argtypes = L.or_collapse_scale.argtypes
            L.or_F_points.argtypes = [ctypes.POINTER(_Tables), vp, i64, i64, vp, vp, i]
            L.or_cubic_largest_root.argtypes = [d, d, d]
            L.or_cubic_largest_root.restype = d
            L.or_tab_node_value.argtypes = [d, d, d]
            L.or_tab_node_value.restype = d
            L.or_tab_node_values.argtypes = [i, vp, i, vp, i, vp, vp]
            L.or_tab_init.argtypes = [ctypes.POINTER(_Tab), i, vp, i, vp, i, vp, vp]
            L.or_tab_free.argtypes = [ctypes.POINTER(_Tab)]
            L.or_tab_query.argtypes = [ctypes.POINTER(_Tab), d, d, d]
            L.or_tab_query.restype = d
            L.or_tab_query_many.argtypes = [ctypes.POINTER(_Tab), vp, vp, vp, i64, vp, i]
            L.or_spline_eval_many.argtypes = [i, vp, vp, vp, vp, i64, vp, i]
            L.or_mlp_forward.argtypes = [vp, vp]
            L.or_mlp_forward.restype = d
            L.or_mlp_loss_grad.argtypes = [vp, vp, vp, i, vp]
            L.or_mlp_loss_grad.restype = d
            L.or_F_tab_points.argtypes = [ctypes.POINTER(_Tables), ctypes.POINTER(_Tab), vp, i64, i64, vp, vp, i]
            L.or_growth_ratios.argtypes = [d, d, i, d, d, vp, vp, vp, vp, vp]
            L.or_ratio_tables_init.argtypes = [ctypes.POINTER(_RatioTables), d, d, i, d, d]
            L.or_ratio_tables_free.argtypes = [ctypes.POINTER(_RatioTables)]
            L.or_ratios_at.argtypes = [ctypes.POINTER(_RatioTables), d, vp]
            L.or_axis_stretch_exact.argtypes = [ctypes.POINTER(_RatioTables), vp, i, d]
            L.or_axis_stretch_exact.restype = d
            L.or_collapse_D_exact.argtypes = [ctypes.POINTER(_RatioTables), vp, ctypes.POINTER(ctypes.c_int)]
            L.or_collapse_D_exact.restype = d
            L.or_F_points_exact.argtypes = [ctypes.POINTER(_RatioTables), vp, i64, i64, vp, vp, i]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- growth / spline
def growth_table(omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0):
    a = np.empty(n_knots)
    D = np.empty(n_knots)
    rc = lib().or_growth_table(omega_m, omega_l, n_knots, a_min, a_max, _p(a), _p(D))
    if rc:
        raise ValueError(f"or_growth_table failed: {rc}")
    return a, D


def growth_at(a, omega_m=0.3, omega_l=0.7) -> float:
    return lib().or_growth_at(omega_m, omega_l, float(a))


def spline_build(x, y, M0=0.0, Mn=0.0) -> np.ndarray:
    x, y = _f64(x), _f64(y)
    M = np.empty_like(x)
    rc = lib().or_spline_build(len(x), _p(x), _p(y), M0, Mn, _p(M))
    if rc:
        raise ValueError(f"or_spline_build failed: {rc}")
    return M


def spline_eval(x, y, M, t) -> np.ndarray:
    x, y, M = _f64(x), _f64(y), _f64(M)
    L = lib()
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.array([L.or_spline_eval(len(x), _p(x), _p(y), _p(M), float(v)) for v in t])


def spline_eval_many(x, y, M, t, nthreads: int = 0) -> np.ndarray:
    """spline_eval at many points in one call (OpenMP over the points)."""
    x, y, M, t = _f64(x), _f64(y), _f64(M), _f64(np.atleast_1d(t))
    out = np.empty(len(t))
    lib().or_spline_eval_many(len(x), _p(x), _p(y), _p(M), _p(t), len(t), _p(out), nthreads)
    return out


def bilinear(xg, yg, z, x, y) -> np.ndarray:
    xg, yg, z = _f64(xg), _f64(yg), _f64(z)
    assert z.shape == (len(xg), len(yg))
    L = lib()
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    return np.array([L.or_bilinear(len(xg), _p(xg), len(yg), _p(yg), _p(z), float(u), float(v))
                     for u, v in zip(x, y)])


# ---------------------------------------------------------------- eigen / collapse
def eigen_jacobi(h) -> np.ndarray:
    h = _f64(h)
    lam = np.empty(3)
    lib().or_eigen_jacobi(_p(h), _p(lam))
    return lam


def eigen_trig(h) -> np.ndarray:
    h = _f64(h)
    lam = np.empty(3)
    lib().or_eigen_trig(_p(h), _p(lam))
    return lam


def axis_stretch(lam, axis: int, D: float) -> float:
    lam = _f64(lam)
    return lib().or_axis_stretch(_p(lam), axis, float(D))


def axis_coeffs(lam, axis: int) -> np.ndarray:
    lam = _f64(lam)
    c = np.empty(4)
    lib().or_axis_coeffs(_p(lam), axis, _p(c))
    return c


def collapse_D(lam, D_top: float):
    lam = _f64(lam)
    f = ctypes.c_int(0)
    Dc = lib().or_collapse_D(_p(lam), float(D_top), ctypes.byref(f))
    return Dc, f.value


class Tables:
    """Growth table and the natural spline of a(D) (owned by the oracle)."""

    def __init__(self, omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0):
        self._t = _Tables()
        rc = lib().or_tables_init(ctypes.byref(self._t), omega_m, omega_l, n_knots, a_min, a_max)
        if rc:
            raise ValueError(f"or_tables_init failed: {rc}")
        self.n = n_knots
        self.a = np.ctypeslib.as_array(self._t.a, shape=(n_knots,)).copy()
        self.D = np.ctypeslib.as_array(self._t.D, shape=(n_knots,)).copy()
        self.M = np.ctypeslib.as_array(self._t.M, shape=(n_knots,)).copy()

    def __del__(self):
        try:
            lib().or_tables_free(ctypes.byref(self._t))
        except Exception:
            pass

    @property
    def D_top(self) -> float:
        return float(self.D[-1])

    def a_of_D(self, D):
        f = ctypes.c_int(0)
        a = lib().or_a_of_D(ctypes.byref(self._t), float(D), ctypes.byref(f))
        return a, f.value

    def F_point(self, h):
        h = _f64(h)
        f = ctypes.c_int(0)
        F = lib().or_F_point(ctypes.byref(self._t), _p(h), ctypes.byref(f))
        return F, f.value

    def F_points(self, hess: np.ndarray, nthreads: int = 0):
        """hess: (6, n) FP64 planes -> (F, flags)."""
        hess = _f64(hess)
        n = hess.shape[1]
        F = np.empty(n)
        flags = np.empty(n, dtype=np.int32)
        lib().or_F_points(ctypes.byref(self._t), _p(hess), n, n, _p(F), _p(flags), nthreads)
        return F, flags

    def collapse_scale(self, hess: np.ndarray, F_max: np.ndarray, idx: np.ndarray, scale_idx: int,
                       nthreads: int = 0) -> np.ndarray:
        """One radius: hess (6, n) FP64 or FP32 planes; updates F_max/idx in place; returns flags."""
        n = hess.shape[1]
        assert F_max.dtype == np.float64 and idx.dtype == np.int32
        assert F_max.flags.c_contiguous and idx.flags.c_contiguous
        flags = np.empty(n, dtype=np.int32)
        if hess.dtype == np.float32:
            h = np.ascontiguousarray(hess)
            lib().or_collapse_scale_f32(ctypes.byref(self._t), _p(h), n, n, _p(F_max), _p(idx),
                                        scale_idx, _p(flags), nthreads)
        else:
            h = _f64(hess)
            lib().or_collapse_scale(ctypes.byref(self._t), _p(h), n, n, _p(F_max), _p(idx),
                                    scale_idx, _p(flags), nthreads)
        return flags

    def collapse_multi(self, hess_stack: np.ndarray, nthreads: int = 0):
        """All radii of a (R, 6, n) stack -> (F_max, idx, flags_or)."""
        R, _, n = hess_stack.shape
        F_max = np.zeros(n)
        idx = np.full(n, -1, dtype=np.int32)
        flags_or = np.zeros(n, dtype=np.int32)
        for r in range(R):
            flags_or |= self.collapse_scale(hess_stack[r], F_max, idx, r, nthreads)
        return F_max, idx, flags_or


# ---------------------------------------------------------------- tabulated collapse
def cubic_largest_root(b, c, d) -> float:
    return lib().or_cubic_largest_root(float(b), float(c), float(d))


def tab_node_value(delta, x, y) -> float:
    return lib().or_tab_node_value(float(delta), float(x), float(y))


def tab_node_values(dg, xg, yg) -> np.ndarray:
    """u = 1/D_c at every node, layout [ix][iy][k] (flattened like the library's)."""
    dg, xg, yg = _f64(dg), _f64(xg), _f64(yg)
    out = np.empty((len(xg), len(yg), len(dg)))
    lib().or_tab_node_values(len(dg), _p(dg), len(xg), _p(xg), len(yg), _p(yg), _p(out))
    return out


class Tab:
    """Table of u = 1/D_c over (delta, x, y) with natural splines along delta."""

    def __init__(self, dg, xg, yg, val):
        self.dg, self.xg, self.yg = _f64(dg), _f64(xg), _f64(yg)
        val = _f64(val).reshape(len(self.xg), len(self.yg), len(self.dg))
        self.val = val
        self._t = _Tab()
        rc = lib().or_tab_init(ctypes.byref(self._t), len(self.dg), _p(self.dg), len(self.xg), _p(self.xg),
                               len(self.yg), _p(self.yg), _p(np.ascontiguousarray(val)))
        if rc:
            raise ValueError(f"or_tab_init failed: {rc}")

    def __del__(self):
        try:
            lib().or_tab_free(ctypes.byref(self._t))
        except Exception:
            pass

    def query(self, delta, x, y) -> np.ndarray:
        L = lib()
        return np.array([L.or_tab_query(ctypes.byref(self._t), float(a), float(b), float(c))
                         for a, b, c in zip(np.atleast_1d(delta), np.atleast_1d(x), np.atleast_1d(y))])

    def query_many(self, delta, x, y, nthreads: int = 0) -> np.ndarray:
        """query at many points in one call (OpenMP over the points)."""
        d, x, y = _f64(np.atleast_1d(delta)), _f64(np.atleast_1d(x)), _f64(np.atleast_1d(y))
        out = np.empty(len(d))
        lib().or_tab_query_many(ctypes.byref(self._t), _p(d), _p(x), _p(y), len(d), _p(out), nthreads)
        return out

    def F_points(self, tables: "Tables", hess: np.ndarray, nthreads: int = 0):
        hess = _f64(hess)
        n = hess.shape[1]
        F = np.empty(n)
        flags = np.empty(n, dtype=np.int32)
        lib().or_F_tab_points(ctypes.byref(tables._t), ctypes.byref(self._t), _p(hess), n, n, _p(F), _p(flags),
                              nthreads)
        return F, flags


# ---------------------------------------------------------------- MLP surrogate reference
MLP_H = 64
MLP_NPARAM = 3 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def mlp_forward(params, z) -> np.ndarray:
    params = _f64(params)
    z = np.atleast_2d(_f64(z))
    L = lib()
    return np.array([L.or_mlp_forward(_p(params), _p(np.ascontiguousarray(row))) for row in z])


def mlp_loss_grad(params, z, t):
    params, z, t = _f64(params), np.ascontiguousarray(_f64(z).reshape(-1, 3)), _f64(t)
    grad = np.empty(MLP_NPARAM)
    loss = lib().or_mlp_loss_grad(_p(params), _p(z), _p(t), len(t), _p(grad))
    return loss, grad


def histogram(F, edges) -> np.ndarray:
    """Counts of F per bin (Sec. 5.5: collapsed points per redshift bin, F = 1 + z_c).

    counts[0] = #{F < e_0} (every non-collapsed point, F = 0, among them),
    counts[1 + k] = #{e_k <= F < e_(k+1)}, counts[nb + 1] = #{F >= e_nb}:
    the slot of a value is the number of edges at or below it."""
    F = np.asarray(F, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.float64)
    slot = np.searchsorted(edges, F, side="right")
    return np.bincount(slot, minlength=len(edges) + 1).astype(np.int64)


# ---------------------------------------------------------------------------
# Field -> smoothed Hessian (the FFT stage ahead of the collapse computation,
# Sec. 3: the second derivatives of the potential that PINOCCHIO's FFTs
# produce). Plain numpy FFTs in FP64.
#
# Conventions (one reading, the paper prints none): an N^3 periodic grid of
# side `box`, cells in C order (x slowest, z fastest), wavenumbers
# k = 2 pi m / box with m the signed DFT frequency; a dimensionless power
# spectrum P(k) = A k^n exp(-(k / k_cut)^2) applied to unit white noise,
# delta_k = DFT(w) sqrt(P(k)), so that var(delta) = mean over the k grid of P;
# Nyquist modes (any |m| = N/2) and k = 0 set to zero; Gaussian smoothing
# G(kR) = exp(-k^2 R^2 / 2); the Hessian of the potential phi with
# laplacian(phi) = delta: H_ij(k) = (k_i k_j / k^2) delta_k G(kR), whose trace
# is the smoothed density.
HESSIAN_COMPONENTS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _kgrid(N: int, box: float):
    m = np.fft.fftfreq(N, 1.0 / N)
    mz = np.arange(N // 2 + 1, dtype=np.float64)
    two_pi = 2.0 * np.pi / box
    kx = (two_pi * m)[:, None, None]
    ky = (two_pi * m)[None, :, None]
    kz = (two_pi * mz)[None, None, :]
    nyq = (np.abs(m)[:, None, None] == N // 2) | (np.abs(m)[None, :, None] == N // 2) | (mz[None, None, :] == N // 2)
    return kx, ky, kz, nyq


def spectrum(k, amplitude: float, index: float, k_cut: float):
    """P(k) = A k^n exp(-(k/k_cut)^2), P(0) = 0."""
    k = np.asarray(k, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = amplitude * np.power(k, index) * np.exp(-(k / k_cut) ** 2)
    return np.where(k > 0, p, 0.0)


def field_delta_k(white, box: float, amplitude: float, index: float, k_cut: float):
    """delta_k = DFT(w) sqrt(P(k)) on the half-complex grid, Nyquist and k = 0 zeroed."""
    white = np.asarray(white, dtype=np.float64)
    N = white.shape[0]
    kx, ky, kz, nyq = _kgrid(N, box)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    dk = np.fft.rfftn(white) * np.sqrt(spectrum(k, amplitude, index, k_cut))
    dk[np.broadcast_to(nyq, dk.shape)] = 0.0
    return dk


def hessian_from_delta_k(dk, N: int, box: float, R: float):
    """(6, N^3) planes H_ij(x) = IDFT[(k_i k_j / k^2) G(kR) delta_k] in component order xx yy zz xy xz yz."""
    kx, ky, kz, _ = _kgrid(N, box)
    kv = (kx, ky, kz)
    k2 = kx * kx + ky * ky + kz * kz
    g = np.exp(-0.5 * k2 * R * R)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    out = np.empty((6, N ** 3))
    for c, (i, j) in enumerate(HESSIAN_COMPONENTS):
        out[c] = np.fft.irfftn(dk * (kv[i] * kv[j] * inv * g), s=(N, N, N), axes=(0, 1, 2)).reshape(-1)
    return out


def field_sigma(N: int, box: float, amplitude: float, index: float, k_cut: float, R: float) -> float:
    """rms of the smoothed density: sqrt(mean over the full k grid of P G^2), Nyquist and k = 0 excluded."""
    m = np.fft.fftfreq(N, 1.0 / N)
    two_pi = 2.0 * np.pi / box
    kx, ky, kz = np.meshgrid(two_pi * m, two_pi * m, two_pi * m, indexing="ij")
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    keep = np.all(np.abs(np.stack(np.meshgrid(m, m, m, indexing="ij"))) != N // 2, axis=0)
    p = spectrum(k, amplitude, index, k_cut) * np.exp(-(k * R) ** 2)
    return float(np.sqrt(np.sum(np.where(keep, p, 0.0)) / N ** 3))


# ---------------------------------------------------------------- exact-background growth ratios
EDS_RATIOS = (-3.0 / 7.0, -1.0 / 3.0, 10.0 / 21.0)


def growth_ratios(omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0):
    """(a_k, D_k, r2_k, r3a_k, r3b_k): second- and third-order growth ratios at the knots."""
    out = [np.empty(n_knots) for _ in range(5)]
    rc = lib().or_growth_ratios(omega_m, omega_l, n_knots, a_min, a_max, *[_p(x) for x in out])
    if rc:
        raise ValueError(f"or_growth_ratios failed: {rc}")
    return tuple(out)


class RatioTables:
    """Tables of the classic path plus natural splines of r2, r3a, r3b in D."""

    def __init__(self, omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0):
        self._t = _RatioTables()
        rc = lib().or_ratio_tables_init(ctypes.byref(self._t), omega_m, omega_l, n_knots, a_min, a_max)
        if rc:
            raise ValueError(f"or_ratio_tables_init failed: {rc}")
        self.n = n_knots

    def __del__(self):
        try:
            lib().or_ratio_tables_free(ctypes.byref(self._t))
        except Exception:
            pass

    @property
    def D_top(self) -> float:
        return self._t.base.D[self.n - 1]

    def ratios_at(self, D) -> np.ndarray:
        r = np.empty(3)
        lib().or_ratios_at(ctypes.byref(self._t), float(D), _p(r))
        return r

    def axis_stretch(self, lam, axis: int, D: float) -> float:
        lam = _f64(lam)
        return lib().or_axis_stretch_exact(ctypes.byref(self._t), _p(lam), axis, float(D))

    def collapse_D(self, lam):
        lam = _f64(lam)
        f = ctypes.c_int(0)
        Dc = lib().or_collapse_D_exact(ctypes.byref(self._t), _p(lam), ctypes.byref(f))
        return Dc, f.value

    def F_points(self, hess: np.ndarray, nthreads: int = 0):
        """hess: (6, n) planes (FP64 or FP32, widened exactly). Returns (F, flags)."""
        hess = np.ascontiguousarray(hess, dtype=np.float64)
        n = hess.shape[1]
        F = np.empty(n)
        fl = np.zeros(n, dtype=np.int32)
        lib().or_F_points_exact(ctypes.byref(self._t), _p(hess), n, n, _p(F), _p(fl), nthreads)
        return F, fl

