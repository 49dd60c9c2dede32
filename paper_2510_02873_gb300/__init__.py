"""GB300-native collapse-time library (arXiv:2510.02873 hot path) -- Python binding.

The names mirror the C-ABI of include/collapse.h (cc_create, cc_collapse_scale,
...); every step of the computation runs in libcollapse's CUDA kernels. This
module only marshals torch tensors (device memory) and CUDA streams into the
C calls. There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import CC_F32, CC_F64, MODES, CcCosmology, CcStats, CollapseError  # noqa: F401

__all__ = [
    "Context", "cc_create", "cc_destroy", "cc_reset_max", "cc_collapse_scale", "cc_collapse_multi",
    "cc_collapse_multi_host", "Batch",
    "cc_get_stats", "cc_reset_stats", "cc_get_growth_table", "cc_build_growth_table", "cc_version", "CollapseError", "build",
]


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return CC_F64
    if t.dtype == torch.float32:
        return CC_F32
    raise TypeError(f"Hessian planes must be float64 or float32, got {t.dtype}")


def _check_outputs(F_max, idx, n: int):
    import torch
    if F_max.dtype != torch.float64 or idx.dtype != torch.int32:
        raise TypeError("F_max must be float64 and idx int32")
    if F_max.numel() < n or idx.numel() < n or not F_max.is_contiguous() or not idx.is_contiguous():
        raise ValueError("F_max/idx must be contiguous with at least n elements")
    if not (F_max.is_cuda and idx.is_cuda):
        raise ValueError("F_max/idx must be CUDA tensors")


# ------------------------------------------------------------------ C-ABI mirrors
def cc_create(omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0, device=0) -> ctypes.c_void_p:
    L = _lib.load()
    h = ctypes.c_void_p()
    cosmo = CcCosmology(omega_m, omega_l, n_knots, a_min, a_max)
    _lib.check(L.cc_create(ctypes.byref(h), ctypes.byref(cosmo), device), "cc_create")
    return h


def cc_destroy(ctx) -> None:
    _lib.load().cc_destroy(ctx)


def cc_build_growth_table(omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0):
    """Host-only: the library's FP64 growth table (a_k, D_k)."""
    a = np.empty(n_knots)
    D = np.empty(n_knots)
    cosmo = CcCosmology(omega_m, omega_l, n_knots, a_min, a_max)
    _lib.check(_lib.load().cc_build_growth_table(ctypes.byref(cosmo), a.ctypes.data, D.ctypes.data),
               "cc_build_growth_table")
    return a, D


def cc_get_growth_table(ctx, n_knots: int):
    a = np.empty(n_knots)
    D = np.empty(n_knots)
    _lib.check(_lib.load().cc_get_growth_table(ctx, a.ctypes.data, D.ctypes.data, n_knots),
               "cc_get_growth_table")
    return a, D


def cc_reset_max(ctx, F_max, idx, n=None, stream=None) -> None:
    n = F_max.numel() if n is None else n
    _check_outputs(F_max, idx, n)
    _lib.check(_lib.load().cc_reset_max(ctx, F_max.data_ptr(), idx.data_ptr(), n, _stream_ptr(stream)),
               "cc_reset_max")


def cc_collapse_scale(ctx, mode, hess, sigma_R: float, F_max, idx, scale_idx: int, stream=None) -> None:
    """hess: CUDA tensor (6, n) (any plane stride with unit inner stride)."""
    if hess.dim() != 2 or hess.shape[0] != 6 or hess.stride(1) != 1:
        raise ValueError("hess must be a (6, n) tensor with unit stride along points")
    if not hess.is_cuda:
        raise ValueError("hess must be a CUDA tensor")
    n = hess.shape[1]
    _check_outputs(F_max, idx, n)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _lib.check(_lib.load().cc_collapse_scale(ctx, m, hess.data_ptr(), _dtype_code(hess), n, hess.stride(0),
                                             float(sigma_R), F_max.data_ptr(), idx.data_ptr(),
                                             int(scale_idx), _stream_ptr(stream)), "cc_collapse_scale")


def cc_collapse_multi(ctx, mode, hess, sigma, F_max, idx, scale_idx0: int = 0, stream=None) -> None:
    """hess: CUDA tensor (R, 6, n) with unit stride along points."""
    if hess.dim() != 3 or hess.shape[1] != 6 or hess.stride(2) != 1:
        raise ValueError("hess must be a (R, 6, n) tensor with unit stride along points")
    if not hess.is_cuda:
        raise ValueError("hess must be a CUDA tensor")
    R, _, n = hess.shape
    sig = (ctypes.c_double * R)(*[float(s) for s in sigma])
    if len(sigma) != R:
        raise ValueError("len(sigma) must equal the number of radii")
    _check_outputs(F_max, idx, n)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _lib.check(_lib.load().cc_collapse_multi(ctx, m, hess.data_ptr(), _dtype_code(hess), n, hess.stride(1),
                                             hess.stride(0), sig, R, F_max.data_ptr(), idx.data_ptr(),
                                             int(scale_idx0), _stream_ptr(stream)), "cc_collapse_multi")


def cc_collapse_multi_host(ctx, mode, hess, sigma, F_max, idx, scale_idx0: int = 0, stream=None) -> None:
    """Host-resident planes and outputs: hess (R, 6, n) CPU tensor or ndarray
    (page-locked for copy/compute overlap), F_max float64 (n,), idx int32 (n,)
    on the host, updated in place. Blocks until the outputs are written."""
    import torch
    to_t = (lambda x: torch.from_numpy(x) if isinstance(x, np.ndarray) else x)
    hess, F_max, idx = to_t(hess), to_t(F_max), to_t(idx)
    if hess.is_cuda or F_max.is_cuda or idx.is_cuda:
        raise ValueError("cc_collapse_multi_host takes host tensors")
    if hess.dim() != 3 or hess.shape[1] != 6 or hess.stride(2) != 1:
        raise ValueError("hess must be a (R, 6, n) tensor with unit stride along points")
    R, _, n = hess.shape
    if len(sigma) != R:
        raise ValueError("len(sigma) must equal the number of radii")
    if F_max.dtype != torch.float64 or idx.dtype != torch.int32 or F_max.numel() < n or idx.numel() < n:
        raise ValueError("F_max must be float64 and idx int32 with at least n elements")
    sig = (ctypes.c_double * R)(*[float(s) for s in sigma])
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _lib.check(_lib.load().cc_collapse_multi_host(ctx, m, hess.data_ptr(), _dtype_code(hess), n, hess.stride(1),
                                                  hess.stride(0), sig, R, F_max.data_ptr(), idx.data_ptr(),
                                                  int(scale_idx0), _stream_ptr(stream)), "cc_collapse_multi_host")


def cc_get_stats(ctx, stream=None) -> dict:
    st = CcStats()
    _lib.check(_lib.load().cc_get_stats(ctx, ctypes.byref(st), _stream_ptr(stream)), "cc_get_stats")
    return st.as_dict()


def cc_reset_stats(ctx, stream=None) -> None:
    _lib.check(_lib.load().cc_reset_stats(ctx, _stream_ptr(stream)), "cc_reset_stats")


def cc_version() -> int:
    return _lib.load().cc_version()


class Batch:
    """A plan for many realizations in one persistent launch (cc_batch_*).

    items: list of (hess (R, 6, n) CUDA tensor, sigma (R,), F_max (n,) float64
    CUDA tensor, idx (n,) int32 CUDA tensor[, scale_idx0]). The tensors must
    outlive the plan."""

    def __init__(self, ctx: "Context", items, mode="mixed"):
        L = _lib.load()
        self._keep = []
        arr = (_lib.CcBatchItem * len(items))()
        for k, it in enumerate(items):
            hess, sigma, F_max, idx = it[:4]
            scale0 = it[4] if len(it) > 4 else 0
            if hess.dim() != 3 or hess.shape[1] != 6 or hess.stride(2) != 1 or not hess.is_cuda:
                raise ValueError("hess must be a CUDA (R, 6, n) tensor with unit stride along points")
            R, _, n = hess.shape
            _check_outputs(F_max, idx, n)
            sig = (ctypes.c_double * R)(*[float(s) for s in sigma])
            self._keep.append(sig)
            arr[k] = _lib.CcBatchItem(hess.data_ptr(), _dtype_code(hess), n, hess.stride(1), hess.stride(0), R,
                                      ctypes.cast(sig, ctypes.POINTER(ctypes.c_double)), F_max.data_ptr(),
                                      idx.data_ptr(), int(scale0))
        self._h = ctypes.c_void_p()
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        _lib.check(L.cc_batch_create(ctx.handle, m, arr, len(items), ctypes.byref(self._h)), "cc_batch_create")
        self.nitems = len(items)

    def autotune(self, cache_path=None, stream=None):
        """Time candidate block sizes and tiles per grid size on these
        realizations and keep the fastest (cc_batch_autotune); with a cache
        file, reuse or record the choice. Overwrites the outputs."""
        path = cache_path.encode() if cache_path else None
        _lib.check(_lib.load().cc_batch_autotune(self._h, path, _stream_ptr(stream)), "cc_batch_autotune")

    def run(self, stream=None):
        """One persistent launch over every realization (cc_batch_run)."""
        _lib.check(_lib.load().cc_batch_run(self._h, _stream_ptr(stream)), "cc_batch_run")

    def run_graph(self, stream=None):
        """The same launch from a CUDA graph, captured on first use and
        replayed afterwards (cc_batch_run_graph)."""
        _lib.check(_lib.load().cc_batch_run_graph(self._h, _stream_ptr(stream)), "cc_batch_run_graph")

    def config(self):
        """(threads per block, [tile points per realization]) in use."""
        blk = ctypes.c_int32()
        tiles = (ctypes.c_int32 * self.nitems)()
        _lib.check(_lib.load().cc_batch_get_config(self._h, ctypes.byref(blk), tiles, self.nitems),
                   "cc_batch_get_config")
        return int(blk.value), list(tiles)

    def close(self):
        """Free the plan (cc_batch_destroy); the caller's tensors are untouched."""
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().cc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ convenience
class Context:
    """Owns one cc_ctx (tables on the device) for the given cosmology."""

    def __init__(self, omega_m=0.3, omega_l=0.7, n_knots=512, a_min=1e-3, a_max=1.0, device=0):
        """Flat LCDM (omega_m + omega_l = 1 not required), growth table of
        n_knots knots log-spaced in a over [a_min, a_max], on CUDA device
        `device` (cc_create)."""
        self.n_knots = n_knots
        self.device = device
        self._h = cc_create(omega_m, omega_l, n_knots, a_min, a_max, device)

    def close(self):
        """Release the device tables and scratch (cc_destroy)."""
        if getattr(self, "_h", None) is not None and self._h.value:
            cc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def growth_table(self):
        """(a_k, D_k) of the growth table, host arrays (cc_get_growth_table)."""
        return cc_get_growth_table(self._h, self.n_knots)

    def reset_max(self, F_max, idx, stream=None):
        """F_max = 0 and idx = -1 on the device (cc_reset_max)."""
        cc_reset_max(self._h, F_max, idx, None, stream)

    def collapse_scale(self, hess, sigma_R, F_max, idx, scale_idx, mode="fp64", stream=None):
        """One radius: hess (6, n) CUDA planes (float64 or float32), sigma_R
        its rms; F_max/idx updated where F > F_max (cc_collapse_scale)."""
        cc_collapse_scale(self._h, mode, hess, sigma_R, F_max, idx, scale_idx, stream)

    def collapse_multi(self, hess, sigma, F_max, idx, scale_idx0=0, mode="fp64", stream=None):
        """All radii in one fused launch: hess (R, 6, n) CUDA planes, sigma
        (R,); the running maximum stays in registers (cc_collapse_multi)."""
        cc_collapse_multi(self._h, mode, hess, sigma, F_max, idx, scale_idx0, stream)

    def collapse_multi_host(self, hess, sigma, F_max, idx, scale_idx0=0, mode="fp64", stream=None):
        """The same from pinned host planes and host F_max/idx: the copies
        of radius r + 1 overlap the launch of radius r; synchronises
        (cc_collapse_multi_host)."""
        cc_collapse_multi_host(self._h, mode, hess, sigma, F_max, idx, scale_idx0, stream)

    # ---- tabulated collapse and interpolation routines
    def set_table(self, dgrid, xgrid, ygrid, values, stream=None):
        """values: (nx, ny, nd) array of u = 1/D_c at the nodes (host)."""
        dg, xg, yg = (np.ascontiguousarray(a, dtype=np.float64) for a in (dgrid, xgrid, ygrid))
        v = np.ascontiguousarray(values, dtype=np.float64).reshape(len(xg), len(yg), len(dg))
        _lib.check(_lib.load().cc_set_table(self._h, dg.ctypes.data, len(dg), xg.ctypes.data, len(xg),
                                            yg.ctypes.data, len(yg), v.ctypes.data, _stream_ptr(stream)),
                   "cc_set_table")

    def table_nodes_rlpt(self, dgrid, xgrid, ygrid, stream=None) -> np.ndarray:
        """u = 1/D_c by R-LPT at every (x, y, delta) node, computed on the device; (nx, ny, nd) host array."""
        dg, xg, yg = (np.ascontiguousarray(a, dtype=np.float64) for a in (dgrid, xgrid, ygrid))
        out = np.empty((len(xg), len(yg), len(dg)))
        _lib.check(_lib.load().cc_table_nodes_rlpt(self._h, dg.ctypes.data, len(dg), xg.ctypes.data, len(xg),
                                                   yg.ctypes.data, len(yg), out.ctypes.data, _stream_ptr(stream)),
                   "cc_table_nodes_rlpt")
        return out

    def table_query(self, d, x, y, out, stream=None):
        """d, x, y, out: float64 CUDA tensors of equal length."""
        m = d.numel()
        _lib.check(_lib.load().cc_table_query(self._h, d.data_ptr(), x.data_ptr(), y.data_ptr(), m,
                                              out.data_ptr(), _stream_ptr(stream)), "cc_table_query")

    def spline_eval(self, xk, yk, q, out, stream=None):
        """xk, yk: host knots; q, out: float64 CUDA tensors."""
        xk, yk = (np.ascontiguousarray(a, dtype=np.float64) for a in (xk, yk))
        _lib.check(_lib.load().cc_spline_eval(self._h, xk.ctypes.data, yk.ctypes.data, len(xk), q.data_ptr(),
                                              q.numel(), out.data_ptr(), _stream_ptr(stream)), "cc_spline_eval")

    def histogram(self, F_max, edges, counts, stream=None):
        """Counts of F_max per bin (cc_histogram). F_max: float64 CUDA tensor;
        edges: host, nbins + 1 increasing positive values; counts: int64 CUDA
        tensor of nbins + 2 (below, bins..., above), overwritten."""
        import torch
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        if F_max.dtype != torch.float64 or not F_max.is_cuda or not F_max.is_contiguous():
            raise TypeError("F_max must be a contiguous float64 CUDA tensor")
        if counts.dtype != torch.int64 or not counts.is_cuda or counts.numel() != len(edges) + 1:
            raise TypeError("counts must be an int64 CUDA tensor of nbins + 2 entries")
        _lib.check(_lib.load().cc_histogram(self._h, F_max.data_ptr(), F_max.numel(), edges.ctypes.data,
                                            len(edges) - 1, counts.data_ptr(), _stream_ptr(stream)),
                   "cc_histogram")

    # ---- learned surrogate
    MLP_NPARAM = 8641

    def surrogate_train(self, hess, sigma, steps=2000, batch=16384, lr=3e-3, seed=1, val_fraction=0.05,
                        stream=None) -> dict:
        """hess: CUDA tensor (6, n) of training Hessians at rms sigma."""
        if hess.dim() != 2 or hess.shape[0] != 6 or hess.stride(1) != 1 or not hess.is_cuda:
            raise ValueError("hess must be a CUDA (6, n) tensor with unit stride along points")
        cfg = _lib.CcTrainConfig(int(steps), int(batch), float(lr), int(seed), float(val_fraction))
        rep = _lib.CcTrainReport()
        _lib.check(_lib.load().cc_surrogate_train(self._h, hess.data_ptr(), _dtype_code(hess), hess.shape[1],
                                                  hess.stride(0), float(sigma), ctypes.byref(cfg), ctypes.byref(rep),
                                                  _stream_ptr(stream)), "cc_surrogate_train")
        return rep.as_dict()

    def surrogate_train_resume(self, hess, sigma, steps, schedule_steps=0, stream=None) -> dict:
        """Continue training from the context's state (after surrogate_train or
        surrogate_restore) for `steps` Adam steps on samples of hess (CUDA
        (6, n) at rms sigma); schedule_steps: length of the learning-rate
        schedule (0 = the stored one, extended to cover the new steps)."""
        if hess.dim() != 2 or hess.shape[0] != 6 or hess.stride(1) != 1 or not hess.is_cuda:
            raise ValueError("hess must be a CUDA (6, n) tensor with unit stride along points")
        rep = _lib.CcTrainReport()
        _lib.check(_lib.load().cc_surrogate_train_resume(self._h, hess.data_ptr(), _dtype_code(hess), hess.shape[1],
                                                         hess.stride(0), float(sigma), int(steps), int(schedule_steps),
                                                         ctypes.byref(rep), _stream_ptr(stream)),
                   "cc_surrogate_train_resume")
        return rep.as_dict()

    def surrogate_checkpoint(self) -> bytes:
        """The training state as a versioned blob (cc_surrogate_checkpoint)."""
        size = ctypes.c_size_t(0)
        _lib.check(_lib.load().cc_surrogate_checkpoint(self._h, None, ctypes.byref(size)), "cc_surrogate_checkpoint")
        buf = ctypes.create_string_buffer(size.value)
        _lib.check(_lib.load().cc_surrogate_checkpoint(self._h, buf, ctypes.byref(size)), "cc_surrogate_checkpoint")
        return buf.raw[:size.value]

    def surrogate_restore(self, blob: bytes):
        """Install a training state written by surrogate_checkpoint (cc_surrogate_restore)."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _lib.check(_lib.load().cc_surrogate_restore(self._h, buf, len(blob)), "cc_surrogate_restore")

    def surrogate_params(self):
        """The network's FP32 master parameters (8641) and training hull (6), host arrays."""
        params = np.empty(self.MLP_NPARAM, dtype=np.float32)
        hull = np.empty(6, dtype=np.float32)
        _lib.check(_lib.load().cc_surrogate_params(self._h, params.ctypes.data, hull.ctypes.data),
                   "cc_surrogate_params")
        return params, hull

    def load_surrogate(self, params, hull):
        """Install a network from host parameters (8641 floats) and hull (lo[3], hi[3])."""
        params = np.ascontiguousarray(params, dtype=np.float32)
        hull = np.ascontiguousarray(hull, dtype=np.float32)
        if params.size != self.MLP_NPARAM or hull.size != 6:
            raise ValueError("params must have 8641 entries and hull 6")
        _lib.check(_lib.load().cc_load_surrogate(self._h, params.ctypes.data, hull.ctypes.data), "cc_load_surrogate")

    SURROGATE_ENGINES = {"mma_sync": 0, "tcgen05": 1}

    def set_surrogate_engine(self, engine: str):
        """Kernel for mode="surrogate": "tcgen05" (default) or "mma_sync"."""
        if engine not in self.SURROGATE_ENGINES:
            raise ValueError(f"engine must be one of {sorted(self.SURROGATE_ENGINES)}")
        _lib.check(_lib.load().cc_set_surrogate_engine(self._h, self.SURROGATE_ENGINES[engine]),
                   "cc_set_surrogate_engine")

    def surrogate_eval(self, z, out, stream=None):
        """z: float32 CUDA tensor (n, 3); out: float32 CUDA tensor (n,)."""
        _lib.check(_lib.load().cc_surrogate_eval(self._h, z.data_ptr(), z.shape[0], out.data_ptr(),
                                                 _stream_ptr(stream)), "cc_surrogate_eval")

    def surrogate_grad(self, z, t):
        """One minibatch gradient of the training kernel on host samples z (n, 3), t (n,): (loss, grad)."""
        z = np.ascontiguousarray(z, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        grad = np.empty(self.MLP_NPARAM, dtype=np.float32)
        loss = ctypes.c_float()
        _lib.check(_lib.load().cc_surrogate_grad(self._h, z.ctypes.data, t.ctypes.data, len(t), grad.ctypes.data,
                                                 ctypes.byref(loss)), "cc_surrogate_grad")
        return float(loss.value), grad

    def stats(self, stream=None) -> dict:
        """Device counters since the last reset_stats (cc_get_stats; synchronises the stream)."""
        return cc_get_stats(self._h, stream)

    def reset_stats(self, stream=None):
        """Zero the device counters (cc_reset_stats)."""
        cc_reset_stats(self._h, stream)


class Field:
    """A Gaussian field kept on the device, smoothed into Hessian planes by FFT
    (cc_field_*). white: contiguous float64 CUDA tensor of N^3 unit white noise
    (C order over x, y, z); P(k) = amplitude k^index exp(-(k/k_cut)^2) on a box of side `box`."""

    def __init__(self, ctx: "Context", white, box: float, amplitude: float, index: float, k_cut: float, stream=None):
        import torch
        if white.dtype != torch.float64 or not white.is_cuda or not white.is_contiguous():
            raise TypeError("white must be a contiguous float64 CUDA tensor")
        N = round(white.numel() ** (1.0 / 3.0))
        if N ** 3 != white.numel():
            raise ValueError("white must hold N^3 values")
        self.N = N
        self._ctx = ctx  # keeps the context alive
        spec = _lib.CcSpectrum(box, amplitude, index, k_cut)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().cc_field_create(ctx._h, white.data_ptr(), N, ctypes.byref(spec), ctypes.byref(h),
                                               _stream_ptr(stream)), "cc_field_create")
        self._h = h.value

    def sigma(self, R: float, stream=None) -> float:
        """rms of delta smoothed at radius R (Gaussian filter), from the device field."""
        out = ctypes.c_double()
        _lib.check(_lib.load().cc_field_sigma(self._h, float(R), ctypes.byref(out), _stream_ptr(stream)),
                   "cc_field_sigma")
        return out.value

    def hessian(self, R: float, planes, stream=None) -> None:
        """planes: CUDA tensor (6, m >= N^3), float64 or float32, unit inner stride."""
        import torch
        if planes.dim() != 2 or planes.shape[0] != 6 or planes.stride(1) != 1 or not planes.is_cuda:
            raise TypeError("planes must be a (6, m) CUDA tensor with unit inner stride")
        dt = CC_F64 if planes.dtype == torch.float64 else CC_F32 if planes.dtype == torch.float32 else None
        if dt is None:
            raise TypeError("planes must be float64 or float32")
        _lib.check(_lib.load().cc_field_hessian(self._h, float(R), planes.data_ptr(), dt, planes.stride(0),
                                                _stream_ptr(stream)), "cc_field_hessian")

    def close(self) -> None:
        """Release the device field (cc_field_destroy)."""
        if self._h:
            _lib.load().cc_field_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

