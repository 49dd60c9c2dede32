"""Device-side Hessian generation (libhessgen.so) for workloads too large to draw on the host.

Same definition as hessgen.hessian_points; used for inputs only.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

from . import C1, C2

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libhessgen.so")
SRC = os.path.join(HERE, "hessgen.cu")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-cudart", "shared", SRC, "-o", tmp]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                build()
            L = ctypes.CDLL(LIB_PATH)
            L.hg_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
            L.hg_fill.restype = ctypes.c_int
            L.hg_fill_correlated.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            L.hg_fill_correlated.restype = ctypes.c_int
            L.hg_white.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p]
            L.hg_white.restype = ctypes.c_int
            _lib = L
    return _lib


def fill(planes, seed: int, realization: int, radius: int, s: float, point_offset: int = 0,
         stream=None) -> None:
    """Fill a CUDA tensor (6, n) (float64 or float32, unit inner stride) in place."""
    import torch
    assert planes.is_cuda and planes.dim() == 2 and planes.shape[0] == 6 and planes.stride(1) == 1
    dtype = 8 if planes.dtype == torch.float64 else 4 if planes.dtype == torch.float32 else None
    if dtype is None:
        raise TypeError("planes must be float64 or float32")
    st = torch.cuda.current_stream() if stream is None else stream
    rc = _load().hg_fill(seed, realization, radius, float(s), C1, C2, planes.shape[1], point_offset,
                         planes.data_ptr(), planes.stride(0), dtype, ctypes.c_void_p(st.cuda_stream))
    if rc:
        raise RuntimeError(f"hg_fill failed with status {rc}")


def fill_correlated(planes, state, seed: int, realization: int, radius: int, s: float, rho: float,
                    first: bool, stream=None) -> None:
    """Correlated-radius fill (same definition as hessgen.hessian_stack_correlated):
    state is a CUDA float64 (6, n) tensor carried from radius to radius."""
    import math

    import torch
    assert planes.is_cuda and planes.dim() == 2 and planes.shape[0] == 6 and planes.stride(1) == 1
    assert state.is_cuda and state.dtype == torch.float64 and state.is_contiguous()
    assert state.shape == (6, planes.shape[1])
    dtype = 8 if planes.dtype == torch.float64 else 4 if planes.dtype == torch.float32 else None
    if dtype is None:
        raise TypeError("planes must be float64 or float32")
    st = torch.cuda.current_stream() if stream is None else stream
    rc = _load().hg_fill_correlated(seed, realization, radius, float(s), C1, C2, float(rho),
                                    math.sqrt(1.0 - rho * rho), planes.shape[1], planes.data_ptr(),
                                    planes.stride(0), dtype, state.data_ptr(), int(bool(first)),
                                    ctypes.c_void_p(st.cuda_stream))
    if rc:
        raise RuntimeError(f"hg_fill_correlated failed with status {rc}")


def white(out, seed: int, realization: int, stream=None) -> None:
    """Fill a contiguous float64 CUDA tensor with unit white noise (hessgen.white_noise)."""
    import torch

    from . import WHITE_SLOT
    assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
    st = torch.cuda.current_stream() if stream is None else stream
    rc = _load().hg_white(seed, realization, WHITE_SLOT, out.numel(), out.data_ptr(), ctypes.c_void_p(st.cuda_stream))
    if rc:
        raise RuntimeError(f"hg_white failed with status {rc}")

