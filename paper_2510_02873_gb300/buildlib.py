"""Build libcollapse.so in-tree for sm_103a (GB300) with nvcc.

Each translation unit is compiled in parallel, then linked against the shared
CUDA runtime so that the library and PyTorch use one runtime instance.
build(debug=True) makes the checking variant in _build_debug/: every kernel
compiled with -DCC_DEBUG, whose table index checks set bit 2 of
cc_stats.error_flags and clamp the index instead of reading outside a table
(the binding loads it when CC_LIBCOLLAPSE_DEBUG=1).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG_DIR, "csrc")
BUILD_DIR = os.path.join(PKG_DIR, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libcollapse.so")
BUILD_DIR_DEBUG = os.path.join(PKG_DIR, "_build_debug")
LIB_PATH_DEBUG = os.path.join(BUILD_DIR_DEBUG, "libcollapse.so")
INCLUDE = os.path.join(os.path.dirname(PKG_DIR), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit multiply-add contraction in device code. Every FMA
# is written out (fma/fmaf), so a device function computes bit-identical
# results in every kernel it is inlined into (the batched kernel reproduces the
# per-realization kernel exactly).
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-fvisibility=hidden",
          f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcollapse")
    return path


def _rpath() -> list[str]:
    """Run-time search path for the toolkit's libraries (cuFFT) next to the nvcc used to build."""
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    dirs = [d for d in (os.path.join(root, "lib64"), os.path.join(root, "targets", "sbsa-linux", "lib"),
                        os.path.join(root, "targets", "x86_64-linux", "lib")) if os.path.isdir(d)]
    return [f"-Xlinker=-rpath,{d}" for d in dirs]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "collapse.h")]


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_PATH_DEBUG if debug else LIB_PATH
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, extra: list[str], build_dir: str = BUILD_DIR) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr}")
    if res.stderr.strip():
        sys.stderr.write(res.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, debug: bool = False) -> str:
    """Compile every .cu/.cpp under csrc/ and link libcollapse.so (the
    checking variant with debug=True)."""
    lib_path, build_dir = (LIB_PATH_DEBUG, BUILD_DIR_DEBUG) if debug else (LIB_PATH, BUILD_DIR)
    if not force and up_to_date(debug):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DCC_DEBUG"] if debug else [])
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", *objs, "-lcufft", *_rpath(), "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
