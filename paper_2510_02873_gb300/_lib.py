"""ctypes declarations of libcollapse (include/collapse.h). Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

from . import buildlib as _build

CC_OK, CC_EINVAL, CC_ECUDA, CC_ENOMEM, CC_ETIMEOUT, CC_ERANGE, CC_ENOTSUP = range(7)
CC_F64, CC_F32 = 8, 4
MODES = {"fp64": 0, "mixed": 1, "surrogate": 2, "tabulated": 3, "f32x2": 4, "exact_growth": 5}

# every symbol the public header declares
EXPORTS = (
    "cc_create", "cc_destroy", "cc_build_growth_table", "cc_get_growth_table", "cc_reset_max", "cc_collapse_scale",
    "cc_collapse_multi", "cc_collapse_multi_host", "cc_collapse_multi_noalloc", "cc_get_stats", "cc_reset_stats", "cc_strerror",
    "cc_last_error_message", "cc_version", "cc_batch_create", "cc_batch_autotune", "cc_batch_run",
    "cc_batch_run_graph", "cc_batch_get_config", "cc_batch_destroy", "cc_set_table", "cc_table_nodes_rlpt",
    "cc_table_query", "cc_spline_eval", "cc_surrogate_train", "cc_surrogate_params", "cc_load_surrogate",
    "cc_set_surrogate_engine", "cc_surrogate_checkpoint", "cc_surrogate_restore", "cc_surrogate_train_resume",
    "cc_surrogate_eval", "cc_surrogate_grad", "cc_histogram", "cc_field_create", "cc_field_sigma",
    "cc_field_hessian", "cc_field_destroy",
)


class CcCosmology(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("n_knots", ctypes.c_int32), ("a_min", ctypes.c_double), ("a_max", ctypes.c_double)]


class CcStats(ctypes.Structure):
    _fields_ = [("evaluations", ctypes.c_uint64), ("collapsed", ctypes.c_uint64),
                ("eds_branch", ctypes.c_uint64), ("refined", ctypes.c_uint64),
                ("fp64_branch", ctypes.c_uint64), ("fallback", ctypes.c_uint64),
                ("error_flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved"}


class CcSpectrum(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("amplitude", ctypes.c_double), ("index", ctypes.c_double),
                ("k_cut", ctypes.c_double)]


class CcBatchItem(ctypes.Structure):
    _fields_ = [("hess", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64),
                ("plane_stride", ctypes.c_int64), ("radius_stride", ctypes.c_int64), ("R", ctypes.c_int32),
                ("sigma", ctypes.POINTER(ctypes.c_double)), ("F_max", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("scale_idx0", ctypes.c_int32)]


class CcTrainConfig(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("val_fraction", ctypes.c_float)]


class CcTrainReport(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_int64), ("train_samples", ctypes.c_int64), ("val_samples", ctypes.c_int64),
                ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float), ("val_rms", ctypes.c_float),
                ("val_max", ctypes.c_float), ("hull_lo", ctypes.c_float * 3), ("hull_hi", ctypes.c_float * 3)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("hull")}
        d["hull_lo"] = list(self.hull_lo)
        d["hull_hi"] = list(self.hull_hi)
        return d


class CollapseError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str):
        super().__init__(f"{what} failed: {detail or 'status ' + str(code)} (code {code})")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    """The release library, or with CC_LIBCOLLAPSE_DEBUG=1 in the environment
    the checking variant (build(debug=True): table index checks that set bit 2
    of cc_stats.error_flags)."""
    return _build.LIB_PATH_DEBUG if os.environ.get("CC_LIBCOLLAPSE_DEBUG") == "1" else _build.LIB_PATH


def load() -> ctypes.CDLL:
    """Load the in-tree libcollapse.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"libcollapse.so not found at {path}: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
        L = ctypes.CDLL(path)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.cc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(CcCosmology), ctypes.c_int]
        L.cc_create.restype = ctypes.c_int
        L.cc_destroy.argtypes = [vp]
        L.cc_destroy.restype = None
        L.cc_build_growth_table.argtypes = [ctypes.POINTER(CcCosmology), vp, vp]
        L.cc_get_growth_table.argtypes = [vp, vp, vp, i32]
        L.cc_reset_max.argtypes = [vp, vp, vp, i64, vp]
        L.cc_collapse_scale.argtypes = [vp, ctypes.c_int, vp, i32, i64, i64, d, vp, vp, i32, vp]
        L.cc_collapse_multi.argtypes = [vp, ctypes.c_int, vp, i32, i64, i64, i64,
                                        ctypes.POINTER(d), i32, vp, vp, i32, vp]
        L.cc_collapse_multi_host.argtypes = L.cc_collapse_multi.argtypes
        L.cc_collapse_multi_noalloc.argtypes = [ctypes.POINTER(CcCosmology), ctypes.c_int, vp, i32, i64, i64, i64,
                                                ctypes.POINTER(d), i32, vp, vp, i32, ctypes.POINTER(CcStats), vp]
        L.cc_get_stats.argtypes = [vp, ctypes.POINTER(CcStats), vp]
        L.cc_batch_create.argtypes = [vp, ctypes.c_int, ctypes.POINTER(CcBatchItem), i32, ctypes.POINTER(vp)]
        L.cc_batch_autotune.argtypes = [vp, ctypes.c_char_p, vp]
        L.cc_batch_run.argtypes = [vp, vp]
        L.cc_batch_run_graph.argtypes = [vp, vp]
        L.cc_batch_get_config.argtypes = [vp, ctypes.POINTER(i32), vp, i32]
        L.cc_batch_destroy.argtypes = [vp]
        L.cc_batch_destroy.restype = None
        L.cc_set_table.argtypes = [vp, vp, i32, vp, i32, vp, i32, vp, vp]
        L.cc_table_nodes_rlpt.argtypes = [vp, vp, i32, vp, i32, vp, i32, vp, vp]
        L.cc_table_query.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.cc_spline_eval.argtypes = [vp, vp, vp, i32, vp, i64, vp, vp]
        L.cc_histogram.argtypes = [vp, vp, i64, vp, i32, vp, vp]
        L.cc_field_create.argtypes = [vp, vp, i32, ctypes.POINTER(CcSpectrum), ctypes.POINTER(vp), vp]
        L.cc_field_sigma.argtypes = [vp, d, ctypes.POINTER(d), vp]
        L.cc_field_hessian.argtypes = [vp, d, vp, i32, i64, vp]
        L.cc_field_destroy.argtypes = [vp]
        L.cc_field_destroy.restype = None
        L.cc_surrogate_train.argtypes = [vp, vp, i32, i64, i64, d, ctypes.POINTER(CcTrainConfig),
                                         ctypes.POINTER(CcTrainReport), vp]
        L.cc_surrogate_params.argtypes = [vp, vp, vp]
        L.cc_load_surrogate.argtypes = [vp, vp, vp]
        L.cc_surrogate_checkpoint.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.cc_surrogate_restore.argtypes = [vp, vp, ctypes.c_size_t]
        L.cc_surrogate_train_resume.argtypes = [vp, vp, i32, i64, i64, d, i32, i32, ctypes.POINTER(CcTrainReport), vp]
        L.cc_set_surrogate_engine.argtypes = [vp, i32]
        L.cc_surrogate_eval.argtypes = [vp, vp, i64, vp, vp]
        L.cc_surrogate_grad.argtypes = [vp, vp, vp, i32, vp, vp]
        L.cc_reset_stats.argtypes = [vp, vp]
        L.cc_strerror.argtypes = [ctypes.c_int]
        L.cc_strerror.restype = ctypes.c_char_p
        L.cc_last_error_message.argtypes = []
        L.cc_last_error_message.restype = ctypes.c_char_p
        L.cc_version.argtypes = []
        for name in ("cc_build_growth_table", "cc_get_growth_table", "cc_reset_max", "cc_collapse_scale",
                     "cc_collapse_multi", "cc_collapse_multi_host", "cc_collapse_multi_noalloc",
                     "cc_get_stats", "cc_reset_stats", "cc_version", "cc_batch_create", "cc_batch_autotune",
                     "cc_batch_run", "cc_batch_run_graph", "cc_batch_get_config", "cc_set_table",
                     "cc_table_nodes_rlpt", "cc_table_query", "cc_spline_eval", "cc_surrogate_train",
                     "cc_surrogate_params", "cc_load_surrogate", "cc_surrogate_eval", "cc_surrogate_grad",
                     "cc_set_surrogate_engine", "cc_surrogate_checkpoint", "cc_surrogate_restore",
                     "cc_surrogate_train_resume", "cc_histogram", "cc_field_create", "cc_field_sigma", "cc_field_hessian"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def check(code: int, what: str) -> None:
    if code != CC_OK:
        detail = load().cc_last_error_message().decode(errors="replace")
        raise CollapseError(code, what, detail)
