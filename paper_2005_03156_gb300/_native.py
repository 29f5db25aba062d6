"""ctypes declarations of libpip.so (include/pip.h). Argument marshalling only:
every step of the join runs in the library's CUDA kernels. Importing this
module fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpip.so")

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U64 = ctypes.c_uint64

STATUS = {0: "PIP_OK", 1: "PIP_EINVAL", 2: "PIP_ENOMEM", 3: "PIP_ECUDA", 4: "PIP_ERANGE",
          5: "PIP_ETIMEOUT", 6: "PIP_EBUSY"}


class PipError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class BuildOpts(ctypes.Structure):
    _fields_ = [("cell_log2", I32), ("max_depth", I32), ("fanout_log2", I32), ("leaf_edges", I32),
                ("size_ratio", I32), ("pts_per_cta", I32), ("stage_depth", I32), ("cand_mode", I32),
                ("approx_units", I32), ("compact_edges", I32),
                ("compact_early", I32), ("bin_residual", I32)]


class SetInfo(ctypes.Structure):
    _fields_ = [("n_poly", I64), ("n_ring", I64), ("n_vert", I64), ("n_levels", I64),
                ("top_cells", I64), ("table_entries", I64), ("leaves", I64),
                ("interior_cells", I64), ("empty_cells", I64), ("superbins", I64),
                ("leaf_cands", I64), ("leaf_edges", I64), ("index_bytes", I64),
                ("max_blob_bytes", I64), ("cell_log2", I32), ("fanout_log2", I32), ("depth", I32),
                ("cand_mode", I32), ("pts_per_cta", I32), ("stage_depth", I32), ("grid_x0", I32),
                ("grid_y0", I32), ("grid_nx", I64), ("grid_ny", I64), ("build_ms", ctypes.c_double),
                ("compact_leaves", I64), ("compact_bytes", I64), ("compact_by_edges", I64 * 8),
                ("size_ratio", I32), ("compact_edges", I32), ("nodes_by_level", I64 * 8)]


class ProjectStats(ctypes.Structure):
    _fields_ = [("n", I64), ("residual", I64), ("items", I64)]


class Query(ctypes.Structure):
    _fields_ = [("set", P), ("lon", P), ("lat", P), ("n", I64), ("out", P)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("n_streams", I32), ("mem_budget_bytes", I64), ("max_batch_points", I64),
                ("max_batch_queries", I32), ("max_pending", I32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", I64), ("completed", I64), ("rejected", I64), ("launches", I64),
                ("points", I64), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mean_batch_queries", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(P, ctypes.c_size_t, P, P)
FREE_FN = ctypes.CFUNCTYPE(None, P, P, P)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", P)]


# name -> (restype, argtypes); mirrors include/pip.h
SIGNATURES = {
    "pip_set_load_i32": (I32, [P, P, I64, P, I64, P, I32, P, I32, P, P, P, P]),
    "pip_set_load_f64": (I32, [P, P, I64, P, I64, P, I32, P, I32, P, P, P, P]),
    "pip_set_rebuild": (I32, [P, P, P]),
    "pip_set_info": (I32, [P, P]),
    "pip_set_free": (I32, [P]),
    "pip_project": (I32, [P, P, P, I64, P, P]),
    "pip_project_ex": (I32, [P, P, P, I64, P, P, P]),
    "pip_project_noalloc": (I32, [P, P, P, I64, P, P]),
    "pip_set_check": (I32, [P, P]),
    "pip_parent_ids": (I32, [P, P, I64, I32, P, P]),
    "pip_plan_create": (I32, [I64, I32, P, P]),
    "pip_plan_run": (I32, [P, P, I32, P]),
    "pip_plan_check": (I32, [P, P]),
    "pip_plan_destroy": (I32, [P]),
    "pip_project_batch": (I32, [P, I32, P]),
    "pip_plan_tune": (I32, [P, P, I32, P, P, P]),
    "pip_set_tune": (I32, [P, P, P, I64, P, P]),
    "pip_server_create": (I32, [P, I32, P, P]),
    "pip_server_submit": (I32, [P, I32, P, P, I64, P, P]),
    "pip_server_wait": (I32, [P, U64, I64]),
    "pip_server_stats": (I32, [P, P, I32]),
    "pip_server_destroy": (None, [P]),
    "pip_quantize": (I32, [P, I64, P, P, P]),
    "pip_selftest_bounded_wait": (I32, [I64, P]),
    "pip_set_top_candidates": (I32, [P, I32, P, P, I64]),
    "pip_profile_enable": (I32, [P, I32]),
    "pip_profile_read": (I32, [P, P, P, P, P]),
    "pip_locate": (I32, [P, P, P, I64, P, P]),
    "pip_kernel_launches": (I64, []),
    "pip_last_error": (ctypes.c_char_p, []),
    "pip_version": (I32, []),
}

_lib = None


def load():
    """Load libpip.so; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libpip.so is not built ({LIB_PATH}); run `python -m paper_2005_03156_gb300.build` "
            "(needs nvcc) - there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != 0:
        msg = load().pip_last_error()
        raise PipError(status, msg.decode() if msg else "")
