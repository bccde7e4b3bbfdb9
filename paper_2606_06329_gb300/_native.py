"""ctypes declarations of the C ABI in include/mecuco.h.

Loading fails loudly (``MecucoNotBuilt``) when lib/libmecuco.so is missing:
there is no CPU or eager fallback behind this package.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmecuco.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_TIMEOUT = range(7)
F32, BF16 = 0, 1
FAST_LITERAL, FAST_HAAR = 0, 1
PREC_FP32, PREC_BF16_MIXED = 0, 1
(OPT_KNN_MARGIN, OPT_JACOBI_FP64, OPT_JACOBI_MAX_SWEEPS, OPT_CHUNK_POINTS, OPT_KNN_QUERY_CHUNK, OPT_PROFILE,
 OPT_KNN_SPLITS, OPT_BATCH_LANES, OPT_TC_SLOTS, OPT_KNN_PAIR, OPT_WAIT_LIMIT, OPT_WORKSPACE_LIMIT,
 OPT_PROFILE_STAGES, OPT_TT_SLOTS, OPT_TT_CTAS, OPT_BATCH_PERSISTENT, OPT_JACOBI_WARP,
 OPT_KNN_SPLIT_BF16) = range(18)
STAGES = ("rownorm", "knn_search", "knn_rerank", "knn_fallback", "gram", "moments", "jacobi", "estimator", "adjoint",
          "basis", "exact", "fidelity", "rotate")


class MecucoNotBuilt(ImportError):
    pass


class MecucoError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: status {status}"
        if _lib is not None:
            msg += f" ({_lib.mecuco_status_string(status).decode()})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class mecuco_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "knn_rows", "knn_uncertified", "knn_fallback_rows", "jacobi_max_sweeps",
        "jacobi_not_converged", "rank_deficient", "kernel_launches", "jacobi_rotations")]


class mecuco_dataset(C.Structure):
    _fields_ = [("X", C.c_void_p), ("N", C.c_int64), ("m", C.c_int64), ("ld", C.c_int64), ("k", C.c_int),
                ("idx", C.c_void_p), ("kappa", C.c_void_p)]


class mecuco_batch_tuning(C.Structure):
    _fields_ = [("lanes", C.c_int), ("knn_pair", C.c_int), ("tt_ctas", C.c_int), ("tt_slots", C.c_int),
                ("ms", C.c_float)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); exactly the functions of include/mecuco.h
_p, _i32, _i64, _st = C.c_void_p, C.c_int, C.c_int64, C.c_int
SIGNATURES = {
    "mecuco_create": (_st, [C.POINTER(C.c_void_p), _i32]),
    "mecuco_destroy": (_st, [_p]),
    "mecuco_set_option": (_st, [_p, _i32, _i64]),
    "mecuco_knn": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _i32, _i32, _p, _p, _p]),
    "mecuco_curvature": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _p, _i32, _i32, _i32, _p, _p, _p, _p, _p]),
    "mecuco_knn_range": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _i32, _i32, _i64, _i64, _p, _p, _p]),
    "mecuco_curvature_range": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _p, _i32, _i32, _i32, _i64, _i64,
                                     _p, _p, _p, _p, _p]),
    "mecuco_curvature_backward": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _p, _i32, _p, _p, _p]),
    "mecuco_tangent_basis": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _p, _i64, _i64, _i32, _p, _p]),
    "mecuco_curvature_exact": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _p, _i32, _i32, _i64, _i64, _p, _p, _p,
                                     _p]),
    "mecuco_curvature_rsvd": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _p, _i32, _i32, _i32, _i32, _i32, _i32, _p,
                                    _p, _p]),
    "mecuco_exact_kappa": (_st, [_p, _p, _p, _i64, _i64, _p, _p]),
    "mecuco_fidelity": (_st, [_p, _p, _p, _i64, _i32, _p, _p]),
    "mecuco_minmax_normalize": (_st, [_p, _p, _i64, _p, _p]),
    "mecuco_curvature_batched": (_st, [_p, C.POINTER(mecuco_dataset), _i32, _i32, _i32, _i32, _i32, _p]),
    "mecuco_autotune_batched": (_st, [_p, C.POINTER(mecuco_dataset), _i32, _i32, _i32, _i32, _i32, _p,
                                      C.POINTER(mecuco_batch_tuning)]),
    "mecuco_curvature_host": (_st, [_p, _p, _i32, _i64, _i64, _i64, _i32, _i32, _i32, _i32, _p, _p, _p]),
    "mecuco_knn_noalloc": (_st, [_p, _i32, _i64, _i64, _i64, _i32, _i32, _p, _p, _p]),
    "mecuco_get_last_status": (_st, [_p, _p]),
    "mecuco_get_stats": (_st, [_p, C.POINTER(mecuco_stats), _p]),
    "mecuco_get_stage_times": (_st, [_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), _p]),
    "mecuco_status_string": (C.c_char_p, [_st]),
    "mecuco_last_error_message": (C.c_char_p, []),
}


def load(path: str | None = None):
    """Load libmecuco.so (building it first is the caller's job:
    ``__graft_entry__.build()`` or ``python -m paper_2606_06329_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise MecucoNotBuilt(f"{p} is missing: build the CUDA library first")
            lib = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int, where: str):
    if status != OK:
        detail = ""
        if status == ERR_CUDA and _lib is not None:
            detail = _lib.mecuco_last_error_message().decode()
        raise MecucoError(status, where, detail)
