"""ctypes front end of the FP64 oracle in ``mecuco_oracle.c``.

Test infrastructure only (see the package docstring).  Inputs are converted to
contiguous float64 arrays (bfloat16 and float32 values widen exactly), so the
oracle sees exactly the values the CUDA path sees.

Functions (paper sections in brackets):
    knn(X, k, rows=None, include_self=False)   brute force [Sec. 3 Step 1; Alg. 1]
    center_patch(X, nb)                        centred patch [Sec. 3 Step 2]
    jacobi_eigh(A)                             own cyclic Jacobi eigensolver
    svd_hestenes(Xc)                           own one-sided Jacobi SVD
    fast_patch(Xc, variant, route)             Alg. 1 Fast branch, term by term
    exact_patch(Xc)                            Theorem 1 (Exact mode)
    naive_patch(Xc, W)                         |tr(-H H^T Sigma)| with explicit H
    hht(W)                                     H H^T from the explicit H
    curvature(X, k, idx, ...)                  Alg. 1 per-point loop
    grad_fd(X, k, idx, coords, h, ...)         FP64 central differences
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "lib_path", "knn", "center_patch", "jacobi_eigh", "svd_hestenes",
    "fast_patch", "exact_patch", "naive_patch", "hht", "curvature", "grad_fd",
    "TERMS", "LITERAL", "HAAR",
]

LITERAL = 0
HAAR = 1
TERMS = ("tau", "t_range", "t_A", "t_B2", "gt2", "t_B", "t_null", "kappa")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mecuco_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction so x86 and Arm
    round the same way)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            d, i64, i32, p = C.c_double, C.c_int64, C.c_int, C.c_void_p
            lib.orc_knn.argtypes = [p, i32, i64, i64, p, i64, i32, i32, p, p, i32]
            lib.orc_knn.restype = i32
            lib.orc_center_patch.argtypes = [p, i64, p, i32, p]
            lib.orc_center_patch.restype = None
            lib.orc_jacobi_eigh.argtypes = [i32, p, p, p, i32]
            lib.orc_jacobi_eigh.restype = i32
            lib.orc_svd_hestenes.argtypes = [i32, i64, p, p, p, i32]
            lib.orc_svd_hestenes.restype = i32
            lib.orc_fast_patch.argtypes = [i32, i64, p, i32, i32, p, p, p]
            lib.orc_fast_patch.restype = i32
            lib.orc_exact_patch.argtypes = [i32, i64, p, p, p]
            lib.orc_exact_patch.restype = d
            lib.orc_hht.argtypes = [i64, p, p]
            lib.orc_hht.restype = None
            lib.orc_naive_patch.argtypes = [i32, i64, p, p]
            lib.orc_naive_patch.restype = d
            lib.orc_curvature.argtypes = [p, i32, i64, i64, i32, p, p, i64, i32, i32, i32, p, p, p, i32]
            lib.orc_curvature.restype = i32
            lib.orc_grad_fd.argtypes = [p, i64, i64, i32, p, i32, i32, p, p, i64, p, p, i32]
            lib.orc_grad_fd.restype = i32
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _typed(X, bf16_bits: bool):
    """(array, element code) for the dataset-level entry points: float32 and
    bfloat16 bit patterns (uint16, with bf16_bits=True) are passed as they
    are and widened exactly to double inside the oracle."""
    X = np.asarray(X)
    if bf16_bits or X.dtype == np.uint16:
        if X.dtype != np.uint16:
            raise TypeError("bf16 inputs must be uint16 bit patterns")
        return np.ascontiguousarray(X), 2
    if X.dtype == np.float32:
        return np.ascontiguousarray(X), 1
    return _f64(X), 0


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def knn(X, k: int, rows=None, include_self: bool = False, nthreads=None, bf16_bits: bool = False):
    """k nearest neighbours of each query row (all rows, or ``rows``) by
    brute force in FP64; returns (idx int32 [q, k], dist float64 [q, k])
    sorted by (distance, index).  X may be float64, float32 or bfloat16 bit
    patterns (uint16); elements are widened exactly to double."""
    X, elt = _typed(X, bf16_bits)
    n, m = X.shape
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nq = n if r is None else r.size
    idx = np.empty((nq, k), dtype=np.int32)
    dist = np.empty((nq, k), dtype=np.float64)
    rc = _load().orc_knn(_ptr(X), elt, n, m, None if r is None else _ptr(r), nq, k,
                         int(bool(include_self)), _ptr(idx), _ptr(dist), _threads(nthreads))
    if rc != 0:
        raise ValueError("oracle knn: invalid k for this n")
    return idx, dist


def center_patch(X, nb):
    X = _f64(X)
    nb = np.ascontiguousarray(nb, dtype=np.int32)
    out = np.empty((nb.size, X.shape[1]), dtype=np.float64)
    _load().orc_center_patch(_ptr(X), X.shape[1], _ptr(nb), nb.size, _ptr(out))
    return out


def jacobi_eigh(A, max_sweeps: int = 100):
    """Eigenvalues (descending) and eigenvectors (columns) of a symmetric
    matrix by the oracle's own cyclic Jacobi; also the sweep count."""
    A = _f64(A).copy()
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    sweeps = _load().orc_jacobi_eigh(n, _ptr(A), _ptr(w), _ptr(V), max_sweeps)
    return w, V, sweeps


def svd_hestenes(Xc, max_sweeps: int = 100):
    """Singular values (descending) and right singular vectors (m x k) of
    the k x m matrix Xc by one-sided Jacobi; also the sweep count."""
    Xc = _f64(Xc)
    k, m = Xc.shape
    s = np.empty(k)
    V = np.empty((m, k))
    sweeps = _load().orc_svd_hestenes(k, m, _ptr(Xc), _ptr(s), _ptr(V), max_sweeps)
    return s, V, sweeps


def fast_patch(Xc, variant: int = LITERAL, route: int = 0, return_v: bool = False):
    """Alg. 1 Fast branch on one centred patch.  Returns a dict of the terms
    (``TERMS``) plus ``p`` and ``lam`` (and ``Vr`` if asked)."""
    Xc = _f64(Xc)
    k, m = Xc.shape
    terms = np.empty(len(TERMS))
    lam = np.empty(k)
    vr = np.empty((m, k)) if return_v else None
    p = _load().orc_fast_patch(k, m, _ptr(Xc), int(variant), int(route), _ptr(terms),
                               _ptr(lam), None if vr is None else _ptr(vr))
    out = dict(zip(TERMS, terms.tolist()))
    out["p"] = int(p)
    out["lam"] = lam
    if return_v:
        out["Vr"] = vr[:, :p]
    return out


def exact_patch(Xc, return_basis: bool = False):
    """Theorem 1 on one centred patch; optionally also (W, v)."""
    Xc = _f64(Xc)
    k, m = Xc.shape
    W = np.empty((m, m))
    v = np.empty(m)
    kappa = _load().orc_exact_patch(k, m, _ptr(Xc), _ptr(W), _ptr(v))
    return (kappa, W, v) if return_basis else kappa


def naive_patch(Xc, W):
    """|tr(-H H^T Sigma)| with H built explicitly from the eigenbasis W."""
    Xc = _f64(Xc)
    W = _f64(W)
    k, m = Xc.shape
    return _load().orc_naive_patch(k, m, _ptr(Xc), _ptr(W))


def hht(W):
    W = _f64(W)
    m = W.shape[0]
    out = np.empty((m, m))
    _load().orc_hht(m, _ptr(W), _ptr(out))
    return out


def curvature(X, k: int, idx, rows=None, mode: str = "fast", variant: int = LITERAL,
              route: int = 0, nthreads=None, return_terms: bool = False, bf16_bits: bool = False):
    """Alg. 1 per-point loop over the query rows (all rows, or ``rows``)
    with frozen neighbour lists ``idx`` (n x k).  X as for ``knn``."""
    X, elt = _typed(X, bf16_bits)
    n, m = X.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nq = n if r is None else r.size
    kappa = np.empty(nq)
    terms = np.empty((nq, len(TERMS))) if return_terms else None
    lam = np.empty((nq, k)) if return_terms else None
    _load().orc_curvature(_ptr(X), elt, n, m, k, _ptr(idx), None if r is None else _ptr(r), nq,
                          1 if mode == "exact" else 0, int(variant), int(route),
                          _ptr(kappa), None if terms is None else _ptr(terms),
                          None if lam is None else _ptr(lam), _threads(nthreads))
    if return_terms:
        return kappa, terms, lam
    return kappa


def grad_fd(X, k: int, idx, coords, h, variant: int = LITERAL, route: int = 0, nthreads=None):
    """Central differences of sum_i K_i w.r.t. X[ci, ca] for each (ci, ca) in
    ``coords`` with step(s) ``h``; neighbour lists frozen."""
    X = _f64(X)
    n, m = X.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 2)
    ci = np.ascontiguousarray(coords[:, 0])
    ca = np.ascontiguousarray(coords[:, 1])
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), ci.shape))
    out = np.empty(ci.size)
    _load().orc_grad_fd(_ptr(X), n, m, k, _ptr(idx), int(variant), int(route), _ptr(ci),
                        _ptr(ca), ci.size, _ptr(hh), _ptr(out), _threads(nthreads))
    return out
