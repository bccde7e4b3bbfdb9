"""Python binding of the C ABI (argument marshalling only).

Every function here forwards torch tensors' device pointers and the current
CUDA stream to the same-named entry point of libmecuco.so; all arithmetic of
the path runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N

_PREC = {"fp32": N.PREC_FP32, "bf16_mixed": N.PREC_BF16_MIXED}
_VAR = {"literal": N.FAST_LITERAL, "haar": N.FAST_HAAR}


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return N.F32
    if t.dtype == torch.bfloat16:
        return N.BF16
    raise TypeError(f"X must be float32 or bfloat16, got {t.dtype}")


def _check_x(X: torch.Tensor, device: int):
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D tensor with unit column stride")
    if not X.is_cuda or X.device.index != device:
        raise ValueError(f"X must live on cuda:{device}")


def _stream(device: int):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Context:
    """Owns one ``mecuco_t`` handle (device workspace, status word)."""

    def __init__(self, device: int = 0):
        self.lib = N.load()
        self.device = int(device)
        h = C.c_void_p()
        N.check(self.lib.mecuco_create(C.byref(h), self.device), "mecuco_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mecuco_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, opt: int, value: int):
        N.check(self.lib.mecuco_set_option(self.handle, int(opt), int(value)), "mecuco_set_option")

    # -- entry points -------------------------------------------------------
    def mecuco_knn(self, X: torch.Tensor, k: int, include_self: bool = False, precision: str = "fp32",
                   return_dist: bool = False):
        _check_x(X, self.device)
        n, m = X.shape
        idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
        dist = torch.empty((n, k), dtype=torch.float32, device=X.device) if return_dist else None
        st = self.lib.mecuco_knn(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                 int(bool(include_self)), _PREC[precision], _ptr(idx), _ptr(dist),
                                 _stream(self.device))
        N.check(st, "mecuco_knn")
        return (idx, dist) if return_dist else idx

    def mecuco_curvature(self, X: torch.Tensor, k: int, idx: torch.Tensor | None = None,
                         include_self: bool = False, variant: str = "literal", precision: str = "fp32",
                         return_lambda: bool = False, return_U: bool = False, return_s: bool = False):
        _check_x(X, self.device)
        n, m = X.shape
        if idx is not None:
            if idx.dtype != torch.int32 or tuple(idx.shape) != (n, k) or not idx.is_contiguous():
                raise ValueError("idx must be a contiguous int32 (N, k) tensor")
        dev = X.device
        kappa = torch.empty(n, dtype=torch.float32, device=dev)
        lam = torch.empty((n, k), dtype=torch.float32, device=dev) if return_lambda else None
        U = torch.empty((n, k, k), dtype=torch.float32, device=dev) if return_U else None
        s = torch.empty((n, k), dtype=torch.float32, device=dev) if return_s else None
        st = self.lib.mecuco_curvature(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                       _ptr(idx), int(bool(include_self)), _VAR[variant], _PREC[precision],
                                       _ptr(kappa), _ptr(lam), _ptr(U), _ptr(s), _stream(self.device))
        N.check(st, "mecuco_curvature")
        out = {"kappa": kappa}
        if return_lambda:
            out["lambda"] = lam
        if return_U:
            out["U"] = U
        if return_s:
            out["s"] = s
        return out if (return_lambda or return_U or return_s) else kappa

    def mecuco_knn_range(self, X: torch.Tensor, k: int, row_begin: int, row_end: int, include_self: bool = False,
                         precision: str = "fp32", return_dist: bool = False):
        _check_x(X, self.device)
        n, m = X.shape
        nr = row_end - row_begin
        idx = torch.empty((nr, k), dtype=torch.int32, device=X.device)
        dist = torch.empty((nr, k), dtype=torch.float32, device=X.device) if return_dist else None
        st = self.lib.mecuco_knn_range(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                       int(bool(include_self)), _PREC[precision], int(row_begin), int(row_end),
                                       _ptr(idx), _ptr(dist), _stream(self.device))
        N.check(st, "mecuco_knn_range")
        return (idx, dist) if return_dist else idx

    def mecuco_curvature_range(self, X: torch.Tensor, k: int, row_begin: int, row_end: int,
                               idx: torch.Tensor | None = None, include_self: bool = False,
                               variant: str = "literal", precision: str = "fp32"):
        _check_x(X, self.device)
        n, m = X.shape
        nr = row_end - row_begin
        if idx is not None and (idx.dtype != torch.int32 or tuple(idx.shape) != (nr, k) or not idx.is_contiguous()):
            raise ValueError("idx must be a contiguous int32 (row_end - row_begin, k) tensor")
        kappa = torch.empty(nr, dtype=torch.float32, device=X.device)
        st = self.lib.mecuco_curvature_range(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                             _ptr(idx), int(bool(include_self)), _VAR[variant], _PREC[precision],
                                             int(row_begin), int(row_end), _ptr(kappa), None, None, None,
                                             _stream(self.device))
        N.check(st, "mecuco_curvature_range")
        return kappa

    def mecuco_curvature_exact(self, X: torch.Tensor, k: int, idx=None, include_self: bool = False,
                               precision: str = "fp32", row_begin: int = 0, row_end=None, return_basis: bool = False):
        """Exact-mode (Theorem 1) curvature of rows [row_begin, row_end); with return_basis also the
        covariance eigenvalues v (rows x m) and eigenvectors W (rows x m x m) it used."""
        _check_x(X, self.device)
        n, m = X.shape
        re = n if row_end is None else int(row_end)
        rows = re - int(row_begin)
        if idx is not None and (idx.dtype != torch.int32 or tuple(idx.shape) != (n, k) or not idx.is_contiguous()):
            raise ValueError("idx must be a contiguous int32 (N, k) tensor")
        kap = torch.empty(rows, dtype=torch.float32, device=X.device)
        v = torch.empty((rows, m), dtype=torch.float32, device=X.device) if return_basis else None
        W = torch.empty((rows, m, m), dtype=torch.float32, device=X.device) if return_basis else None
        st = self.lib.mecuco_curvature_exact(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                             _ptr(idx) if idx is not None else None, int(bool(include_self)),
                                             _PREC[precision], int(row_begin), re, _ptr(kap),
                                             _ptr(v) if v is not None else None, _ptr(W) if W is not None else None,
                                             _stream(self.device))
        N.check(st, "mecuco_curvature_exact")
        return (kap, v, W) if return_basis else kap

    def mecuco_curvature_rsvd(self, X: torch.Tensor, k: int, rank: int, sketch_cols: int | None = None,
                              power_iters: int = 2, omega: torch.Tensor | None = None, seed: int = 0,
                              idx: torch.Tensor | None = None, include_self: bool = False, variant: str = "literal",
                              precision: str = "fp32") -> torch.Tensor:
        """Fast-mode curvature with a randomised rank-`rank` SVD of each patch.  omega is the
        k x sketch_cols Gaussian test matrix (default: rank + min(8, k - rank) columns drawn
        from numpy's default_rng(seed))."""
        _check_x(X, self.device)
        n, m = X.shape
        if idx is not None and (idx.dtype != torch.int32 or tuple(idx.shape) != (n, k) or not idx.is_contiguous()):
            raise ValueError("idx must be a contiguous int32 (N, k) tensor")
        if omega is None:
            import numpy as np
            cols = sketch_cols if sketch_cols is not None else rank + min(8, k - rank)
            omega = torch.from_numpy(np.random.default_rng(seed).standard_normal((k, cols)).astype(np.float32))
        omega = omega.to(device=X.device, dtype=torch.float32).contiguous()
        if omega.dim() != 2 or omega.shape[0] != k:
            raise ValueError("omega must be (k, sketch_cols)")
        kappa = torch.empty(n, dtype=torch.float32, device=X.device)
        st = self.lib.mecuco_curvature_rsvd(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                            _ptr(idx), int(bool(include_self)), _VAR[variant], _PREC[precision],
                                            int(rank), int(omega.shape[1]), int(power_iters), _ptr(omega),
                                            _ptr(kappa), _stream(self.device))
        N.check(st, "mecuco_curvature_rsvd")
        return kappa

    def mecuco_exact_kappa(self, v: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
        """Theorem 1 on supplied eigenpairs: v (np, m), W (np, m, m), column s = eigenvector s."""
        dev = f"cuda:{self.device}"
        v = v.to(device=dev, dtype=torch.float32).contiguous()
        W = W.to(device=dev, dtype=torch.float32).contiguous()
        if v.dim() != 2 or W.shape != (v.shape[0], v.shape[1], v.shape[1]):
            raise ValueError("v must be (np, m) and W (np, m, m)")
        kappa = torch.empty(v.shape[0], dtype=torch.float32, device=dev)
        st = self.lib.mecuco_exact_kappa(self.handle, _ptr(v), _ptr(W), v.shape[1], v.shape[0], _ptr(kappa),
                                         _stream(self.device))
        N.check(st, "mecuco_exact_kappa")
        return kappa

    def mecuco_fidelity(self, kappa_ref: torch.Tensor, kappa: torch.Tensor, normalize: bool = False):
        """(MAE, Spearman rho_S, Chatterjee xi) of kappa against kappa_ref."""
        a = kappa_ref.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        b = kappa.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        if a.numel() != b.numel():
            raise ValueError("the two vectors differ in length")
        out = torch.empty(3, dtype=torch.float64, device=a.device)
        st = self.lib.mecuco_fidelity(self.handle, _ptr(a), _ptr(b), a.numel(), int(bool(normalize)), _ptr(out),
                                      _stream(self.device))
        N.check(st, "mecuco_fidelity")
        mae, rho, xi = out.cpu().tolist()
        return mae, rho, xi

    def mecuco_minmax_normalize(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(dtype=torch.float32).contiguous()
        y = torch.empty_like(x)
        st = self.lib.mecuco_minmax_normalize(self.handle, _ptr(x), x.numel(), _ptr(y), _stream(self.device))
        N.check(st, "mecuco_minmax_normalize")
        return y

    def curvature_auto(self, X: torch.Tensor, k: int, idx=None, **kw):
        """The paper's automatic mode: Exact (Theorem 1) for m < 50, Fast otherwise."""
        if X.shape[1] < 50:
            return self.mecuco_curvature_exact(X, k, idx=idx, include_self=kw.get("include_self", False),
                                               precision=kw.get("precision", "fp32"))
        return self.mecuco_curvature(X, k, idx=idx, **kw)

    def _datasets(self, Xs, ks, idx_out):
        if len(Xs) != len(ks) or not Xs:
            raise ValueError("one k per dataset")
        dt = _dtype_code(Xs[0])
        arr = (N.mecuco_dataset * len(Xs))()
        kappas = []
        for i, (X, k) in enumerate(zip(Xs, ks)):
            _check_x(X, self.device)
            if _dtype_code(X) != dt:
                raise ValueError("all datasets of a batch share one dtype")
            n, m = X.shape
            kap = torch.empty(n, dtype=torch.float32, device=X.device)
            kappas.append(kap)
            iv = idx_out[i] if idx_out is not None else None
            if iv is not None and (iv.dtype != torch.int32 or tuple(iv.shape) != (n, int(k)) or not iv.is_contiguous()):
                raise ValueError("idx_out[i] must be a contiguous int32 (N, k) tensor")
            arr[i] = N.mecuco_dataset(_ptr(X), n, m, X.stride(0), int(k), _ptr(iv) if iv is not None else None,
                                      _ptr(kap))
        return arr, dt, kappas

    def mecuco_curvature_batched(self, Xs, ks, include_self: bool = False, variant: str = "literal",
                                 precision: str = "fp32", idx_out=None):
        """Curvature of several datasets in one call; returns one kappa tensor per dataset
        (neighbour lists written to idx_out[i] when given)."""
        arr, dt, kappas = self._datasets(Xs, ks, idx_out)
        st = self.lib.mecuco_curvature_batched(self.handle, arr, len(Xs), dt, int(bool(include_self)), _VAR[variant],
                                               _PREC[precision], _stream(self.device))
        N.check(st, "mecuco_curvature_batched")
        return kappas

    def mecuco_autotune_batched(self, Xs, ks, include_self: bool = False, variant: str = "literal",
                                precision: str = "fp32") -> dict:
        """Time the batched call over its tuning space (BF16-mixed: kNN tile form and the
        third-moment pass's CTAs per SM and TMEM slots; FP32: 1..32 lanes); keep the fastest
        for this batch signature and return it as a dict."""
        arr, dt, _ = self._datasets(Xs, ks, None)
        out = N.mecuco_batch_tuning()
        st = self.lib.mecuco_autotune_batched(self.handle, arr, len(Xs), dt, int(bool(include_self)), _VAR[variant],
                                              _PREC[precision], _stream(self.device), C.byref(out))
        N.check(st, "mecuco_autotune_batched")
        return {f: getattr(out, f) for f, _ in N.mecuco_batch_tuning._fields_}

    def mecuco_tangent_basis(self, X: torch.Tensor, k: int, idx: torch.Tensor, d_out: int, row_begin: int = 0,
                             row_end=None) -> torch.Tensor:
        """First d_out tangent directions V_r (m x d_out per point) of rows [row_begin, row_end)."""
        _check_x(X, self.device)
        n, m = X.shape
        if idx.dtype != torch.int32 or tuple(idx.shape) != (n, k) or not idx.is_contiguous():
            raise ValueError("idx must be a contiguous int32 (N, k) tensor")
        re = n if row_end is None else int(row_end)
        V = torch.empty((re - int(row_begin), m, int(d_out)), dtype=torch.float32, device=X.device)
        st = self.lib.mecuco_tangent_basis(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k), _ptr(idx),
                                           int(row_begin), re, int(d_out), _ptr(V), _stream(self.device))
        N.check(st, "mecuco_tangent_basis")
        return V

    def mecuco_curvature_backward(self, X: torch.Tensor, k: int, idx: torch.Tensor, dkappa: torch.Tensor,
                                  variant: str = "literal"):
        """dX = d(sum_i dkappa_i K_i)/dX with the neighbour lists idx frozen (float32, N x m)."""
        _check_x(X, self.device)
        n, m = X.shape
        if idx.dtype != torch.int32 or tuple(idx.shape) != (n, k) or not idx.is_contiguous():
            raise ValueError("idx must be a contiguous int32 (N, k) tensor")
        dk = dkappa.to(device=X.device, dtype=torch.float32).contiguous()
        dX = torch.empty((n, m), dtype=torch.float32, device=X.device)
        st = self.lib.mecuco_curvature_backward(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                                _ptr(idx), _VAR[variant], _ptr(dk), _ptr(dX),
                                                _stream(self.device))
        N.check(st, "mecuco_curvature_backward")
        return dX

    def mecuco_get_stage_times(self) -> dict:
        ms = (C.c_double * len(N.STAGES))()
        cnt = (C.c_int64 * len(N.STAGES))()
        N.check(self.lib.mecuco_get_stage_times(self.handle, ms, cnt, _stream(self.device)), "mecuco_get_stage_times")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(N.STAGES)}

    def mecuco_curvature_host(self, X: torch.Tensor, k: int, include_self: bool = False,
                              variant: str = "literal", precision: str = "fp32", return_idx: bool = False,
                              kappa_out: torch.Tensor | None = None, idx_out: torch.Tensor | None = None):
        """Host (CPU, ideally pinned) tensors in and out; copies happen inside the call."""
        if X.is_cuda or X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("X must be a 2-D CPU tensor with unit column stride")
        n, m = X.shape
        kappa = kappa_out if kappa_out is not None else torch.empty(n, dtype=torch.float32)
        idx = idx_out if idx_out is not None else (torch.empty((n, k), dtype=torch.int32) if return_idx else None)
        st = self.lib.mecuco_curvature_host(self.handle, _ptr(X), _dtype_code(X), n, m, X.stride(0), int(k),
                                            int(bool(include_self)), _VAR[variant], _PREC[precision],
                                            _ptr(kappa), _ptr(idx), _stream(self.device))
        N.check(st, "mecuco_curvature_host")
        return (kappa, idx) if (return_idx or idx_out is not None) else kappa

    def mecuco_get_last_status(self) -> int:
        return int(self.lib.mecuco_get_last_status(self.handle, _stream(self.device)))

    def mecuco_get_stats(self) -> dict:
        st = N.mecuco_stats()
        N.check(self.lib.mecuco_get_stats(self.handle, C.byref(st), _stream(self.device)), "mecuco_get_stats")
        return {f: getattr(st, f) for f, _ in N.mecuco_stats._fields_}


_default = {}


def context(device: int = 0) -> Context:
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def mecuco_knn(X, k, **kw):
    return context(X.device.index or 0).mecuco_knn(X, k, **kw)


def mecuco_curvature(X, k, **kw):
    return context(X.device.index or 0).mecuco_curvature(X, k, **kw)


def mecuco_curvature_host(X, k, device: int = 0, **kw):
    return context(device).mecuco_curvature_host(X, k, **kw)
