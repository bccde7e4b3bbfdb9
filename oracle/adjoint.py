"""Reference gradient of the Fast-mode curvature in FP64: d(sum_i w_i K_i)/dX
with the neighbour lists frozen, by reverse-mode differentiation (PyTorch CPU
autograd, float64) of Alg. 1's Fast branch written term by term (test
infrastructure only, like the rest of this package).

Per query point i the patch is X_c = X[idx_i] - mean (Sec. 3 Step 2); its
Gram G = X_c X_c^T is eigendecomposed with torch.linalg.eigh (a library
routine; its backward is the first-order perturbation formula of symmetric
eigenpairs, valid for distinct eigenvalues); the top p pairs give
V_r = X_c^T U_p diag(s)^-1 and lambda_r = s^2/(k-1), and then, as printed:
    tau = sum lambda_r,  t_range = |X_c V_r^{o2}|_F^2/(k-1),  d_P = 1 - V_r^{o2} 1,
    t_A = |X_c d_P|^2/(k-1),  t_B2 = |X_c V_r|_F^2/(k-1),
    G_tens[j,l1,l2] = sum_a X_c[j,a] V_r[a,l1] V_r[a,l2],
    literal: t_B = tau - 2 t_B2 + |G_tens|^2/(k-1),  t_null = (t_A + 2 t_B)/(m - p)
    Haar:    t_B = tau - 2 sum_{j,a} X_c[j,a]^2 (1 - d_P[a])/(k-1) + |G_tens|^2/(k-1),
             t_null = (t_A + 2 t_B)/(m - p + 2)
    K = |(t_range + t_null)/2 + tau/2|.
p = min(k - 1, m, #{eigenvalues > k m 2^-52 of the largest}), the C oracle's
rule, taken for each point from the unperturbed values (p is piecewise
constant in X).  All points are processed as one batch.
"""
from __future__ import annotations

import numpy as np

__all__ = ["curvature_fast", "grad_adjoint"]


def _fast_batch(Xc, variant: str):
    """K for a batch of centred patches Xc (B x k x m, float64 torch tensor)."""
    import torch
    B, k, m = Xc.shape
    km1 = k - 1.0
    G = Xc @ Xc.transpose(1, 2)
    w, U = torch.linalg.eigh(G)                       # ascending
    w = torch.flip(w, dims=[1])
    U = torch.flip(U, dims=[2])
    with torch.no_grad():
        pmax = min(k - 1, m)
        thr = k * m * 2.0 ** -52 * torch.clamp(w[:, :1], min=0.0)
        rank = (w > thr).sum(dim=1)
    ps = torch.clamp(rank, max=pmax)
    kappas = []
    for p in torch.unique(ps).tolist():               # a batch per truncation rank
        sel = (ps == p).nonzero(as_tuple=True)[0]
        Xs = Xc[sel]
        Up = U[sel, :, :p]
        s2 = w[sel, :p]
        Vr = Xs.transpose(1, 2) @ Up / torch.sqrt(s2)[:, None, :]        # B x m x p
        tau = s2.sum(dim=1) / km1
        t_range = ((Xs @ Vr ** 2) ** 2).sum(dim=(1, 2)) / km1
        dP = 1.0 - (Vr ** 2).sum(dim=2)                                   # B x m
        t_A = ((Xs @ dP[:, :, None]) ** 2).sum(dim=(1, 2)) / km1
        t_B2 = ((Xs @ Vr) ** 2).sum(dim=(1, 2)) / km1
        G_tens = torch.einsum("bja,bal,ban->bjln", Xs, Vr, Vr)
        gt2 = (G_tens ** 2).sum(dim=(1, 2, 3))
        q = m - p
        if variant == "haar":
            h = (Xs ** 2 * (1.0 - dP)[:, None, :]).sum(dim=(1, 2))
            t_B = tau - 2.0 * h / km1 + gt2 / km1
            t_null = (t_A + 2.0 * t_B) / (q + 2) if q > 0 else torch.zeros_like(tau)
        else:
            t_B = tau - 2.0 * t_B2 + gt2 / km1
            t_null = (t_A + 2.0 * t_B) / q if q > 0 else torch.zeros_like(tau)
        kappas.append((sel, torch.abs(0.5 * (t_range + t_null) + 0.5 * tau)))
    parts = torch.zeros(B, dtype=Xc.dtype)
    for sel, kap in kappas:
        parts = parts.index_put((sel,), kap)
    return parts


def curvature_fast(X, idx, variant: str = "literal"):
    """K of every point (numpy float64 out) with frozen neighbour lists idx (n x k)."""
    import torch
    Xt = torch.as_tensor(np.asarray(X, dtype=np.float64))
    nb = Xt[torch.as_tensor(np.asarray(idx, dtype=np.int64))]            # n x k x m
    Xc = nb - nb.mean(dim=1, keepdim=True)
    with torch.no_grad():
        return _fast_batch(Xc, variant).numpy()


def grad_adjoint(X, idx, weights=None, variant: str = "literal"):
    """d(sum_i w_i K_i)/dX (n x m float64), neighbour lists idx frozen."""
    import torch
    Xt = torch.tensor(np.asarray(X, dtype=np.float64), requires_grad=True)
    nb = Xt[torch.as_tensor(np.asarray(idx, dtype=np.int64))]
    Xc = nb - nb.mean(dim=1, keepdim=True)
    kap = _fast_batch(Xc, variant)
    w = torch.ones_like(kap) if weights is None else torch.as_tensor(np.asarray(weights, dtype=np.float64))
    (kap * w).sum().backward()
    return Xt.grad.numpy()
