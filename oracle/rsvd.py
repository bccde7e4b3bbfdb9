"""Randomised low-rank variant of the Fast mode, in FP64 with NumPy (test
infrastructure only, like the rest of this package).

The paper's future work (Sec. Conclusions) proposes replacing the Fast mode's
truncated SVD by a randomised low-rank approximation.  Here the range finder
of Halko, Martinsson & Tropp (SIAM Review 53, 2011; Alg. 4.3 with q power
iterations, Alg. 4.4's re-orthonormalisation, then the Rayleigh-Ritz step of
their Sec. 5) runs on the patch Gram G = X_c X_c^T with a k x l Gaussian test
matrix Omega:

    Y = G Omega;  q times: Q = orth(Y), Y = G Q;  Q = orth(Y)
    B = Q^T G Q = V_B diag(s2) V_B^T,  U = Q V_B,  keep the r largest

and the Fast estimator (Alg. 1, Fast branch; eqs. tA, tB, tnull, fast_curv)
runs with p = r on those Ritz pairs: V_r = X_c^T U_r diag(s)^-1.

    fast_from_eig(Xc, U, s2, variant)   Alg. 1's Fast terms from given eigenpairs
                                        (U: k x p orthonormal columns, s2: Gram
                                        eigenvalues), every term from V_r as printed
    rsvd_eig(G, omega, rank, power)     the range finder and Rayleigh-Ritz step
    rsvd_patch(Xc, omega, rank, power, variant)

orth() is numpy's QR; B's eigenpairs come from numpy.linalg.eigh.  Where Y is
rank-deficient (G has rank <= k - 1: the rows of X_c sum to zero) QR's extra
columns only add directions; the r largest Ritz pairs are unaffected when r
is below the rank of Y.
"""
from __future__ import annotations

import numpy as np

__all__ = ["fast_from_eig", "rsvd_eig", "rsvd_patch"]


def fast_from_eig(Xc, U, s2, variant: str = "literal") -> dict:
    """Alg. 1 Fast branch on one centred patch Xc (k x m) with the truncated
    SVD replaced by the given eigenpairs of G = Xc Xc^T: U (k x p), s2 (p)."""
    Xc = np.asarray(Xc, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    s2 = np.asarray(s2, dtype=np.float64)
    k, m = Xc.shape
    p = U.shape[1]
    km1 = k - 1.0
    Vr = Xc.T @ U / np.sqrt(s2)[None, :]            # m x p
    lam = s2 / km1
    tau = lam.sum()
    t_range = np.sum((Xc @ (Vr ** 2)) ** 2) / km1
    dP = 1.0 - (Vr ** 2).sum(axis=1)
    t_A = np.sum((Xc @ dP) ** 2) / km1
    t_B2 = np.sum((Xc @ Vr) ** 2) / km1
    G_tens = np.einsum("ja,al,an->jln", Xc, Vr, Vr)
    gt2 = np.sum(G_tens ** 2)
    q = m - p
    if variant == "haar":
        h = np.sum(Xc ** 2 * (1.0 - dP)[None, :])
        t_B = tau - 2.0 * h / km1 + gt2 / km1
        t_null = (t_A + 2.0 * t_B) / (q + 2) if q > 0 else 0.0
    else:
        t_B = tau - 2.0 * t_B2 + gt2 / km1
        t_null = (t_A + 2.0 * t_B) / q if q > 0 else 0.0
    kappa = abs(0.5 * (t_range + t_null) + 0.5 * tau)
    return dict(tau=tau, t_range=t_range, t_A=t_A, t_B2=t_B2, gt2=gt2, t_B=t_B, t_null=t_null, kappa=kappa)


def rsvd_eig(G, omega, rank: int, power: int):
    """(U_r, s2_r): the rank largest Ritz pairs of G from the range of G^(power+1) omega."""
    G = np.asarray(G, dtype=np.float64)
    Y = G @ np.asarray(omega, dtype=np.float64)
    for _ in range(power):
        Q, _ = np.linalg.qr(Y)
        Y = G @ Q
    Q, _ = np.linalg.qr(Y)
    B = Q.T @ G @ Q
    B = 0.5 * (B + B.T)
    w, V = np.linalg.eigh(B)
    order = np.argsort(-w)[:rank]
    return Q @ V[:, order], w[order]


def rsvd_patch(Xc, omega, rank: int, power: int, variant: str = "literal") -> float:
    """K of one centred patch with the randomised rank-`rank` SVD; eigenvalues at
    or below k m 2^-52 of the largest are dropped (the exact Fast mode's rule)."""
    Xc = np.asarray(Xc, dtype=np.float64)
    k, m = Xc.shape
    U, s2 = rsvd_eig(Xc @ Xc.T, omega, rank, power)
    keep = s2 > k * m * 2.0 ** -52 * max(s2[0], 0.0)
    return fast_from_eig(Xc, U[:, keep], s2[keep], variant)["kappa"]
