"""Agreement metrics of the paper's curvature-fidelity experiments, in FP64
with NumPy (test infrastructure only, like the rest of this package).

The experiments section compares two curvature vectors (the original method
as reference ``a``, MeCuCo as ``b``) by the mean absolute error, Spearman's
rank correlation rho_S and Chatterjee's xi (Chatterjee, "A new coefficient of
correlation", JASA 2021), and repeats the comparison after each vector is
min-max normalised to [0, 1] ("The Effect of Normalization").

Each function is the definition written out:
    minmax_normalize(x)   (x - min x) / (max x - min x); all zeros when max = min
    mae(a, b)             mean of |a_i - b_i|
    average_ranks(x)      rank 1..n, tied values share the mean of their positions
    spearman(a, b)        Pearson correlation of average_ranks(a) and average_ranks(b)
    chatterjee_xi(a, b)   Chatterjee's xi_n in the form that allows ties (his Eq. 1.2):
                          order the pairs by a (ties in a by index), r_i = #{j: b_j <= b_(i)},
                          l_i = #{j: b_j >= b_(i)},
                          xi = 1 - n sum_{i<n} |r_{i+1} - r_i| / (2 sum_i l_i (n - l_i))
    fidelity(a, b, normalize)   (MAE, rho_S, xi); the ranks of a strictly increasing
                          transform are those of its argument, so rho_S and xi are
                          taken on the raw vectors and only the MAE on normalised ones.

Degenerate cases (readings where the definitions divide by zero): rho_S = 0
when either vector is constant; xi = 0 when b is constant.
"""
from __future__ import annotations

import numpy as np

__all__ = ["minmax_normalize", "mae", "average_ranks", "spearman", "chatterjee_xi", "fidelity"]


def _vec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())


def minmax_normalize(x) -> np.ndarray:
    x = _vec(x)
    lo, hi = x.min(), x.max()
    if hi == lo:
        return np.zeros_like(x)
    return (x - lo) / (hi - lo)


def mae(a, b) -> float:
    a, b = _vec(a), _vec(b)
    return float(np.mean(np.abs(a - b)))


def average_ranks(x) -> np.ndarray:
    """A value with `less` smaller values and `leq` values <= it occupies the
    sorted positions less+1 .. leq; its rank is their mean (less + 1 + leq) / 2."""
    x = _vec(x)
    s = np.sort(x)
    less = np.searchsorted(s, x, side="left")
    leq = np.searchsorted(s, x, side="right")
    return 0.5 * (less + 1 + leq)


def _pearson(u, v) -> float:
    du, dv = u - u.mean(), v - v.mean()
    su, sv = np.sqrt(np.sum(du * du)), np.sqrt(np.sum(dv * dv))
    if su == 0.0 or sv == 0.0:
        return 0.0
    return float(np.sum(du * dv) / (su * sv))


def spearman(a, b) -> float:
    return _pearson(average_ranks(a), average_ranks(b))


def chatterjee_xi(a, b) -> float:
    a, b = _vec(a), _vec(b)
    n = a.size
    order = np.argsort(a, kind="stable")          # pairs by a, equal a by index
    bs = np.sort(b)
    b_ord = b[order]
    r = np.searchsorted(bs, b_ord, side="right")  # #{j: b_j <= b_(i)}
    l = n - np.searchsorted(bs, b_ord, side="left")  # #{j: b_j >= b_(i)}
    num = np.sum(np.abs(np.diff(r)).astype(np.float64))
    den = 2.0 * np.sum(l.astype(np.float64) * (n - l))
    if den == 0.0:
        return 0.0
    return float(1.0 - n * num / den)


def fidelity(a, b, normalize: bool = False):
    """(MAE, rho_S, xi) of b against the reference a."""
    a, b = _vec(a), _vec(b)
    if a.size != b.size or a.size < 2:
        raise ValueError("need two vectors of the same length >= 2")
    ea, eb = (minmax_normalize(a), minmax_normalize(b)) if normalize else (a, b)
    return mae(ea, eb), spearman(a, b), chatterjee_xi(a, b)
