"""A host-side check of the a-priori rounding bound in the kNN certificate
(csrc/knn_simt.cu, knn_rerank_kernel; the rounding terms come from
row_norm_warp).

For FP32 rows the tensor-core search multiplies BF16 copies: with one
rounding (x = h + d, h = bf16(x)) it forms h_x . h_y; with the three-term
split (x = h + l + r, l = bf16(x - h)) the query copy [h | h | l] against the
candidate copy [h | l | h] forms h_x.h_y + h_x.l_y + l_x.h_y.  The certificate
bounds what that leaves out, for any candidate y of the dataset, by
Cauchy-Schwarz with the query's |x| and rounding-term norms and the dataset's
largest |y| and rounding-term norms:
    single:  (|x| + t1) m1 + t1 (|y|max + m1) + t1 m1
    split:   t1 m1 + (|x| + t2) m2 + t2 (|y|max + m2) + t2 m2
(t1, t2 the query's |d| or |l|, |r|, each raised by 2^-10; m1, m2 the largest
of those over the dataset).  Here the omitted part is computed exactly
(FP64, math.fsum) for random, wide-range, sparse and aligned-residual
vectors and must never exceed the bound; the bound is tight (over 90 % of it
is reached) and a bound with one of its leading terms dropped is caught.  The
FP32 accumulation of the search is covered separately (by the certificate's
estimate from the candidates) and is not modelled here."""
import math

import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

UP = 1.0 + 2.0 ** -10


def _bf16(x):
    return synth.bf16_bits_to_f32(synth.f32_to_bf16_bits(np.asarray(x, np.float32)))


def _terms(x):
    """h, l, r of the three-term split in the kernel's FP32 arithmetic (d = x - h = l + r)."""
    x = np.asarray(x, np.float32)
    h = _bf16(x)
    d = (x - h).astype(np.float32)  # exact in FP32
    l = _bf16(d)
    r = (d - l).astype(np.float32)  # exact in FP32
    return h, d, l, r


def _norm_up(v):
    return math.sqrt(math.fsum(float(a) * float(a) for a in v)) * UP


def _dot(a, b):
    return math.fsum(float(p) * float(q) for p, q in zip(a, b))  # products exact in FP64


def _bound(quant, x, Y, drop=None):
    xq = math.sqrt(_dot(x, x))
    ym = max(math.sqrt(_dot(y, y)) for y in Y)
    if quant == "single":
        t1 = _norm_up(_terms(x)[1])
        m1 = max(_norm_up(_terms(y)[1]) for y in Y)
        parts = [(xq + t1) * m1, t1 * (ym + m1), t1 * m1]
    else:
        _, _, lx, rx = _terms(x)
        t1, t2 = _norm_up(lx), _norm_up(rx)
        m1 = max(_norm_up(_terms(y)[2]) for y in Y)
        m2 = max(_norm_up(_terms(y)[3]) for y in Y)
        parts = [t1 * m1, (xq + t2) * m2, t2 * (ym + m2), t2 * m2]
    if drop is not None:
        parts.pop(drop)
    return sum(parts)


def _omitted(quant, x, y):
    """x.y minus what the search's BF16 products form, exactly."""
    hx, _, lx, _ = _terms(x)
    hy, _, ly, _ = _terms(y)
    full = _dot(x, y)
    if quant == "single":
        return full - _dot(hx, hy)
    return full - math.fsum([_dot(hx, hy), _dot(hx, ly), _dot(lx, hy)])


def _cases(rng, m):
    g = rng.standard_normal((6, m)).astype(np.float32)
    wide = (rng.standard_normal((6, m)) * 10.0 ** rng.uniform(-6, 6, (6, m))).astype(np.float32)
    sparse = np.clip(0.2 + 0.3 * rng.standard_normal((6, m)), 0.0, 1.0).astype(np.float32)
    # aligned residuals: values just below the BF16 halfway points, so every
    # rounding term has the same sign; and a candidate equal to the query
    base = _bf16(rng.uniform(1.0, 2.0, m))
    ulp = (np.float32(2.0) ** (np.floor(np.log2(np.abs(base))) - 7)).astype(np.float32)
    aligned = np.stack([base + np.float32(0.4999) * ulp, base - np.float32(0.4999) * ulp,
                        base + np.float32(0.25) * ulp]).astype(np.float32)
    return [g, wide, sparse, aligned]


@pytest.mark.parametrize("quant", ["single", "split"])
@pytest.mark.parametrize("m", [7, 64, 784])
def test_rounding_bound_covers_the_omitted_products(quant, m):
    rng = np.random.default_rng(m)
    for Y in _cases(rng, m):
        for x in list(Y) + [Y[0] * np.float32(3.0)]:
            b = _bound(quant, x, Y)
            for y in Y:
                assert abs(_omitted(quant, x, y)) <= b


@pytest.mark.parametrize("quant,leading", [("single", (0, 1)), ("split", (0, 1, 2))])
def test_bound_is_tight_and_its_leading_terms_are_needed(quant, leading):
    """On aligned residuals with y = x (where Cauchy-Schwarz is tight) the
    omitted part reaches over 90 % of the bound, and without any one of the
    leading terms (order 2^-9 |x||y| for one rounding, 2^-18 for the split)
    some case escapes.  The last term, of the next order, is covered by the
    slack of |h| <= |x| + |d| in the others."""
    rng = np.random.default_rng(11)
    cases = _cases(rng, 64)
    worst = max(abs(_omitted(quant, x, y)) / _bound(quant, x, Y) for Y in cases for x in Y for y in Y)
    assert 0.9 < worst <= 1.0
    for drop in leading:
        escaped = any(abs(_omitted(quant, x, y)) > _bound(quant, x, Y, drop=drop)
                      for Y in cases for x in Y for y in Y)
        assert escaped, f"term {drop} of the {quant} bound is never needed"
