"""Pins of the agreement-metric oracle (oracle/fidelity.py): library routines
(scipy.stats.spearmanr, rankdata, chatterjeexi) on the cases where they share
the definition, closed forms for monotone pairs, and brute force over pairs on
tiny inputs with ties."""
import numpy as np
import pytest

from oracle import fidelity as F

stats = pytest.importorskip("scipy.stats")


def _brute_avg_ranks(x):
    # rank = mean of the 1-based positions its value takes in the sorted vector
    s = sorted(x)
    return np.array([np.mean([p + 1 for p, v in enumerate(s) if v == xi]) for xi in x])


def _brute_xi(a, b):
    n = len(a)
    order = sorted(range(n), key=lambda i: (a[i], i))
    r = [sum(1 for j in range(n) if b[j] <= b[i]) for i in order]
    l = [sum(1 for j in range(n) if b[j] >= b[i]) for i in order]
    num = sum(abs(r[i + 1] - r[i]) for i in range(n - 1))
    den = 2 * sum(li * (n - li) for li in l)
    return 1.0 - n * num / den


def test_minmax_and_mae_by_hand():
    assert np.array_equal(F.minmax_normalize([2.0, 4.0, 6.0, 3.0]), [0.0, 0.5, 1.0, 0.25])
    assert np.array_equal(F.minmax_normalize([5.0, 5.0, 5.0]), [0.0, 0.0, 0.0])
    assert F.mae([1.0, 2.0, 3.0], [1.5, 1.0, 3.0]) == pytest.approx(0.5)


def test_average_ranks_against_rankdata_and_brute_force():
    rng = np.random.default_rng(0)
    x = rng.integers(0, 7, 40).astype(np.float64)      # many ties
    assert np.array_equal(F.average_ranks(x), stats.rankdata(x, method="average"))
    assert np.array_equal(F.average_ranks(x), _brute_avg_ranks(list(x)))
    assert np.array_equal(F.average_ranks([0.0, -0.0, 1.0]), [1.5, 1.5, 3.0])


@pytest.mark.parametrize("ties", [False, True])
def test_spearman_against_scipy(ties):
    rng = np.random.default_rng(1)
    n = 5000
    a = rng.standard_normal(n)
    b = a + 0.7 * rng.standard_normal(n)
    if ties:
        a, b = np.round(a, 1), np.round(b, 1)
    ref = stats.spearmanr(a, b).statistic
    assert F.spearman(a, b) == pytest.approx(ref, abs=1e-13)


def test_spearman_monotone_closed_forms():
    x = np.random.default_rng(2).standard_normal(300)
    assert F.spearman(x, np.exp(x)) == pytest.approx(1.0, abs=1e-14)
    assert F.spearman(x, -x ** 3) == pytest.approx(-1.0, abs=1e-14)
    assert F.spearman(x, np.full_like(x, 3.0)) == 0.0


@pytest.mark.parametrize("b_ties", [False, True])
def test_xi_against_scipy_without_ties_in_a(b_ties):
    if not hasattr(stats, "chatterjeexi"):
        pytest.skip("scipy without chatterjeexi")
    rng = np.random.default_rng(3)
    n = 4000
    a = rng.standard_normal(n)                              # continuous: no ties in a
    b = np.sin(3 * a) + 0.3 * rng.standard_normal(n)
    if b_ties:
        b = np.round(b, 1)
    ref = stats.chatterjeexi(a, b, y_continuous=False).statistic
    assert F.chatterjee_xi(a, b) == pytest.approx(ref, abs=1e-13)


def test_xi_closed_forms():
    # b a strictly monotone function of a: r_i = i (or n + 1 - i), no ties,
    # so xi = 1 - 3 (n - 1) / (n^2 - 1) = 1 - 3 / (n + 1) for either direction
    n = 101
    a = np.random.default_rng(4).permutation(n).astype(np.float64)
    assert F.chatterjee_xi(a, 2 * a + 1) == pytest.approx(1 - 3 / (n + 1), abs=1e-14)
    assert F.chatterjee_xi(a, -a) == pytest.approx(1 - 3 / (n + 1), abs=1e-14)
    assert F.chatterjee_xi(a, np.ones(n)) == 0.0
    # xi is not symmetric: b = a^2 on a symmetric grid is a function of a, not a of b
    g = np.linspace(-1, 1, 201)
    assert F.chatterjee_xi(g, g ** 2) > 0.95
    assert F.chatterjee_xi(g ** 2, g) < 0.2


def test_xi_brute_force_with_ties_in_both():
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(2, 14))
        a = list(rng.integers(0, 4, n).astype(float))
        b = list(rng.integers(0, 3, n).astype(float))
        if len(set(b)) == 1:
            continue
        assert F.chatterjee_xi(a, b) == pytest.approx(_brute_xi(a, b), abs=1e-14)


def test_fidelity_normalisation_changes_only_mae():
    rng = np.random.default_rng(6)
    a = rng.gamma(2.0, 3.0, 1000)
    b = 0.5 * a + rng.gamma(1.0, 1.0, 1000)
    m0, r0, x0 = F.fidelity(a, b)
    m1, r1, x1 = F.fidelity(a, b, normalize=True)
    assert (r0, x0) == (r1, x1)
    assert m0 == pytest.approx(np.mean(np.abs(a - b)))
    na = (a - a.min()) / (a.max() - a.min())
    nb = (b - b.min()) / (b.max() - b.min())
    assert m1 == pytest.approx(np.mean(np.abs(na - nb)), rel=1e-14)


def test_planted_mistakes_are_caught():
    # each plausible slip in xi (strict < for r, l from <=, dropping the n factor)
    # moves the value on a tied example by far more than rounding
    a = [0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0]
    b = [1.0, 0.0, 1.0, 2.0, 1.0, 2.0, 0.0, 2.0]
    good = _brute_xi(a, b)
    n = len(a)
    r_strict = [sum(1 for j in range(n) if b[j] < b[i]) for i in range(n)]
    num = sum(abs(r_strict[i + 1] - r_strict[i]) for i in range(n - 1))
    l = [sum(1 for j in range(n) if b[j] >= b[i]) for i in range(n)]
    bad = 1 - n * num / (2 * sum(li * (n - li) for li in l))
    assert abs(bad - good) > 1e-3
    assert F.chatterjee_xi(a, b) == pytest.approx(good, abs=1e-14)
