"""Pins of the randomised-SVD oracle (oracle/rsvd.py): the Fast terms from
given eigenpairs against the C oracle's Fast mode (its own Jacobi SVD), the
range finder with a sketch spanning the Gram's range against the exact
truncated SVD, convergence of the power iterations to the exact rank-r
truncation, and the printed t_B2 (not tau) for Ritz vectors."""
import numpy as np
import pytest

from oracle import rsvd as R


def _patch(rng, k, m, d=4, noise=1e-2):
    # k points near a curved d-dimensional patch in R^m: a clear spectral gap after d + 1
    u = rng.standard_normal((k, d))
    h = 0.5 * np.sum(u ** 2, axis=1, keepdims=True) * 0.3
    Q, _ = np.linalg.qr(rng.standard_normal((m, d + 1)))
    X = np.concatenate([u, h], axis=1) @ Q.T + noise * rng.standard_normal((k, m))
    return X - X.mean(axis=0)


@pytest.mark.parametrize("variant", ["literal", "haar"])
def test_fast_from_exact_eigenpairs_matches_c_oracle(orc, variant):
    rng = np.random.default_rng(0)
    for k, m in ((10, 32), (16, 40), (24, 100)):
        Xc = _patch(rng, k, m)
        w, V = np.linalg.eigh(Xc @ Xc.T)
        order = np.argsort(-w)[:k - 1]
        got = R.fast_from_eig(Xc, V[:, order], w[order], variant)
        ref = orc.fast_patch(Xc, variant=orc.HAAR if variant == "haar" else orc.LITERAL)
        for t in ("tau", "t_range", "t_A", "t_B2", "t_B", "t_null", "kappa"):
            assert got[t] == pytest.approx(ref[t], rel=1e-9, abs=1e-12 * abs(ref["tau"])), t


@pytest.mark.parametrize("variant", ["literal", "haar"])
def test_full_sketch_equals_exact_fast(orc, variant):
    rng = np.random.default_rng(1)
    for k, m in ((12, 50), (20, 64)):
        Xc = _patch(rng, k, m)
        omega = rng.standard_normal((k, k))
        got = R.rsvd_patch(Xc, omega, k - 1, 0, variant)
        ref = orc.fast_patch(Xc, variant=orc.HAAR if variant == "haar" else orc.LITERAL)["kappa"]
        assert got == pytest.approx(ref, rel=1e-8)


def test_power_iterations_converge_to_exact_rank_r():
    rng = np.random.default_rng(2)
    k, m, d = 24, 80, 4
    Xc = _patch(rng, k, m, d=d, noise=1e-3)
    r = d + 1
    w, V = np.linalg.eigh(Xc @ Xc.T)
    order = np.argsort(-w)[:r]
    exact = R.fast_from_eig(Xc, V[:, order], w[order])["kappa"]
    omega = rng.standard_normal((k, r + 4))
    errs = [abs(R.rsvd_patch(Xc, omega, r, q) - exact) / exact for q in (0, 1, 3, 8)]
    assert errs[-1] < 1e-10
    assert errs[0] >= errs[-1]


def test_ritz_vectors_use_printed_t_b2():
    # with a coarse sketch the Ritz vectors are not eigenvectors of G: |X_c V_r|^2 / (k-1) != tau
    rng = np.random.default_rng(3)
    k, m = 20, 60
    Xc = _patch(rng, k, m, d=6, noise=0.05)
    U, s2 = R.rsvd_eig(Xc @ Xc.T, rng.standard_normal((k, 5)), 4, 0)
    t = R.fast_from_eig(Xc, U, s2)
    assert abs(t["t_B2"] - t["tau"]) > 1e-6 * t["tau"]
    # and for exact eigenpairs the two agree
    w, V = np.linalg.eigh(Xc @ Xc.T)
    order = np.argsort(-w)[:4]
    t = R.fast_from_eig(Xc, V[:, order], w[order])
    assert t["t_B2"] == pytest.approx(t["tau"], rel=1e-12)
