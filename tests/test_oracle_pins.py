"""Pins for the FP64 oracle: each check ties the oracle to something other than
itself (a library routine, a second formula from the paper's derivation, a
special case where two modes must agree, an invariant, a Monte Carlo estimate
of the Haar expectation, a closed-form golden patch, brute force).

Paper references: Sec. 3 (Steps 1-5), Sec. 4 (eqs. HHt_final, C_def,
Theorem 1), the Fast-mode subsection (eqs. svd_cov, split, gnull_exp, tnull,
tA, tB, fast_curv) and Alg. 1.
"""
import glob
import os

import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _centered(rng, k, m, scale=1.0):
    x = scale * rng.standard_normal((k, m))
    return x - x.mean(axis=0, keepdims=True)


def _haar(rng, m, d):
    return synth.haar_frame(m, d, rng)


# --------------------------------------------------------------------------
# Step 1: kNN (P1) - brute force against a full sort of numpy distances
# --------------------------------------------------------------------------
def test_knn_matches_full_row_sort(orc):
    rng = np.random.default_rng(11)
    X = rng.standard_normal((400, 9))
    idx, dist = orc.knn(X, 7)
    D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    ref = np.argsort(D, axis=1, kind="stable")[:, :7]
    assert np.array_equal(idx, ref)
    assert np.allclose(dist, np.take_along_axis(D, ref, 1), rtol=1e-13, atol=0)


def test_knn_ties_go_to_lower_index_and_self_flag(orc):
    # integer grid with duplicated points: many exact distance ties
    rng = np.random.default_rng(12)
    base = rng.integers(0, 3, size=(60, 3)).astype(np.float64)
    X = np.concatenate([base, base[:20]], axis=0)
    for include_self in (False, True):
        idx, dist = orc.knn(X, 6, include_self=include_self)
        D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        if not include_self:
            np.fill_diagonal(D, np.inf)
        # lexicographic (distance, index): stable argsort on exact integers
        ref = np.argsort(D, axis=1, kind="stable")[:, :6]
        assert np.array_equal(idx, ref)
    idx, _ = orc.knn(X, 6, rows=[3, 70, 5])
    full, _ = orc.knn(X, 6)
    assert np.array_equal(idx, full[[3, 70, 5]])


# --------------------------------------------------------------------------
# Own eigensolver and SVD routes (P2) - against numpy's LAPACK routines
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 7, 33, 64])
def test_jacobi_eigh_matches_lapack(orc, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, V, sweeps = orc.jacobi_eigh(A)
    assert sweeps > 0
    assert np.allclose(w, np.linalg.eigvalsh(A)[::-1], rtol=0, atol=1e-12 * np.abs(w).max())
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    assert np.abs(A @ V - V * w[None, :]).max() < 1e-12 * np.abs(w).max()


@pytest.mark.parametrize("k,m", [(5, 12), (10, 32), (16, 9), (32, 256)])
def test_svd_routes_agree_with_lapack(orc, k, m):
    rng = np.random.default_rng(k * 1000 + m)
    Xc = _centered(rng, k, m)
    s_ref = np.linalg.svd(Xc, compute_uv=False)
    s, V, _ = orc.svd_hestenes(Xc)
    r = min(k, m)
    assert np.allclose(s[:r], s_ref, rtol=0, atol=1e-12 * s_ref[0])
    assert np.all(s[r:] < 1e-12 * s_ref[0])
    f0 = orc.fast_patch(Xc, route=0, return_v=True)
    f1 = orc.fast_patch(Xc, route=1, return_v=True)
    p = f0["p"]
    assert p == f1["p"] == min(k - 1, m)
    _, _, Vt = np.linalg.svd(Xc, full_matrices=False)
    for Vr in (f0["Vr"], f1["Vr"]):
        cos = np.abs(np.sum(Vr * Vt[:p].T, axis=0))
        assert np.allclose(cos, 1.0, atol=1e-10)
    for t in ("kappa", "t_range", "t_A", "gt2", "t_null"):
        assert f0[t] == pytest.approx(f1[t], rel=1e-10, abs=1e-12)


# --------------------------------------------------------------------------
# Sec. 4: eq. HHt_final (P3) and Theorem 1 = naive form (P4, Remark 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [3, 8, 24, 40])
def test_hht_identity(orc, m):
    rng = np.random.default_rng(100 + m)
    W = _haar(rng, m, m)
    W2 = W ** 2
    ref = 0.5 * W2 @ W2.T + 0.5 * np.eye(m)
    assert np.abs(orc.hht(W) - ref).max() < 1e-13


@pytest.mark.parametrize("k,m", [(6, 12), (10, 32), (40, 20), (8, 40)])
def test_naive_equals_theorem1_same_basis(orc, k, m):
    rng = np.random.default_rng(200 + k + m)
    Xc = _centered(rng, k, m)
    kap, W, v = orc.exact_patch(Xc, return_basis=True)
    naive = orc.naive_patch(Xc, W)
    assert abs(naive - kap) / kap < 1e-12


def test_exact_bounds_half_tau_to_tau(orc):
    # W^{o2} is doubly stochastic, so sum_l C_sl^2 lies in [0, 1]
    rng = np.random.default_rng(7)
    for _ in range(20):
        k, m = rng.integers(3, 12), rng.integers(2, 20)
        Xc = _centered(rng, k, m, scale=rng.uniform(0.1, 10))
        kap = orc.exact_patch(Xc)
        tau = np.sum(Xc ** 2) / (k - 1)
        assert 0.5 * tau * (1 - 1e-12) <= kap <= tau * (1 + 1e-12)


# --------------------------------------------------------------------------
# Fast = Exact special cases (P5)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k,m", [(5, 3), (10, 9), (12, 4)])
def test_fast_equals_exact_without_null_space(orc, k, m):
    rng = np.random.default_rng(300 + k + m)
    Xc = _centered(rng, k, m)
    exact = orc.exact_patch(Xc)
    for variant in (orc.LITERAL, orc.HAAR):
        f = orc.fast_patch(Xc, variant=variant)
        assert f["p"] == m and f["t_null"] == 0.0
        assert f["kappa"] == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("k,m", [(5, 12), (8, 30), (10, 11)])
def test_fast_equals_exact_on_coordinate_subspace(orc, k, m):
    # the patch spans a (k-1)-dimensional coordinate subspace with a full,
    # non-diagonal covariance inside it: C_sl = 0 for every null direction l,
    # t_A = t_B = 0 in both variants, so Fast must equal Exact
    rng = np.random.default_rng(400 + k + m)
    p = k - 1
    support = rng.choice(m, size=p, replace=False)
    Xc = np.zeros((k, m))
    Xc[:, support] = _centered(rng, k, p)
    exact = orc.exact_patch(Xc)
    for variant in (orc.LITERAL, orc.HAAR):
        f = orc.fast_patch(Xc, variant=variant)
        assert f["p"] == p
        assert abs(f["t_A"]) < 1e-12 * f["tau"] and abs(f["t_B"]) < 1e-12 * f["tau"]
        assert f["kappa"] == pytest.approx(exact, rel=1e-11)


def test_diagonal_covariance_gives_tau(orc):
    # axis-aligned patch with distinct variances: W = I, C = I, K = tau
    rng = np.random.default_rng(8)
    k, m = 9, 20
    Xc = np.zeros((k, m))
    cols = rng.choice(m, size=4, replace=False)
    # orthogonal centred columns (rows of a Hadamard-like design)
    H = np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], float)
    design = np.concatenate([H, -H, np.zeros((1, 4))], axis=0)  # 9 x 4, centred
    Xc[:, cols] = design * np.array([3.0, 2.0, 1.5, 0.5])
    tau = np.sum(Xc ** 2) / (k - 1)
    assert orc.exact_patch(Xc) == pytest.approx(tau, rel=1e-12)
    for variant in (orc.LITERAL, orc.HAAR):
        assert orc.fast_patch(Xc, variant=variant)["kappa"] == pytest.approx(tau, rel=1e-12)


# --------------------------------------------------------------------------
# Each Fast term against a second formula from the derivation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k,m", [(6, 14), (10, 32), (20, 64)])
def test_fast_terms_against_derivation(orc, k, m):
    rng = np.random.default_rng(500 + k + m)
    Xc = _centered(rng, k, m)
    for variant in (orc.LITERAL, orc.HAAR):
        f = orc.fast_patch(Xc, variant=variant, return_v=True)
        Vr, p = f["Vr"], f["p"]
        lam = f["lam"][:p]
        q = m - p
        # tau = tr(Sigma)
        assert f["tau"] == pytest.approx(np.sum(Xc ** 2) / (k - 1), rel=1e-12)
        # eq. split: t_range = sum_{s,l in range} lambda_s C_r[s,l]^2, C_r = V_r^T V_r^{o2}
        Cr = Vr.T @ Vr ** 2
        assert f["t_range"] == pytest.approx(np.sum(lam[:, None] * Cr ** 2), rel=1e-11)
        # eq. tA: d_P = diag(P_perp); t_A = d_P^T Sigma d_P
        Sigma = Xc.T @ Xc / (k - 1)
        P = np.eye(m) - Vr @ Vr.T
        dP = np.diag(P)
        assert f["t_A"] == pytest.approx(dP @ Sigma @ dP, rel=1e-10, abs=1e-13)
        # |X_c V_r|_F^2 = (k-1) tau: the literal middle term equals tau
        assert f["t_B2"] == pytest.approx(f["tau"], rel=1e-12)
        # |G_tens|_F^2 = sum_{a,b} (X_c^T X_c)_ab (V_r V_r^T)_ab^2
        R = Vr @ Vr.T
        assert f["gt2"] == pytest.approx(np.sum((Xc.T @ Xc) * R ** 2), rel=1e-11)
        if variant == orc.HAAR:
            # expectation form: t_null^H = [t_A + 2 sum_{ab} Sigma_ab P_ab^2] / (q + 2)
            ref = (dP @ Sigma @ dP + 2 * np.sum(Sigma * P ** 2)) / (q + 2)
            assert f["t_null"] == pytest.approx(ref, rel=1e-10)
            assert f["t_B"] >= -1e-12 * f["tau"]
        else:
            assert f["t_B"] == pytest.approx(f["gt2"] / (k - 1) - f["tau"], rel=1e-10, abs=1e-12)
        kappa = abs(0.5 * (f["t_range"] + f["t_null"]) + 0.5 * f["tau"])
        assert f["kappa"] == pytest.approx(kappa, rel=1e-14)


# --------------------------------------------------------------------------
# eq. gnull_exp (P7): Monte Carlo over Haar null-space bases
# --------------------------------------------------------------------------
def test_haar_expectation_monte_carlo(orc):
    rng = np.random.default_rng(2024)
    k, m = 5, 12
    Xc = _centered(rng, k, m)
    _, s, Vt = np.linalg.svd(Xc)
    p = k - 1
    q = m - p
    Vr = Vt[:p].T
    lam = s[:p] ** 2 / (k - 1)
    N0 = np.linalg.svd(np.eye(m) - Vr @ Vr.T)[0][:, :q]  # basis of null(V_r^T)
    Cr = Vr.T @ Vr ** 2
    t_range = np.sum(lam[:, None] * Cr ** 2)
    tau = lam.sum()
    draws, batch = 400_000, 50_000
    vals = []
    for _ in range(draws // batch):
        g = rng.standard_normal((batch, q, q))
        Q, Rm = np.linalg.qr(g)
        Q = Q * np.sign(np.diagonal(Rm, axis1=1, axis2=2))[:, None, :]
        V0 = np.einsum("aq,dql->dal", N0, Q)
        Crn = np.einsum("as,dal->dsl", Vr, V0 ** 2)
        t_null = np.einsum("s,dsl->d", lam, Crn ** 2)
        vals.append(0.5 * (t_range + t_null) + 0.5 * tau)
    vals = np.concatenate(vals)
    mean, se = vals.mean(), vals.std(ddof=1) / np.sqrt(vals.size)
    haar = orc.fast_patch(Xc, variant=orc.HAAR)["kappa"]
    literal = orc.fast_patch(Xc, variant=orc.LITERAL)["kappa"]
    assert abs(haar - mean) < 4 * se, (haar, mean, se)
    # the algorithm as printed (middle term |X_c V_r|_F^2, denominator m - p)
    # is not the Haar expectation, whose middle term is
    # sum_{j,a} X_c[j,a]^2 (1 - d_P[a]) and whose denominator is m - p + 2
    assert abs(literal - mean) > 20 * se


# --------------------------------------------------------------------------
# Invariants (P6)
# --------------------------------------------------------------------------
def test_translation_permutation_homogeneity(orc):
    rng = np.random.default_rng(9)
    X = synth.sphere(n=300, m=16, seed=3).astype(np.float64)
    idx, _ = orc.knn(X, 10)
    rows = np.arange(0, 300, 7)
    for variant in (orc.LITERAL, orc.HAAR):
        base = orc.curvature(X, 10, idx, rows=rows, variant=variant)
        shift = orc.curvature(X + rng.standard_normal(16) * 5, 10, idx, rows=rows, variant=variant)
        assert np.allclose(shift, base, rtol=1e-9)
        perm = rng.permutation(16)
        permuted = orc.curvature(X[:, perm], 10, idx, rows=rows, variant=variant)
        assert np.allclose(permuted, base, rtol=1e-10)
        scaled = orc.curvature(3.0 * X, 10, idx, rows=rows, variant=variant)
        assert np.allclose(scaled, 9.0 * base, rtol=1e-11)
    # the neighbour lists are unchanged by translation, permutation and scaling
    assert np.array_equal(orc.knn(3.0 * X[:, perm] + 1.0, 10)[0], idx)


def test_rank_deficient_patch_uses_numerical_rank(orc):
    # duplicated rows: rank 3 < k - 1 = 5, so p = 3 (reading of Alg. 1's p)
    rng = np.random.default_rng(10)
    base = rng.standard_normal((4, 10))
    Xp = np.concatenate([base, base[:2]], axis=0)
    Xc = Xp - Xp.mean(0)
    for route in (0, 1):
        f = orc.fast_patch(Xc, route=route)
        assert f["p"] == 3
        assert np.isfinite(f["kappa"])
    assert orc.fast_patch(Xc, route=0)["kappa"] == pytest.approx(orc.fast_patch(Xc, route=1)["kappa"], rel=1e-9)


# --------------------------------------------------------------------------
# Closed-form golden patches
# --------------------------------------------------------------------------
def _read_golden(path):
    rec = {"points": []}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "point":
            rec["points"].append([float(v) for v in vals])
        else:
            rec[key] = float(vals[0])
    rec["points"] = np.array(rec["points"])
    return rec


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "patch_*.txt"))))
def test_golden_patches(orc, path):
    g = _read_golden(path)
    P = g["points"]
    k = int(g["k"])
    assert P.shape == (k, int(g["m"]))
    Xc = orc.center_patch(P, np.arange(k))
    kap, W, v = orc.exact_patch(Xc, return_basis=True)
    assert kap == pytest.approx(g["kappa_exact"], rel=1e-13)
    assert orc.naive_patch(Xc, W) == pytest.approx(g["kappa_naive"], rel=1e-13)
    for route in (0, 1):
        lit = orc.fast_patch(Xc, variant=orc.LITERAL, route=route)
        assert lit["kappa"] == pytest.approx(g["kappa_fast_literal"], rel=1e-13)
        assert lit["tau"] == pytest.approx(g["tau"], rel=1e-13)
        assert orc.fast_patch(Xc, variant=orc.HAAR, route=route)["kappa"] == pytest.approx(
            g["kappa_fast_haar"], rel=1e-13)


# Hand-derived patches with a null space (q > 0) on which t_A, t_B and t_null
# are all non-zero: they fix the null-space combination of Alg. 1 (eq. tnull,
# denominator m - p) and its Haar counterpart (denominator q + 2), term by term,
# including a rank-deficient patch (p = numerical rank < k - 1).
@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "nullspace_*.txt"))),
                         ids=os.path.basename)
def test_golden_null_space_terms(orc, path):
    g = _read_golden(path)
    P = g["points"]
    k, m = int(g["k"]), int(g["m"])
    assert P.shape == (k, m)
    Xc = orc.center_patch(P, np.arange(k))
    # absolute slack for terms that cancel to a small value
    tol = dict(rel=1e-12, abs=1e-11 * g["tau"])
    for route in (0, 1):
        lit = orc.fast_patch(Xc, variant=orc.LITERAL, route=route)
        haar = orc.fast_patch(Xc, variant=orc.HAAR, route=route)
        assert lit["p"] == haar["p"] == int(g["p"])
        for r in (lit, haar):
            assert r["tau"] == pytest.approx(g["tau"], **tol)
            assert r["t_range"] == pytest.approx(g["t_range"], **tol)
            assert r["t_A"] == pytest.approx(g["t_A"], **tol)
            assert r["t_B2"] == pytest.approx(g["t_B2"], **tol)
            assert r["gt2"] == pytest.approx(g["gtens_sq"], **tol)
        assert lit["t_B"] == pytest.approx(g["literal_t_B"], **tol)
        assert lit["t_null"] == pytest.approx(g["literal_t_null"], **tol)
        assert lit["kappa"] == pytest.approx(g["kappa_fast_literal"], **tol)
        assert haar["t_B"] == pytest.approx(g["haar_t_B"], **tol)
        assert haar["t_null"] == pytest.approx(g["haar_t_null"], **tol)
        assert haar["kappa"] == pytest.approx(g["kappa_fast_haar"], **tol)
        # the two variants must differ here, or the fixture pins nothing
        assert abs(lit["kappa"] - haar["kappa"]) > 0.1 * g["tau"]
    if "kappa_exact" in g:
        assert orc.exact_patch(Xc) == pytest.approx(g["kappa_exact"], rel=1e-12)
    # the same patch as one point's neighbourhood of the dataset-level loop
    # (every point is its own neighbour's patch when the k points are all of X)
    ref = orc.curvature(P, k, np.tile(np.arange(k, dtype=np.int32), (k, 1)), variant=orc.LITERAL)
    assert np.allclose(ref, g["kappa_fast_literal"], rtol=1e-12, atol=1e-11 * g["tau"])


# --------------------------------------------------------------------------
# Reference gradient (P8): central differences are O(h^2)
# --------------------------------------------------------------------------
def test_fd_gradient_is_second_order(orc):
    X = synth.mlp_decoder(n=120, m=12, latent=3, seed=5).astype(np.float64)
    k = 6
    idx, _ = orc.knn(X, k)
    rng = np.random.default_rng(3)
    coords = np.stack([rng.integers(0, 120, 12), rng.integers(0, 12, 12)], axis=1)
    scale = np.sqrt(np.mean(X ** 2))
    g1 = orc.grad_fd(X, k, idx, coords, 1e-4 * scale)
    g2 = orc.grad_fd(X, k, idx, coords, 0.5e-4 * scale)
    g3 = orc.grad_fd(X, k, idx, coords, 0.25e-4 * scale)
    # successive differences shrink ~4x (second-order) until rounding takes over
    d12, d23 = np.abs(g1 - g2), np.abs(g2 - g3)
    big = d12 > 1e-7 * (np.abs(g2) + 1)
    assert np.all(d23[big] < 0.4 * d12[big])
    assert np.allclose(g2, g3, rtol=1e-4, atol=1e-8)


# --------------------------------------------------------------------------
# Conditioning floor (P9): spread of K under 1e-7 relative input noise
# --------------------------------------------------------------------------
def test_conditioning_floor_sphere(orc):
    X = synth.sphere(n=600, m=32, seed=1).astype(np.float64)
    k = 10
    idx, _ = orc.knn(X, k)
    rows = np.arange(0, 600, 5)
    base = orc.curvature(X, k, idx, rows=rows)
    rng = np.random.default_rng(4)
    rms = np.sqrt(np.mean(X ** 2))
    pert = orc.curvature(X + 1e-7 * rms * rng.standard_normal(X.shape), k, idx, rows=rows)
    spread = np.max(np.abs(pert - base) / base)
    # FP32 parity is judged at 1e-4 relative; the estimator itself must be far
    # better conditioned than that on this workload
    assert spread < 1e-4
