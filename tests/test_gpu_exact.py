"""Exact mode (Theorem 1) on the GPU (mecuco_curvature_exact).  Where the
covariance has a null space the curvature depends on the eigenbasis, so the
GPU value is checked against the oracle's naive H-form evaluated on the GPU's
own basis W (Remark 1: naive = identity on the same W), W against the FP64
covariance, and the bounds tau/2 <= K <= tau; with well-separated spectra and
no null space it is compared with the oracle's Exact mode directly."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

from gpu_helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _anisotropic(n, m, seed):
    # Gaussian cloud with well-separated per-coordinate scales (distinct covariance eigenvalues)
    rng = np.random.default_rng(seed)
    scales = np.linspace(1.0, 0.3, m)
    return (rng.standard_normal((n, m)) * scales).astype(np.float32)


def test_exact_matches_oracle_without_null_space(ctx, orc):
    X = _anisotropic(3000, 12, seed=1)
    k = 40                                   # m = 12 <= k - 1: no null space
    X64 = X.astype(np.float64)
    idx, _ = orc.knn(X64, k)
    kap = ctx.mecuco_curvature_exact(torch.from_numpy(X).cuda(), k, idx=torch.from_numpy(idx).cuda())
    torch.cuda.synchronize()
    rows = np.random.default_rng(0).choice(3000, 64, replace=False)
    ref = orc.curvature(X64, k, idx, rows=rows, mode="exact")
    err = rel_err(kap.cpu().numpy()[rows], ref)
    print(f"exact (no null space): max rel err {err.max():.2e}")
    assert err.max() < KAPPA_TOL


def test_exact_with_null_space_on_own_basis(ctx, orc):
    X = synth.sphere(n=2000, m=32, seed=1)  # C1: m = 32 > k - 1 = 9
    k = 10
    X64 = X.astype(np.float64)
    idx, _ = orc.knn(X64, k)
    kap, v, W = ctx.mecuco_curvature_exact(torch.from_numpy(X).cuda(), k, idx=torch.from_numpy(idx).cuda(),
                                           return_basis=True)
    torch.cuda.synchronize()
    kap, v, W = kap.cpu().numpy(), v.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64)
    worst_k = worst_w = 0.0
    for r in np.random.default_rng(1).choice(2000, 40, replace=False):
        Xc = orc.center_patch(X64, idx[r])
        S = Xc.T @ Xc / (k - 1)
        Wr = W[r]
        assert np.allclose(Wr.T @ Wr, np.eye(32), atol=2e-6)
        resid = np.abs(Wr @ np.diag(v[r]) @ Wr.T - S).max() / np.abs(S).max()
        worst_w = max(worst_w, resid)
        ref = orc.naive_patch(Xc, Wr)          # |tr(-H H^T Sigma)| on the same W
        worst_k = max(worst_k, abs(kap[r] - ref) / ref)
        tau = v[r].sum()
        assert 0.5 * tau * (1 - 1e-5) <= kap[r] <= tau * (1 + 1e-5)
    print(f"exact (null space): K vs naive-on-same-W {worst_k:.2e}, eigen residual {worst_w:.2e}")
    assert worst_k < KAPPA_TOL and worst_w < 1e-5


def test_auto_mode_picks_exact_below_50(ctx):
    X = torch.from_numpy(synth.sphere(n=800, m=32, seed=2)).cuda()
    idx = ctx.mecuco_knn(X, 10)
    a = ctx.curvature_auto(X, 10, idx=idx)
    b = ctx.mecuco_curvature_exact(X, 10, idx=idx)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_exact_row_range_and_computed_neighbours(ctx):
    X = torch.from_numpy(_anisotropic(1500, 20, seed=3)).cuda()
    full = ctx.mecuco_curvature_exact(X, 24)
    part = ctx.mecuco_curvature_exact(X, 24, row_begin=500, row_end=900)
    torch.cuda.synchronize()
    assert torch.equal(full[500:900], part)
