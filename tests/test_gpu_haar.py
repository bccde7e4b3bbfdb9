"""The Fast mode's null-space term on the GPU against its definition.

eq. gnull_exp replaces the null-space eigenvectors that an eigensolver would
return by their expectation under the Haar measure.  So with the range
eigenpairs of a patch fixed and the null-space columns rotated by Haar-random
orthogonal matrices, the mean of Theorem 1's K over the draws (mecuco_exact_kappa
on the GPU) estimates what MECUCO_FAST_HAAR computes; the printed algorithm
(MECUCO_FAST_LITERAL) differs from it by thousands of standard errors.

The relative error of Fast against Exact as D/k grows (the paper's O(p/D)
bias bound, eq. error_bound) is measured on the GPU for both variants."""
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


def _haar(rng, draws, d):
    # QR of a Gaussian matrix with the signs of R's diagonal moved into Q (Mezzadri 2007)
    Q, R = np.linalg.qr(rng.standard_normal((draws, d, d)))
    return Q * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]


def _theorem1(v, W):
    C = np.einsum("dis,dil->dsl", W, W * W)
    return np.abs(0.5 * np.einsum("ds,dsl->d", v, C * C) + 0.5 * v.sum(1))


def test_exact_kappa_on_supplied_bases(ctx):
    rng = np.random.default_rng(0)
    for m in (1, 7, 33, 64):
        W = _haar(rng, 50, m)
        v = rng.gamma(1.0, 1.0, (50, m))
        got = ctx.mecuco_exact_kappa(torch.from_numpy(v), torch.from_numpy(W)).cpu().numpy()
        ref = _theorem1(v.astype(np.float32).astype(np.float64), W.astype(np.float32).astype(np.float64))
        assert rel_err(got, ref).max() < 1e-5


def test_haar_variant_is_the_monte_carlo_mean(ctx, orc):
    m, k = 24, 8
    p = k - 1
    X = synth.sphere(n=600, m=m, seed=4)
    idx, _ = orc.knn(X.astype(np.float64), k)
    Xg, ig = torch.from_numpy(X).cuda(), torch.from_numpy(idx).cuda()
    _, v, W = ctx.mecuco_curvature_exact(Xg, k, idx=ig, return_basis=True)
    fast_h = ctx.mecuco_curvature(Xg, k, idx=ig, variant="haar").cpu().numpy()
    fast_l = ctx.mecuco_curvature(Xg, k, idx=ig, variant="literal").cpu().numpy()
    v, W = v.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(11)
    draws = 65536
    for r in (0, 100, 200, 300):
        Q = _haar(rng, draws, m - p)
        Wd = np.concatenate([np.broadcast_to(W[r][:, :p], (draws, m, p)), W[r][:, p:] @ Q], axis=2)
        vd = np.zeros((draws, m))
        vd[:, :p] = v[r][:p]
        kd = ctx.mecuco_exact_kappa(torch.from_numpy(vd), torch.from_numpy(Wd)).cpu().numpy().astype(np.float64)
        mean, se = kd.mean(), kd.std() / np.sqrt(draws)
        ref_h = orc.fast_patch(orc.center_patch(X.astype(np.float64), idx[r]), variant=orc.HAAR)["kappa"]
        print(f"row {r}: MC mean {mean:.6g} (SE {se / mean:.1e} rel); haar {(fast_h[r] - mean) / se:+.2f} SE, "
              f"literal {(fast_l[r] - mean) / se:+.0f} SE")
        assert abs(fast_h[r] - ref_h) / ref_h < KAPPA_TOL
        assert abs(fast_h[r] - mean) < 4 * se + KAPPA_TOL * mean
        assert abs(fast_l[r] - mean) > 100 * se


def test_fast_vs_exact_error_against_d_over_k(ctx):
    k = 5
    curve = []
    for m in (16, 32, 64):
        X = torch.from_numpy(synth.sphere(n=3000, m=m, seed=1)).cuda()
        idx = ctx.mecuco_knn(X, k)
        ex = ctx.mecuco_curvature_exact(X, k, idx=idx).cpu().numpy().astype(np.float64)
        fl = ctx.mecuco_curvature(X, k, idx=idx, variant="literal").cpu().numpy()
        fh = ctx.mecuco_curvature(X, k, idx=idx, variant="haar").cpu().numpy()
        el, eh = rel_err(fl, ex).mean(), rel_err(fh, ex).mean()
        curve.append((m / k, el, eh))
        print(f"D/k = {m / k:5.1f}: mean relative error literal {el:.4f}, haar {eh:.4f}")
    lit = [c[1] for c in curve]
    assert lit[0] > lit[1] > lit[2]                 # the bias falls as D/k grows
    assert all(c[2] < c[1] for c in curve)          # the Haar expectation is the closer one
