"""Tangent bases (mecuco_tangent_basis) against the FP64 oracle's right
singular vectors V_r of each patch (Alg. 1 SVD_p): subspace projectors must
agree, and single columns wherever their singular value is well separated."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROJ_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _oracle_basis(orc, X64, idx, row):
    Xc = orc.center_patch(X64, idx[row])
    out = orc.fast_patch(Xc, return_v=True)
    return Xc, out["Vr"], out["lam"][:out["p"]]


def _check(ctx, orc, X, k, d_out, rows, row_begin=0):
    n, m = X.shape
    X64 = X.astype(np.float64)
    idx, _ = orc.knn(X64, k)
    Xd = torch.from_numpy(X).cuda()
    idd = torch.from_numpy(idx).cuda()
    V = ctx.mecuco_tangent_basis(Xd, k, idd, d_out, row_begin=row_begin).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert V.shape == (n - row_begin, m, d_out)
    worst_proj = worst_col = 0.0
    for r in rows:
        Xc, Vo, lam = _oracle_basis(orc, X64, idx, r)
        Vg = V[r - row_begin]
        d = min(d_out, Vo.shape[1])
        # orthonormal columns
        assert np.allclose(Vg[:, :d].T @ Vg[:, :d], np.eye(d), atol=1e-4)
        # the subspace: compare projectors where the d-th gap separates it
        if d == Vo.shape[1] or lam[d - 1] > 1.01 * lam[d]:
            Pg = Vg[:, :d] @ Vg[:, :d].T
            Po = Vo[:, :d] @ Vo[:, :d].T
            worst_proj = max(worst_proj, np.abs(Pg - Po).max())
        # single columns with a separated singular value, sign by the convention
        for l in range(d):
            lo = lam[l + 1] if l + 1 < len(lam) else 0.0
            hi = lam[l - 1] if l > 0 else np.inf
            if lam[l] < 1.01 * lo or hi < 1.01 * lam[l]:
                continue
            u = Xc @ Vo[:, l]
            j = int(np.argmax(np.abs(u)))
            vo = Vo[:, l] * (1.0 if u[j] > 0 else -1.0)
            worst_col = max(worst_col, np.abs(Vg[:, l] - vo).max())
    return worst_proj, worst_col


def test_basis_sphere(ctx, orc):
    X = synth.sphere(n=2000, m=32, seed=1)
    rows = np.random.default_rng(0).choice(2000, 40, replace=False)
    for d_out in (2, 9):
        wp, wc = _check(ctx, orc, X, 10, d_out, rows)
        print(f"basis sphere d_out={d_out}: projector {wp:.2e}, columns {wc:.2e}")
        assert wp < PROJ_TOL and wc < 1e-3


def test_basis_mlp_decoder_row_range(ctx, orc):
    X = synth.mlp_decoder(n=6000, m=256, seed=2)
    rows = np.random.default_rng(1).choice(np.arange(1000, 6000), 24, replace=False)
    wp, wc = _check(ctx, orc, X, 32, 10, rows, row_begin=1000)
    print(f"basis mlp_decoder d_out=10: projector {wp:.2e}, columns {wc:.2e}")
    assert wp < PROJ_TOL and wc < 1e-3


def test_basis_rejects_bad_width(ctx):
    from paper_2606_06329_gb300 import _native as N
    X = torch.from_numpy(synth.sphere(n=200, m=32, seed=2)).cuda()
    idx = ctx.mecuco_knn(X, 10)
    for bad in (0, 10):
        with pytest.raises(N.MecucoError):
            ctx.mecuco_tangent_basis(X, 10, idx, bad)
