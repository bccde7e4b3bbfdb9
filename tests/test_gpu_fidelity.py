"""Agreement metrics on the GPU (mecuco_fidelity, mecuco_minmax_normalize)
against the FP64 oracle on the same FP32 vectors.

Ranks are integers decided by comparisons of the same FP32 values on both
sides, so rho_S and xi agree to FP64 summation-order rounding (1e-10 here).
The raw MAE sums |a_i - b_i| exactly formed in FP64 (rel 1e-12).  Normalised
values are FP32 on the GPU: (x - min) and the division each round by at most
2^-24 relative, so each entry is within 2 * 2^-24 of the FP64 value in [0, 1]
and the normalised MAE within twice that (abs 2.5e-7)."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RANK_TOL = 1e-10
NORM_TOL = 2.5e-7


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def F():
    from oracle import fidelity
    return fidelity


def _pair(n, seed, ties):
    rng = np.random.default_rng(seed)
    a = rng.gamma(2.0, 2.0, n)
    b = a * (1 + 0.2 * rng.standard_normal(n)) + 0.5 * rng.gamma(1.0, 1.0, n)
    if ties:
        a, b = np.round(a, 1), np.round(b, 1)
    return a.astype(np.float32), b.astype(np.float32)


def _check(ctx, F, a, b, normalize):
    got = ctx.mecuco_fidelity(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), normalize=normalize)
    ref = F.fidelity(a, b, normalize=normalize)
    if normalize:
        assert abs(got[0] - ref[0]) < NORM_TOL, (got, ref)
    else:
        assert got[0] == pytest.approx(ref[0], rel=1e-12, abs=0), (got, ref)
    assert abs(got[1] - ref[1]) < RANK_TOL, (got, ref)
    assert abs(got[2] - ref[2]) < RANK_TOL, (got, ref)
    return got


@pytest.mark.parametrize("n", [2, 3, 257, 5 * 2048 + 37, (1 << 20) + 3])
@pytest.mark.parametrize("ties", [False, True])
@pytest.mark.parametrize("normalize", [False, True])
def test_metrics_match_oracle(ctx, F, n, ties, normalize):
    a, b = _pair(n, seed=n + 7 * ties, ties=ties)
    _check(ctx, F, a, b, normalize)


def test_degenerate_inputs(ctx, F):
    a = np.array([0.0, -0.0, 1.0, 2.0, -0.0], np.float32)      # -0 and +0 tie
    b = np.array([3.0, 1.0, -0.0, 0.0, 2.0], np.float32)
    _check(ctx, F, a, b, False)
    const = np.full(1000, 2.5, np.float32)
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    got = _check(ctx, F, x, const, True)
    assert got[1] == 0.0 and got[2] == 0.0
    got = _check(ctx, F, x, x, False)
    assert got[0] == 0.0 and got[1] == pytest.approx(1.0, abs=1e-12)
    assert got[2] == pytest.approx(1 - 3 / 1001, abs=1e-12)
    from paper_2606_06329_gb300._native import MecucoError
    with pytest.raises(MecucoError):
        ctx.mecuco_fidelity(torch.ones(1, device="cuda"), torch.ones(1, device="cuda"))


@pytest.mark.parametrize("n", [1, 1000, (1 << 18) + 5])
def test_minmax_normalize(ctx, F, n):
    x = np.random.default_rng(n).gamma(2.0, 3.0, n).astype(np.float32)
    y = ctx.mecuco_minmax_normalize(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = F.minmax_normalize(x)
    assert np.abs(y.astype(np.float64) - ref).max() <= NORM_TOL
    if n > 1:
        assert y.min() == 0.0 and y.max() == 1.0


def test_fast_against_exact_curvature(ctx, F):
    # the paper's protocol on one synthetic set: Exact mode as reference,
    # Fast mode compared by MAE, rho_S and xi, raw and normalised
    X = torch.from_numpy(synth.sphere(n=4000, m=24, seed=3)).cuda()
    k = 12
    idx = ctx.mecuco_knn(X, k)
    exact = ctx.mecuco_curvature_exact(X, k, idx=idx)
    fast = ctx.mecuco_curvature(X, k, idx=idx)
    torch.cuda.synchronize()
    a, b = exact.cpu().numpy(), fast.cpu().numpy()
    for normalize in (False, True):
        got = _check(ctx, F, a, b, normalize)
        print(f"fast vs exact (normalize={normalize}): MAE {got[0]:.4g} rho_S {got[1]:.4f} xi {got[2]:.4f}")


def test_report_tables(ctx, capsys):
    from paper_2606_06329_gb300 import report
    report.main([])
    out = capsys.readouterr().out
    assert "min-max normalised scores" in out and "D/k" in out
    with capsys.disabled():
        print(out)
