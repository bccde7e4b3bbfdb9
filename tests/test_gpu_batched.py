"""Batched entry point (mecuco_curvature_batched): many uneven datasets in one
call must give exactly what one mecuco_curvature call per dataset gives, match
the FP64 oracle on sampled rows, replay identically from a CUDA graph, and
keep working after the lane-count autotuner has run."""
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


def _small_batch(nsets=12, seed=3):
    return synth.batched_mlp_datasets(nsets=nsets, seed=seed, n_range=(300, 2500), m_choices=(64, 128, 256),
                                      k_range=(10, 40))


def _sampled_parity(orc, sets, Xs, idx_out, kappas, rows_per_set, rng):
    worst = 0.0
    for d, X, idx, kap in zip(sets, Xs, idx_out, kappas):
        n = X.shape[0]
        rows = rng.choice(n, min(rows_per_set, n), replace=False)
        X64 = d["X"].astype(np.float64)
        ref_idx, _ = orc.knn(X64, d["k"], rows=rows)
        assert np.array_equal(idx.cpu().numpy()[rows], ref_idx)
        full = np.zeros((n, d["k"]), dtype=np.int32)
        full[rows] = ref_idx
        ref = orc.curvature(X64, d["k"], full, rows=rows)
        worst = max(worst, rel_err(kap.cpu().numpy()[rows], ref).max())
    return worst


@pytest.mark.parametrize("precision", ["fp32", "bf16_mixed"])
def test_batched_matches_single_calls(ctx, precision):
    sets = _small_batch()
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    kb = ctx.mecuco_curvature_batched(Xs, ks, precision=precision, idx_out=idx_out)
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == 0
    for X, k, kap, idx in zip(Xs, ks, kb, idx_out):
        ref_idx = ctx.mecuco_knn(X, k, precision=precision)
        ref = ctx.mecuco_curvature(X, k, idx=ref_idx, precision=precision)
        assert torch.equal(idx, ref_idx)
        assert torch.equal(kap, ref)


def test_batched_parity_and_graph_replay(ctx, orc):
    sets = _small_batch(nsets=16, seed=4)
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    eager = ctx.mecuco_curvature_batched(Xs, ks, idx_out=idx_out)
    torch.cuda.synchronize()
    worst = _sampled_parity(orc, sets, Xs, idx_out, eager, 3, np.random.default_rng(0))
    print(f"batched sampled parity: max rel err {worst:.2e}")
    assert worst < KAPPA_TOL
    # the same call captured into a CUDA graph (workspace and tables already exist)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            captured = ctx.mecuco_curvature_batched(Xs, ks, idx_out=idx_out)
    for c in captured:
        c.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, captured):
        assert torch.equal(a, b)


def test_autotune_then_batched(ctx):
    sets = _small_batch(nsets=10, seed=5)
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    before = ctx.mecuco_curvature_batched(Xs, ks)
    lanes = ctx.mecuco_autotune_batched(Xs, ks)
    assert lanes in (1, 2, 4, 8, 16, 32)
    after = ctx.mecuco_curvature_batched(Xs, ks)
    torch.cuda.synchronize()
    print(f"autotuned lanes: {lanes}")
    for a, b in zip(before, after):
        assert torch.equal(a, b)


def test_batched_256_uneven_datasets(ctx, orc):
    """256 datasets, N in [500, 20000], m in {64..1024}, k in [10, 64]."""
    sets = synth.batched_mlp_datasets(nsets=256, seed=1)
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    kap = ctx.mecuco_curvature_batched(Xs, ks, idx_out=idx_out)
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == 0
    pick = np.random.default_rng(1).choice(256, 12, replace=False)
    worst = _sampled_parity(orc, [sets[i] for i in pick], [Xs[i] for i in pick], [idx_out[i] for i in pick],
                            [kap[i] for i in pick], 2, np.random.default_rng(2))
    print(f"256-set batch sampled parity: max rel err {worst:.2e}")
    assert worst < KAPPA_TOL
    for i in pick[:3]:
        ref = ctx.mecuco_curvature(Xs[i], ks[i], idx=idx_out[i])
        assert torch.equal(kap[i], ref)
