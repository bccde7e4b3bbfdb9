"""Batched entry point (mecuco_curvature_batched): many uneven datasets in one
call must give exactly what one mecuco_curvature call per dataset gives, in
both batched forms (BF16-mixed: one launch per stage over device tables of all
datasets; FP32 or with the persistent form off: stream lanes), match the FP64
oracle on sampled rows, replay identically from a CUDA graph, and keep working
after the autotuner has run."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

from gpu_helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA_TOL = 1e-4


BF16_U = 2.0 ** -9  # unit roundoff of BF16 (8 significand bits, round to nearest)


def bf16_kappa_tol(orc, X64, nb, ref, rng, draws=3):
    """Bound on the BF16-mixed form's relative curvature error at one point.
    That form computes K, up to FP32 accumulation, for a patch whose centred
    entries carry a relative rounding error of at most u = 2^-9 (the BF16
    operands of the Gram and rotation GEMMs) and whose rotated coordinates
    carry another (the BF16 operand of the third-moment GEMM).  How far that
    moves K depends on the patch (small singular values amplify it), so the
    bound is measured with the oracle: K of the centred patch with every entry
    scaled by (1 + 2u xi), xi uniform in [-1, 1] (twice the rounding, standing
    for both roundings), over a few draws; the bound is 4x the largest relative
    change seen, and not below 2e-5."""
    Xc = orc.center_patch(X64, nb)
    worst = 0.0
    for _ in range(draws):
        pert = Xc * (1.0 + 2.0 * BF16_U * rng.uniform(-1.0, 1.0, Xc.shape))
        worst = max(worst, abs(orc.fast_patch(pert)["kappa"] - ref) / abs(ref))
    return max(4.0 * worst, 2e-5)


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


def _sampled_parity(orc, sets, Xs, idx_out, kappas, rows_per_set, rng, precision="fp32"):
    """Largest relative curvature error on sampled rows, as a fraction of the
    precision's bound (fp32: KAPPA_TOL; bf16_mixed: bf16_kappa_tol per row)."""
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
        err = rel_err(kap.cpu().numpy()[rows], ref)
        for r_i, q in enumerate(rows):
            tol = KAPPA_TOL if precision == "fp32" else bf16_kappa_tol(orc, X64, full[q], ref[r_i], rng)
            worst = max(worst, err[r_i] / tol)
    return worst


def _check_against_single_calls(ctx, Xs, ks, kb, idx_out, precision, include_self=False, variant="literal"):
    for X, k, kap, idx in zip(Xs, ks, kb, idx_out):
        ref_idx = ctx.mecuco_knn(X, k, precision=precision, include_self=include_self)
        ref = ctx.mecuco_curvature(X, k, idx=ref_idx, precision=precision, include_self=include_self,
                                   variant=variant)
        assert torch.equal(idx, ref_idx)
        assert torch.equal(kap, ref)


@pytest.mark.parametrize("precision,persistent", [("fp32", 1), ("bf16_mixed", 1), ("bf16_mixed", 0)])
def test_batched_matches_single_calls(ctx, precision, persistent):
    from paper_2606_06329_gb300 import _native as N
    sets = _small_batch()
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    ctx.set_option(N.OPT_BATCH_PERSISTENT, persistent)
    try:
        kb = ctx.mecuco_curvature_batched(Xs, ks, precision=precision, idx_out=idx_out)
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == 0
    finally:
        ctx.set_option(N.OPT_BATCH_PERSISTENT, 1)
    _check_against_single_calls(ctx, Xs, ks, kb, idx_out, precision)


@pytest.mark.parametrize("case", ["bf16_storage", "cta_pairs", "small_chunks", "haar_self"])
def test_one_launch_per_stage_forms(ctx, case):
    """The one-launch-per-stage form over its variants: BF16 storage (rows used
    in place where aligned, copied where m is not a multiple of 8), the kNN as
    CTA pairs, estimator chunks that cut datasets into several segments and
    launches, and the Haar variant with the query among its neighbours."""
    from paper_2606_06329_gb300 import _native as N
    m_choices = (64, 100, 256) if case == "bf16_storage" else (64, 128, 256)
    sets = synth.batched_mlp_datasets(nsets=9, seed=11, n_range=(300, 2200), m_choices=m_choices, k_range=(10, 64))
    dtype = torch.bfloat16 if case == "bf16_storage" else torch.float32
    Xs = [torch.from_numpy(d["X"]).cuda().to(dtype) for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    include_self = case == "haar_self"
    variant = "haar" if case == "haar_self" else "literal"
    opts = {"cta_pairs": (N.OPT_KNN_PAIR, 1, -1), "small_chunks": (N.OPT_CHUNK_POINTS, 700, 0)}.get(case)
    if opts:
        ctx.set_option(opts[0], opts[1])
    try:
        kb = ctx.mecuco_curvature_batched(Xs, ks, precision="bf16_mixed", idx_out=idx_out, include_self=include_self,
                                          variant=variant)
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == 0
        launches = ctx.mecuco_get_stats()["kernel_launches"]
        _check_against_single_calls(ctx, Xs, ks, kb, idx_out, "bf16_mixed", include_self, variant)
    finally:
        if opts:
            ctx.set_option(opts[0], opts[2])
    # output patch; kNN: row norms, (BF16 copy,) search, re-rank, fallback;
    # estimator: 5 per chunk
    if case != "small_chunks":
        assert launches <= 1 + 5 + 5


@pytest.mark.parametrize("precision", ["fp32", "bf16_mixed"])
def test_batched_parity_and_graph_replay(ctx, orc, precision):
    sets = _small_batch(nsets=16, seed=4)
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    eager = ctx.mecuco_curvature_batched(Xs, ks, idx_out=idx_out, precision=precision)
    torch.cuda.synchronize()
    worst = _sampled_parity(orc, sets, Xs, idx_out, eager, 3, np.random.default_rng(0), precision)
    print(f"batched sampled parity ({precision}): max rel err / bound {worst:.2f}")
    assert worst < 1.0
    # the same call captured into a CUDA graph (workspace and tables already exist)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            captured = ctx.mecuco_curvature_batched(Xs, ks, idx_out=idx_out, precision=precision)
    for c in captured:
        c.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, captured):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "bf16_mixed"])
def test_autotune_then_batched(ctx, precision):
    sets = _small_batch(nsets=10, seed=5)
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    before = ctx.mecuco_curvature_batched(Xs, ks, precision=precision)
    tuned = ctx.mecuco_autotune_batched(Xs, ks, precision=precision)
    print(f"autotuned ({precision}): {tuned}")
    assert tuned["ms"] > 0
    if precision == "fp32":
        assert tuned["lanes"] in (1, 2, 4, 8, 16, 32)
    else:
        assert tuned["lanes"] == 1 and tuned["knn_pair"] in (0, 1)
        assert (tuned["tt_ctas"], tuned["tt_slots"]) in ((2, 2), (2, 4), (1, 4), (1, 8))
    after = ctx.mecuco_curvature_batched(Xs, ks, precision=precision)
    torch.cuda.synchronize()
    for a, b in zip(before, after):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "bf16_mixed"])
def test_batched_256_uneven_datasets(ctx, orc, precision):
    """256 datasets, N in [500, 20000], m in {64..1024}, k in [10, 64]."""
    sets = synth.batched_mlp_datasets(nsets=256, seed=1)
    Xs = [torch.from_numpy(d["X"]).cuda() for d in sets]
    ks = [d["k"] for d in sets]
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    kap = ctx.mecuco_curvature_batched(Xs, ks, idx_out=idx_out, precision=precision)
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == 0
    pick = np.random.default_rng(1).choice(256, 12, replace=False)
    worst = _sampled_parity(orc, [sets[i] for i in pick], [Xs[i] for i in pick], [idx_out[i] for i in pick],
                            [kap[i] for i in pick], 2, np.random.default_rng(2), precision)
    print(f"256-set batch sampled parity ({precision}): max rel err / bound {worst:.2f}")
    assert worst < 1.0
    for i in pick[:3]:
        ref_idx = ctx.mecuco_knn(Xs[i], ks[i], precision=precision)
        ref = ctx.mecuco_curvature(Xs[i], ks[i], idx=ref_idx, precision=precision)
        assert torch.equal(idx_out[i], ref_idx)
        assert torch.equal(kap[i], ref)


@pytest.mark.parametrize("dtype,include_self", [("f32", False), ("bf16", False), ("f32", True)])
def test_one_launch_per_stage_edge_datasets(ctx, dtype, include_self):
    """Corners of the batch tables: datasets smaller than one search tile
    (N down to 3), k at its largest for N (N - 1, or N with the query itself),
    m = 1, odd m, m just past a 64-column chunk, and rows whose leading
    dimension exceeds m (views); every dataset must come out as a single call
    gives it, bit for bit."""
    rng = np.random.default_rng(17)
    shapes = [(3, 5, 2), (40, 1, 5), (257, 3, 64), (300, 65, 20), (129, 33, 64), (1000, 130, 17), (64, 8, 63)]
    Xs, ks = [], []
    for n, m, k in shapes:
        if include_self and k == n - 1:
            k = n
        k = min(k, n if include_self else n - 1, 64)
        base = rng.standard_normal((n, m + 3)).astype(np.float32)
        X = torch.from_numpy(base).cuda()[:, :m]  # leading dimension m + 3
        if dtype == "bf16":
            X = X.to(torch.bfloat16)
        Xs.append(X)
        ks.append(k)
    idx_out = [torch.empty((X.shape[0], k), dtype=torch.int32, device="cuda") for X, k in zip(Xs, ks)]
    kb = ctx.mecuco_curvature_batched(Xs, ks, precision="bf16_mixed", include_self=include_self, idx_out=idx_out)
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == 0
    _check_against_single_calls(ctx, Xs, ks, kb, idx_out, "bf16_mixed", include_self)
