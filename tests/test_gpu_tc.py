"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) candidate search:
after the exact re-rank its neighbour lists must equal the FP64 brute force
(tie rule as for the plain path), with the candidate margin certified for
every row (no row may need the exact full-scan fallback on these inputs, which
would mask a wrong distance GEMM)."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

from gpu_helpers import knn_mismatches, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _bf16(bits):
    return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16)


def _check(ctx, orc, Xt, X64, k, rows=None, max_uncert=0):
    Xd = Xt.cuda()
    idx = ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
    torch.cuda.synchronize()
    st = ctx.mecuco_get_stats()
    assert ctx.mecuco_get_last_status() == 0
    idx = idx.cpu().numpy()
    ref_idx, ref_d = orc.knn(X64, k, rows=rows)
    got = idx if rows is None else idx[rows]
    assert knn_mismatches(X64, got, ref_idx, ref_d, rows=rows) == []
    assert st["knn_uncertified"] <= max_uncert, st
    assert st["knn_fallback_rows"] == st["knn_uncertified"]
    return idx


@pytest.mark.parametrize("n,m,k", [(1000, 128, 8), (1037, 200, 16), (300, 64, 64), (700, 4096, 32)])
def test_tc_knn_bf16_storage(ctx, orc, n, m, k):
    bits = synth.curved_patches(n=n, m=m, n_patches=3, seed=n + m)
    _check(ctx, orc, _bf16(bits), synth.bf16_bits_to_f32(bits).astype(np.float64), k)


def test_tc_knn_fp32_input_small_m(ctx, orc):
    X = synth.sphere(n=2000, m=32, seed=1)
    _check(ctx, orc, torch.from_numpy(X), X.astype(np.float64), 10)


@pytest.mark.parametrize("split", [1, 0])
def test_tc_knn_sparse_clusters(ctx, orc, split):
    """FP32 rows through the tensor-core search, as the three-term BF16 split
    (default) and as one rounding: the lists are the oracle's either way.  One
    rounding perturbs d~ by ~1e-2 here and its a-priori bound leaves rows
    uncertified (the exact scan re-solves them); the split's bound is ~2^8
    smaller and certifies all but a few."""
    from paper_2606_06329_gb300 import _native as N
    X = synth.sparse_clusters(n=6000, m=784, seed=2)
    ctx.set_option(N.OPT_KNN_SPLIT_BF16, split)
    try:
        _check(ctx, orc, torch.from_numpy(X), X.astype(np.float64), 50, max_uncert=6 if split else 6000)
        print(f"split={split}: uncertified {ctx.mecuco_get_stats()['knn_uncertified']} of 6000")
    finally:
        ctx.set_option(N.OPT_KNN_SPLIT_BF16, 1)


@pytest.mark.parametrize("n,m,k", [(1037, 200, 16), (700, 4096, 32), (3000, 256, 64)])
def test_tc_knn_cta_pairs(ctx, orc, n, m, k):
    # CTA pairs sharing two-SM (cta_group::2) MMAs: the same lists as one CTA
    # per SM, and the oracle's neighbours (n not a multiple of the pair's 256 rows)
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=n, m=m, n_patches=3, seed=n + 2 * m)
    Xd = _bf16(bits).cuda()
    ctx.set_option(N.OPT_KNN_PAIR, 1)
    try:
        pair = _check(ctx, orc, _bf16(bits), synth.bf16_bits_to_f32(bits).astype(np.float64), k)
        pi, pdist = ctx.mecuco_knn(Xd, k, precision="bf16_mixed", return_dist=True)
    finally:
        ctx.set_option(N.OPT_KNN_PAIR, 0)
    si, sdist = ctx.mecuco_knn(Xd, k, precision="bf16_mixed", return_dist=True)
    ctx.set_option(N.OPT_KNN_PAIR, -1)
    assert np.array_equal(pair, si.cpu().numpy())
    assert torch.equal(pi, si) and torch.equal(pdist, sdist)


def test_tc_knn_matches_plain_path(ctx):
    bits = synth.curved_patches(n=20000, m=512, n_patches=8, seed=3)
    Xd = _bf16(bits).cuda()
    a = ctx.mecuco_knn(Xd, 24, precision="bf16_mixed")
    b = ctx.mecuco_knn(Xd, 24, precision="fp32")
    assert torch.equal(a, b)


# BF16-mixed form: the centred values are rounded to BF16 once and each pair
# product once more (unit roundoff u = 2^-9 each), with FP32 accumulation.  K
# is a degree-2 function of the patch, so coherent rounding could move it by
# ~4u = 8e-3; the roundings are independent and average over the k m entries
# of a patch, and the measured error against the FP64 oracle is 5-8e-5 at
# k = 10..64.  The bounds below are ~6x the largest measured value for the
# maximum (a bug moving K by 1e-3 fails) and 1e-4 for the median.
BF16_KAPPA_TOL = 5e-4
BF16_KAPPA_MEDIAN_TOL = 1e-4


def _bf16_mixed_vs_oracle(ctx, orc, bits, k, variant, n_rows=48, seed=0):
    n = bits.shape[0]
    Xd = _bf16(bits).cuda()
    out = ctx.mecuco_curvature(Xd, k, precision="bf16_mixed", variant=variant, return_lambda=True)
    idx = ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == 0
    rows = np.random.default_rng(seed).choice(n, n_rows, replace=False)
    ref, _, ref_lam = orc.curvature(bits, k, idx.cpu().numpy(), rows=rows, return_terms=True,
                                    variant=orc.HAAR if variant == "haar" else orc.LITERAL, bf16_bits=True)
    err = rel_err(out["kappa"].cpu().numpy()[rows], ref)
    print(f"bf16_mixed n={n} m={bits.shape[1]} k={k} {variant}: max rel err {err.max():.3e}, "
          f"median {np.median(err):.3e}")
    assert err.max() < BF16_KAPPA_TOL
    assert np.median(err) < BF16_KAPPA_MEDIAN_TOL
    lam = out["lambda"].cpu().numpy()[rows]
    # first-order eigenvalue shift of a BF16 rounding of the centred entries:
    # ~2u/sqrt(3km) of lambda_0 (~1e-5 here); 10x that as the absolute slack
    assert np.allclose(lam[:, :k - 1], ref_lam[:, :k - 1], rtol=BF16_KAPPA_TOL, atol=1e-4 * ref_lam[:, 0:1])
    return idx, rows


@pytest.mark.parametrize("k,variant", [(32, "literal"), (64, "literal"), (20, "haar"), (10, "literal")])
def test_tc_curvature_bf16_mixed(ctx, orc, k, variant):
    bits = synth.curved_patches(n=3000, m=1024, n_patches=3, seed=5 + k)
    _bf16_mixed_vs_oracle(ctx, orc, bits, k, variant)


def test_tc_curvature_bf16_mixed_headline_shape(ctx, orc):
    # the benchmark's patch shape (m = 4096, k = 64) on 20,000 curved-patch
    # points: the kNN lists of the sampled rows against the FP64 brute force
    # over all points, and K against the oracle on those lists
    bits = synth.curved_patches(n=20000, m=4096, n_patches=8, seed=21)
    idx, rows = _bf16_mixed_vs_oracle(ctx, orc, bits, 64, "literal", n_rows=32, seed=1)
    X64 = synth.bf16_bits_to_f32(bits).astype(np.float64)
    ref_idx, ref_d = orc.knn(bits, 64, rows=rows, bf16_bits=True)
    assert knn_mismatches(X64, idx.cpu().numpy()[rows], ref_idx, ref_d, rows=rows) == []


@pytest.mark.parametrize("precision", ["bf16_mixed", "fp32"])
def test_chunked_launches_give_the_same_results(ctx, orc, precision):
    # query chunks (several kNN launches, each with its own output offsets and
    # reused candidate buffers) and estimator chunks (several moment / Jacobi /
    # estimator rounds) at test size: results bit-identical to one launch each,
    # and the kNN lists equal the FP64 brute force
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=5000, m=512, n_patches=4, seed=31)
    Xd = _bf16(bits).cuda()
    k = 32
    idx0, d0 = ctx.mecuco_knn(Xd, k, precision=precision, return_dist=True)
    kap0 = ctx.mecuco_curvature(Xd, k, precision=precision)
    try:
        ctx.set_option(N.OPT_KNN_QUERY_CHUNK, 1000)
        ctx.set_option(N.OPT_CHUNK_POINTS, 700)
        idx1, d1 = ctx.mecuco_knn(Xd, k, precision=precision, return_dist=True)
        kap1 = ctx.mecuco_curvature(Xd, k, precision=precision)
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == 0
    finally:
        ctx.set_option(N.OPT_KNN_QUERY_CHUNK, 0)
        ctx.set_option(N.OPT_CHUNK_POINTS, 0)
    assert torch.equal(idx0, idx1) and torch.equal(d0, d1)
    assert torch.equal(kap0, kap1)
    X64 = synth.bf16_bits_to_f32(bits).astype(np.float64)
    ref_idx, ref_d = orc.knn(X64, k)
    assert knn_mismatches(X64, idx1.cpu().numpy(), ref_idx, ref_d) == []


@pytest.mark.parametrize("k,variant", [(64, "haar"), (10, "literal")])
def test_tc_moment_slots_do_not_change_results(ctx, k, variant):
    # the row-product operand's TMEM slots (handed between warps in pairs) only
    # change the schedule: every tile accumulates its K chunks in the same
    # order, so kappa is bit-identical for 2, 4, 6 and 8 slots; odd counts are
    # rejected
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=2000, m=1000, n_patches=3, seed=7 + k)
    Xd = _bf16(bits).cuda()
    idx = ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
    outs = []
    try:
        for slots in (2, 4, 6, 8):
            ctx.set_option(N.OPT_TC_SLOTS, slots)
            outs.append(ctx.mecuco_curvature(Xd, k, idx=idx, precision="bf16_mixed", variant=variant))
            torch.cuda.synchronize()
            assert ctx.mecuco_get_last_status() == 0
        for bad in (1, 3, 7, 10):
            with pytest.raises(Exception):
                ctx.set_option(N.OPT_TC_SLOTS, bad)
    finally:
        ctx.set_option(N.OPT_TC_SLOTS, 4)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])



@pytest.mark.parametrize("k,variant", [(64, "literal"), (20, "haar")])
def test_third_moment_pass_schedules_give_the_same_results(ctx, k, variant):
    # the BF16-mixed third-moment pass with 1 or 2 CTAs per SM and 2..8 TMEM
    # slots: the tiles, passes and hand-over change, the sums are formed in a
    # fixed order, so kappa is bit-identical
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=2000, m=1000, n_patches=3, seed=11 + k)
    Xd = _bf16(bits).cuda()
    idx = ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
    outs = []
    try:
        for ctas, slots in ((1, 2), (1, 4), (1, 8), (2, 2), (2, 4)):
            ctx.set_option(N.OPT_TT_CTAS, ctas)
            ctx.set_option(N.OPT_TT_SLOTS, slots)
            outs.append(ctx.mecuco_curvature(Xd, k, idx=idx, precision="bf16_mixed", variant=variant))
            torch.cuda.synchronize()
            assert ctx.mecuco_get_last_status() == 0
        for bad in ((N.OPT_TT_CTAS, 3), (N.OPT_TT_SLOTS, 5)):
            with pytest.raises(Exception):
                ctx.set_option(*bad)
    finally:
        ctx.set_option(N.OPT_TT_CTAS, 2)
        ctx.set_option(N.OPT_TT_SLOTS, 4)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
