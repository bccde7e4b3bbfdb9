"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, plain FP32
form.  kNN lists must match the FP64 brute force exactly except where two
distances agree within 1e-6 relative; curvature must match within 1e-4
relative (the FP32 tolerance of the target), on the same seeded inputs."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

from gpu_helpers import knn_mismatches, rel_err

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


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _run(ctx, X, k, variant="literal", include_self=False, idx=None):
    Xd = _dev(X)
    if idx is None:
        idx_d = ctx.mecuco_knn(Xd, k, include_self=include_self)
    else:
        idx_d = _dev(idx.astype(np.int32))
    out = ctx.mecuco_curvature(Xd, k, idx=idx_d, include_self=include_self, variant=variant,
                               return_lambda=True)
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == 0
    return idx_d.cpu().numpy(), out["kappa"].cpu().numpy(), out["lambda"].cpu().numpy()


def _as64(X):
    if X.dtype == np.uint16:
        return synth.bf16_bits_to_f32(X).astype(np.float64)
    return X.astype(np.float64)


# --------------------------------------------------------------------------
# Sphere in R^32, N=2000, k=10: every row, both variants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["literal", "haar"])
def test_sphere_full_parity(ctx, orc, variant):
    X = synth.sphere(n=2000, m=32, seed=1)
    k = 10
    X64 = _as64(X)
    ref_idx, ref_d = orc.knn(X64, k)
    idx, kappa, lam = _run(ctx, X, k, variant=variant)
    assert knn_mismatches(X64, idx, ref_idx, ref_d) == []
    ref_k, terms, ref_lam = orc.curvature(X64, k, ref_idx, variant=orc.HAAR if variant == "haar" else orc.LITERAL,
                                          return_terms=True)
    # the same neighbour lists on both sides (they are identical here)
    assert np.array_equal(idx, ref_idx)
    err = rel_err(kappa, ref_k)
    assert err.max() < KAPPA_TOL, err.max()
    assert np.allclose(lam, ref_lam, rtol=1e-4, atol=1e-6 * ref_lam.max())


# --------------------------------------------------------------------------
# Sparse clusters (MNIST-class rows), reduced N: all kNN rows, sampled kappa
# --------------------------------------------------------------------------
def test_sparse_clusters_reduced(ctx, orc):
    X = synth.sparse_clusters(n=6000, m=784, seed=2)
    k = 50
    X64 = _as64(X)
    ref_idx, ref_d = orc.knn(X64, k)
    idx, kappa, _ = _run(ctx, X, k)
    assert knn_mismatches(X64, idx, ref_idx, ref_d) == []
    rows = np.random.default_rng(0).choice(6000, 96, replace=False)
    ref = orc.curvature(X64, k, idx, rows=rows)
    assert rel_err(kappa[rows], ref).max() < KAPPA_TOL


def test_sparse_clusters_full_size_sampled(ctx, orc):
    X = synth.sparse_clusters(n=70000, m=784, seed=1)
    k = 50
    X64 = _as64(X)
    idx, kappa, _ = _run(ctx, X, k)
    rows = np.random.default_rng(1).choice(70000, 48, replace=False)
    ref_idx, ref_d = orc.knn(X64, k, rows=rows)
    assert knn_mismatches(X64, idx[rows], ref_idx, ref_d, rows=rows) == []
    ref = orc.curvature(X64, k, idx, rows=rows)
    assert rel_err(kappa[rows], ref).max() < KAPPA_TOL
    st = ctx.mecuco_get_stats()
    assert st["knn_fallback_rows"] == st["knn_uncertified"]


def test_mlp_decoder_full_size_sampled(ctx, orc):
    X = synth.mlp_decoder(n=50000, m=256, seed=1)
    k = 32
    X64 = _as64(X)
    idx, kappa, _ = _run(ctx, X, k)
    rows = np.random.default_rng(2).choice(50000, 64, replace=False)
    ref_idx, ref_d = orc.knn(X64, k, rows=rows)
    assert knn_mismatches(X64, idx[rows], ref_idx, ref_d, rows=rows) == []
    ref = orc.curvature(X64, k, idx, rows=rows)
    assert rel_err(kappa[rows], ref).max() < KAPPA_TOL


# --------------------------------------------------------------------------
# Edge cases: ragged sizes, odd k, no null space, minimum N, self-inclusion,
# duplicated points (exact ties and rank-deficient patches), BF16 storage,
# wide patches (m = 4096, k = 64)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,k", [(129, 37, 7), (300, 5, 10), (11, 3, 10), (257, 1, 3), (200, 130, 64)])
def test_edge_shapes(ctx, orc, n, m, k):
    rng = np.random.default_rng(n * 7 + m)
    X = rng.standard_normal((n, m)).astype(np.float32)
    X64 = _as64(X)
    ref_idx, ref_d = orc.knn(X64, k)
    idx, kappa, _ = _run(ctx, X, k)
    assert knn_mismatches(X64, idx, ref_idx, ref_d) == []
    for variant in ("literal", "haar"):
        _, kap, _ = _run(ctx, X, k, variant=variant, idx=ref_idx)
        ref = orc.curvature(X64, k, ref_idx, variant=orc.HAAR if variant == "haar" else orc.LITERAL)
        assert rel_err(kap, ref).max() < KAPPA_TOL, (variant, rel_err(kap, ref).max())


def test_include_self(ctx, orc):
    X = synth.sphere(n=500, m=32, seed=3)
    k = 12
    X64 = _as64(X)
    ref_idx, ref_d = orc.knn(X64, k, include_self=True)
    idx, kappa, _ = _run(ctx, X, k, include_self=True)
    assert knn_mismatches(X64, idx, ref_idx, ref_d) == []
    assert np.all(idx[:, 0] == np.arange(500))
    ref = orc.curvature(X64, k, idx)
    assert rel_err(kappa, ref).max() < KAPPA_TOL


def test_duplicates_ties_and_rank_deficiency(ctx, orc):
    rng = np.random.default_rng(5)
    base = rng.integers(-2, 3, size=(150, 6)).astype(np.float32)
    X = np.concatenate([base, base[:60]], axis=0)
    k = 8
    X64 = _as64(X)
    ref_idx, ref_d = orc.knn(X64, k)
    idx, kappa, _ = _run(ctx, X, k, idx=None)
    assert knn_mismatches(X64, idx, ref_idx, ref_d) == []
    _, kap, _ = _run(ctx, X, k, idx=ref_idx)
    ref = orc.curvature(X64, k, ref_idx)
    ok = np.abs(ref) > 1e-12
    assert rel_err(kap[ok], ref[ok]).max() < KAPPA_TOL
    assert np.all(np.abs(kap[~ok]) < 1e-5)


def test_bf16_storage(ctx, orc):
    Xb = synth.curved_patches(n=4000, m=256, n_patches=4, seed=2)
    X = torch.from_numpy(Xb.view(np.int16)).view(torch.bfloat16)
    k = 16
    X64 = _as64(Xb)
    Xd = X.cuda()
    idx = ctx.mecuco_knn(Xd, k)
    kappa = ctx.mecuco_curvature(Xd, k, idx=idx)
    torch.cuda.synchronize()
    idx, kappa = idx.cpu().numpy(), kappa.cpu().numpy()
    rows = np.random.default_rng(3).choice(4000, 128, replace=False)
    ref_idx, ref_d = orc.knn(X64, k, rows=rows)
    assert knn_mismatches(X64, idx[rows], ref_idx, ref_d, rows=rows) == []
    ref = orc.curvature(X64, k, idx, rows=rows)
    assert rel_err(kappa[rows], ref).max() < KAPPA_TOL


def test_wide_patches_k64(ctx, orc):
    Xb = synth.curved_patches(n=1500, m=4096, n_patches=3, seed=4)
    k = 64
    X64 = _as64(Xb)
    X = torch.from_numpy(Xb.view(np.int16)).view(torch.bfloat16).cuda()
    idx = ctx.mecuco_knn(X, k)
    kappa = ctx.mecuco_curvature(X, k, idx=idx)
    torch.cuda.synchronize()
    idx, kappa = idx.cpu().numpy(), kappa.cpu().numpy()
    rows = np.random.default_rng(4).choice(1500, 24, replace=False)
    ref_idx, ref_d = orc.knn(X64, k, rows=rows)
    assert knn_mismatches(X64, idx[rows], ref_idx, ref_d, rows=rows) == []
    ref = orc.curvature(X64, k, idx, rows=rows)
    assert rel_err(kappa[rows], ref).max() < KAPPA_TOL


def test_host_buffer_entry_point_matches_device_path(ctx):
    X = synth.sphere(n=1000, m=32, seed=9)
    k = 10
    Xd = _dev(X)
    kd = ctx.mecuco_curvature(Xd, k).cpu().numpy()
    kh, ih = ctx.mecuco_curvature_host(torch.from_numpy(X).pin_memory(), k, return_idx=True)
    assert np.array_equal(kh.numpy(), kd)
    assert np.array_equal(ih.numpy(), ctx.mecuco_knn(Xd, k).cpu().numpy())


def test_invalid_arguments_enqueue_nothing(ctx):
    from paper_2606_06329_gb300 import _native as N
    X = _dev(np.zeros((10, 4), np.float32))
    with pytest.raises(N.MecucoError) as e:
        ctx.mecuco_knn(X, 10)  # k > N - 1
    assert e.value.status == N.ERR_INVALID_ARG
    with pytest.raises(N.MecucoError):
        ctx.mecuco_knn(X, 65)


# --------------------------------------------------------------------------
# The forms of the FP32 Jacobi sweeps (the fused form with 1, 2 (default) or
# 4 warps per patch; the three-pass CTA form) apply the same rotations in a
# different rounding order: the plain FP32 curvatures agree far inside the
# FP32 tolerance (1e-5), and all match the oracle.  In the BF16-mixed form the
# eigenvectors rotate the patch before its BF16 rounding, so an eigenvector
# change in the last bits flips roundings of the rotated patch (2^-9 relative
# each): there the forms agree within that form's bound against the oracle
# (5e-4).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [10, 33, 64])
def test_jacobi_forms_agree(ctx, orc, k):
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=3000, m=256, n_patches=4, seed=21 + k)
    X = synth.bf16_bits_to_f32(bits)
    Xd = _dev(X)
    idx = ctx.mecuco_knn(Xd, k)
    out = {}
    forms = (2, 1, 4, 0)
    for form in forms:
        ctx.set_option(N.OPT_JACOBI_WARP, form)
        try:
            for prec in ("fp32", "bf16_mixed"):
                kap = ctx.mecuco_curvature(Xd, k, idx=idx, precision=prec)
                torch.cuda.synchronize()
                assert ctx.mecuco_get_last_status() == 0
                out[(form, prec)] = kap.cpu().numpy()
        finally:
            ctx.set_option(N.OPT_JACOBI_WARP, 2)
    for form in forms[1:]:
        for prec, tol in (("fp32", 1e-5), ("bf16_mixed", 5e-4)):
            d = rel_err(out[(form, prec)], out[(2, prec)])
            print(f"k={k} {prec}: form {form} vs form 2 max rel diff {d.max():.2e}")
            assert d.max() < tol
    rows = np.random.default_rng(k).choice(X.shape[0], 24, replace=False)
    ref = orc.curvature(X.astype(np.float64), k, idx.cpu().numpy(), rows=rows)
    for form in forms:
        assert rel_err(out[(form, "fp32")][rows], ref).max() < KAPPA_TOL
