"""The seeded input generators (paper_2606_06329_gb300/synth.py), the one
module the oracle's tests and the CUDA path share: the stated shapes, ranges
and structure of each workload, determinism in the seed (and independence of
the thread count), and the BF16 rounding against torch's own conversion."""
import numpy as np
import pytest
import torch

from paper_2606_06329_gb300 import synth


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-20, 20, 20000),
        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, -1.5e-38], np.float32),
    ])
    # ties: values exactly halfway between two BF16 neighbours round to even
    halves = (np.arange(1, 200, dtype=np.uint32) << np.uint32(16)) | np.uint32(0x8000)
    x = np.concatenate([x, (halves + np.uint32(0x3F800000)).view(np.float32)])
    ours = synth.f32_to_bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    back = synth.bf16_bits_to_f32(ours)
    assert np.array_equal(back, torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy())


def test_sphere_lies_near_a_unit_sphere_in_a_3d_subspace():
    x = synth.sphere(n=2000, m=32, noise=0.01, seed=5)
    assert x.shape == (2000, 32) and x.dtype == np.float32
    s = np.linalg.svd(x.astype(np.float64), compute_uv=False)
    assert s[2] > 20 * s[3]  # three directions carry the sphere, the rest is noise
    _, _, vt = np.linalg.svd(x.astype(np.float64), full_matrices=False)
    r = np.linalg.norm(x @ vt[:3].T, axis=1)
    assert abs(r.mean() - 1.0) < 0.01 and r.std() < 0.03
    assert np.array_equal(x, synth.sphere(n=2000, m=32, noise=0.01, seed=5))
    assert not np.array_equal(x, synth.sphere(n=2000, m=32, noise=0.01, seed=6))


def test_sparse_clusters_range_zero_fraction_and_clusters():
    x = synth.sparse_clusters(n=3000, m=784, seed=2)
    assert x.shape == (3000, 784) and x.dtype == np.float32
    assert x.min() >= 0.0 and x.max() <= 1.0
    assert 0.75 < synth.zero_fraction(x) < 0.85  # about 80 % exact zeros
    # ten cluster means: after centring, 9 between-cluster directions stand
    # far above the within-cluster spread
    s = np.linalg.svd(x - x.mean(axis=0, dtype=np.float64), compute_uv=False)
    assert s[8] > 10 * s[9]
    assert np.array_equal(x, synth.sparse_clusters(n=3000, m=784, seed=2))


def test_mlp_images_are_deterministic_and_finite():
    a = synth.mlp_image(500, 64, 3, seed=4)
    assert a.shape == (500, 64) and a.dtype == np.float32 and np.isfinite(a).all()
    assert np.array_equal(a, synth.mlp_image(500, 64, 3, seed=4))
    assert not np.array_equal(a, synth.mlp_image(500, 64, 3, seed=5))
    d = synth.mlp_decoder(n=400, m=256, latent=10, seed=1)
    assert d.shape == (400, 256) and np.isfinite(d).all()
    assert np.array_equal(d, synth.mlp_decoder(n=400, m=256, latent=10, seed=1))


def test_batched_datasets_follow_the_stated_ranges():
    sets = synth.batched_mlp_datasets(nsets=12, seed=3, n_range=(500, 700))
    assert len(sets) == 12
    for s in sets:
        n, m = s["X"].shape
        assert 500 <= n <= 700 and m in (64, 128, 256, 512, 1024)
        assert 10 <= s["k"] <= 64 and 2 <= s["d"] <= 16
        assert s["X"].dtype == np.float32 and np.isfinite(s["X"]).all()
    assert len({s["X"].shape[1] for s in sets}) > 1  # uneven m across the batch


def test_curved_patches_are_bf16_and_independent_of_threads():
    a = synth.curved_patches(n=3000, m=64, n_patches=4, seed=7, threads=1)
    b = synth.curved_patches(n=3000, m=64, n_patches=4, seed=7, threads=4)
    assert a.dtype == np.uint16 and a.shape == (3000, 64)
    assert np.array_equal(a, b)
    x = synth.bf16_bits_to_f32(a).astype(np.float64)
    assert np.isfinite(x).all()
    # each patch spans 9 directions (8 intrinsic + the quadratic height) at
    # its own offset: after centring, 4 * 9 + 3 directions, then the
    # N(0, 0.005^2) noise (singular values near 0.005 sqrt(n), BF16 rounding on top)
    s = np.linalg.svd(x - x.mean(axis=0), compute_uv=False)
    assert s[38] > 10 * s[39]
    assert 0.5 * 0.005 * np.sqrt(3000) < s[39] < 2 * 0.005 * np.sqrt(3000)
    assert not np.array_equal(a, synth.curved_patches(n=3000, m=64, n_patches=4, seed=8, threads=1))


@pytest.mark.parametrize("gen", ["sphere", "sparse_clusters"])
def test_generators_draw_nothing_from_global_state(gen):
    np.random.seed(0)
    torch.manual_seed(0)
    kw = dict(n=300, m=16) if gen == "sphere" else dict(n=300, m=32)
    a = getattr(synth, gen)(seed=1, **kw)
    np.random.seed(123)
    torch.manual_seed(123)
    assert np.array_equal(a, getattr(synth, gen)(seed=1, **kw))
