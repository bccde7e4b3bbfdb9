"""Pins of the FP64 reference gradient (oracle/adjoint.py, autograd through
Alg. 1's Fast branch): its forward values equal the C oracle's Fast mode, and
its gradient equals the C oracle's central differences extrapolated to h -> 0
(Richardson: (4 g(h/2) - g(h)) / 3 removes the O(h^2) term)."""
import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

pytest.importorskip("torch")

from oracle import adjoint as A  # noqa: E402


def _case(seed=3, n=400, m=16, k=8):
    X = synth.mlp_decoder(n=n, m=m, latent=3, seed=seed).astype(np.float64)
    return X, k


@pytest.mark.parametrize("variant", ["literal", "haar"])
def test_forward_matches_c_oracle(orc, variant):
    X, k = _case()
    idx, _ = orc.knn(X, k)
    got = A.curvature_fast(X, idx, variant)
    ref = orc.curvature(X, k, idx, variant=orc.HAAR if variant == "haar" else orc.LITERAL)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("variant", ["literal", "haar"])
def test_gradient_matches_extrapolated_differences(orc, variant):
    X, k = _case()
    n, m = X.shape
    idx, _ = orc.knn(X, k)
    g = A.grad_adjoint(X, idx, variant=variant)
    rng = np.random.default_rng(4)
    coords = np.stack([rng.integers(0, n, 40), rng.integers(0, m, 40)], axis=1)
    h = 1e-4 * np.sqrt(np.mean(X ** 2))  # (4 g(h/2) - g(h)) / 3 agrees to ~4e-8 here; 1e-3 leaves O(h^4)
    var = orc.HAAR if variant == "haar" else orc.LITERAL
    g1 = orc.grad_fd(X, k, idx, coords, h, variant=var)
    g2 = orc.grad_fd(X, k, idx, coords, 0.5 * h, variant=var)
    fd = (4.0 * g2 - g1) / 3.0
    got = g[coords[:, 0], coords[:, 1]]
    scale = np.maximum(np.abs(fd), 1e-2 * np.sqrt(np.mean(fd ** 2)))
    err = np.abs(got - fd) / scale
    print(f"autograd vs extrapolated FD ({variant}): max {err.max():.2e}")
    assert err.max() < 1e-6


def test_weights_are_linear(orc):
    X, k = _case(n=200)
    idx, _ = orc.knn(X, k)
    w = np.random.default_rng(1).random(X.shape[0])
    g1 = A.grad_adjoint(X, idx, w)
    g2 = A.grad_adjoint(X, idx, 2.0 * w)
    assert np.allclose(g2, 2.0 * g1, rtol=1e-12, atol=0)
