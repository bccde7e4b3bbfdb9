"""Seeded synthetic point clouds shaped like the paper's workloads.

This module is the one piece of code shared by the FP64 oracle's tests and the
CUDA path's tests and benchmark: it draws inputs and holds none of the
estimator's arithmetic.  Every generator takes an integer seed and uses
numpy's counter-based Philox bit generator, with one spawned child stream per
independent block (cluster, dataset, layer), so the bytes produced do not
depend on thread scheduling.

Workload shapes (the paper measures on OpenML tables, which are not used here;
these seeded clouds stand in for them):

* ``sphere``          - unit 2-sphere in R^3 mapped into R^m by a Haar frame,
                        plus Gaussian noise (small exact-vs-fast workload).
* ``sparse_clusters`` - [0,1]-valued rows with ~80 % exact zeros from seeded
                        Gaussian clusters, shaped like the 70,000 x 784
                        MNIST-class rows of the paper's Table 3.
* ``mlp_image``       - random tanh-MLP images of low-dimensional Gaussian
                        latents (curved manifolds of chosen intrinsic dim).
* ``curved_patches``  - mixture of quadratic-graph patches rotated into R^m,
                        stored in BF16 (the large 1M x 4096 workload).
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

__all__ = [
    "haar_frame", "sphere", "sparse_clusters", "mlp_image", "mlp_decoder",
    "batched_mlp_datasets", "curved_patches", "f32_to_bf16_bits",
    "bf16_bits_to_f32", "zero_fraction",
]


def _gen(seed_seq: np.random.SeedSequence) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed_seq))


def _children(seed: int, n: int, tag: int = 0) -> list:
    return np.random.SeedSequence([int(seed), int(tag)]).spawn(n)


def haar_frame(m: int, d: int, rng: np.random.Generator) -> np.ndarray:
    """m x d matrix with orthonormal columns, Haar distributed: QR of a
    Gaussian matrix with the signs of R's diagonal folded into Q."""
    g = rng.standard_normal((m, d))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even) and
    return the 16-bit patterns.  Inputs here are finite."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    bias = ((u >> np.uint32(16)) & np.uint32(1)) + np.uint32(0x7FFF)
    return ((u + bias) >> np.uint32(16)).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    """Exact widening of bfloat16 bit patterns to float32."""
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def zero_fraction(x: np.ndarray) -> float:
    return float(np.count_nonzero(x == 0)) / x.size


def sphere(n: int = 2000, m: int = 32, noise: float = 0.01, seed: int = 1) -> np.ndarray:
    """Points uniform on the unit 2-sphere, embedded in R^m by the first three
    columns of a Haar orthogonal matrix, plus i.i.d. N(0, noise^2)."""
    rng = _gen(_children(seed, 1, tag=101)[0])
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    q = haar_frame(m, 3, rng)
    x = u @ q.T + noise * rng.standard_normal((n, m))
    return x.astype(np.float32)


def sparse_clusters(n: int = 70000, m: int = 784, n_clusters: int = 10,
                    sigma: float = 0.15, support: float = 0.18,
                    off_mean: float = -0.30, seed: int = 1) -> np.ndarray:
    """[0,1]-valued rows from seeded Gaussian clusters.  Each cluster mean has a
    random support (fraction ``support`` of coordinates, values U(0.25, 1));
    off-support coordinates have mean ``off_mean`` < 0 so that clipping at 0
    produces exact zeros.  With the defaults the zero fraction is ~0.80.
    Rows are placed in a seeded random order."""
    kids = _children(seed, n_clusters + 1, tag=202)
    perm = _gen(kids[-1]).permutation(n)
    x = np.empty((n, m), dtype=np.float32)
    bounds = np.linspace(0, n, n_clusters + 1).astype(np.int64)
    for c in range(n_clusters):
        rng = _gen(kids[c])
        mask = rng.random(m) < support
        mu = np.where(mask, rng.uniform(0.25, 1.0, m), off_mean)
        rows = perm[bounds[c]:bounds[c + 1]]
        blk = mu[None, :] + sigma * rng.standard_normal((rows.size, m))
        x[rows] = np.clip(blk, 0.0, 1.0).astype(np.float32)
    return x


def _tanh_mlp(z: np.ndarray, widths: list, rng: np.random.Generator,
              bias_sd: float = 0.1) -> np.ndarray:
    """Random tanh MLP: weights N(0, 1/fan_in), biases N(0, bias_sd^2), tanh on
    hidden layers, linear output layer."""
    h = z
    for li, w_out in enumerate(widths):
        a = rng.standard_normal((h.shape[1], w_out)) / np.sqrt(h.shape[1])
        b = bias_sd * rng.standard_normal(w_out)
        h = h @ a + b
        if li + 1 < len(widths):
            h = np.tanh(h)
    return h


def mlp_image(n: int, m: int, d: int, hidden: int = 64, noise: float = 0.01,
              seed: int = 1, tag: int = 303) -> np.ndarray:
    """2-layer tanh MLP image of d-dimensional standard-normal latents in R^m,
    plus i.i.d. N(0, noise^2)."""
    rng = _gen(_children(seed, 1, tag=tag)[0])
    z = rng.standard_normal((n, d))
    x = _tanh_mlp(z, [hidden, m], rng)
    x = x + noise * rng.standard_normal((n, m))
    return x.astype(np.float32)


def mlp_decoder(n: int = 50000, m: int = 256, latent: int = 10, seed: int = 1) -> np.ndarray:
    """3-layer tanh decoder latent -> 64 -> 128 -> m of standard-normal
    latents (no added noise)."""
    rng = _gen(_children(seed, 1, tag=404)[0])
    z = rng.standard_normal((n, latent))
    return _tanh_mlp(z, [64, 128, m], rng).astype(np.float32)


def batched_mlp_datasets(nsets: int = 256, seed: int = 1, n_range=(500, 20000),
                         m_choices=(64, 128, 256, 512, 1024), k_range=(10, 64),
                         d_range=(2, 16)) -> list:
    """Many independent datasets of uneven size: returns a list of dicts with
    keys ``X`` (N x m float32), ``k`` and ``d``."""
    meta = _gen(_children(seed, 1, tag=505)[0])
    out = []
    for s in range(nsets):
        n = int(meta.integers(n_range[0], n_range[1] + 1))
        m = int(meta.choice(np.asarray(m_choices)))
        k = int(meta.integers(k_range[0], k_range[1] + 1))
        d = int(meta.integers(d_range[0], d_range[1] + 1))
        x = mlp_image(n, m, d, seed=seed * 100003 + s, tag=506)
        out.append({"X": x, "k": k, "d": d})
    return out


def _curved_block(args):
    (kid, rows, m, intrinsic, offset_sd, noise, out) = args
    rng = _gen(kid)
    nb = rows.size
    # symmetric with N(0,1) entries: fill the upper triangle, mirror it
    a = np.triu(rng.standard_normal((intrinsic, intrinsic)))
    a = a + np.triu(a, 1).T
    frame = haar_frame(m, intrinsic + 1, rng).astype(np.float32)
    offset = (offset_sd * rng.standard_normal(m)).astype(np.float32)
    chunk = 8192
    for c0 in range(0, nb, chunk):
        c1 = min(nb, c0 + chunk)
        u = rng.uniform(-1.0, 1.0, (c1 - c0, intrinsic))
        h = 0.5 * np.einsum("ni,ij,nj->n", u, a, u)
        loc = np.concatenate([u, h[:, None]], axis=1).astype(np.float32)
        blk = loc @ frame.T
        blk += offset[None, :]
        blk += np.float32(noise) * rng.standard_normal((c1 - c0, m), dtype=np.float32)
        out[rows[c0:c1]] = f32_to_bf16_bits(blk)
    return None


def curved_patches(n: int = 1_000_000, m: int = 4096, n_patches: int = 32,
                   intrinsic: int = 8, offset_sd: float = 0.5, noise: float = 0.005,
                   seed: int = 1, threads: int | None = None) -> np.ndarray:
    """Mixture of ``n_patches`` curved patches stored as bfloat16 bit patterns
    (uint16, shape n x m).  Patch c: u ~ U[-1,1]^intrinsic, h(u) = u^T A_c u / 2
    with A_c symmetric N(0,1); the point (u, h) is mapped into R^m by a Haar
    frame F_c, shifted by o_c ~ N(0, offset_sd^2 I), plus N(0, noise^2) noise,
    then rounded to bfloat16.  Rows are placed in a seeded random order."""
    kids = _children(seed, n_patches + 1, tag=606)
    perm = _gen(kids[-1]).permutation(n)
    out = np.empty((n, m), dtype=np.uint16)
    bounds = np.linspace(0, n, n_patches + 1).astype(np.int64)
    jobs = [(kids[c], perm[bounds[c]:bounds[c + 1]], m, intrinsic, offset_sd, noise, out)
            for c in range(n_patches)]
    nt = threads or min(len(jobs), max(1, os.cpu_count() or 1))
    if nt <= 1:
        for j in jobs:
            _curved_block(j)
    else:
        with _cf.ThreadPoolExecutor(max_workers=nt) as ex:
            list(ex.map(_curved_block, jobs))
    return out
