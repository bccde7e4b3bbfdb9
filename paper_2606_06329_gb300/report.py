"""Curvature-fidelity report on the GPU, in the layout of the paper's
experiment tables: per dataset the mean and standard deviation of the Exact
(Theorem 1) and Fast (Alg. 1) curvatures with their times, and MAE, Spearman
rho_S and Chatterjee xi of Fast against Exact, on raw scores and after min-max
normalisation to [0, 1]; then the mean relative error of Fast against Exact as
D/k grows (eq. error_bound).  k = round(log2 n) as in the paper's protocol.
The inputs are seeded synthetic sets from ``synth`` (Exact mode here takes
m <= 64).

    python -m paper_2606_06329_gb300.report [--variant literal|haar]
"""
from __future__ import annotations

import argparse
import math

import numpy as np
import torch

from . import api, synth


def _timed(fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return out, a.elapsed_time(b) * 1e-3


def datasets():
    """(name, X) pairs: seeded synthetic clouds with m <= 64."""
    return [
        ("sphere-m16", synth.sphere(n=4000, m=16, seed=1)),
        ("sphere-m32", synth.sphere(n=8000, m=32, seed=2)),
        ("sphere-m64", synth.sphere(n=8000, m=64, seed=3)),
        ("mlp-image-d4-m48", synth.mlp_image(n=10000, m=48, d=4, seed=4)),
        ("mlp-image-d8-m64", synth.mlp_image(n=20000, m=64, d=8, seed=5)),
        ("clusters-m40", synth.sparse_clusters(n=10000, m=40, n_clusters=6, seed=6)),
    ]


def fidelity_rows(ctx: api.Context, variant: str = "literal"):
    rows = []
    for name, Xn in datasets():
        X = torch.from_numpy(np.ascontiguousarray(Xn, dtype=np.float32)).cuda()
        n, m = X.shape
        k = max(3, int(round(math.log2(n))))
        idx = ctx.mecuco_knn(X, k)
        ex, t_ex = _timed(lambda: ctx.mecuco_curvature_exact(X, k, idx=idx))
        fa, t_fa = _timed(lambda: ctx.mecuco_curvature(X, k, idx=idx, variant=variant))
        raw = ctx.mecuco_fidelity(ex, fa, normalize=False)
        nrm = ctx.mecuco_fidelity(ex, fa, normalize=True)
        ne, nf = ctx.mecuco_minmax_normalize(ex), ctx.mecuco_minmax_normalize(fa)
        rows.append(dict(name=name, n=n, m=m, k=k,
                         exact=(ex.mean().item(), ex.std().item(), t_ex),
                         fast=(fa.mean().item(), fa.std().item(), t_fa),
                         exact_norm=(ne.mean().item(), ne.std().item()),
                         fast_norm=(nf.mean().item(), nf.std().item()),
                         raw=raw, normalized=nrm))
    return rows


def error_curve(ctx: api.Context, k: int = 5, ms=(8, 16, 24, 32, 48, 64), n: int = 4000):
    out = []
    for m in ms:
        X = torch.from_numpy(synth.sphere(n=n, m=m, seed=7)).cuda()
        idx = ctx.mecuco_knn(X, k)
        ex = ctx.mecuco_curvature_exact(X, k, idx=idx).double()
        errs = []
        for variant in ("literal", "haar"):
            fa = ctx.mecuco_curvature(X, k, idx=idx, variant=variant).double()
            errs.append(((fa - ex).abs() / ex.abs()).mean().item())
        out.append((m, m / k, errs[0], errs[1]))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--variant", choices=("literal", "haar"), default="literal")
    a = ap.parse_args(argv)
    with api.Context(0) as ctx:
        rows = fidelity_rows(ctx, a.variant)
        hdr = f"{'dataset':18s} {'n':>6s} {'m':>3s} {'k':>3s} | {'Exact mean':>10s} {'std':>9s} {'s':>7s} | " \
              f"{'Fast mean':>10s} {'std':>9s} {'s':>7s} | {'MAE':>9s} {'rho_S':>7s} {'xi':>7s}"
        for key, title in (("raw", "raw scores"), ("normalized", "min-max normalised scores")):
            print(f"\nFast ({a.variant}) against Exact, {title}")
            print(hdr)
            for r in rows:
                if key == "raw":
                    e, f = r["exact"], r["fast"]
                else:
                    e, f = r["exact_norm"] + (r["exact"][2],), r["fast_norm"] + (r["fast"][2],)
                mae, rho, xi = r[key]
                print(f"{r['name']:18s} {r['n']:6d} {r['m']:3d} {r['k']:3d} | {e[0]:10.4g} {e[1]:9.3g} {e[2]:7.3f} | "
                      f"{f[0]:10.4g} {f[1]:9.3g} {f[2]:7.3f} | {mae:9.4g} {rho:7.4f} {xi:7.4f}")
        print("\nmean relative error of Fast against Exact (sphere, k = 5)")
        print(f"{'m':>4s} {'D/k':>6s} {'literal':>9s} {'haar':>9s}")
        for m, r, el, eh in error_curve(ctx):
            print(f"{m:4d} {r:6.1f} {el:9.4f} {eh:9.4f}")


if __name__ == "__main__":
    main()
