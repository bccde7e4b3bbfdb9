"""The hand-derived null-space patches of tests/golden/nullspace_*.txt through
the C ABI: each fixture's k points form a dataset of N = k points whose every
neighbourhood (include_self) is the fixture's patch, so every point's
curvature must equal the closed-form value for both Fast variants (Alg. 1;
eqs. tA, tB, tnull, fast_curv; eq. gnull_exp), in both arithmetic forms.  The
points and centred values are small integers, exact in BF16.

The plain form must match to 1e-4 relative.  The BF16-mixed form rounds the
rotated patch Y = U^T X_c (irrational here) to BF16 and forms each third
moment from three such values and one rounded product: to first order every
term of T^ moves by at most 4u of its size (u = 2^-9), so every sum of
squares the estimator combines moves by at most 8u of its size, and
|K - K_exact| <= 8u (t_range/2 + |t_null|/2 + tau/2).  With m = 3 or 4 no
averaging over columns reduces this, and the literal q = 1 patch is a
cancellation (|-44/81| from terms of size ~20), so the bound is on the terms'
scale, not on K; at the benchmark's m the same form is within 1e-4 of the
FP64 oracle (test_gpu_tc)."""
import glob
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(path):
    rec = {"points": []}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "point":
            rec["points"].append([float(v) for v in vals])
        else:
            rec[key] = float(vals[0])
    rec["points"] = np.array(rec["points"])
    return rec


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16_mixed"])
@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "nullspace_*.txt"))),
                         ids=os.path.basename)
def test_golden_null_space_patch_on_gpu(ctx, path, precision):
    g = _read(path)
    k = int(g["k"])
    X = torch.from_numpy(g["points"].astype(np.float32)).cuda()
    if precision == "bf16_mixed":
        X = X.to(torch.bfloat16)
    for variant, key, tnull in (("literal", "kappa_fast_literal", "literal_t_null"),
                                ("haar", "kappa_fast_haar", "haar_t_null")):
        out = ctx.mecuco_curvature(X, k, include_self=True, variant=variant, precision=precision,
                                   return_lambda=True)
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == 0
        kap = out["kappa"].cpu().numpy().astype(np.float64)
        if precision == "fp32":
            # K of the q = 1 literal case is a cancellation (|-44/81| from terms of
            # size 18), which scales FP32 rounding by ~35: 1e-4 still holds
            assert np.allclose(kap, g[key], rtol=1e-4, atol=0), (variant, kap, g[key])
        else:
            scale = 0.5 * (g["t_range"] + abs(g[tnull]) + g["tau"])
            err = np.abs(kap - g[key]).max()
            print(f"{os.path.basename(path)} bf16_mixed {variant}: |dK| = {err:.3e} = "
                  f"{err / scale / 2 ** -9:.2f} u of the terms' scale")
            assert err <= 8 * 2 ** -9 * scale, (variant, kap, g[key])
        lam = out["lambda"].cpu().numpy()
        assert np.isclose(lam[:, :int(g["p"])].sum(1), g["tau"], rtol=1e-5).all()
        # lambda past the numerical rank is reported as 0
        assert np.all(lam[:, int(g["p"]):] == 0.0)
