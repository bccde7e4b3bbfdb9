"""The hand-derived null-space patches of tests/golden/nullspace_*.txt through
the C ABI: each fixture's k points form a dataset of N = k points whose every
neighbourhood (include_self) is the fixture's patch, so every point's
curvature must equal the closed-form value for both Fast variants (Alg. 1;
eqs. tA, tB, tnull, fast_curv; eq. gnull_exp), in both arithmetic forms.  The
points are small integers, exact in BF16, and so are the centred values and
their pair products, so the BF16-mixed form sees exact moments here."""
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
    for variant, key in (("literal", "kappa_fast_literal"), ("haar", "kappa_fast_haar")):
        out = ctx.mecuco_curvature(X, k, include_self=True, variant=variant, precision=precision,
                                   return_lambda=True)
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == 0
        kap = out["kappa"].cpu().numpy().astype(np.float64)
        # K of the q = 1 literal case is a cancellation (|-44/81| from terms of
        # size 18), which scales FP32 rounding by ~35: 1e-4 still holds
        assert np.allclose(kap, g[key], rtol=1e-4, atol=0), (variant, kap, g[key])
        lam = out["lambda"].cpu().numpy()
        assert np.isclose(lam[:, :int(g["p"])].sum(1), g["tau"], rtol=1e-5).all()
        # lambda past the numerical rank is reported as 0
        assert np.all(lam[:, int(g["p"]):] == 0.0)
