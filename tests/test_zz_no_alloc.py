"""mecuco_knn_noalloc: the allocation-free kNN entry point, for callers that
cannot allocate device memory (a framework-owned memory pool, a fixed device
budget, or code that must not pay cudaMalloc's implicit synchronisation).  It
must return the same neighbour lists as mecuco_knn (plain FP32 form) on two
calls in a row through the C ABI, and reject sizes beyond its fixed scratch.
Kept in a file collected last, so a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2606_06329_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import api, build, _native
    build.build()
    lib = _native.load()
    ctx = api.Context(0)
    yield lib, ctx
    ctx.close()


def _noalloc(lib, X, k, include_self=False):
    from paper_2606_06329_gb300 import _native as N
    n, m = X.shape
    idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    dt = N.BF16 if X.dtype == torch.bfloat16 else N.F32
    st = lib.mecuco_knn_noalloc(C.c_void_p(X.data_ptr()), dt, n, m, X.stride(0), k, int(include_self),
                                C.c_void_p(idx.data_ptr()), C.c_void_p(dist.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(st, "mecuco_knn_noalloc")
    return idx, dist


def test_noalloc_matches_context_entry_point_twice(lib_ctx):
    lib, ctx = lib_ctx
    cases = [(torch.from_numpy(synth.sphere(n=3000, m=32, seed=11)).cuda(), 10, False),
             (torch.from_numpy(synth.curved_patches(n=5000, m=256, n_patches=4, seed=12).view(np.int16))
              .view(torch.bfloat16).cuda(), 24, True)]
    for X, k, inc in cases:  # two calls in a row, different shapes, shared scratch
        idx_a, dist_a = _noalloc(lib, X, k, inc)
        idx_b, dist_b = ctx.mecuco_knn(X, k, include_self=inc, precision="fp32", return_dist=True)
        torch.cuda.synchronize()
        assert torch.equal(idx_a, idx_b)
        assert torch.allclose(dist_a, dist_b, rtol=1e-6, atol=0)
    # a repeat of the first case after the scratch held another problem
    X, k, inc = cases[0]
    idx_c, _ = _noalloc(lib, X, k, inc)
    torch.cuda.synchronize()
    assert torch.equal(idx_c, ctx.mecuco_knn(X, k, include_self=inc))


def test_noalloc_crosses_its_query_chunks(lib_ctx):
    # N above the entry point's 16,384-row query chunk: three launches writing
    # at row offsets, and a candidate split different from mecuco_knn's plan;
    # after the exact re-rank the lists and distances must still be the same
    lib, ctx = lib_ctx
    X = torch.from_numpy(synth.sphere(n=40000, m=32, seed=13)).cuda()
    for _ in range(2):
        idx_a, dist_a = _noalloc(lib, X, 10)
        idx_b, dist_b = ctx.mecuco_knn(X, 10, precision="fp32", return_dist=True)
        torch.cuda.synchronize()
        assert torch.equal(idx_a, idx_b)
        assert torch.allclose(dist_a, dist_b, rtol=1e-6, atol=0)


def test_noalloc_rejects_oversized_problems(lib_ctx):
    lib, _ = lib_ctx
    from paper_2606_06329_gb300 import _native as N
    X = torch.zeros((4, 8), device="cuda")
    idx = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    # N beyond the fixed scratch: rejected before any device work
    st = lib.mecuco_knn_noalloc(C.c_void_p(X.data_ptr()), N.F32, (1 << 22) + 1, 8, 8, 2, 0,
                                C.c_void_p(idx.data_ptr()), None, None)
    assert st == N.ERR_INVALID_ARG
    assert b"exceeds the maximum" in lib.mecuco_last_error_message()
