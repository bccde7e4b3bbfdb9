"""Failure paths, made to happen without faulting the GPU: an eigensolver
sweep cap (MECUCO_ERR_NOT_CONVERGED, results still written), bounded waits in
the tensor-core kernels made to run out by a short limit
(MECUCO_ERR_TIMEOUT: the launch returns, frees its tensor memory, and the
context keeps working), and a device allocation refused by the context's
allocation cap (MECUCO_ERR_OOM before any allocation)."""
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


@pytest.mark.parametrize("precision", ["fp32", "bf16_mixed"])
def test_sweep_cap_reports_not_converged(ctx, precision):
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=2000, m=256, n_patches=3, seed=41)
    Xd = _bf16(bits).cuda()
    idx = ctx.mecuco_knn(Xd, 32, precision=precision)
    ref = ctx.mecuco_curvature(Xd, 32, idx=idx, precision=precision)
    assert ctx.mecuco_get_last_status() == N.OK
    try:
        ctx.set_option(N.OPT_JACOBI_MAX_SWEEPS, 1)
        kap = ctx.mecuco_curvature(Xd, 32, idx=idx, precision=precision)
        torch.cuda.synchronize()
        stats = ctx.mecuco_get_stats()
        assert ctx.mecuco_get_last_status() == N.ERR_NOT_CONVERGED
    finally:
        ctx.set_option(N.OPT_JACOBI_MAX_SWEEPS, 40)
    assert stats["jacobi_not_converged"] > 0 and stats["jacobi_max_sweeps"] == 1
    # the capped eigenpairs are still written and give finite curvatures
    assert torch.isfinite(kap).all()
    # the status word was cleared by the query: the next call is clean
    again = ctx.mecuco_curvature(Xd, 32, idx=idx, precision=precision)
    assert ctx.mecuco_get_last_status() == N.OK
    assert torch.equal(again, ref)


def test_short_wait_limit_times_out_and_the_context_recovers(ctx, orc):
    from paper_2606_06329_gb300 import _native as N
    bits = synth.curved_patches(n=3000, m=512, n_patches=3, seed=42)
    Xd = _bf16(bits).cuda()
    k = 32
    idx0 = ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
    kap0 = ctx.mecuco_curvature(Xd, k, idx=idx0, precision="bf16_mixed")
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == N.OK
    try:
        # a limit of one clock cycle: the first wait that has to spin runs out
        ctx.set_option(N.OPT_WAIT_LIMIT, 1)
        ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == N.ERR_TIMEOUT
        ctx.mecuco_curvature(Xd, k, idx=idx0, precision="bf16_mixed")
        torch.cuda.synchronize()
        assert ctx.mecuco_get_last_status() == N.ERR_TIMEOUT
    finally:
        ctx.set_option(N.OPT_WAIT_LIMIT, 0)
    # every launch freed its tensor memory (a leak would stall the next
    # allocation) and the results are again those of the clean run
    idx1 = ctx.mecuco_knn(Xd, k, precision="bf16_mixed")
    kap1 = ctx.mecuco_curvature(Xd, k, idx=idx1, precision="bf16_mixed")
    torch.cuda.synchronize()
    assert ctx.mecuco_get_last_status() == N.OK
    assert torch.equal(idx0, idx1) and torch.equal(kap0, kap1)
    X64 = synth.bf16_bits_to_f32(bits).astype(np.float64)
    rows = np.arange(0, 3000, 97)
    ref_idx, ref_d = orc.knn(X64, k, rows=rows)
    assert knn_mismatches(X64, idx1.cpu().numpy()[rows], ref_idx, ref_d, rows=rows) == []


def test_allocation_cap_reports_oom_and_leaves_the_context_usable(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06329_gb300 import _native as N
    from paper_2606_06329_gb300 import api
    X = synth.sphere(n=2000, m=32, seed=43)
    Xd = torch.from_numpy(X).cuda()
    with api.Context(0) as c:
        c.set_option(N.OPT_WORKSPACE_LIMIT, 1 << 16)  # 64 KB: below this call's workspace
        with pytest.raises(N.MecucoError) as ei:
            c.mecuco_curvature(Xd, 10)
        assert ei.value.status == N.ERR_OOM
        assert b"allocation limit" in c.lib.mecuco_last_error_message()
        c.set_option(N.OPT_WORKSPACE_LIMIT, 0)
        kap = c.mecuco_curvature(Xd, 10)
        torch.cuda.synchronize()
        assert c.mecuco_get_last_status() == N.OK
    ref_idx, _ = orc.knn(X, 10)
    ref = orc.curvature(X, 10, ref_idx)
    assert rel_err(kap.cpu().numpy(), ref).max() < 1e-4
