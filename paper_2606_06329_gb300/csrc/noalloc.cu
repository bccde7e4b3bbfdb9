// noalloc.cu - mecuco_knn_noalloc: the k-nearest-neighbour search of
// mecuco_knn for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under a framework that owns
// every byte of device memory through its own pool, services with a fixed
// device-memory budget decided at start-up, and code paths where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable.  For them
// this entry point takes no context and allocates nothing: its scratch (row
// norms, per-row candidate lists, certification flags, counters) lives in one
// file-scope __device__ array of NOALLOC_BYTES, which every GPU whose module
// copy is loaded holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress once per device and context
// (on that device, under a lock) and passed to the kernels.  The first call on
// a device does that lookup (which may load this module) and should therefore
// come before any stream capture.  The cache is keyed on the current CUDA
// context, so after a cudaDeviceReset (which destroys the primary context and
// this module's copy of the array with it) the next call looks the address up
// again in the new context instead of using a stale one.  All calls share the array and it keeps the last
// call's contents: the counters are cleared at the start of each call, and
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the array and must be serialised by the
// caller.  The work is the plain FP32 candidate search, the exact re-rank and
// the exact full-scan fallback of mecuco_knn, so the lists are the same as
// mecuco_knn(..., MECUCO_PREC_FP32, ...) returns.
#include <cuda.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {
namespace {

constexpr size_t NOALLOC_BYTES = (size_t)32 << 20;      // 32 MiB
constexpr int64_t NOALLOC_MAX_N = (int64_t)1 << 22;      // 4,194,304 rows (16 MiB of norms)
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
CUcontext g_noalloc_ctx[NOALLOC_MAX_DEVICES] = {};

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// cuCtxGetCurrent from the driver the runtime already loaded (no -lcuda).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

// Device address of the scratch array on the current device (looked up once
// per device and context).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    CUcontext cur = nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
    if (!g_noalloc_addr[dev] || !get || !cur || cur != g_noalloc_ctx[dev]) {
        // the lookup binds the device's primary context if none is current yet,
        // so the context is read again after it
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
        g_noalloc_addr[dev] = p;
        g_noalloc_ctx[dev] = cur;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace mecuco

using namespace mecuco;

extern "C" MECUCO_API mecuco_status mecuco_knn_noalloc(const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                                                       int64_t ld, int k, int include_self, int32_t *idx_out,
                                                       float *dist_out, void *stream) {
    if (!X || !idx_out) return MECUCO_ERR_INVALID_ARG;
    if (dt != MECUCO_F32 && dt != MECUCO_BF16) return MECUCO_ERR_INVALID_ARG;
    if (include_self != 0 && include_self != 1) return MECUCO_ERR_INVALID_ARG;
    if (N < 2 || m < 1 || ld < m || k < 2 || k > 64 || (int64_t)k > N - (include_self ? 0 : 1))
        return MECUCO_ERR_INVALID_ARG;
    if (N > NOALLOC_MAX_N) {
        char msg[160];
        snprintf(msg, sizeof(msg), "mecuco_knn_noalloc: N = %lld exceeds the maximum of %lld rows of its fixed scratch",
                 (long long)N, (long long)NOALLOC_MAX_N);
        set_error_text(msg);
        return MECUCO_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return MECUCO_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MECUCO_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MECUCO_ERR_CUDA;

    // candidate capacity and work split as mecuco_knn's plain form (margin 32)
    int kc = (k + 32 + 31) / 32 * 32;
    if (kc > 128) kc = 128;
    // layout: counters | norms (N) | flags (qchunk) | cand_d, cand_i (qchunk * nsplit * kc)
    const size_t fixed = up256(sizeof(DevCounters)) + up256((size_t)N * sizeof(float));
    int64_t qchunk = std::min<int64_t>(N, 16384);
    const int64_t qblocks = (qchunk + 127) / 128;
    int nsplit = 1;
    if (qblocks < 2LL * sms) nsplit = (int)std::min<int64_t>((2LL * sms + qblocks - 1) / qblocks, 1024 / kc);
    while (nsplit > 1 && (N + nsplit - 1) / nsplit < kc) --nsplit;
    auto need = [&](int64_t qc, int ns) {
        return fixed + up256((size_t)qc * sizeof(int32_t)) + 2 * up256((size_t)qc * ns * kc * sizeof(float));
    };
    while (nsplit > 1 && need(qchunk, nsplit) > NOALLOC_BYTES) --nsplit;
    while (qchunk > 128 && need(qchunk, nsplit) > NOALLOC_BYTES) qchunk /= 2;
    if (need(qchunk, nsplit) > NOALLOC_BYTES) {
        char msg[160];
        snprintf(msg, sizeof(msg), "mecuco_knn_noalloc: N = %lld needs more than the %zu bytes of its fixed scratch",
                 (long long)N, NOALLOC_BYTES);
        set_error_text(msg);
        return MECUCO_ERR_INVALID_ARG;
    }

    char *p = static_cast<char *>(base);
    DevCounters *ctr = reinterpret_cast<DevCounters *>(p);
    p += up256(sizeof(DevCounters));
    float *norms = reinterpret_cast<float *>(p);
    p += up256((size_t)N * sizeof(float));
    int32_t *flags = reinterpret_cast<int32_t *>(p);
    p += up256((size_t)qchunk * sizeof(int32_t));
    float *cand_d = reinterpret_cast<float *>(p);
    p += up256((size_t)qchunk * nsplit * kc * sizeof(float));
    int32_t *cand_i = reinterpret_cast<int32_t *>(p);

    if (cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s) != cudaSuccess) return MECUCO_ERR_CUDA;
    if (launch_rownorm(X, dt, N, m, ld, norms, s) != cudaSuccess) return MECUCO_ERR_CUDA;
    for (int64_t q0 = 0; q0 < N; q0 += qchunk) {
        const int64_t nq = std::min(qchunk, N - q0);
        int32_t *io = idx_out + q0 * k;
        float *dout = dist_out ? dist_out + q0 * k : nullptr;
        if (launch_knn_simt(X, dt, N, m, ld, norms, q0, nq, kc, nsplit, include_self, cand_d, cand_i, s) !=
            cudaSuccess)
            return MECUCO_ERR_CUDA;
        if (launch_knn_rerank(X, dt, N, m, ld, norms, q0, nq, kc, nsplit, k, cand_d, cand_i, io, dout, flags, ctr,
                              s) != cudaSuccess)
            return MECUCO_ERR_CUDA;
        if (launch_knn_fallback(X, dt, N, m, ld, q0, nq, k, include_self, flags, io, dout, ctr, s) != cudaSuccess)
            return MECUCO_ERR_CUDA;
    }
    return MECUCO_OK;
}
