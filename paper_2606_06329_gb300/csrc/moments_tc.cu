// moments_tc.cu - Steps 2-3 for the BF16-mixed form: gather and centre each
// patch and produce, on the 5th-generation tensor cores, every moment the
// estimator needs:
//   M[a][b][t] = sum_c X_c[a,c] X_c[b,c] X_c[t,c]   (pairs a <= b, all t)
//   G[a][b]    = sum_c X_c[a,c] X_c[b,c]             (= X_c X_c^T, eq. svd_cov)
//   Q[a][b]    = sum_c w_c X_c[a,c] X_c[b,c],  w_c = sum_j X_c[j,c]^2 (Haar term)
//   R[a]       = sum_c X_c[a,c]
// as one GEMM per 128-pair tile: D = Z B^T with
//   Z[(a,b), c] = X_c[a,c] X_c[b,c]  (rows in pair order, pair(a,b) = a k - a(a-1)/2 + b - a)
//   B = [X_c ; 1 ; w]                  (k + 2 rows, zero-padded to N = 16 ceil((k+2)/16))
// so D[(a,b), t] = M[a][b][t], D[(a,b), k] = G[a][b], D[(a,b), k+1] = Q[a][b].
//
// One CTA (512 threads) per patch.  The columns of the patch are streamed in
// 64-column chunks: the CUDA cores gather the k neighbour rows (the next
// chunk's loads are issued before the current chunk is processed, so their
// latency hides behind it), centre each column (x - mean over the k rows) in
// FP32, accumulate R, form w, and write Z and B as BF16 into a 128-byte-
// swizzled K-major operand buffer (two buffers: building chunk i+1 overlaps
// the MMAs of chunk i); one thread issues tcgen05.mma (M=128, N, K=16) for
// every tile of the current pass into TMEM (FP32 accumulation).  TMEM holds up
// to TPP tiles, so the tiles are covered in passes over the columns (re-reading
// the patch from L2).  After a pass the warps drain TMEM through shared memory
// so each tile's 128 pair rows (contiguous in the pair-major M buffer) leave as
// coalesced stores.  Every mbarrier wait is bounded (MECUCO_ERR_TIMEOUT, no
// trap).
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int MT_THREADS = 512;
constexpr int MT_CH = 64;                  // columns per chunk (one 128-byte swizzle row of BF16)
constexpr int MT_TPP = 5;                  // tiles per pass (shared-memory bound)
constexpr int MT_TILE_BYTES = 128 * 128;   // 128 rows x 128 bytes
constexpr int MT_BMAX_ROWS = 80;           // k <= 64 -> N <= 80
constexpr int MT_B_BYTES = MT_BMAX_ROWS * 128;
constexpr int MT_BUF_BYTES = MT_TPP * MT_TILE_BYTES + MT_B_BYTES;
constexpr int MT_XS_LD = 68;               // FP32 staging row stride (floats)
constexpr int MT_XS_FLOATS = 64 * MT_XS_LD;
constexpr long long MT_WAIT = 1000000000LL;

__device__ __forceinline__ uint32_t sw128(int row, int unit16) {
    // byte offset of 16-byte unit `unit16` (0..7) of `row` in a 128B-swizzled K-major tile
    return (uint32_t)(row * 128 + ((unit16 ^ (row & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Raw gather of one 8-column unit of one row (zero past m).
template <typename T>
struct Unit8;
template <>
struct Unit8<__nv_bfloat16> {
    uint4 v;
    __device__ __forceinline__ void load(const __nv_bfloat16 *row, int64_t a, int64_t m, bool vec) {
        if (vec && a + 8 <= m) {
            v = __ldg(reinterpret_cast<const uint4 *>(row + a));
        } else {
            uint32_t h[8];
            for (int e = 0; e < 8; ++e)
                h[e] = (a + e < m) ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(row) + a + e) : 0u;
            v = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
    }
    __device__ __forceinline__ void zero() { v = make_uint4(0, 0, 0, 0); }
    __device__ __forceinline__ void store(float *dst) const {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        float f[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            f[2 * e] = __uint_as_float(w[e] << 16);
            f[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
        }
        reinterpret_cast<float4 *>(dst)[0] = make_float4(f[0], f[1], f[2], f[3]);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(f[4], f[5], f[6], f[7]);
    }
};
template <>
struct Unit8<float> {
    float4 lo, hi;
    __device__ __forceinline__ void load(const float *row, int64_t a, int64_t m, bool vec) {
        if (vec && a + 8 <= m) {
            lo = __ldg(reinterpret_cast<const float4 *>(row + a));
            hi = __ldg(reinterpret_cast<const float4 *>(row + a) + 1);
        } else {
            float f[8];
            for (int e = 0; e < 8; ++e) f[e] = (a + e < m) ? __ldg(row + a + e) : 0.f;
            lo = make_float4(f[0], f[1], f[2], f[3]);
            hi = make_float4(f[4], f[5], f[6], f[7]);
        }
    }
    __device__ __forceinline__ void zero() { lo = hi = make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ void store(float *dst) const {
        reinterpret_cast<float4 *>(dst)[0] = lo;
        reinterpret_cast<float4 *>(dst)[1] = hi;
    }
};
}  // namespace

__host__ __device__ inline int moments_tc_n(int k) { return ((k + 2 + 15) / 16) * 16; }

size_t moments_tc_smem_bytes() {
    return 1024 + 2 * (size_t)MT_BUF_BYTES + 2 * (size_t)MT_XS_FLOATS * sizeof(float) + 64 * sizeof(float) +
           MT_CH * sizeof(float) + 8 * 64 * sizeof(float) + 64;
}

template <typename T>
__global__ void __launch_bounds__(MT_THREADS, 1)
moments_tc_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx, int k,
                  const int32_t *__restrict__ pair_ab, float *__restrict__ M, float *__restrict__ G,
                  float *__restrict__ R, float *__restrict__ Q, DevCounters *ctr) {
    extern __shared__ __align__(1024) uint8_t msm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(msm_raw) + 1023) & ~(uintptr_t)1023);
    float *Xs0 = reinterpret_cast<float *>(base + 2 * MT_BUF_BYTES);  // two [64][MT_XS_LD] staging chunks
    float *Rs = Xs0 + 2 * MT_XS_FLOATS;                                // [64]
    float *Ws = Rs + 64;                                               // [MT_CH] column weights w_c
    float *Part = Ws + MT_CH;                                          // [8][64] centring partials
    __shared__ uint64_t mma_done[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int rows[64];
    __shared__ int abort_flag, never;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t pt = blockIdx.x;
    const int npairs = k * (k + 1) / 2;
    const int ntiles = (npairs + 127) / 128;
    const int Nb = moments_tc_n(k);
    const int tpp = min(MT_TPP, 512 / Nb);
    const int nchunks = (int)((m + MT_CH - 1) / MT_CH);
    const uint32_t idesc = tc::idesc_bf16_f32(128, Nb);
    const bool vec = (ld % 8 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

    if (tid < 64) {
        int r = 0;
        if (tid < k) {
            r = idx[pt * k + tid];
            if (r < 0 || (int64_t)r >= N) { atomicOr(&ctr->status, (unsigned)DEV_INVALID); r = 0; }
        }
        rows[tid] = r;
        Rs[tid] = 0.f;
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mma_done[0]), 1);
        tc::mbar_init(tc::smem_u32(&mma_done[1]), 1);
        abort_flag = (*(volatile unsigned *)&ctr->status & DEV_TIMEOUT) ? 1 : 0;
        never = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), 512);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abortp = &abort_flag;
    uint32_t commits0 = 0, commits1 = 0;  // commits issued on mma_done[0] / [1] (uniform across threads)

    // gather unit of this thread: row gj, 8-column group gg (64 rows x 8 groups = 512 units)
    const int gj = tid >> 3, gg = tid & 7;
    const T *grow = X + (int64_t)rows[gj] * ld;
    Unit8<T> pre;

    for (int t0 = 0; t0 < ntiles && !*abortp; t0 += tpp) {
        const int nt = min(tpp, ntiles - t0);
        // prologue: chunk 0 into staging 0
        if (gj < k) pre.load(grow, gg * 8, m, vec); else pre.zero();
        pre.store(Xs0 + gj * MT_XS_LD + gg * 8);
        for (int ci = 0; ci < nchunks; ++ci) {
            const int b = ci & 1;
            float *Xs = Xs0 + b * MT_XS_FLOATS;
            uint8_t *ob = base + b * MT_BUF_BYTES;
            const int64_t a0 = (int64_t)ci * MT_CH;
            // issue the next chunk's loads now; they land while this chunk is processed
            const bool has_next = ci + 1 < nchunks;
            if (has_next) {
                if (gj < k) pre.load(grow, a0 + MT_CH + gg * 8, m, vec); else pre.zero();
            }
            __syncthreads();  // staging b complete
            // ---- centre each column over the k rows: thread (column cc, row group rg)
            // owns rows 8 rg .. 8 rg + 7; column sums and sums of squares go through
            // shared partials (8 groups per column)
            {
                const int cc = tid & 63, rg = tid >> 6;
                float v[8], s = 0.f;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    v[e] = Xs[(rg * 8 + e) * MT_XS_LD + cc];  // rows >= k hold zeros
                    s += v[e];
                }
                Part[rg * 64 + cc] = s;
                __syncthreads();
                float tot = 0.f;
#pragma unroll
                for (int g = 0; g < 8; ++g) tot += Part[g * 64 + cc];
                const float mean = tot / (float)k;
                float w = 0.f, rsum[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const bool real = rg * 8 + e < k;
                    const float x = real ? v[e] - mean : 0.f;
                    Xs[(rg * 8 + e) * MT_XS_LD + cc] = x;
                    w = fmaf(x, x, w);
                    rsum[e] = x;
                }
                __syncthreads();  // every thread has read Part
                Part[rg * 64 + cc] = w;
                // row sums R (first pass only): warp-reduce each of the 8 rows over 32 columns
                if (t0 == 0) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float r = warp_sum(rsum[e]);
                        if (lane == 0 && rg * 8 + e < k) atomicAdd(&Rs[rg * 8 + e], r);
                    }
                }
                __syncthreads();
                if (rg == 0) {
                    float ws = 0.f;
#pragma unroll
                    for (int g = 0; g < 8; ++g) ws += Part[g * 64 + cc];
                    Ws[cc] = (a0 + cc < m) ? ws : 0.f;
                }
            }
            // operand buffer b is free once the MMAs of the chunk that last used it completed
            const uint32_t cb = b ? commits1 : commits0;
            if (tid == 0 && cb > 0) {
                if (!tc::mbar_wait(tc::smem_u32(&mma_done[b]), (cb - 1) & 1, abortp, MT_WAIT)) {
                    atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
                    abort_flag = 1;
                }
            }
            __syncthreads();
            // ---- B operand: rows 0..k-1 = X_c, row k = 1, row k+1 = w, rest 0
            uint8_t *bb = ob + MT_TPP * MT_TILE_BYTES;
            for (int u = tid; u < Nb * 8; u += MT_THREADS) {
                const int r = u >> 3, g = u & 7;
                float v[8];
                if (r < k) {
                    const float4 lo = reinterpret_cast<const float4 *>(Xs + r * MT_XS_LD + g * 8)[0];
                    const float4 hi = reinterpret_cast<const float4 *>(Xs + r * MT_XS_LD + g * 8)[1];
                    v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
                    v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
                } else if (r == k) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = (a0 + g * 8 + e < m) ? 1.f : 0.f;
                } else if (r == k + 1) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = Ws[g * 8 + e];
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = 0.f;
                }
                *reinterpret_cast<uint4 *>(bb + sw128(r, g)) =
                    make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                               pack_bf16x2(v[6], v[7]));
            }
            // ---- A operand: Z rows of this pass's tiles
            for (int u = tid; u < nt * 128 * 8; u += MT_THREADS) {
                const int rl = u >> 3, g = u & 7;  // row within the pass, 16-byte unit
                const int pr = t0 * 128 + rl;
                uint4 pk = make_uint4(0, 0, 0, 0);
                if (pr < npairs) {
                    const int code = __ldg(pair_ab + pr);
                    const int pa = code & 0xffff, pb = code >> 16;
                    const float4 *xa = reinterpret_cast<const float4 *>(Xs + pa * MT_XS_LD + g * 8);
                    const float4 *xb = reinterpret_cast<const float4 *>(Xs + pb * MT_XS_LD + g * 8);
                    const float4 a_lo = xa[0], a_hi = xa[1], b_lo = xb[0], b_hi = xb[1];
                    pk = make_uint4(pack_bf16x2(a_lo.x * b_lo.x, a_lo.y * b_lo.y),
                                    pack_bf16x2(a_lo.z * b_lo.z, a_lo.w * b_lo.w),
                                    pack_bf16x2(a_hi.x * b_hi.x, a_hi.y * b_hi.y),
                                    pack_bf16x2(a_hi.z * b_hi.z, a_hi.w * b_hi.w));
                }
                *reinterpret_cast<uint4 *>(ob + (rl >> 7) * MT_TILE_BYTES + sw128(rl & 127, g)) = pk;
            }
            // the next chunk's raw values go to the other staging buffer
            if (has_next) pre.store(Xs0 + (b ^ 1) * MT_XS_FLOATS + gj * MT_XS_LD + gg * 8);
            // make the generic-proxy stores visible to the tensor core, then issue
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0 && !*abortp) {
                tc::fence_after();
                const uint32_t bsa = tc::smem_u32(bb);
                for (int t = 0; t < nt; ++t) {
                    const uint32_t asa = tc::smem_u32(ob + t * MT_TILE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < MT_CH / 16; ++kk)
                        tc::mma_f16(tmem + (uint32_t)(t * Nb), tc::sdesc_sw128(asa + kk * 32),
                                    tc::sdesc_sw128(bsa + kk * 32), idesc, (ci | kk) != 0);
                }
                tc::commit(tc::smem_u32(&mma_done[b]));
            }
            if (b) ++commits1; else ++commits0;
        }
        // ---- wait for the last MMAs of the pass (bounded), then drain TMEM
        if (tid == 0) {
            if (commits0 > 0) tc::mbar_wait(tc::smem_u32(&mma_done[0]), (commits0 - 1) & 1, &never, MT_WAIT);
            if (commits1 > 0) tc::mbar_wait(tc::smem_u32(&mma_done[1]), (commits1 - 1) & 1, &never, MT_WAIT);
        }
        __syncthreads();
        tc::fence_after();
        // warp group wg = warp / 4 drains tiles wg, wg + 4, ... into its own staging
        // slot (128 x k floats) in the now idle operand buffers
        const int quarter = warp & 3, wg = warp >> 2;
        const size_t slot_bytes = 128 * 64 * sizeof(float);
        float *stage = reinterpret_cast<float *>(base + (size_t)wg * slot_bytes);
        for (int tb = 0; tb < nt; tb += 4) {
            const int t = tb + wg;
            const bool active = t < nt;
            const int row = quarter * 32 + lane;
            const int pr = (t0 + t) * 128 + row;
            const bool valid = active && pr < npairs;
            int pa = 0, pb = 0;
            if (valid) { const int code = __ldg(pair_ab + pr); pa = code & 0xffff; pb = code >> 16; }
            if (active) {
                for (int c0 = 0; c0 < Nb; c0 += 16) {
                    uint32_t r16[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                        : "=r"(r16[0]), "=r"(r16[1]), "=r"(r16[2]), "=r"(r16[3]), "=r"(r16[4]), "=r"(r16[5]),
                          "=r"(r16[6]), "=r"(r16[7]), "=r"(r16[8]), "=r"(r16[9]), "=r"(r16[10]), "=r"(r16[11]),
                          "=r"(r16[12]), "=r"(r16[13]), "=r"(r16[14]), "=r"(r16[15])
                        : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * Nb + c0)));
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = c0 + j;
                        const float v = __uint_as_float(r16[j]);
                        if (col < k) stage[row * k + col] = v;
                        else if (valid && col == k) {
                            G[pt * k * k + pa * k + pb] = v;
                            G[pt * k * k + pb * k + pa] = v;
                        } else if (valid && col == k + 1 && Q) {
                            Q[pt * k * k + pa * k + pb] = v;
                            Q[pt * k * k + pb * k + pa] = v;
                        }
                    }
                }
            }
            __syncthreads();
            // coalesced copy of the staged tiles: rows [r0, min(npairs, r0 + 128)) x k floats are contiguous
            for (int g4 = 0; g4 < 4; ++g4) {
                const int tt = tb + g4;
                if (tt >= nt) break;
                const int r0 = (t0 + tt) * 128;
                const int nf = min(128, npairs - r0) * k;
                const float *src = reinterpret_cast<const float *>(base + (size_t)g4 * slot_bytes);
                float *dst = M + (pt * (int64_t)npairs + r0) * k;
                for (int e = tid; e < nf; e += MT_THREADS) dst[e] = src[e];
            }
            __syncthreads();
        }
        tc::fence_before();
        __syncthreads();
    }
    if (tid < k) R[pt * k + tid] = Rs[tid];
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

void moments_tc_build_pairs(int k, int32_t *pair_ab) {
    int n = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a; b < k; ++b) pair_ab[n++] = a | (b << 16);
}

cudaError_t launch_moments_tc(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                              int k, int64_t np, const int32_t *pair_ab, float *M, float *G, float *R, float *Q,
                              DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64 || k < 2) return cudaErrorInvalidValue;
    const size_t smem = moments_tc_smem_bytes();
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(moments_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        moments_tc_kernel<<<(unsigned)np, MT_THREADS, smem, s>>>((const __nv_bfloat16 *)X, N, m, ld, idx, k, pair_ab,
                                                                 M, G, R, Q, ctr);
    } else {
        e = cudaFuncSetAttribute(moments_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        moments_tc_kernel<<<(unsigned)np, MT_THREADS, smem, s>>>((const float *)X, N, m, ld, idx, k, pair_ab, M, G,
                                                                 R, Q, ctr);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
