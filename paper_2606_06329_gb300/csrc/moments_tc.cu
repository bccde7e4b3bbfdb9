// moments_tc.cu - Steps 2-3 for the BF16-mixed form: gather and centre each
// patch once per pass and produce, on the 5th-generation tensor cores, every
// moment the estimator needs:
//   M[a][b][t] = sum_c X_c[a,c] X_c[b,c] X_c[t,c]   (pairs a <= b, all t)
//   G[a][b]    = sum_c X_c[a,c] X_c[b,c]             (= X_c X_c^T, eq. svd_cov)
//   Q[a][b]    = sum_c w_c X_c[a,c] X_c[b,c],  w_c = sum_j X_c[j,c]^2 (Haar term)
//   R[a]       = sum_c X_c[a,c]
// as one GEMM per 128-pair tile: D = Z B^T with
//   Z[(a,b), c] = X_c[a,c] X_c[b,c]  (rows in pair order, pair(a,b) = a k - a(a-1)/2 + b - a)
//   B = [X_c ; 1 ; w]                  (k + 2 rows, zero-padded to N = 16 ceil((k+2)/16))
// so D[(a,b), t] = M[a][b][t], D[(a,b), k] = G[a][b], D[(a,b), k+1] = Q[a][b].
//
// One CTA (256 threads) per patch.  The column range of the patch is streamed
// in 64-column chunks: the CUDA cores gather the k neighbour rows, centre each
// column (x - mean over the k rows) in FP32, accumulate R, form w, and write Z
// and B as BF16 into a 128-byte-swizzled, K-major operand buffer (two buffers,
// so building chunk i+1 overlaps the MMAs of chunk i); one thread then issues
// tcgen05.mma (M=128, N, K=16) for every tile of the current pass into TMEM
// with FP32 accumulation.  TMEM holds up to TPP tiles, so the tiles are covered
// in passes over the columns (re-reading the patch from L2).  After a pass the
// 8 warps drain TMEM straight to the pair-major M buffer, G and Q.
// Every mbarrier wait is bounded (MECUCO_ERR_TIMEOUT, no trap).
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int MT_THREADS = 256;
constexpr int MT_CH = 64;              // columns per chunk (one 128-byte swizzle row of BF16)
constexpr int MT_TPP = 5;              // tiles per pass (shared-memory bound)
constexpr int MT_TILE_BYTES = 128 * 128;   // 128 rows x 128 bytes
constexpr int MT_BMAX_ROWS = 80;           // k <= 64 -> N <= 80
constexpr int MT_B_BYTES = MT_BMAX_ROWS * 128;
constexpr int MT_BUF_BYTES = MT_TPP * MT_TILE_BYTES + MT_B_BYTES;
constexpr int MT_XS_LD = 68;               // FP32 staging row stride (floats)
constexpr long long MT_WAIT = 1000000000LL;

__device__ __forceinline__ uint32_t sw128(int row, int unit16) {
    // byte offset of 16-byte unit `unit16` (0..7) of `row` in a 128B-swizzled K-major tile
    return (uint32_t)(row * 128 + ((unit16 ^ (row & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
}  // namespace

__host__ __device__ inline int moments_tc_n(int k) { return ((k + 2 + 15) / 16) * 16; }

size_t moments_tc_smem_bytes() {
    return 1024 + 2 * (size_t)MT_BUF_BYTES + (size_t)64 * MT_XS_LD * sizeof(float) + 64 * sizeof(float) +
           MT_CH * sizeof(float) + 64;
}

template <typename T>
__global__ void __launch_bounds__(MT_THREADS, 1)
moments_tc_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx, int k,
                  const int32_t *__restrict__ pair_ab, float *__restrict__ M, float *__restrict__ G,
                  float *__restrict__ R, float *__restrict__ Q, DevCounters *ctr) {
    extern __shared__ __align__(1024) uint8_t msm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(msm_raw) + 1023) & ~(uintptr_t)1023);
    float *Xs = reinterpret_cast<float *>(base + 2 * MT_BUF_BYTES);  // [64][MT_XS_LD] centred chunk
    float *Rs = Xs + 64 * MT_XS_LD;                                  // [64]
    float *Ws = Rs + 64;                                             // [MT_CH] column weights w_c
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
    // commits issued so far on mma_done[0] / mma_done[1] (uniform across threads)
    uint32_t commits0 = 0, commits1 = 0;

    for (int t0 = 0; t0 < ntiles && !*abortp; t0 += tpp) {
        const int nt = min(tpp, ntiles - t0);
        for (int ci = 0; ci < nchunks; ++ci) {
            const int b = ci & 1;
            uint8_t *ob = base + b * MT_BUF_BYTES;
            const int64_t a0 = (int64_t)ci * MT_CH;
            const uint32_t cb = b ? commits1 : commits0;
            // buffer b is free once the MMAs of the chunk that used it completed
            if (cb > 0) {
                if (!tc::mbar_wait(tc::smem_u32(&mma_done[b]), (cb - 1) & 1, abortp, MT_WAIT)) {
                    if (tid == 0) { atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT); abort_flag = 1; }
                }
            }
            // ---- gather the k rows of this chunk into FP32 staging (8 columns per unit)
            for (int u = tid; u < 64 * 8; u += MT_THREADS) {
                const int j = u >> 3, g = u & 7;
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = 0.f;
                if (j < k) {
                    const T *src = X + (int64_t)rows[j] * ld + a0 + g * 8;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (a0 + g * 8 + e < m) v[e] = load_elem(src + e);
                }
                float4 *dst = reinterpret_cast<float4 *>(Xs + j * MT_XS_LD + g * 8);
                dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                dst[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
            __syncthreads();
            // ---- centre each column, column weights w_c, row sums R
            if (tid < MT_CH) {
                float s = 0.f;
                for (int j = 0; j < k; ++j) s += Xs[j * MT_XS_LD + tid];
                const float mean = s / (float)k;
                float w = 0.f;
                for (int j = 0; j < k; ++j) {
                    const float x = Xs[j * MT_XS_LD + tid] - mean;
                    Xs[j * MT_XS_LD + tid] = x;
                    w = fmaf(x, x, w);
                }
                Ws[tid] = (a0 + tid < m) ? w : 0.f;
            }
            __syncthreads();
            if (t0 == 0 && tid < k) {
                float s = 0.f;
                for (int c = 0; c < MT_CH; ++c) s += Xs[tid * MT_XS_LD + c];
                Rs[tid] += s;
            }
            // ---- B operand: rows 0..k-1 = X_c, row k = 1, row k+1 = w, rest 0
            uint8_t *bb = ob + MT_TPP * MT_TILE_BYTES;
            for (int u = tid; u < Nb * 8; u += MT_THREADS) {
                const int r = u >> 3, g = u & 7;
                float v[8];
                if (r < k) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = Xs[r * MT_XS_LD + g * 8 + e];
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
                uint4 pk = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                                      pack_bf16x2(v[6], v[7]));
                *reinterpret_cast<uint4 *>(bb + sw128(r, g)) = pk;
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
                const int tile = rl >> 7, row = rl & 127;
                *reinterpret_cast<uint4 *>(ob + tile * MT_TILE_BYTES + sw128(row, g)) = pk;
            }
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
        if (commits0 > 0) tc::mbar_wait(tc::smem_u32(&mma_done[0]), (commits0 - 1) & 1, &never, MT_WAIT);
        if (commits1 > 0) tc::mbar_wait(tc::smem_u32(&mma_done[1]), (commits1 - 1) & 1, &never, MT_WAIT);
        tc::fence_after();
        const int quarter = warp & 3, half = warp >> 2;
        for (int t = half; t < nt; t += 2) {
            const int pr = (t0 + t) * 128 + quarter * 32 + lane;
            const bool valid = pr < npairs;
            int pa = 0, pb = 0;
            if (valid) { const int code = __ldg(pair_ab + pr); pa = code & 0xffff; pb = code >> 16; }
            float *mrow = M + (pt * (int64_t)npairs + (valid ? pr : 0)) * k;
            for (int c0 = 0; c0 < Nb; c0 += 16) {
                uint32_t r[32];
                // 16 columns per load: use the x32 form on 32-column groups when possible
                if (c0 + 32 <= Nb && (c0 & 31) == 0) {
                    tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * Nb + c0), r);
                    tc::tmem_ld_wait();
                    if (valid) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = c0 + j;
                            const float v = __uint_as_float(r[j]);
                            if (col < k) mrow[col] = v;
                            else if (col == k) { G[pt * k * k + pa * k + pb] = v; G[pt * k * k + pb * k + pa] = v; }
                            else if (col == k + 1 && Q) { Q[pt * k * k + pa * k + pb] = v; Q[pt * k * k + pb * k + pa] = v; }
                        }
                    }
                    c0 += 16;
                } else {
                    uint32_t r16[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                        : "=r"(r16[0]), "=r"(r16[1]), "=r"(r16[2]), "=r"(r16[3]), "=r"(r16[4]), "=r"(r16[5]),
                          "=r"(r16[6]), "=r"(r16[7]), "=r"(r16[8]), "=r"(r16[9]), "=r"(r16[10]), "=r"(r16[11]),
                          "=r"(r16[12]), "=r"(r16[13]), "=r"(r16[14]), "=r"(r16[15])
                        : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * Nb + c0)));
                    tc::tmem_ld_wait();
                    if (valid) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int col = c0 + j;
                            const float v = __uint_as_float(r16[j]);
                            if (col < k) mrow[col] = v;
                            else if (col == k) { G[pt * k * k + pa * k + pb] = v; G[pt * k * k + pb * k + pa] = v; }
                            else if (col == k + 1 && Q) { Q[pt * k * k + pa * k + pb] = v; Q[pt * k * k + pb * k + pa] = v; }
                        }
                    }
                }
                (void)r;
            }
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
