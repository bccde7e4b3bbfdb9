// gram_tc.cu - the Gram pass of the BF16-mixed estimator (Sec. 3 Step 2;
// eq. svd_cov; Alg. 1 Fast branch): per patch, on the tensor cores,
//   G = X_c X_c^T                          (k x k)
//   Q = X_c diag(w) X_c^T, w_c = sum_j X_c[j,c]^2   (k x k, Haar variant)
// and on the CUDA cores R = X_c 1_m.
//
// One CTA per patch.  8 producer warps gather the k neighbour rows of each
// 64-column chunk (the next chunk's loads in flight), centre every column in
// FP32 (pg::centre_chunk, as the rotation pass does) and write a 128-row
// K-major tile with the 128-byte swizzle: rows 0..63 the BF16 patch X_c (rows
// past k zero), rows 64..127 the BF16 products w (.) x_j (HMUL2 of BF16 w and
// BF16 x_j; zero for the literal variant).  One MMA thread accumulates
// D = tile * X_c^T over the chunks (M = 128, N = 16 ceil(k / 16), B = the
// tile's first rows), so D's rows 0..k-1 are G and rows 64..64+k-1 are Q.
// The tile is double-buffered; after the last chunk the producer warps read D
// (tcgen05.ld) and store G and Q.  Every wait is bounded (MECUCO_ERR_TIMEOUT,
// no trap) and the MMA thread waits for its last MMAs before tensor memory is
// freed.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "patch_gather.cuh"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int GT_PRODUCER_WARPS = 8;
constexpr int GT_THREADS = (GT_PRODUCER_WARPS + 1) * 32;  // + the MMA warp
constexpr int GT_CH = 64;
constexpr int GT_XS_LD = 68;
constexpr int GT_TILE = 128 * 128;  // 128 rows x 64 K (BF16)
constexpr long long GT_WAIT = 1000000000LL;
using pg::load_halves;
using pg::pack_bf16x2;
using pg::sw128;
using pg::Unit8;
}  // namespace

size_t gram_tc_smem_bytes() { return 1024 + 2 * (size_t)GT_TILE + 64 * (size_t)GT_XS_LD * 4 + 4 * 64 * 4; }

// two CTAs per SM (113 registers a thread): the gather needs warps in flight
template <typename T>
__global__ void __launch_bounds__(GT_THREADS, 2)
gram_tc_kernel(const __grid_constant__ PatchSeg one, const PatchSeg *__restrict__ tab, int ntab, int with_q,
               long long wait_limit, DevCounters *ctr) {
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *Tile0 = base;                                           // 2 x 128-row tile
    float *Xs = reinterpret_cast<float *>(Tile0 + 2 * GT_TILE);     // [64][68] FP32 staging
    float *Part = Xs + 64 * GT_XS_LD;                                // [4][64] column partials
    __shared__ uint64_t t_full[2], t_empty[2], d_full, mma_fin;
    __shared__ uint32_t tmem_slot;
    __shared__ int rows[64];
    __shared__ int abort_flag, never;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int local;
    const PatchSeg &seg = find_seg(one, tab, ntab, (int)blockIdx.x, local);
    const T *X = static_cast<const T *>(seg.X);
    const int64_t N = seg.N, m = seg.m, ld = seg.ld, pt = local;
    const int k = seg.k;
    const int32_t *idx = seg.idx;
    float *G = seg.G, *R = seg.R, *Q = with_q ? seg.Q : nullptr;
    const int nchunks = (int)((m + GT_CH - 1) / GT_CH);
    const int Nb = k <= 16 ? 16 : ((k + 15) / 16) * 16;
    const uint32_t idesc = tc::idesc_bf16_f32(128, Nb);
    const bool vec = (ld % 8 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

    if (tid < 64) {
        int r = 0;
        if (tid < k) {
            r = idx[pt * k + tid];
            if (r < 0 || (int64_t)r >= N) { atomicOr(&ctr->status, (unsigned)DEV_INVALID); r = 0; }
        }
        rows[tid] = r;
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tc::smem_u32(&t_full[b]), 1);
            tc::mbar_init(tc::smem_u32(&t_empty[b]), 1);
        }
        tc::mbar_init(tc::smem_u32(&d_full), 1);
        tc::mbar_init(tc::smem_u32(&mma_fin), 1);
        abort_flag = (*(volatile unsigned *)&ctr->status & DEV_TIMEOUT) ? 1 : 0;
        never = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), 64);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abortp = &abort_flag;
    auto fail = [&]() {
        atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
        abort_flag = 1;
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (!*abortp && !tc::mbar_wait(tc::smem_u32(bar), parity, abortp, wait_limit)) fail();
    };

    if (warp < GT_PRODUCER_WARPS) {
        // ============ producers: gather, centre, tile; read G and Q back ============
        const int ptid = tid;
        const int gr0 = ptid >> 3, gg = ptid & 7;
        const T *grow0 = X + (int64_t)rows[gr0] * ld;
        const T *grow1 = X + (int64_t)rows[gr0 + 32] * ld;
        const bool live0 = gr0 < k, live1 = gr0 + 32 < k;
        const int cc = ptid & 63, rg = ptid >> 6;
        const float inv_k = 1.f / (float)k;
        float racc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) racc[e] = 0.f;
        Unit8<T> pre0, pre1;
        if (live0) pre0.load(grow0, gg * 8, m, vec); else pre0.zero();
        if (live1) pre1.load(grow1, gg * 8, m, vec); else pre1.zero();
        for (int ci = 0; ci < nchunks; ++ci) {
            const int b = ci & 1;
            pre0.store(Xs + gr0 * GT_XS_LD + gg * 8, gg >= 4);
            pre1.store(Xs + (gr0 + 32) * GT_XS_LD + gg * 8, gg >= 4);
            if (ci + 1 < nchunks) {
                const int64_t an = (int64_t)(ci + 1) * GT_CH + gg * 8;
                if (live0) pre0.load(grow0, an, m, vec); else pre0.zero();
                if (live1) pre1.load(grow1, an, m, vec); else pre1.zero();
            }
            float xc[16];
            pg::centre_chunk<GT_XS_LD>(Xs, Part, cc, rg, k, inv_k, xc);
            float w = 0.f;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                w = fmaf(xc[e], xc[e], w);
                racc[e] += xc[e];
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");  // every thread has read the mean's partials
            Part[rg * 64 + cc] = w;
            // tile b is free once the MMAs of chunk ci - 2 are done with it
            if (ptid == 0 && ci >= 2) wait(&t_empty[b], (uint32_t)((ci >> 1) - 1) & 1u);
            asm volatile("bar.sync 1, 256;" ::: "memory");
            float wsum = 0.f;
            if (ptid < 64) wsum = Part[ptid] + Part[64 + ptid] + Part[128 + ptid] + Part[192 + ptid];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (ptid < 64) Part[ptid] = wsum;  // w_c of the chunk, FP32
            asm volatile("bar.sync 1, 256;" ::: "memory");
            uint8_t *tile = Tile0 + b * GT_TILE;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = gr0 + 32 * h;
                float4 lo, hi;
                load_halves(Xs + r * GT_XS_LD + gg * 8, lo, hi, gg >= 4);
                const uint32_t xw[4] = {pack_bf16x2(lo.x, lo.y), pack_bf16x2(lo.z, lo.w), pack_bf16x2(hi.x, hi.y),
                                        pack_bf16x2(hi.z, hi.w)};
                *reinterpret_cast<uint4 *>(tile + sw128(r, gg)) = make_uint4(xw[0], xw[1], xw[2], xw[3]);
                uint32_t qw[4] = {0u, 0u, 0u, 0u};
                if (with_q) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t wv = pack_bf16x2(Part[gg * 8 + 2 * e], Part[gg * 8 + 2 * e + 1]);
                        __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162 *>(&xw[e]);
                        __nv_bfloat162 w2 = *reinterpret_cast<const __nv_bfloat162 *>(&wv);
                        __nv_bfloat162 pr = __hmul2(x2, w2);
                        qw[e] = *reinterpret_cast<uint32_t *>(&pr);
                    }
                }
                *reinterpret_cast<uint4 *>(tile + sw128(64 + r, gg)) = make_uint4(qw[0], qw[1], qw[2], qw[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (ptid == 0) tc::mbar_arrive(tc::smem_u32(&t_full[b]));
        }
        // R = X_c 1: the column threads' partial sums, reduced per row
#pragma unroll
        for (int e = 0; e < 16; ++e) Xs[(rg * 16 + e) * GT_XS_LD + cc] = racc[e];
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (ptid < k) {
            float r = 0.f;
            for (int c = 0; c < 64; ++c) r += Xs[ptid * GT_XS_LD + c];
            R[pt * k + ptid] = r;
        }
        // G (TMEM lanes 0..k-1) and Q (lanes 64..64+k-1): warp w reads lane
        // quarter w & 3, columns [32 (w >> 2), +32) of the Nb accumulated ones
        if (lane == 0) wait(&d_full, 0u);
        __syncwarp();
        tc::fence_after();
        const int qd = warp & 3, ch = warp >> 2;
        const int lrow = qd * 32 + lane;
        if (ch * 32 < Nb) {
            uint32_t r16[16];
            for (int c0 = ch * 32; c0 < min(Nb, ch * 32 + 32); c0 += 16) {
                tc::tmem_ld_32x32b_x16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0, r16);
                tc::tmem_ld_wait();
                float *dst = nullptr;
                if (lrow < k) dst = G + (pt * k + lrow) * (int64_t)k;
                else if (with_q && lrow >= 64 && lrow - 64 < k) dst = Q + (pt * k + (lrow - 64)) * (int64_t)k;
                if (dst) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c0 + e < k) dst[c0 + e] = __uint_as_float(r16[e]);
                }
            }
        }
        tc::fence_before();
    } else if (lane == 0) {
        // ================= MMA thread =================
        bool ok = true;
        for (int ci = 0; ci < nchunks && ok; ++ci) {
            const int b = ci & 1;
            if (!tc::mbar_wait(tc::smem_u32(&t_full[b]), (uint32_t)(ci >> 1) & 1u, abortp, wait_limit)) {
                fail();
                ok = false;
                break;
            }
            tc::fence_after();
            const uint64_t ad = tc::sdesc_sw128(tc::smem_u32(Tile0 + b * GT_TILE));
#pragma unroll
            for (int kk = 0; kk < GT_CH / 16; ++kk)
                tc::mma_f16(tmem, ad + (uint64_t)(2 * kk), ad + (uint64_t)(2 * kk), idesc, (ci | kk) != 0);
            tc::commit(tc::smem_u32(&t_empty[b]));
        }
        tc::commit(tc::smem_u32(&d_full));
        // every MMA has completed before TMEM is freed (a barrier used once)
        tc::commit(tc::smem_u32(&mma_fin));
        if (!tc::mbar_wait(tc::smem_u32(&mma_fin), 0u, &never, GT_WAIT)) fail();
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 64);
    }
}

cudaError_t launch_gram_tc(mecuco_dtype dt, const PatchSeg &one, const PatchSeg *tab, int ntab, int64_t np,
                           int with_q, long long wait_limit, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (ntab == 0 && (one.k > 64 || one.k < 2)) return cudaErrorInvalidValue;
    if (wait_limit <= 0) wait_limit = GT_WAIT;
    const size_t smem = gram_tc_smem_bytes();
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(gram_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        gram_tc_kernel<__nv_bfloat16><<<(unsigned)np, GT_THREADS, smem, s>>>(one, tab, ntab, with_q, wait_limit, ctr);
    } else {
        e = cudaFuncSetAttribute(gram_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gram_tc_kernel<float><<<(unsigned)np, GT_THREADS, smem, s>>>(one, tab, ntab, with_q, wait_limit, ctr);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
