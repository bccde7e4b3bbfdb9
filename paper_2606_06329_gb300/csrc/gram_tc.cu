// gram_tc.cu - the Gram pass of the BF16-mixed estimator (Sec. 3 Step 2;
// eq. svd_cov; Alg. 1 Fast branch): per patch, on the tensor cores,
//   G = X_c X_c^T                          (k x k)
//   Q = X_c diag(w) X_c^T, w_c = sum_j X_c[j,c]^2   (k x k, Haar variant)
// and on the CUDA cores R = X_c 1_m.
//
// One CTA per patch.  The 256 producer threads gather the k neighbour rows of
// each 64-column chunk into a ring of raw stages with cp.async (five chunks
// in flight for BF16 rows, two for FP32 rows).  Producer warp u then owns
// columns 8u .. 8u + 7 of the chunk, lane l rows l and l + 32: it centres its
// columns in FP32 (pg::centre_lane, as the rotation pass does; the column
// means come from warp shuffles, so a chunk costs the CTA one barrier) and
// writes its units of a 128-row K-major tile with the 128-byte swizzle: rows
// 0..63 the BF16 patch X_c (rows past k zero), rows 64..127 the BF16 products
// w (.) x_j (HMUL2 of BF16 w and BF16 x_j; zero, written once, for the literal
// variant).  One MMA thread accumulates D = tile * X_c^T over the chunks
// (M = 128, N = 16 ceil(k / 16), B = the tile's first rows), so D's rows
// 0..k-1 are G and rows 64..64+k-1 are Q.  The tile is double-buffered, each
// producer warp signalling its part of a tile and waiting for the tile's
// release itself; after the last chunk the producer warps read D
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
constexpr int GT_TILE = 128 * 128;  // 128 rows x 64 K (BF16)
constexpr long long GT_WAIT = 1000000000LL;
// gather ring depth: 6 x 8 KB stages of BF16 rows, 3 x 16 KB of FP32 rows
template <typename T>
__host__ __device__ constexpr int gt_stages() {
    return sizeof(T) == 2 ? 6 : 3;
}
using pg::pack_bf16x2;
using pg::sw128;
}  // namespace

template <typename T>
size_t gram_tc_smem_bytes() {
    return 1024 + 2 * (size_t)GT_TILE + 8 * 64 * 4 + (size_t)gt_stages<T>() * pg::raw_stage_bytes<T>();
}

// two CTAs per SM (~84 KB of shared memory each)
template <typename T>
__global__ void __launch_bounds__(GT_THREADS, 2)
gram_tc_kernel(const __grid_constant__ PatchSeg one, const PatchSeg *__restrict__ tab, int ntab, int with_q,
               long long wait_limit, DevCounters *ctr) {
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *Tile0 = base;                                           // 2 x 128-row tile
    float *Red = reinterpret_cast<float *>(Tile0 + 2 * GT_TILE);    // [8][64] row sums per producer warp
    uint8_t *Raw = reinterpret_cast<uint8_t *>(Red + 8 * 64);        // gather ring
    constexpr int S = gt_stages<T>(), RB = pg::raw_stage_bytes<T>();
    __shared__ uint64_t t_full[2], t_empty[2], d_full, mma_fin;
    __shared__ uint32_t tmem_slot;
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

    if (tid < k) {
        const int r = idx[pt * k + tid];
        if (r < 0 || (int64_t)r >= N) atomicOr(&ctr->status, (unsigned)DEV_INVALID);
    }
    // gather units of producer thread tid: rows gr0 and gr0 + 32, 8-column unit gg
    // (an invalid index reads row 0); the first S - 1 chunks go in flight now
    const int gr0 = (tid & 255) >> 3, gg = tid & 7;
    const bool glive0 = gr0 < k, glive1 = gr0 + 32 < k;
    auto nbr = [&](bool live, int j) -> const T * {
        int r = live ? idx[pt * k + j] : 0;
        if (r < 0 || (int64_t)r >= N) r = 0;
        return X + (int64_t)r * ld;
    };
    const T *grow0 = nbr(glive0, gr0), *grow1 = nbr(glive1, gr0 + 32);
    auto issue = [&](int j) {  // chunk j into stage j % S (an empty group past the last chunk)
        if (j < nchunks) {
            uint8_t *st = Raw + (j % S) * RB;
            const int64_t a = (int64_t)j * GT_CH + gg * 8;
            pg::raw_issue(st, gr0, gg, grow0, glive0, a, m, vec);
            pg::raw_issue(st, gr0 + 32, gg, grow1, glive1, a, m, vec);
        }
        pg::cp_async_commit();
    };
    if (warp < GT_PRODUCER_WARPS) {
        for (int j = 0; j < S - 1; ++j) issue(j);
        if (!with_q)  // the products' rows of both tiles stay zero
            for (int e = tid; e < 2 * 64 * 8; e += 256)
                *reinterpret_cast<uint4 *>(Tile0 + (e >> 9) * GT_TILE + sw128(64 + ((e >> 3) & 63), e & 7)) =
                    make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tc::smem_u32(&t_full[b]), GT_PRODUCER_WARPS);
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
        const int u = warp;  // columns 8u .. 8u + 7 of every chunk; rows lane, lane + 32
        const float inv_k = 1.f / (float)k;
        float racc0 = 0.f, racc1 = 0.f;
        for (int ci = 0; ci < nchunks; ++ci) {
            const int b = ci & 1;
            pg::cp_async_wait<S - 2>();  // this thread's copies of chunk ci have landed
            // every producer's copies of chunk ci are visible, and every read
            // of stage (ci - 1) % S is done, so it takes chunk ci + S - 1
            asm volatile("bar.sync 1, 256;" ::: "memory");
            issue(ci + S - 1);
            float x0[8], x1[8];
            pg::centre_lane<T>(Raw + (ci % S) * RB, lane, u, k, inv_k, x0, x1);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                racc0 += x0[e];
                racc1 += x1[e];
            }
            // tile b is free once the MMAs of chunk ci - 2 are done with it
            if (ci >= 2) {
                if (lane == 0) wait(&t_empty[b], (uint32_t)((ci >> 1) - 1) & 1u);
                __syncwarp();
            }
            uint8_t *tile = Tile0 + b * GT_TILE;
            uint32_t xw0[4], xw1[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                xw0[e] = pack_bf16x2(x0[2 * e], x0[2 * e + 1]);
                xw1[e] = pack_bf16x2(x1[2 * e], x1[2 * e + 1]);
            }
            *reinterpret_cast<uint4 *>(tile + sw128(lane, u)) = make_uint4(xw0[0], xw0[1], xw0[2], xw0[3]);
            *reinterpret_cast<uint4 *>(tile + sw128(lane + 32, u)) = make_uint4(xw1[0], xw1[1], xw1[2], xw1[3]);
            if (with_q) {
                float w[8];  // w_c over the k rows, FP32
#pragma unroll
                for (int e = 0; e < 8; ++e) w[e] = fmaf(x0[e], x0[e], x1[e] * x1[e]);
                pg::warp_colsum8(w, lane);
                uint32_t q0[4], q1[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t wv = pack_bf16x2(w[2 * e], w[2 * e + 1]);
                    const __nv_bfloat162 w2 = *reinterpret_cast<const __nv_bfloat162 *>(&wv);
                    __nv_bfloat162 p0 = __hmul2(*reinterpret_cast<const __nv_bfloat162 *>(&xw0[e]), w2);
                    __nv_bfloat162 p1 = __hmul2(*reinterpret_cast<const __nv_bfloat162 *>(&xw1[e]), w2);
                    q0[e] = *reinterpret_cast<uint32_t *>(&p0);
                    q1[e] = *reinterpret_cast<uint32_t *>(&p1);
                }
                *reinterpret_cast<uint4 *>(tile + sw128(64 + lane, u)) = make_uint4(q0[0], q0[1], q0[2], q0[3]);
                *reinterpret_cast<uint4 *>(tile + sw128(96 + lane, u)) = make_uint4(q1[0], q1[1], q1[2], q1[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&t_full[b]));
        }
        // R = X_c 1: every warp's row sums over its columns, reduced per row
        Red[u * 64 + lane] = racc0;
        Red[u * 64 + 32 + lane] = racc1;
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (tid < k) {
            float r = 0.f;
#pragma unroll
            for (int w = 0; w < GT_PRODUCER_WARPS; ++w) r += Red[w * 64 + tid];
            R[pt * k + tid] = r;
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
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        const size_t smem = gram_tc_smem_bytes<__nv_bfloat16>();
        e = cudaFuncSetAttribute(gram_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        gram_tc_kernel<__nv_bfloat16><<<(unsigned)np, GT_THREADS, smem, s>>>(one, tab, ntab, with_q, wait_limit, ctr);
    } else {
        const size_t smem = gram_tc_smem_bytes<float>();
        e = cudaFuncSetAttribute(gram_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gram_tc_kernel<float><<<(unsigned)np, GT_THREADS, smem, s>>>(one, tab, ntab, with_q, wait_limit, ctr);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
