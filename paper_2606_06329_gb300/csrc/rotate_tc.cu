// rotate_tc.cu - the rotated patch of the BF16-mixed estimator: for every
// patch, Y = U^T X_c (k x m), U the k x k eigenvector matrix of the patch Gram
// G = X_c X_c^T (eq. svd_cov; Alg. 1 SVD_p).  Row l of Y is s_l v_l^T: the
// l-th right singular vector scaled by its singular value, so the tangent
// basis V_r = X_c^T U_p S^-1 of Alg. 1 is Y's first p rows divided by s_l, and
// X_c = U Y exactly for the full orthogonal U.  The third-moment pass of the
// Fast estimator works on Y (tthird_tc.cu).
//
// One CTA per patch.  The 256 producer threads gather the k neighbour rows of
// each 64-column chunk into a ring of raw stages with cp.async (four chunks in
// flight for BF16 rows, one for FP32 rows; the first ones while U is staged).
// Producer warp u then owns columns 8u .. 8u + 7 of the chunk, lane l rows l
// and l + 32: it centres them in FP32 (pg::centre_lane, as the Gram pass
// does, so both see identical BF16 values) and writes them transposed into
// X_c^T (64 columns x 64 rows, BF16, K-major with the 128-byte swizzle), the
// B operand; a chunk costs the CTA one barrier.  One MMA thread
// computes D = [U_hi^T | U_lo^T] [X_c^T | X_c^T]^T on the tensor cores: U is
// split into two BF16 terms (U_hi = bf16(U), U_lo = bf16(U - U_hi), together
// U to ~2^-17 relative) placed side by side along K, so one FP32 accumulator
// sums both products; BF16 x BF16 products are exact in FP32.  Rows 64..127 of
// the MMA's A operand repeat rows 0..63, so TMEM lanes 64..127 hold a second
// copy of the chunk of Y: two drain warps, confined to TMEM lane quarters 1
// and 2, read rows 32..63 and (the copy of) rows 0..31, round to BF16 and
// store the chunk of Y while the producers already centre the next ones.
// Accumulators and B operands are double-buffered; every wait is bounded
// (MECUCO_ERR_TIMEOUT, no trap) and the MMA thread waits for its last MMAs
// before tensor memory is freed.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "patch_gather.cuh"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int RT_PRODUCER_WARPS = 8;
constexpr int RT_MMA_WARP = RT_PRODUCER_WARPS;             // warp 8; warps 9, 10 drain
constexpr int RT_DRAIN_WARPS = 2;
constexpr int RT_THREADS = (RT_PRODUCER_WARPS + 1 + RT_DRAIN_WARPS) * 32;
constexpr int RT_CH = 64;                                  // columns per chunk
constexpr int RT_XS_LD = 68;                               // FP32 staging row stride (floats)
constexpr int RT_A_TILE = 128 * 128;                       // one A tile: 128 rows x 64 K (BF16), 16 KB
constexpr int RT_B_BYTES = 64 * 128;                       // X_c^T chunk: 64 rows x 64 K (BF16), 8 KB
constexpr int RT_U_BYTES = 64 * RT_XS_LD * 4;              // U staged in FP32 (A operand set-up)
constexpr long long RT_WAIT = 1000000000LL;
// gather ring depth: 5 x 8 KB stages of BF16 rows, 2 x 16 KB of FP32 rows
// (two CTAs per SM)
template <typename T>
__host__ __device__ constexpr int rt_stages() {
    return sizeof(T) == 2 ? 5 : 2;
}
using pg::pack_bf16x2;
using pg::sw128;
}  // namespace

template <typename T>
size_t rotate_tc_smem_bytes() {
    return 1024 + 2 * (size_t)RT_A_TILE + 2 * (size_t)RT_B_BYTES + (size_t)RT_U_BYTES +
           (size_t)rt_stages<T>() * pg::raw_stage_bytes<T>();
}

// two CTAs per SM (~108 KB of shared memory each, 76 registers a thread)
template <typename T>
__global__ void __launch_bounds__(RT_THREADS, 2)
rotate_tc_kernel(const __grid_constant__ PatchSeg one, const PatchSeg *__restrict__ tab, int ntab,
                 __nv_bfloat16 *__restrict__ Y, int64_t ldy, long long wait_limit, DevCounters *ctr) {
    extern __shared__ __align__(1024) uint8_t rsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(rsm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *Aop = base;                                             // 2 A tiles (U_hi^T, U_lo^T)
    uint8_t *Bop0 = base + 2 * RT_A_TILE;                            // 2 x B operand
    float *Xs = reinterpret_cast<float *>(Bop0 + 2 * RT_B_BYTES);    // [64][68] U in FP32
    uint8_t *Raw = reinterpret_cast<uint8_t *>(Xs) + RT_U_BYTES;     // gather ring
    constexpr int S = rt_stages<T>(), RB = pg::raw_stage_bytes<T>();
    __shared__ uint64_t b_full[2], b_empty[2], d_full[2], d_empty[2], mma_fin;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag, never;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int local;
    const PatchSeg &seg = find_seg(one, tab, ntab, (int)blockIdx.x, local);
    const T *X = static_cast<const T *>(seg.X);
    const int64_t N = seg.N, m = seg.m, ld = seg.ld, pt = local;
    const int k = seg.k;
    const int32_t *idx = seg.idx;
    const float *U = seg.U;
    const int64_t yp = blockIdx.x;  // Y is indexed by the launch's point (uniform ldy)
    const int nchunks = (int)((m + RT_CH - 1) / RT_CH);
    const uint32_t idesc = tc::idesc_bf16_f32(128, 64);
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
            const int64_t a = (int64_t)j * RT_CH + gg * 8;
            pg::raw_issue(st, gr0, gg, grow0, glive0, a, m, vec);
            pg::raw_issue(st, gr0 + 32, gg, grow1, glive1, a, m, vec);
        }
        pg::cp_async_commit();
    };
    if (warp < RT_PRODUCER_WARPS)
        for (int j = 0; j < S - 1; ++j) issue(j);
    // U (row j, column l) staged as Xs[j][l], zero outside k x k
    const float *Up = U + pt * (int64_t)k * k;
    for (int e = tid; e < 64 * 64; e += RT_THREADS) {
        const int j = e >> 6, l = e & 63;
        Xs[j * RT_XS_LD + l] = (j < k && l < k) ? Up[j * k + l] : 0.f;
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tc::smem_u32(&b_full[b]), RT_PRODUCER_WARPS);
            tc::mbar_init(tc::smem_u32(&b_empty[b]), 1);
            tc::mbar_init(tc::smem_u32(&d_full[b]), 1);
            tc::mbar_init(tc::smem_u32(&d_empty[b]), RT_DRAIN_WARPS);
        }
        tc::mbar_init(tc::smem_u32(&mma_fin), 1);
        abort_flag = (*(volatile unsigned *)&ctr->status & DEV_TIMEOUT) ? 1 : 0;
        never = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), 128);  // two 64-column accumulators
        tc::tmem_relinquish();
    }
    __syncthreads();
    // A operand: rows l and 64 + l hold U[:, l] (the l-th column of U) split in
    // two BF16 terms, the high term in tile 0 and the low term in tile 1
    // (K = j).  Thread (row, unit) reads a column of the staged U.
    for (int e = tid; e < 128 * 8; e += RT_THREADS) {
        const int l = e & 127, un = e >> 7;  // row, 16-byte unit (8 values of j)
        const int lc = l & 63;               // column of U
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float u0 = Xs[(8 * un + 2 * q) * RT_XS_LD + lc], u1 = Xs[(8 * un + 2 * q + 1) * RT_XS_LD + lc];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(u0), h1 = __float2bfloat16_rn(u1);
            hw[q] = pack_bf16x2(__bfloat162float(h0), __bfloat162float(h1));
            lw[q] = pack_bf16x2(u0 - __bfloat162float(h0), u1 - __bfloat162float(h1));
        }
        *reinterpret_cast<uint4 *>(Aop + sw128(l, un)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(Aop + RT_A_TILE + sw128(l, un)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

    if (warp < RT_PRODUCER_WARPS) {
        // ============ producers: gather, centre, transposed pack ============
        const int u = warp;  // columns 8u .. 8u + 7 of every chunk; rows lane, lane + 32
        const float inv_k = 1.f / (float)k;
        // this lane's K positions (rows j = lane, lane + 32) in a row of X_c^T
        const uint32_t kb0 = (uint32_t)((lane & 7) * 2);
        const int ku0 = lane >> 3, ku1 = 4 + (lane >> 3);
        for (int ci = 0; ci < nchunks; ++ci) {
            const int b = ci & 1;
            pg::cp_async_wait<S - 2>();  // this thread's copies of chunk ci have landed
            // every producer's copies of chunk ci are visible, and every read
            // of stage (ci - 1) % S is done, so it takes chunk ci + S - 1
            asm volatile("bar.sync 1, 256;" ::: "memory");
            issue(ci + S - 1);
            float x0[8], x1[8];
            pg::centre_lane<T>(Raw + (ci % S) * RB, lane, u, k, inv_k, x0, x1);
            // buffer b is free once the MMAs of chunk ci - 2 are done with it
            if (ci >= 2) {
                if (lane == 0) wait(&b_empty[b], (uint32_t)((ci >> 1) - 1) & 1u);
                __syncwarp();
            }
            uint8_t *Bop = Bop0 + b * RT_B_BYTES;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int c = 8 * u + e;  // row of X_c^T
                *reinterpret_cast<__nv_bfloat16 *>(Bop + sw128(c, ku0) + kb0) = __float2bfloat16_rn(x0[e]);
                *reinterpret_cast<__nv_bfloat16 *>(Bop + sw128(c, ku1) + kb0) = __float2bfloat16_rn(x1[e]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&b_full[b]));
        }
    } else if (warp > RT_MMA_WARP) {
        // ============ drain: TMEM lane quarter dq, rows 32 (dq & 1) + lane of Y ============
        const int dq = warp & 3;  // 1 (rows 32..63) or 2 (the copy of rows 0..31)
        __nv_bfloat16 *yrow = Y + (yp * 64 + (dq & 1) * 32 + lane) * ldy;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            if (lane == 0) wait(&d_full[b], (uint32_t)(c >> 1) & 1u);
            __syncwarp();
            tc::fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t r32[32];
                tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(dq * 32) << 16) + (uint32_t)(b * 64 + h * 32), r32);
                tc::tmem_ld_wait();
                uint32_t pk[16];
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    pk[e] = pack_bf16x2(__uint_as_float(r32[2 * e]), __uint_as_float(r32[2 * e + 1]));
                uint4 *dst = reinterpret_cast<uint4 *>(yrow + (int64_t)c * RT_CH + h * 32);
#pragma unroll
                for (int e = 0; e < 4; ++e) dst[e] = make_uint4(pk[4 * e], pk[4 * e + 1], pk[4 * e + 2], pk[4 * e + 3]);
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&d_empty[b]));
        }
    } else if (lane == 0) {
        // ================= MMA thread =================
        const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(Aop)), a1 = tc::sdesc_sw128(tc::smem_u32(Aop + RT_A_TILE));
        bool ok = true;
        for (int ci = 0; ci < nchunks && ok; ++ci) {
            const int b = ci & 1;
            if (!tc::mbar_wait(tc::smem_u32(&b_full[b]), (uint32_t)(ci >> 1) & 1u, abortp, wait_limit) ||
                (ci >= 2 &&
                 !tc::mbar_wait(tc::smem_u32(&d_empty[b]), (uint32_t)((ci >> 1) - 1) & 1u, abortp, wait_limit))) {
                fail();
                ok = false;
                break;
            }
            tc::fence_after();
            const uint64_t bd = tc::sdesc_sw128(tc::smem_u32(Bop0 + b * RT_B_BYTES));
            const uint32_t d = tmem + (uint32_t)(b * 64);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) tc::mma_f16(d, a0 + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, kk != 0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) tc::mma_f16(d, a1 + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, 1u);
            tc::commit(tc::smem_u32(&b_empty[b]));
            tc::commit(tc::smem_u32(&d_full[b]));
        }
        // every MMA has completed before TMEM is freed (a barrier used once)
        tc::commit(tc::smem_u32(&mma_fin));
        if (!tc::mbar_wait(tc::smem_u32(&mma_fin), 0u, &never, RT_WAIT)) fail();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 128);
    }
}

cudaError_t launch_rotate_tc(mecuco_dtype dt, const PatchSeg &one, const PatchSeg *tab, int ntab, int64_t np, void *Y,
                             int64_t ldy, long long wait_limit, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    // every segment's m must fit ldy (the caller's contract for tables)
    if ((ntab == 0 && (one.k > 64 || one.k < 2 || ldy < (one.m + RT_CH - 1) / RT_CH * RT_CH)) || (ldy % 8) != 0 ||
        (reinterpret_cast<uintptr_t>(Y) & 15))
        return cudaErrorInvalidValue;
    if (wait_limit <= 0) wait_limit = RT_WAIT;
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        const size_t smem = rotate_tc_smem_bytes<__nv_bfloat16>();
        e = cudaFuncSetAttribute(rotate_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        rotate_tc_kernel<__nv_bfloat16><<<(unsigned)np, RT_THREADS, smem, s>>>(one, tab, ntab, (__nv_bfloat16 *)Y,
                                                                              ldy, wait_limit, ctr);
    } else {
        const size_t smem = rotate_tc_smem_bytes<float>();
        e = cudaFuncSetAttribute(rotate_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        rotate_tc_kernel<float><<<(unsigned)np, RT_THREADS, smem, s>>>(one, tab, ntab, (__nv_bfloat16 *)Y, ldy,
                                                                      wait_limit, ctr);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
