// tthird_tc.cu - Step 4 of the BF16-mixed form (eqs. tnull, tA, tB,
// fast_curv; Alg. 1 Fast branch) from the rotated patch Y = U^T X_c
// (rotate_tc.cu), on the 5th-generation tensor cores.
//
// With U the k x k orthogonal eigenvector matrix of G = X_c X_c^T, row l of Y
// is y_l = X_c^T u_l = s_l v_l, and X_c = U Y.  The tangent basis of Alg. 1 is
// V_r = [y_r / s_r]_{r < p}.  Put
//   T^[(r,t), l] = sum_a (Y_ra / s_r)(Y_ta / s_t) Y_la      (r, t < p; all l < k).
// Then G_tens[j] = V_r^T diag(x_j) V_r = sum_l U_jl T^[., l] and, U having
// orthonormal columns,
//   |G_tens|_F^2        = sum_{r,t < p} sum_l T^[(r,t), l]^2,
//   |X_c V_r^{o2}|_F^2  = sum_{r < p} sum_l T^[(r,r), l]^2          (t_range),
//   X_c V_r^{o2} 1_p    = U c,  c_l = sum_{r < p} T^[(r,r), l]       (X_c d_P = R - U c),
// so every term of the estimator is a sum of squares of T^ or a k-vector
// product - nothing m-sized and no third-moment tensor is stored.  |X_c V_r|_F^2
// = sum_{l<p} s_l^2 = (k-1) tau; the Haar term is sum_{l<p} u_l^T Q u_l / s_l^2.
//
// T^ is the GEMM D = Z Y^T over the columns a, Z the row products
// Z[(r,t), a] = Y_ra Y_ta (r <= t, 8 x 8 pair blocks as in the moment kernel)
// and the scale 1/(s_r s_t) applied in FP32 when D is read.  One CTA per point:
//   TMA warp     loads 64-column chunks of the point's Y (64 rows x 128 B,
//                128-byte swizzle) into a ring of stages;
//   8 formers    form the products of each tile row (HMUL2 on BF16 pairs read
//                from the stage) into TMEM slots (the MMA's A operand) and,
//                after each pass over the columns, read the accumulators back,
//                scale them and accumulate the sums;
//   MMA thread   issues tcgen05.mma with A in TMEM and B = the stage itself.
// The accumulators of up to (512 - 32 slots)/N tiles fit in TMEM, so the
// tiles are covered in passes over the chunks.  All sums are formed in a fixed
// order (deterministic).  Every wait is bounded (MECUCO_ERR_TIMEOUT, no trap).
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int TT_FORMER_WARPS = 8;
constexpr int TT_THREADS = (TT_FORMER_WARPS + 2) * 32;  // formers, the TMA warp, the MMA warp
constexpr int TT_TMA_WARP = TT_FORMER_WARPS, TT_MMA_WARP = TT_FORMER_WARPS + 1;
constexpr int TT_CH = 64;                  // columns per chunk
constexpr int TT_STAGE = 64 * 128;         // a chunk of Y: 64 rows x 64 columns BF16
constexpr int TT_NS = 6;                   // ring stages
constexpr int TT_MAX_SLOTS = 8;
constexpr int TT_SLOT_COLS = TT_CH / 2;    // 32-bit TMEM columns per slot
constexpr int TT_GROUP = 2;                // tiles per slot hand-over
constexpr int TT_DLD = 65;                 // row stride of the diagonal rows kept for the final sums
constexpr long long TT_WAIT = 1000000000LL;

enum : int { ROW_NONE = 0, ROW_PAIR = 1 };

__host__ __device__ inline int tthird_n(int k) { return k <= 16 ? 16 : ((k + 15) / 16) * 16; }
}  // namespace

__host__ __device__ int tthird_rows(int k) {
    const int kb = (k + 7) / 8;
    return (kb * (kb + 1) / 2 * 64 + 127) / 128 * 128;
}

// Pairs r <= t in 8 x 8 blocks (r-block <= t-block): a 32-row quarter of a
// block holds 4 values of r and 8 of t, so along a row of blocks a lane keeps
// its r (the formers reload only Y_t).  Code = r | t << 8 | kind << 16.
void tthird_build_rows(int k, int32_t *codes) {
    const int kb = (k + 7) / 8;
    const int nrows = tthird_rows(k);
    int n = 0;
    for (int A = 0; A < kb; ++A)
        for (int B = A; B < kb; ++B)
            for (int r = 0; r < 64; ++r) {
                const int h = r / 32, L = r % 32;
                const int a = 8 * A + 4 * h + L / 8, b = 8 * B + L % 8;
                const bool valid = a < k && b < k && (A < B || a <= b);
                codes[n++] = valid ? (int32_t)(a | (b << 8) | (ROW_PAIR << 16)) : 0;
            }
    for (; n < nrows; ++n) codes[n] = 0;
}

// ctas = CTAs per SM, each allocating 512 / ctas TMEM columns.  With one CTA
// the request is raised to 120 KB so that no second CTA becomes resident (it
// would only wait in its allocation).
size_t tthird_smem_bytes(int k, int ctas) {
    const size_t need = 1024 + (size_t)TT_NS * TT_STAGE + (size_t)tthird_rows(k) * 8 + 64 * (size_t)TT_DLD * 4;
    return (ctas == 1 && need < ((size_t)120 << 10)) ? ((size_t)120 << 10) : need;
}

// two CTAs per SM by default (102 registers a thread at most)
__global__ void __launch_bounds__(TT_THREADS, 2)
tthird_tc_kernel(const __grid_constant__ CUtensorMap map_y, const __grid_constant__ PatchSeg one,
                 const PatchSeg *__restrict__ tab, int ntab, int variant, int nslots, int tcols, long long wait_limit,
                 DevCounters *ctr) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int local;
    const PatchSeg &seg = find_seg(one, tab, ntab, (int)blockIdx.x, local);
    const int64_t pt = local, m = seg.m;
    const int k = seg.k;
    const int nrows = tthird_rows(k);
    const int32_t *rowtab = seg.rowtab;
    const float *sigma = seg.sig, *U = seg.U, *R = seg.R, *Q = seg.Q;
    float *kappa = seg.kappa, *lambda_out = seg.lambda, *s_out = seg.s;
    // numerical-rank threshold of a Gram accumulated from BF16 products
    const float rank_eps = 8.f * sqrtf((float)m) * 5.9604644775390625e-08f;
    extern __shared__ __align__(1024) uint8_t tsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = base;                                                        // TT_NS stages
    int32_t *codes = reinterpret_cast<int32_t *>(ring + TT_NS * TT_STAGE);     // [nrows]
    float *diag = reinterpret_cast<float *>(codes + nrows);                     // [64][TT_DLD] rows T^[(r,r), .]
    float *rowsq = diag + 64 * TT_DLD;                                          // [nrows] w |T^ row|^2
    __shared__ uint64_t full[TT_NS], empty[TT_NS], slot_full[TT_MAX_SLOTS], slot_empty[TT_MAX_SLOTS];
    __shared__ uint64_t pass_done, d_free, mma_fin;
    __shared__ uint32_t tmem_slot;
    __shared__ float inv_s[64], c_s[64];
    __shared__ double red[TT_THREADS / 32][4];
    __shared__ int s_p, abort_flag, never;

    const int ntiles = nrows / 128;
    const int Nb = tthird_n(k);
    const int dcols = tcols - nslots * TT_SLOT_COLS;  // accumulator columns; the A slots follow
    const int tpp = min(ntiles, dcols / Nb);
    const int npass = (ntiles + tpp - 1) / tpp;
    const int nchunks = (int)((m + TT_CH - 1) / TT_CH);
    const uint32_t idesc = tc::idesc_bf16_f32(128, Nb);
    const float *sg = sigma + pt * k;

    for (int e = tid; e < nrows; e += TT_THREADS) codes[e] = __ldg(rowtab + e);
    for (int e = tid; e < 64 * TT_DLD; e += TT_THREADS) diag[e] = 0.f;
    if (tid == 0) {
        // numerical rank: eigenvalues above rank_eps * s_0 (the Gram's rounding scale)
        int pmax = k - 1;
        if ((int64_t)pmax > m) pmax = (int)m;
        const float s0 = fmaxf(sg[0], 0.f);
        int rank = 0;
        for (int l = 0; l < k; ++l) rank += (sg[l] > rank_eps * s0) && (sg[l] > 0.f);
        s_p = rank < pmax ? rank : pmax;
        if (s_p < pmax) atomicAdd(&ctr->rank_deficient, 1ull);
        for (int s = 0; s < TT_NS; ++s) {
            tc::mbar_init(tc::smem_u32(&full[s]), 1);
            tc::mbar_init(tc::smem_u32(&empty[s]), 1);
        }
        for (int s = 0; s < nslots; ++s) {
            tc::mbar_init(tc::smem_u32(&slot_full[s]), TT_FORMER_WARPS);
            tc::mbar_init(tc::smem_u32(&slot_empty[s]), 1);
        }
        tc::mbar_init(tc::smem_u32(&pass_done), 1);
        tc::mbar_init(tc::smem_u32(&d_free), TT_FORMER_WARPS);
        tc::mbar_init(tc::smem_u32(&mma_fin), 1);
        abort_flag = (*(volatile unsigned *)&ctr->status & DEV_TIMEOUT) ? 1 : 0;
        never = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map_y);
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), (uint32_t)tcols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int p = s_p;
    if (tid < 64) inv_s[tid] = tid < p ? (float)(1.0 / sqrt((double)sg[tid])) : 0.f;
    const uint32_t tmem = tmem_slot;
    volatile int *abortp = &abort_flag;
    auto fail = [&]() {
        atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
        abort_flag = 1;
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (!*abortp && !tc::mbar_wait(tc::smem_u32(bar), parity, abortp, wait_limit)) fail();
    };
    __syncthreads();  // inv_s

    if (warp < TT_FORMER_WARPS) {
        // ================= formers: row products into TMEM; drain and sums =================
        const int qd = warp & 3, half = warp >> 2;  // TMEM lane quarter, K half
        const int trow = qd * 32 + lane;
        const uint32_t ngs = (uint32_t)(nslots / TT_GROUP);
        uint32_t gs = 0, gph = 0, gq = 0, st = 0, sph = 0;  // slot group state; stage and phase
        for (int ps = 0; ps < npass; ++ps) {
            const int t0 = ps * tpp, nt = min(tpp, ntiles - t0);
            for (int ci = 0; ci < nchunks; ++ci) {
                if (lane == 0) wait(&full[st], sph);
                __syncwarp();
                const uint8_t *stage = ring + st * TT_STAGE;
                uint4 xa[4];
                int ka = -1;
                for (int t = 0; t < nt; t += TT_GROUP, ++gq) {
                    const int cnt = min(TT_GROUP, nt - t);
                    if (gq >= ngs && lane == 0) wait(&slot_empty[gs], gph ^ 1u);
                    __syncwarp();
                    tc::fence_after();
                    for (int u = 0; u < cnt; ++u) {
                        const int code = codes[(t0 + t + u) * 128 + trow];
                        const int ra = code & 0xff, rb = (code >> 8) & 0xff;
                        // row r's 16-byte unit v (K = 8v .. 8v + 7) sits at r*128 + ((v ^ (r & 7)) << 4)
                        if (ra != ka) {
                            ka = ra;
#pragma unroll
                            for (int e4 = 0; e4 < 4; ++e4)
                                xa[e4] = *reinterpret_cast<const uint4 *>(stage + ra * 128 +
                                                                          (((half * 4 + e4) ^ (ra & 7)) << 4));
                        }
                        uint32_t z[16];
#pragma unroll
                        for (int e4 = 0; e4 < 4; ++e4) {
                            const uint4 bv = *reinterpret_cast<const uint4 *>(stage + rb * 128 +
                                                                              (((half * 4 + e4) ^ (rb & 7)) << 4));
                            const uint4 av = xa[e4];
                            const uint32_t aw[4] = {av.x, av.y, av.z, av.w};
                            const uint32_t bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162 *>(&aw[e]);
                                __nv_bfloat162 y = *reinterpret_cast<const __nv_bfloat162 *>(&bw[e]);
                                __nv_bfloat162 pr = __hmul2(x, y);
                                z[e4 * 4 + e] = *reinterpret_cast<uint32_t *>(&pr);
                            }
                        }
                        tc::tmem_st_32x32b_x16(tmem + ((uint32_t)(qd * 32) << 16) +
                                                   (uint32_t)(dcols + ((int)gs * TT_GROUP + u) * TT_SLOT_COLS +
                                                              half * 16),
                                               z);
                    }
                    tc::tmem_st_wait();
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(tc::smem_u32(&slot_full[gs]));
                    if (++gs == ngs) { gs = 0; gph ^= 1u; }
                }
                if (++st == (uint32_t)TT_NS) { st = 0; sph ^= 1u; }
            }
            // ---- read the pass's accumulators: this warp takes tiles half, half + 2, ...
            if (lane == 0) wait(&pass_done, ps & 1);
            __syncwarp();
            tc::fence_after();
            for (int t = half; t < nt; t += 2) {
                const int code = codes[(t0 + t) * 128 + trow];
                const int ra = code & 0xff, rb = (code >> 8) & 0xff;
                const bool live = ((code >> 16) & 3) == ROW_PAIR && ra < p && rb < p;
                const float f = live ? inv_s[ra] * inv_s[rb] : 0.f;
                float sq = 0.f;
                for (int c0 = 0; c0 < Nb; c0 += 16) {
                    uint32_t r16[16];
                    tc::tmem_ld_32x32b_x16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(t * Nb + c0), r16);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float v = f * __uint_as_float(r16[e]);
                        sq = fmaf(v, v, sq);
                        if (live && ra == rb) diag[ra * TT_DLD + c0 + e] = v;
                    }
                }
                rowsq[(t0 + t) * 128 + trow] = live ? (ra == rb ? 1.f : 2.f) * sq : 0.f;
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&d_free));
        }
    } else if (warp == TT_TMA_WARP) {
        // ================= TMA producer (one thread) =================
        if (lane == 0) {
            uint32_t st = 0, sph = 0;
            int issued = 0;
            bool ok = true;
            const uint32_t ring0 = tc::smem_u32(ring), full0 = tc::smem_u32(&full[0]),
                           empty0 = tc::smem_u32(&empty[0]);
            for (int ps = 0; ps < npass && ok; ++ps) {
                for (int ci = 0; ci < nchunks; ++ci) {
                    if (!tc::mbar_wait(empty0 + 8 * st, sph ^ 1u, abortp, wait_limit)) {
                        if (!*abortp) fail();
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(full0 + 8 * st, TT_STAGE);
                    tc::tma_load_2d(ring0 + st * TT_STAGE, &map_y, full0 + 8 * st, ci * TT_CH, (int)(blockIdx.x * 64));
                    ++issued;
                    if (++st == (uint32_t)TT_NS) { st = 0; sph ^= 1u; }
                }
            }
            // every load issued has landed before the CTA can exit (bounded by time only)
            for (int j = issued - TT_NS; j < issued; ++j)
                if (j >= 0) tc::mbar_wait(tc::smem_u32(&full[j % TT_NS]), (uint32_t)(j / TT_NS) & 1u, &never, TT_WAIT);
        }
    } else {
        // ================= MMA thread =================
        if (lane == 0) {
            uint32_t s = 0, ph = 0, st = 0, sph = 0;
            const uint32_t ngs = (uint32_t)(nslots / TT_GROUP);
            bool ok = true;
            const uint32_t a_base = tmem + (uint32_t)dcols;
            const uint32_t slot_full0 = tc::smem_u32(&slot_full[0]), slot_empty0 = tc::smem_u32(&slot_empty[0]);
            for (int ps = 0; ps < npass && ok; ++ps) {
                const int nt = min(tpp, ntiles - ps * tpp);
                if (ps > 0) {
                    wait(&d_free, (ps - 1) & 1);  // the formers have read the previous pass
                    ok = !*abortp;
                    tc::fence_after();
                }
                for (int ci = 0; ci < nchunks && ok; ++ci) {
                    if (!tc::mbar_wait(tc::smem_u32(&full[st]), sph, abortp, wait_limit)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint64_t bd0 = tc::sdesc_sw128(tc::smem_u32(ring + st * TT_STAGE));
                    uint32_t d = tmem;
                    for (int t = 0; t < nt; t += TT_GROUP, d += (uint32_t)(TT_GROUP * Nb)) {
                        if (!tc::mbar_wait(slot_full0 + 8 * s, ph, abortp, wait_limit)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t a_g = a_base + s * (uint32_t)(TT_GROUP * TT_SLOT_COLS);
                        if (t + TT_GROUP <= nt) {
#pragma unroll
                            for (int u = 0; u < TT_GROUP; ++u)
#pragma unroll
                                for (int kk = 0; kk < TT_CH / 16; ++kk)
                                    tc::mma_f16_ts(d + (uint32_t)(u * Nb), a_g + (uint32_t)(u * TT_SLOT_COLS + kk * 8),
                                                   bd0 + (uint64_t)(2 * kk), idesc, (ci | kk) != 0);
                        } else {  // a pass whose tile count is not a multiple of TT_GROUP
                            for (int u = 0; u < nt - t; ++u)
#pragma unroll
                                for (int kk = 0; kk < TT_CH / 16; ++kk)
                                    tc::mma_f16_ts(d + (uint32_t)(u * Nb), a_g + (uint32_t)(u * TT_SLOT_COLS + kk * 8),
                                                   bd0 + (uint64_t)(2 * kk), idesc, (ci | kk) != 0);
                        }
                        tc::commit(slot_empty0 + 8 * s);
                        if (++s == ngs) { s = 0; ph ^= 1u; }
                    }
                    tc::commit(tc::smem_u32(&empty[st]));  // the stage is free once these MMAs complete
                    if (++st == (uint32_t)TT_NS) { st = 0; sph ^= 1u; }
                }
                tc::commit(tc::smem_u32(&pass_done));
            }
            // every MMA has completed before TMEM is freed (a barrier used once)
            tc::commit(tc::smem_u32(&mma_fin));
            if (!tc::mbar_wait(tc::smem_u32(&mma_fin), 0u, &never, TT_WAIT)) fail();
        }
        __syncwarp();
    }
    // ================= final sums (all threads) =================
    tc::fence_before();
    __syncthreads();
    // |G_tens|^2: each thread sums a fixed set of table rows (the schedule of
    // tiles over passes and warps does not change the order)
    double gsum = 0.0;
    for (int e = tid; e < nrows; e += TT_THREADS) gsum += (double)rowsq[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    // U and Q of the point, staged in the (now idle) ring: U[j][l] at Us[j*65 + l]
    float *Us = reinterpret_cast<float *>(ring), *Qs = Us + 64 * 65;
    const float *ug = U + pt * (int64_t)k * k;
    for (int e = tid; e < k * k; e += TT_THREADS) Us[(e / k) * 65 + e % k] = ug[e];
    if (variant == MECUCO_FAST_HAAR) {
        const float *qg = Q + pt * (int64_t)k * k;
        for (int e = tid; e < k * k; e += TT_THREADS) Qs[(e / k) * 65 + e % k] = qg[e];
    }
    __syncthreads();
    double dsum = 0.0, xa2 = 0.0, hsum = 0.0;
    if (tid < k) {
        // c_l = sum_{r<p} T^[(r,r), l] and t_range's sum, in a fixed order over r
        const int l = tid;
        float cl = 0.f;
        double d2 = 0.0;
        for (int r = 0; r < p; ++r) {
            const float v = diag[r * TT_DLD + l];
            cl += v;
            d2 += (double)v * v;
        }
        c_s[l] = cl;
        dsum = d2;
    }
    if (variant == MECUCO_FAST_HAAR && tid >= 64 && tid < 64 + p) {
        // u_l^T Q u_l / s_l^2
        const int l = tid - 64;
        double acc = 0.0;
        for (int a = 0; a < k; ++a) {
            float qu = 0.f;
            for (int b = 0; b < k; ++b) qu = fmaf(Qs[a * 65 + b], Us[b * 65 + l], qu);
            acc += (double)Us[a * 65 + l] * qu;
        }
        hsum = acc / (double)sg[l];
    }
    __syncthreads();
    if (tid < k) {
        // X_c d_P = R - U c
        const int j = tid;
        float uc = 0.f;
        for (int l = 0; l < k; ++l) uc = fmaf(Us[j * 65 + l], c_s[l], uc);
        const double xd = (double)R[pt * k + j] - (double)uc;
        xa2 = xd * xd;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        xa2 += __shfl_xor_sync(0xffffffffu, xa2, o);
        hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
    }
    if (lane == 0) { red[warp][0] = gsum; red[warp][1] = dsum; red[warp][2] = xa2; red[warp][3] = hsum; }
    __syncthreads();
    if (tid == 0) {
        double gt2 = 0.0, d2 = 0.0, a2 = 0.0, h = 0.0;
        for (int w = 0; w < TT_THREADS / 32; ++w) { gt2 += red[w][0]; d2 += red[w][1]; a2 += red[w][2]; h += red[w][3]; }
        const double km1 = (double)(k - 1);
        double tau = 0.0;
        for (int l = 0; l < p; ++l) tau += (double)sg[l];
        tau /= km1;
        const double t_range = d2 / km1, t_A = a2 / km1;
        const int64_t q = m - p;
        double t_null = 0.0;
        if (q > 0) {
            if (variant == MECUCO_FAST_HAAR) {
                const double tB = tau - 2.0 * h / km1 + gt2 / km1;
                t_null = (t_A + 2.0 * tB) / (double)(q + 2);
            } else {
                const double tB = tau - 2.0 * tau + gt2 / km1;  // |X_c V_r|_F^2 / (k-1) = tau
                t_null = (t_A + 2.0 * tB) / (double)q;
            }
        }
        kappa[pt] = (float)fabs(0.5 * (t_range + t_null) + 0.5 * tau);
    }
    if (lambda_out)
        for (int l = tid; l < k; l += TT_THREADS)
            lambda_out[pt * k + l] = (l < p) ? fmaxf(sg[l], 0.f) / (float)(k - 1) : 0.f;
    if (s_out)
        for (int l = tid; l < k; l += TT_THREADS) s_out[pt * k + l] = sqrtf(fmaxf(sg[l], 0.f));
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, (uint32_t)tcols);
    }
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tt_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) ==
                cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
    }
    return fn;
}
}  // namespace

cudaError_t launch_tthird_tc(const PatchSeg &one, const PatchSeg *tab, int ntab, int kmax, int64_t np, const void *Y,
                             int64_t ldy, int variant, int nslots, int ctas, long long wait_limit, DevCounters *ctr,
                             cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    const int tcols = ctas == 2 ? 256 : 512;
    if (kmax > 64 || kmax < 2 || (ctas != 1 && ctas != 2) || nslots < TT_GROUP || nslots > TT_MAX_SLOTS ||
        nslots % TT_GROUP != 0 || (tcols - nslots * TT_SLOT_COLS) < tthird_n(kmax) || (ldy % 8) != 0 ||
        (ntab == 0 && (one.k != kmax || ldy < (one.m + TT_CH - 1) / TT_CH * TT_CH ||
                       (variant == MECUCO_FAST_HAAR && !one.Q))) ||
        (reinterpret_cast<uintptr_t>(Y) & 15) || np * 64 >= ((int64_t)1 << 31))
        return cudaErrorInvalidValue;
    if (wait_limit <= 0) wait_limit = TT_WAIT;
    auto fn = tt_encode_fn();
    if (!fn) return cudaErrorInvalidValue;
    // Y of the chunk: (np * 64) rows of ldy BF16 columns; boxes of 64 rows x 64 columns
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)ldy, (cuuint64_t)(np * 64)};
    cuuint64_t strides[1] = {(cuuint64_t)ldy * 2};
    cuuint32_t box[2] = {(cuuint32_t)TT_CH, 64u};
    cuuint32_t estr[2] = {1, 1};
    if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(Y), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = tthird_smem_bytes(kmax, ctas);
    cudaError_t e = cudaFuncSetAttribute(tthird_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tthird_tc_kernel<<<(unsigned)np, TT_THREADS, smem, s>>>(map, one, tab, ntab, variant, nslots, tcols, wait_limit,
                                                            ctr);
    return cudaGetLastError();
}

}  // namespace mecuco
