// moments_tc.cu - Steps 2-3 for the BF16-mixed form: gather and centre each
// patch and produce, on the 5th-generation tensor cores, every moment the
// estimator needs:
//   M[a][b][t] = sum_c X_c[a,c] X_c[b,c] X_c[t,c]   (pairs a <= b, all t)
//   G[a][t]    = sum_c X_c[a,c] X_c[t,c]             (= X_c X_c^T, eq. svd_cov)
//   Q[a][t]    = sum_c w_c X_c[a,c] X_c[t,c],  w_c = sum_j X_c[j,c]^2 (Haar term)
//   R[a]       = sum_c X_c[a,c]                      (CUDA cores, while centring)
// as GEMMs D = Z B^T with B = X_c (N = 16 ceil(k/16) rows, zero-padded) and Z
// the row products Z[r, c] = X_c[a_r, c] y_r[c], y_r = X_c[b_r, :] (an M row),
// the all-ones vector (a G row) or w (a Q row).
//
// Row order.  The pairs a <= b are grouped in 8 x 8 blocks (a-block <= b-block;
// a 32-row quarter of a block holds 4 values of a and 8 of b, so a warp reads
// few distinct rows of the patch); the rows a > b that the diagonal blocks
// leave free carry the G and Q rows.  Two blocks form a 128-row MMA tile.
// The host builds the table of row codes once per k.
//
// One CTA per patch, three warp roles connected by mbarriers:
//   8 producer warps  gather the k neighbour rows of the next 64-column chunk
//                     (loads in flight while the current chunk is processed),
//                     centre each column in FP32, accumulate R and w, and
//                     write the chunk as packed BF16 pairs and as the K-major,
//                     128-byte-swizzled B operand (two buffers);
//   8 former warps    for every tile of the current pass, each thread forms
//                     32 products of its tile row (HMUL2 on BF16 pairs) and
//                     writes them with tcgen05.st straight into a TMEM slot
//                     holding the A operand (2, 4, 6 or 8 slots of 64
//                     K-columns);
//   1 MMA warp        issues tcgen05.mma with A in TMEM, B in shared memory and
//                     FP32 accumulators in TMEM, and releases each slot and
//                     chunk buffer with tcgen05.commit (a chunk's commit follows
//                     every former's reads of it, so it alone frees the buffer).
// Formers and the MMA warp hand tiles over in groups of MT_GROUP slots: an
// mbarrier wait or arrive issued after tcgen05 work costs the issuing thread a
// few hundred cycles, so each side takes one wait and one arrive per group
// rather than per tile (the MMA thread then queues 4 MT_GROUP MMAs per wait).
// TMEM holds the accumulators of up to (512 - 32 slots)/N tiles, so the tiles are covered
// in passes over the columns (the patch is re-read from L2).  After a pass the
// formers read the accumulators back (tcgen05.ld) and store each row to its
// destination.  Every wait is bounded (MECUCO_ERR_TIMEOUT, no trap; the
// limit of the waits in the work loops is a launch argument, default ~0.5 s);
// the MMA warp waits for its last MMAs (always with the default limit) before
// TMEM is freed.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "patch_gather.cuh"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int MT_PRODUCER_WARPS = 8;                  // gather, centre, pack
constexpr int MT_FORMER_WARPS = 8;                     // row products into TMEM, drain
constexpr int MT_THREADS = (MT_PRODUCER_WARPS + MT_FORMER_WARPS + 1) * 32;  // + the MMA warp
constexpr int MT_CH = 64;                              // columns per chunk
constexpr int MT_MAX_SLOTS = 8;                        // A slots in TMEM (runtime count, 2..8)
constexpr int MT_SLOT_COLS = MT_CH / 2;                // 32-bit TMEM columns per slot
constexpr int MT_GROUP = 2;                            // tiles per slot hand-over (slots come in groups)
constexpr int MT_XS_LD = 68;                           // FP32 staging row stride (floats)
constexpr int MT_XP_LD = 36;                           // packed BF16x2 row stride (words)
constexpr int MT_ROW_ONES = 64, MT_ROW_W = 65, MT_ROW_ZERO = 66, MT_XP_ROWS = 67;
constexpr int MT_B_BYTES = 64 * 128;                   // B operand: up to 64 rows x 128 bytes
constexpr long long MT_WAIT = 1000000000LL;

enum : int { ROW_NONE = 0, ROW_PAIR = 1, ROW_G = 2, ROW_Q = 3 };
using pg::load_halves;
using pg::pack_bf16x2;
using pg::sw128;
using pg::Unit8;

}  // namespace

__host__ __device__ inline int moments_tc_n(int k) { return k <= 16 ? 16 : ((k + 15) / 16) * 16; }

// Rows of the row table: the 8 x 8 pair blocks, or more if their free rows
// cannot hold the 2k G and Q rows, rounded up to whole 128-row tiles.
int moments_tc_rows(int k) {
    const int kb = (k + 7) / 8;
    const int rows = std::max(kb * (kb + 1) / 2 * 64, k * (k + 1) / 2 + 2 * k);
    return (rows + 127) / 128 * 128;
}

void moments_tc_build_rows(int k, int32_t *codes) {
    const int kb = (k + 7) / 8;
    const int nrows = moments_tc_rows(k);
    auto code = [](int a, int b, int kind) { return (int32_t)(a | (b << 8) | (kind << 16)); };
    int n = 0;
    for (int A = 0; A < kb; ++A)
        for (int B = A; B < kb; ++B)
            for (int r = 0; r < 64; ++r) {
                const int h = r / 32, L = r % 32;
                const int a = 8 * A + 4 * h + L / 8, b = 8 * B + L % 8;
                const bool valid = a < k && b < k && (A < B || a <= b);
                codes[n++] = valid ? code(a, b, ROW_PAIR) : code(MT_ROW_ZERO, MT_ROW_ZERO, ROW_NONE);
            }
    for (; n < nrows; ++n) codes[n] = code(MT_ROW_ZERO, MT_ROW_ZERO, ROW_NONE);
    // G and Q rows go into free slots
    int next = 0;
    for (int which = 0; which < 2; ++which)
        for (int a = 0; a < k; ++a) {
            while (((codes[next] >> 16) & 3) != ROW_NONE) ++next;
            codes[next] = which == 0 ? code(a, MT_ROW_ONES, ROW_G) : code(a, MT_ROW_W, ROW_Q);
        }
}

size_t moments_tc_smem_bytes(int k) {
    return 1024 + 2 * (size_t)MT_B_BYTES + 2 * (size_t)MT_XP_ROWS * MT_XP_LD * 4 + 64 * (size_t)MT_XS_LD * 4 +
           4 * 64 * 4 + (size_t)moments_tc_rows(k) * 4;
}

template <typename T>
__global__ void __launch_bounds__(MT_THREADS, 1)
moments_tc_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx, int k,
                  const int32_t *__restrict__ rowtab, int nrows, float *__restrict__ M, float *__restrict__ G,
                  float *__restrict__ R, float *__restrict__ Q, int nslots, long long wait_limit,
                  DevCounters *ctr) {
    extern __shared__ __align__(1024) uint8_t msm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(msm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *Bop0 = base;                                                       // 2 x B operand
    uint32_t *Xp0 = reinterpret_cast<uint32_t *>(base + 2 * MT_B_BYTES);        // 2 x [67][36] packed pairs
    float *Xs = reinterpret_cast<float *>(Xp0 + 2 * MT_XP_ROWS * MT_XP_LD);     // [64][68] FP32 staging
    float *Part = Xs + 64 * MT_XS_LD;                                           // [4][64] column partials
    int32_t *codes = reinterpret_cast<int32_t *>(Part + 4 * 64);                // [nrows]
    __shared__ uint64_t slot_full[MT_MAX_SLOTS], slot_empty[MT_MAX_SLOTS];
    __shared__ uint64_t chunk_ready[2], chunk_done[2], pass_done, d_free, mma_fin;
    __shared__ uint32_t tmem_slot;
    __shared__ int rows[64];
    __shared__ int abort_flag, never;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t pt = blockIdx.x;
    const int npairs = k * (k + 1) / 2;
    const int ntiles = nrows / 128;
    const int Nb = moments_tc_n(k);
    const int dcols = 512 - nslots * MT_SLOT_COLS;  // accumulator columns; the A slots follow
    const int tpp = min(ntiles, dcols / Nb);
    const int npass = (ntiles + tpp - 1) / tpp;
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
    }
    for (int e = tid; e < nrows; e += MT_THREADS) codes[e] = __ldg(rowtab + e);
    // constant rows of both packed buffers: ones (BF16 1.0 pairs) and zeros
    for (int e = tid; e < 2 * MT_XP_LD; e += MT_THREADS) {
        uint32_t *xp = Xp0 + (e / MT_XP_LD) * MT_XP_ROWS * MT_XP_LD;
        xp[MT_ROW_ONES * MT_XP_LD + e % MT_XP_LD] = 0x3f803f80u;
        xp[MT_ROW_ZERO * MT_XP_LD + e % MT_XP_LD] = 0u;
    }
    if (tid == 0) {
        for (int s = 0; s < nslots; ++s) {
            tc::mbar_init(tc::smem_u32(&slot_full[s]), MT_FORMER_WARPS);
            tc::mbar_init(tc::smem_u32(&slot_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tc::smem_u32(&chunk_ready[b]), 1);
            tc::mbar_init(tc::smem_u32(&chunk_done[b]), 1);
        }
        tc::mbar_init(tc::smem_u32(&pass_done), 1);
        tc::mbar_init(tc::smem_u32(&d_free), MT_FORMER_WARPS);
        tc::mbar_init(tc::smem_u32(&mma_fin), 1);
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
    auto fail = [&]() {
        atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
        abort_flag = 1;
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (!*abortp && !tc::mbar_wait(tc::smem_u32(bar), parity, abortp, wait_limit)) fail();
    };

    if (warp < MT_PRODUCER_WARPS) {
        // ================= producers: gather, centre, pack =================
        const int ptid = tid;                                  // 0 .. 255
        const int gr0 = ptid >> 3, gg = ptid & 7;              // gather units (row gr0 / gr0 + 32, group gg)
        const T *grow0 = X + (int64_t)rows[gr0] * ld;
        const T *grow1 = X + (int64_t)rows[gr0 + 32] * ld;
        const bool live0 = gr0 < k, live1 = gr0 + 32 < k;
        const int cc = ptid & 63, rg = ptid >> 6;              // centring: column cc, rows 16 rg .. 16 rg + 15
        const float inv_k = 1.f / (float)k;
        float racc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) racc[e] = 0.f;
        Unit8<T> pre0, pre1;
        if (live0) pre0.load(grow0, gg * 8, m, vec); else pre0.zero();
        if (live1) pre1.load(grow1, gg * 8, m, vec); else pre1.zero();
        uint32_t gc = 0;
        for (int ps = 0; ps < npass; ++ps) {
            for (int ci = 0; ci < nchunks; ++ci, ++gc) {
                const int b = gc & 1;
                const uint32_t use = gc >> 1;
                pre0.store(Xs + gr0 * MT_XS_LD + gg * 8, gg >= 4);
                pre1.store(Xs + (gr0 + 32) * MT_XS_LD + gg * 8, gg >= 4);
                // next chunk (wrapping into the next pass) is loaded while this one is processed
                const bool more = ci + 1 < nchunks || ps + 1 < npass;
                if (more) {
                    const int64_t an = (ci + 1 < nchunks ? (int64_t)(ci + 1) * MT_CH : 0) + gg * 8;
                    if (live0) pre0.load(grow0, an, m, vec); else pre0.zero();
                    if (live1) pre1.load(grow1, an, m, vec); else pre1.zero();
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");
                float v[16], sum = 0.f;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    v[e] = Xs[(rg * 16 + e) * MT_XS_LD + cc];
                    sum += v[e];
                }
                Part[rg * 64 + cc] = sum;
                asm volatile("bar.sync 1, 256;" ::: "memory");
                const float mean = (Part[cc] + Part[64 + cc] + Part[128 + cc] + Part[192 + cc]) * inv_k;
                float w = 0.f;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const float x = (rg * 16 + e < k) ? v[e] - mean : 0.f;
                    Xs[(rg * 16 + e) * MT_XS_LD + cc] = x;
                    w = fmaf(x, x, w);
                    if (ps == 0) racc[e] += x;
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");  // every thread has read Part
                Part[rg * 64 + cc] = w;
                // buffer b is free once the MMAs of its previous chunk are done with it:
                // they ran after every former warp had formed its tiles of that chunk
                // (each slot group's MMAs wait for all formers' arrivals), so the
                // formers are done with it too
                if (ptid == 0 && use >= 1) wait(&chunk_done[b], (use - 1) & 1);
                asm volatile("bar.sync 1, 256;" ::: "memory");
                uint32_t *Xp = Xp0 + b * MT_XP_ROWS * MT_XP_LD;
                uint8_t *Bop = Bop0 + b * MT_B_BYTES;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = gr0 + 32 * h;
                    float4 lo, hi;
                    load_halves(Xs + r * MT_XS_LD + gg * 8, lo, hi, gg >= 4);
                    const uint4 pk = make_uint4(pack_bf16x2(lo.x, lo.y), pack_bf16x2(lo.z, lo.w),
                                                pack_bf16x2(hi.x, hi.y), pack_bf16x2(hi.z, hi.w));
                    *reinterpret_cast<uint4 *>(Xp + r * MT_XP_LD + gg * 4) = pk;
                    if (r < Nb) *reinterpret_cast<uint4 *>(Bop + sw128(r, gg)) = pk;
                }
                if (ptid < 32) {
                    const int c0 = 2 * ptid;
                    const float w0 = Part[c0] + Part[64 + c0] + Part[128 + c0] + Part[192 + c0];
                    const float w1 = Part[c0 + 1] + Part[65 + c0] + Part[129 + c0] + Part[193 + c0];
                    Xp[MT_ROW_W * MT_XP_LD + ptid] = pack_bf16x2(w0, w1);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("bar.sync 1, 256;" ::: "memory");
                if (ptid == 0) tc::mbar_arrive(tc::smem_u32(&chunk_ready[b]));
            }
        }
        // R = X_c 1: per-thread partial sums of pass 0, reduced over the 64 column threads
#pragma unroll
        for (int e = 0; e < 16; ++e) Xs[(rg * 16 + e) * MT_XS_LD + cc] = racc[e];
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (ptid < k) {
            float r = 0.f;
            for (int c = 0; c < 64; ++c) r += Xs[ptid * MT_XS_LD + c];
            R[pt * k + ptid] = r;
        }
    } else if (warp < MT_PRODUCER_WARPS + MT_FORMER_WARPS) {
        // ================= formers: row products into TMEM; drain =================
        const int qd = warp & 3, half = (warp - MT_PRODUCER_WARPS) >> 2;  // TMEM lane quarter, K half
        const int trow = qd * 32 + lane;
        const uint32_t ngs = (uint32_t)(nslots / MT_GROUP);  // slot groups
        uint32_t gs = 0, gph = 0, gq = 0, gc = 0;             // group slot, its phase, groups formed, chunks
        for (int ps = 0; ps < npass; ++ps) {
            const int t0 = ps * tpp, nt = min(tpp, ntiles - t0);
            for (int ci = 0; ci < nchunks; ++ci, ++gc) {
                const int b = gc & 1;
                if (lane == 0) wait(&chunk_ready[b], (gc >> 1) & 1);
                __syncwarp();
                const uint32_t *Xp = Xp0 + b * MT_XP_ROWS * MT_XP_LD;
                // x_a of the lane's previous tile: along a row of 8 x 8 pair blocks a
                // lane keeps its a, so only x_b is reloaded (shared-memory traffic,
                // not arithmetic, bounds the formers)
                uint4 xa[4];
                int ka = -1;
                // tiles in groups of MT_GROUP: one wait for the group's slots, the
                // group's products stored back to back, one store wait and one
                // arrive (forming the products before the wait was measured slower)
                for (int t = 0; t < nt; t += MT_GROUP, ++gq) {
                    const int cnt = min(MT_GROUP, nt - t);
                    if (gq >= ngs && lane == 0) wait(&slot_empty[gs], gph ^ 1u);
                    __syncwarp();
                    tc::fence_after();
                    for (int u = 0; u < cnt; ++u) {
                        const int code = codes[(t0 + t + u) * 128 + trow];
                        if ((code & 0xff) != ka) {
                            ka = code & 0xff;
                            const uint4 *pa = reinterpret_cast<const uint4 *>(Xp + ka * MT_XP_LD + half * 16);
#pragma unroll
                            for (int e4 = 0; e4 < 4; ++e4) xa[e4] = pa[e4];
                        }
                        const uint4 *pb =
                            reinterpret_cast<const uint4 *>(Xp + ((code >> 8) & 0xff) * MT_XP_LD + half * 16);
                        uint32_t z[16];
#pragma unroll
                        for (int e4 = 0; e4 < 4; ++e4) {
                            const uint4 av = xa[e4], bv = pb[e4];
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
                                                   (uint32_t)(dcols + ((int)gs * MT_GROUP + u) * MT_SLOT_COLS +
                                                              half * 16),
                                               z);
                    }
                    tc::tmem_st_wait();
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(tc::smem_u32(&slot_full[gs]));
                    if (++gs == ngs) { gs = 0; gph ^= 1u; }
                }
            }
            // ---- drain the pass's accumulators: this warp takes tiles half, half + 2, ...
            if (lane == 0) wait(&pass_done, ps & 1);
            __syncwarp();
            tc::fence_after();
            for (int t = half; t < nt; t += 2) {
                const int code = codes[(t0 + t) * 128 + trow];
                const int ra = code & 0xff, rb = (code >> 8) & 0xff, kind = (code >> 16) & 3;
                float *dst = nullptr;
                if (kind == ROW_PAIR) dst = M + (pt * (int64_t)npairs + pair_index(ra, rb, k)) * k;
                else if (kind == ROW_G) dst = G + (pt * k + ra) * (int64_t)k;
                else if (kind == ROW_Q && Q) dst = Q + (pt * k + ra) * (int64_t)k;
                for (int c0 = 0; c0 < Nb; c0 += 16) {
                    uint32_t r16[16];
                    tc::tmem_ld_32x32b_x16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(t * Nb + c0), r16);
                    tc::tmem_ld_wait();
                    if (dst) {
                        if ((k & 3) == 0 && c0 + 16 <= k) {
#pragma unroll
                            for (int e = 0; e < 16; e += 4)
                                *reinterpret_cast<float4 *>(dst + c0 + e) =
                                    make_float4(__uint_as_float(r16[e]), __uint_as_float(r16[e + 1]),
                                                __uint_as_float(r16[e + 2]), __uint_as_float(r16[e + 3]));
                        } else {
#pragma unroll
                            for (int e = 0; e < 16; ++e)
                                if (c0 + e < k) dst[c0 + e] = __uint_as_float(r16[e]);
                        }
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&d_free));
        }
    } else {
        // ================= MMA warp (lane 0 issues) =================
        if (lane == 0) {
            // A single thread issues every MMA, so its loop is kept free of
            // long dependent chains: the slot group and its phase are running
            // counters (no division), the B descriptor is built once per chunk
            // and advanced by adding the 32-byte K step (>> 4) to its address
            // field, and the abort flag is read only when a wait has to spin.
            uint32_t gc = 0, s = 0, ph = 0;
            const uint32_t ngs = (uint32_t)(nslots / MT_GROUP);
            bool ok = true;
            const uint32_t a_base = tmem + (uint32_t)dcols;
            const uint32_t slot_full0 = tc::smem_u32(&slot_full[0]), slot_empty0 = tc::smem_u32(&slot_empty[0]);
            for (int ps = 0; ps < npass && ok; ++ps) {
                const int nt = min(tpp, ntiles - ps * tpp);
                if (ps > 0) {
                    wait(&d_free, (ps - 1) & 1);  // the formers have drained the previous pass
                    ok = !*abortp;
                    tc::fence_after();
                }
                for (int ci = 0; ci < nchunks && ok; ++ci, ++gc) {
                    const uint64_t bd0 = tc::sdesc_sw128(tc::smem_u32(Bop0 + (gc & 1) * MT_B_BYTES));
                    uint32_t d = tmem;
                    for (int t = 0; t < nt; t += MT_GROUP, d += (uint32_t)(MT_GROUP * Nb)) {
                        if (!tc::mbar_wait(slot_full0 + 8 * s, ph, abortp, wait_limit)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t a_g = a_base + s * (uint32_t)(MT_GROUP * MT_SLOT_COLS);
                        if (t + MT_GROUP <= nt) {
#pragma unroll
                            for (int u = 0; u < MT_GROUP; ++u)
#pragma unroll
                                for (int kk = 0; kk < MT_CH / 16; ++kk)
                                    tc::mma_f16_ts(d + (uint32_t)(u * Nb), a_g + (uint32_t)(u * MT_SLOT_COLS + kk * 8),
                                                   bd0 + (uint64_t)(2 * kk), idesc, (ci | kk) != 0);
                        } else {  // a pass whose tile count is not a multiple of MT_GROUP
                            for (int u = 0; u < nt - t; ++u)
#pragma unroll
                                for (int kk = 0; kk < MT_CH / 16; ++kk)
                                    tc::mma_f16_ts(d + (uint32_t)(u * Nb), a_g + (uint32_t)(u * MT_SLOT_COLS + kk * 8),
                                                   bd0 + (uint64_t)(2 * kk), idesc, (ci | kk) != 0);
                        }
                        tc::commit(slot_empty0 + 8 * s);
                        if (++s == ngs) { s = 0; ph ^= 1u; }
                    }
                    tc::commit(tc::smem_u32(&chunk_done[gc & 1]));
                }
                tc::commit(tc::smem_u32(&pass_done));
            }
            // every MMA has completed before TMEM is freed, whatever happened
            // elsewhere: a commit tracks all earlier MMAs of this thread, and a
            // barrier used once has an unambiguous phase 0 (after an abort,
            // pass_done may have two commits pending, and a parity wait there can
            // name a phase that completed earlier).  The wait keeps the long
            // default limit: MMAs in flight always complete.
            tc::commit(tc::smem_u32(&mma_fin));
            if (!tc::mbar_wait(tc::smem_u32(&mma_fin), 0u, &never, MT_WAIT)) fail();
        }
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

cudaError_t launch_moments_tc(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                              int k, int64_t np, const int32_t *rowtab, float *M, float *G, float *R, float *Q,
                              int nslots, long long wait_limit, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (wait_limit <= 0) wait_limit = MT_WAIT;
    if (k > 64 || k < 2) return cudaErrorInvalidValue;
    if (nslots < MT_GROUP || nslots > MT_MAX_SLOTS || nslots % MT_GROUP != 0 ||
        (512 - nslots * MT_SLOT_COLS) < moments_tc_n(k))
        return cudaErrorInvalidValue;
    const int nrows = moments_tc_rows(k);
    const size_t smem = moments_tc_smem_bytes(k);
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(moments_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        moments_tc_kernel<<<(unsigned)np, MT_THREADS, smem, s>>>((const __nv_bfloat16 *)X, N, m, ld, idx, k, rowtab,
                                                                 nrows, M, G, R, Q, nslots, wait_limit, ctr);
    } else {
        e = cudaFuncSetAttribute(moments_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        moments_tc_kernel<<<(unsigned)np, MT_THREADS, smem, s>>>((const float *)X, N, m, ld, idx, k, rowtab, nrows, M,
                                                                 G, R, Q, nslots, wait_limit, ctr);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
