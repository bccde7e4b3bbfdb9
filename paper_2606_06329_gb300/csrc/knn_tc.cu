// knn_tc.cu - Step 1 (Sec. 3 Step 1, eq. knn; Alg. 1 kNN-Graph) candidate
// search on the 5th-generation tensor cores: BF16 x BF16 -> FP32 distance GEMM
// with the per-row candidate selection fused into the TMEM drain.
//
// Persistent CTAs (one per SM); a work item = 128 query rows (the MMA's M, one
// TMEM lane each) against one split of the candidate rows, swept in tiles of
// 256 (the MMA's N).  Warp roles:
//   warp 0      TMA producer: for every (candidate tile, TBK-wide K block) loads
//               the 128 x TBK query slice and the 256 x TBK candidate slice
//               (swizzled by the width of a TBK row, zero-filled past the
//               matrix edges) into a NSTAGE-deep ring of shared-memory stages.
//   warp 1      allocates 512 TMEM columns (two 256-column FP32 accumulators)
//               and issues tcgen05.mma (M=128, N=256, K=16) from one lane,
//               committing each stage back to the producer and each finished
//               tile to the epilogue.
//   warps 2-9   epilogue: drain one accumulator while the MMA fills the other;
//               the two warps of a TMEM lane quarter take one query row per
//               thread and half of the tile's 256 columns each, every (row,
//               half) with its own kc-slot candidate list (distances in shared
//               memory as a max-heap, indices straight to global), so a row leaves with
//               TC_HALVES lists per candidate split; d~ = |x|^2 + |y|^2 - 2 x.y;
//               values below a list's admission threshold enter it.
// CTA pairs (optional, for 256 or more query rows): two CTAs of a
// thread-block cluster share one 256 x 256 tcgen05.mma (cta_group::2, M = 256)
// per K step.  Each CTA loads its own 128 query rows and one 128-row half of
// the candidate tile (16 KB a stage instead of 24 KB, nine stages in the same
// shared memory); both CTAs' loads complete on the even CTA's stage barrier
// (cta_group::2 TMA), whose warp 1 issues the MMAs and commits (multicast) to
// both CTAs' barriers; each CTA drains its own 128 accumulator rows, and the eight
// epilogue warps of both CTAs release an accumulator at the even CTA.  The
// lists are those of the single-CTA form.  Measured on GB300 it ties the
// single-CTA form at 1M x 4096 (8.0 s per search) and is 5% slower at 100k,
// so single CTAs are the default.
// Every mbarrier wait is bounded; a timeout sets MECUCO_ERR_TIMEOUT in the
// device status word, raises a CTA-wide abort flag, drains the copies and MMAs
// already in flight (also bounded), frees TMEM and returns.  The limit of the
// waits in the work loops is a launch argument (default WAIT_LIMIT); the drains
// always use WAIT_LIMIT, since the copies and MMAs they wait for complete.
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace mecuco {

namespace {
constexpr int TBM = 128;        // query rows per CTA (MMA M)
constexpr int TBN = 256;        // candidate rows per tile (MMA N)
// K elements per stage: 32 (one 64-byte swizzle row) in 6 stages of 24 KB
// rather than 64 in 3 stages of 48 KB - the same shared memory, but 5/6 of it
// in flight while the MMA consumes a stage instead of 2/3
constexpr int TBK = 32;
constexpr int NSTAGE = 6;
constexpr int A_BYTES = TBM * TBK * 2;   // 8 KB
constexpr int B_BYTES = TBN * TBK * 2;   // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
static_assert(TBK == 64 || TBK == 32, "stage rows are one 128- or 64-byte swizzle row");
// K-major operand descriptor of a stage (swizzle width = the stage's row)
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) {
    return TBK == 64 ? tc::sdesc_sw128(saddr) : tc::sdesc_sw64(saddr);
}
constexpr int TC_THREADS = 320;  // TMA warp, MMA warp, 8 epilogue warps
constexpr int TC_HALVES = 2;     // epilogue warps per TMEM lane quarter (column halves)
constexpr long long WAIT_LIMIT = 1000000000LL;  // ~0.5 s of SM clock per wait

struct ListState {
    float thr;  // admission threshold: the largest distance held once the list is full
    int cnt;    // entries in use
};

// Rare path of the drain: the row's list is a binary max-heap of kc distances
// in shared memory (position p at Ld[p * TBM + row]); Ls[p * TBM + row] is the
// slot of the global index array out[] that holds the entry's candidate, so
// entries move inside the heap without touching global memory.  Filling appends
// and sifts up; once full, a candidate below the root replaces it and sifts
// down (O(log kc) instead of a scan for the new maximum).
__device__ __noinline__ ListState list_insert(ListState st, float d, int c, float *Ld, uint8_t *Ls, int32_t *out,
                                              int row, int kc) {
    if (st.cnt < kc) {
        int pos = st.cnt;
        while (pos > 0) {
            const int par = (pos - 1) >> 1;
            const float pd = Ld[par * TBM + row];
            if (pd >= d) break;
            Ld[pos * TBM + row] = pd;
            Ls[pos * TBM + row] = Ls[par * TBM + row];
            pos = par;
        }
        Ld[pos * TBM + row] = d;
        Ls[pos * TBM + row] = (uint8_t)st.cnt;
        out[st.cnt] = c;
        ++st.cnt;
        if (st.cnt == kc) st.thr = Ld[row];
        return st;
    }
    const uint8_t slot = Ls[row];
    out[slot] = c;
    int pos = 0;
    for (;;) {
        const int l = 2 * pos + 1;
        if (l >= kc) break;
        const float dl = Ld[l * TBM + row];
        const float dr = l + 1 < kc ? Ld[(l + 1) * TBM + row] : -INFINITY;
        const int ch = dr > dl ? l + 1 : l;
        const float dc = dr > dl ? dr : dl;
        if (dc <= d) break;
        Ld[pos * TBM + row] = dc;
        Ls[pos * TBM + row] = Ls[ch * TBM + row];
        pos = ch;
    }
    Ld[pos * TBM + row] = d;
    Ls[pos * TBM + row] = slot;
    st.thr = Ld[row];
    return st;
}

constexpr int MAX_NSTAGE = 9;
constexpr int PEND = 16;        // register buffer of admitted candidates per (row, half)
constexpr int PEND_TILES = 16;  // tiles of an item drained through the buffer (2,048 candidates per list)
constexpr int PEND_ALL_TILES = 256;  // items of at most this many tiles use the buffer throughout

// Per-variant layout.  Single CTA: a work item is 128 query rows; each stage
// holds the 128-row query slice and the 256-row candidate slice (24 KB at
// K = 32), six stages.  CTA pair (cta_group::2, M = 256): a work item is 256
// query rows, 128 per CTA; each CTA's stage holds its 128 query rows and its
// 128 of the tile's 256 candidate rows (16 KB), nine stages in the same
// shared memory, and one 256 x 256 MMA per K step covers both.
template <bool PAIR>
struct KCfg {
    static constexpr int B_ROWS = PAIR ? TBN / 2 : TBN;
    static constexpr int STAGE = A_BYTES + B_ROWS * TBK * 2;
    static constexpr int NST = PAIR ? 9 : 6;
    static constexpr int QROWS = PAIR ? 2 * TBM : TBM;
    static constexpr uint32_t IDESC = tc::idesc_bf16_f32(PAIR ? 2 * TBM : TBM, TBN);
};
static_assert(KCfg<false>::NST * KCfg<false>::STAGE == KCfg<true>::NST * KCfg<true>::STAGE, "same ring size");

// Geometry of one work item: query block, candidate split and the operand's
// description (a single launch: the kernel's arguments; a batched launch: the
// item's dataset in the device table).
struct ItemGeo {
    const CUtensorMap *ma, *mb;
    const float *norms;
    float *cand_d;
    int32_t *cand_i;
    int64_t N, q0, qend, qb, cbeg, cend;
    int ntiles, nkb, split, nsplit, kc, include_self;
};

struct TcShared {
    uint64_t full[MAX_NSTAGE];
    uint64_t empty[MAX_NSTAGE];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint32_t tmem_base;
    int abort;
};
}  // namespace

template <bool PAIR, bool BATCH, bool BUF>
__global__ void __launch_bounds__(TC_THREADS, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int64_t N,
              int64_t m, const float *__restrict__ norms, int64_t q0, int64_t nq, int kc, int nsplit,
              int include_self, float *__restrict__ cand_d, int32_t *__restrict__ cand_i, long long wait_limit,
              DevCounters *ctr, const KnnSet *__restrict__ sets, int nsets, int64_t nitems_all) {
    // Persistent: CTA (pair) b takes work items b, b + G, b + 2G, ... (G CTAs or
    // pairs), item = (query block item / nsplit, candidate split item % nsplit).
    // All start their items together and every item has the same number of
    // tiles, so they sweep the same candidate tiles in lockstep (each tile comes
    // from HBM about once per wave).
    using C = KCfg<PAIR>;
    constexpr int NST = C::NST;
    constexpr int STAGE = C::STAGE;
    extern __shared__ __align__(1024) uint8_t tsm_raw[];
    // 1024-byte aligned stage ring, then candidate distances [kc][TBM], then barriers
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *stages = base;
    float *Ld0 = reinterpret_cast<float *>(base + NST * STAGE);  // [TC_HALVES][kc][TBM] heaps
    uint8_t *Ls0 = reinterpret_cast<uint8_t *>(Ld0 + (size_t)TC_HALVES * kc * TBM);  // [TC_HALVES][kc][TBM]
    TcShared *sh = reinterpret_cast<TcShared *>(Ls0 + (size_t)TC_HALVES * kc * TBM);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? tc::cluster_ctarank() : 0u;
    const int64_t nitems = BATCH ? nitems_all : ((nq + C::QROWS - 1) / C::QROWS) * nsplit;
    const int64_t first = PAIR ? blockIdx.x / 2 : blockIdx.x, stride = PAIR ? gridDim.x / 2 : gridDim.x;
    // a batched launch reads each item's dataset from the table (items of a
    // dataset are consecutive; the table is sorted by first item)
    auto geo = [&](int64_t item) {
        ItemGeo g;
        int64_t li = item;
        if constexpr (BATCH) {
            int lo = 0, hi = nsets - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sets[mid].item_begin <= item) lo = mid;
                else hi = mid - 1;
            }
            const KnnSet &d = sets[lo];
            li = item - d.item_begin;
            g.ma = &d.map_a;
            g.mb = &d.map_b;
            g.norms = d.norms;
            g.cand_d = d.cand_d;
            g.cand_i = d.cand_i;
            g.N = d.N;
            g.q0 = 0;
            g.qend = d.N;
            g.nsplit = d.nsplit;
            g.kc = d.kcl;
            g.nkb = (int)((d.mk + TBK - 1) / TBK);
            g.include_self = d.include_self;
        } else {
            g.ma = &map_a;
            g.mb = &map_b;
            g.norms = norms;
            g.cand_d = cand_d;
            g.cand_i = cand_i;
            g.N = N;
            g.q0 = q0;
            g.qend = q0 + nq;
            g.nsplit = nsplit;
            g.kc = kc;
            g.nkb = (int)((m + TBK - 1) / TBK);
            g.include_self = include_self;
        }
        const int64_t per = (g.N + g.nsplit - 1) / g.nsplit;
        g.split = (int)(li % g.nsplit);
        g.qb = g.q0 + (li / g.nsplit) * C::QROWS;
        g.cbeg = (int64_t)g.split * per;
        g.cend = min(g.N, g.cbeg + per);
        g.ntiles = g.cend > g.cbeg ? (int)((g.cend - g.cbeg + TBN - 1) / TBN) : 0;
        return g;
    };
    volatile int *abort_flag = &sh->abort;
    __shared__ int never;  // a flag that stays 0: drain waits are bounded by time only

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            tc::mbar_init(tc::smem_u32(&sh->full[s]), 1);
            tc::mbar_init(tc::smem_u32(&sh->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(tc::smem_u32(&sh->tfull[a]), 1);
            // pair: one arrival per epilogue warp of both CTAs (at the even CTA)
            tc::mbar_init(tc::smem_u32(&sh->tempty[a]), PAIR ? 2 * 4 * TC_HALVES : 4 * TC_HALVES * 32);
        }
        // circuit breaker: once any CTA of this launch timed out, later CTAs skip
        // the work (their lists come out empty) instead of timing out one by one
        // (a pair decides once, below)
        sh->abort = (!PAIR && (*(volatile unsigned *)&ctr->status & DEV_TIMEOUT)) ? 1 : 0;
        never = 0;
        tc::fence_mbar_init();
        if constexpr (!BATCH) {
            tc::prefetch_tmap(&map_a);
            tc::prefetch_tmap(&map_b);
        }
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            tc::tmem_alloc2(tc::smem_u32(&sh->tmem_base), 512);
        } else {
            tc::tmem_alloc(tc::smem_u32(&sh->tmem_base), 512);
            tc::tmem_relinquish();
        }
    }
    tc::fence_before();
    __syncthreads();
    if constexpr (PAIR) {
        __syncwarp();
        tc::cluster_sync();  // both CTAs' barriers initialised before any remote arrive
        if (rank == 0 && threadIdx.x == 0) {
            const uint32_t ab = (*(volatile unsigned *)&ctr->status & DEV_TIMEOUT) ? 1u : 0u;
            tc::st_cluster_u32(tc::mapa(tc::smem_u32(&sh->abort), 0), ab);
            tc::st_cluster_u32(tc::mapa(tc::smem_u32(&sh->abort), 1), ab);
        }
        __syncwarp();
        tc::cluster_sync();
    }
    tc::fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        // ------------------------------ TMA producer ----------------------------
        if (lane == 0) {
            // one thread issues every load: stage index and phase are running
            // counters, so the loop carries no division
            int it = 0;
            uint32_t s = 0, ph = 0;
            bool ok = true;
            const uint32_t st0 = tc::smem_u32(stages), full0 = tc::smem_u32(&sh->full[0]),
                           empty0 = tc::smem_u32(&sh->empty[0]);
            // pair: both CTAs' loads complete on the even CTA's barrier, which
            // expects the bytes of both
            const uint32_t pfull0 = PAIR ? tc::mapa(full0, 0) : 0u;
            const CUtensorMap *last_map = nullptr;
            for (int64_t item = first; item < nitems && ok && !*abort_flag; item += stride) {
            const ItemGeo g = geo(item);
            const int64_t qb = g.qb + (int64_t)rank * TBM;
            const CUtensorMap *map_q = g.ma, *map_c = g.mb;
            if constexpr (BATCH) {
                // the table's maps were written by a host copy: fence each dataset's
                // pair once before its first load
                if (map_q != last_map) {
                    tc::fence_tmap_acquire(map_q);
                    if (map_c != map_q) tc::fence_tmap_acquire(map_c);
                    last_map = map_q;
                }
            }
            for (int t = 0; t < g.ntiles && ok && !*abort_flag; ++t) {
                const int c0 = (int)(g.cbeg + (int64_t)t * TBN) + (int)rank * C::B_ROWS;
                for (int kb = 0; kb < g.nkb; ++kb, ++it) {
                    if (!tc::mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag, wait_limit)) { ok = false; break; }
                    const uint32_t sa = st0 + s * (uint32_t)STAGE;
                    if constexpr (PAIR) {
                        if (rank == 0) tc::mbar_expect_tx(full0 + 8 * s, 2 * STAGE);
                        tc::tma_load_2d_pair(sa, map_q, pfull0 + 8 * s, kb * TBK, (int)qb);
                        tc::tma_load_2d_pair(sa + A_BYTES, map_c, pfull0 + 8 * s, kb * TBK, c0);
                    } else {
                        const uint32_t fb = full0 + 8 * s;
                        tc::mbar_expect_tx(fb, STAGE);
                        tc::tma_load_2d(sa, map_q, fb, kb * TBK, (int)qb);
                        tc::tma_load_2d(sa + A_BYTES, map_c, fb, kb * TBK, c0);
                    }
                    if (++s == (uint32_t)NST) { s = 0; ph ^= 1u; }
                }
            }
            }
            if (!ok) {
                atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
                sh->abort = 1;
            }
            // drain: every issued stage must have landed before the CTA can exit
            // (bounded by time only: the abort flag must not cut this wait short);
            // a pair waits until the pair MMA has released them (they landed
            // before it ran), so that no read of this CTA's stages or commit to
            // its barriers is outstanding
            const int issued = it;
            for (int j = issued - NST; j < issued; ++j) {
                if (j < 0) continue;
                if (PAIR)
                    tc::mbar_wait(tc::smem_u32(&sh->empty[j % NST]), (j / NST) & 1, &never, WAIT_LIMIT);
                else
                    tc::mbar_wait(tc::smem_u32(&sh->full[j % NST]), (j / NST) & 1, &never, WAIT_LIMIT);
            }
        }
    } else if (warp == 1) {
        if (PAIR && rank == 1) {
            // odd CTA of a pair: the even CTA issues the pair MMAs
        } else {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            // lean issue loop (a single thread): running stage / phase counters,
            // descriptors as base + stage offset + K step (address field >> 4)
            int it = 0;
            uint32_t s = 0, ph = 0;
            bool ok = true;
            int t = 0;  // tiles issued so far by this CTA (all items)
            const uint32_t st0 = tc::smem_u32(stages), full0 = tc::smem_u32(&sh->full[0]),
                           empty0 = tc::smem_u32(&sh->empty[0]);
            const uint64_t ad0 = kdesc(st0), bd0 = kdesc(st0 + A_BYTES);
            for (int64_t item = first; item < nitems && ok && !*abort_flag; item += stride) {
            const ItemGeo g = geo(item);
            const int nkb = g.nkb;
            for (int tt = 0; tt < g.ntiles && ok && !*abort_flag; ++tt, ++t) {
                const int acc = t & 1;
                const uint32_t te = tc::smem_u32(&sh->tempty[acc]);
                const uint32_t tpar = ((t >> 1) & 1) ^ 1;
                if (!(PAIR ? tc::mbar_wait_cluster(te, tpar, abort_flag, wait_limit)
                           : tc::mbar_wait(te, tpar, abort_flag, wait_limit))) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * TBN);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    if (!(PAIR ? tc::mbar_wait_cluster(full0 + 8 * s, ph, abort_flag, wait_limit)
                               : tc::mbar_wait(full0 + 8 * s, ph, abort_flag, wait_limit))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint64_t off = (uint64_t)(s * (uint32_t)(STAGE >> 4));
#pragma unroll
                    for (int kk = 0; kk < TBK / 16; ++kk) {
                        if constexpr (PAIR)
                            tc::mma2_f16(dt, ad0 + off + (uint64_t)(2 * kk), bd0 + off + (uint64_t)(2 * kk),
                                         C::IDESC, (kb | kk) != 0);
                        else
                            tc::mma_f16(dt, ad0 + off + (uint64_t)(2 * kk), bd0 + off + (uint64_t)(2 * kk),
                                        C::IDESC, (kb | kk) != 0);
                    }
                    if constexpr (PAIR) tc::commit2_mc(empty0 + 8 * s, (uint16_t)3);
                    else tc::commit(empty0 + 8 * s);
                    if (++s == (uint32_t)NST) { s = 0; ph ^= 1u; }
                }
                if (ok) {
                    if constexpr (PAIR) tc::commit2_mc(tc::smem_u32(&sh->tfull[acc]), (uint16_t)3);
                    else tc::commit(tc::smem_u32(&sh->tfull[acc]));
                }
            }
            }
            if (!ok) {
                atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
                sh->abort = 1;
            }
            // drain: the last commit covers every MMA issued by this thread
            if (it > 0) {
                const int j = it - 1;
                tc::mbar_wait(tc::smem_u32(&sh->empty[j % NST]), (j / NST) & 1, &never, WAIT_LIMIT);
            }
        }
        __syncwarp();
        }
    } else {
        // ------------------------------ epilogue ---------------------------------
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        const int half = (warp - 2) >> 2;  // columns [128 half, 128 half + 128) of each tile
        const int row = quarter * 32 + lane;
        float *Ld = Ld0 + (size_t)half * kc * TBM;
        uint8_t *Ls = Ls0 + (size_t)half * kc * TBM;
        const uint32_t tempty_even0 = PAIR ? tc::mapa(tc::smem_u32(&sh->tempty[0]), 0) : 0u;
        int t = 0;  // tiles drained so far by this CTA (all items)
        for (int64_t item = first; item < nitems && !*abort_flag; item += stride) {
            const ItemGeo g = geo(item);
            const int64_t qb = g.qb + (int64_t)rank * TBM;
            const int64_t cbeg = g.cbeg, cend = g.cend, N = g.N;
            const int ntiles = g.ntiles, kc = g.kc;
            const int include_self = g.include_self;
            const float *norms = g.norms;
            const int64_t gq = qb + row;
            const bool valid_row = gq < g.qend;
            const float qn = valid_row ? norms[gq] : 0.f;
            const int64_t out_base =
                valid_row ? (((gq - g.q0) * g.nsplit + g.split) * TC_HALVES + half) * (int64_t)kc : 0;
            ListState st{valid_row ? INFINITY : -INFINITY, 0};
            int32_t *out_i = g.cand_i + out_base;
            // In the first PEND_TILES tiles of an item, candidates below the
            // threshold wait in registers (newest first) and go into the heap
            // together: a warp flushes before a group of 8 candidates once any
            // lane holds more than PEND - 8, so a heap pass serves every lane's
            // pending entries instead of one candidate column at a time.  32
            // rows' independent lists otherwise take a divergent pass whenever
            // any of them admits a candidate, which is most candidates while the
            // lists fill (the first ~32 kc per list); later tiles of long items
            // admit rarely and insert directly (the buffer's extra instructions
            // slowed a 1M-point search by 15%), while items of up to
            // PEND_ALL_TILES tiles keep the buffer throughout (a 19,647-point
            // search: 6.89 ms direct, 6.13 with 16 buffered tiles, 4.89 with all)
            float pd[PEND];
            int pc[PEND];
            int np = 0;
            const int pend_tiles = BUF ? (ntiles <= PEND_ALL_TILES ? ntiles : PEND_TILES) : 0;
            auto flush = [&]() {
#pragma unroll
                for (int i = 0; i < PEND; ++i)
                    if (i < np && pd[i] < st.thr) st = list_insert(st, pd[i], pc[i], Ld, Ls, out_i, row, kc);
                np = 0;
            };
            for (int tt = 0; tt < ntiles && !*abort_flag; ++tt, ++t) {
                const int acc = t & 1;
                if (!tc::mbar_wait(tc::smem_u32(&sh->tfull[acc]), (t >> 1) & 1, abort_flag, wait_limit)) {
                    atomicOr(&ctr->status, (unsigned)DEV_TIMEOUT);
                    sh->abort = 1;
                    break;
                }
                tc::fence_after();
                const int64_t c0 = cbeg + (int64_t)tt * TBN;
                const bool masked = (c0 + TBN > cend) || (!include_self && gq >= c0 && gq < c0 + TBN);
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * TBN);
#pragma unroll 1
                for (int ch = half * (TBN / 32 / TC_HALVES); ch < (half + 1) * (TBN / 32 / TC_HALVES); ++ch) {
                    uint32_t r[32];
                    tc::tmem_ld_32x32b_x32(taddr + ch * 32, r);
                    tc::tmem_ld_wait();
                    const int64_t cb = c0 + ch * 32;
                    const float *cnp = norms + cb;
                    if (BUF && tt < pend_tiles) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if ((j & 7) == 0 && __any_sync(0xffffffffu, np > PEND - 8)) flush();
                            const int64_t c = cb + j;
                            const float cn = (c < N) ? __ldg(cnp + j) : 0.f;
                            float d = fmaf(-2.f, __uint_as_float(r[j]), qn + cn);
                            if (masked && (c >= cend || (!include_self && c == gq))) d = INFINITY;
                            const bool adm = d < st.thr;
                            // the vote keeps the (predicated) shift off the common path
                            if (__any_sync(0xffffffffu, adm) && adm) {
#pragma unroll
                                for (int i = PEND - 1; i > 0; --i) {
                                    pd[i] = pd[i - 1];
                                    pc[i] = pc[i - 1];
                                }
                                pd[0] = d;
                                pc[0] = (int)c;
                                ++np;
                            }
                        }
                    } else {
                        // past the first tiles admissions are rare: straight into the heap
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int64_t c = cb + j;
                            const float cn = (c < N) ? __ldg(cnp + j) : 0.f;
                            float d = fmaf(-2.f, __uint_as_float(r[j]), qn + cn);
                            if (masked && (c >= cend || (!include_self && c == gq))) d = INFINITY;
                            if (d < st.thr) st = list_insert(st, d, (int)c, Ld, Ls, out_i, row, kc);
                        }
                    }
                }
                if (BUF && tt + 1 == pend_tiles) flush();
                tc::fence_before();
                if constexpr (PAIR) {
                    // one arrival per warp at the even CTA, once every lane has read its rows
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive_cluster(tempty_even0 + 8 * acc);
                } else {
                    tc::mbar_arrive(tc::smem_u32(&sh->tempty[acc]));
                }
            }
            if constexpr (BUF) flush();
            if (valid_row) {
                for (int p = 0; p < st.cnt; ++p) g.cand_d[out_base + Ls[p * TBM + row]] = Ld[p * TBM + row];
                for (int s2 = st.cnt; s2 < kc; ++s2) {
                    g.cand_d[out_base + s2] = INFINITY;
                    out_i[s2] = -1;
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if constexpr (PAIR) {
        // no remote arrive, commit or MMA read targets either CTA past here
        __syncwarp();
        tc::cluster_sync();
    }
    if (warp == 1) {
        tc::fence_after();
        if constexpr (PAIR) tc::tmem_dealloc2(tmem, 512);
        else tc::tmem_dealloc(tmem, 512);
    }
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *map, const void *Xb, int64_t N, int64_t m, int64_t ldb, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)ldb * 2};
    cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(Xb), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, TBK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}
}  // namespace

size_t knn_tc_smem_bytes(int kc) {
    return 1024 + (size_t)NSTAGE * STAGE_BYTES + (size_t)TC_HALVES * kc * TBM * (sizeof(float) + 1) + sizeof(TcShared) +
           64;
}

int knn_tc_halves() { return TC_HALVES; }
int knn_tc_item_rows(int pair) { return pair ? KCfg<true>::QROWS : KCfg<false>::QROWS; }

cudaError_t launch_knn_tc(const void *Xa, const void *Xb, int64_t N, int64_t m, int64_t ldb, const float *norms,
                          int64_t q0, int64_t nq, int kc, int nsplit, int include_self, float *cand_d, int32_t *cand_i,
                          int pair, long long wait_limit, DevCounters *ctr, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    if (wait_limit <= 0) wait_limit = WAIT_LIMIT;
    if ((reinterpret_cast<uintptr_t>(Xa) & 15) || (reinterpret_cast<uintptr_t>(Xb) & 15) || (ldb % 8) != 0 || kc > 64)
        return cudaErrorInvalidValue;
    // queries from Xa (128-row boxes); candidates from Xb, in 256-row boxes for
    // single CTAs and 128-row halves for CTA pairs
    CUtensorMap ma, mb, mb2;
    if (!make_map(&ma, Xa, N, m, ldb, TBM) || !make_map(&mb, Xb, N, m, ldb, TBN) || !make_map(&mb2, Xb, N, m, ldb, TBM))
        return cudaErrorInvalidValue;
    const size_t smem = knn_tc_smem_bytes(kc);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // short sweeps (items of at most PEND_ALL_TILES candidate tiles) drain
    // through the register buffer; long ones take the direct form, whose
    // leaner loop a 1M-point search needs
    const bool buf = (N + TBN - 1) / TBN <= PEND_ALL_TILES;
    if (pair && nq >= 2 * TBM) {
        // CTA pairs (cta_group::2): 256 query rows per item; each CTA's candidate
        // half uses the 128-row box of the query map
        auto kern = buf ? knn_tc_kernel<true, false, true> : knn_tc_kernel<true, false, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (nclusters > 0) {
            const int64_t items = ((nq + 2 * TBM - 1) / (2 * TBM)) * nsplit;
            cfg.gridDim = dim3((unsigned)(2 * (items < nclusters ? items : nclusters)));
            // the pair form keeps the default limit: its cross-CTA arrivals are
            // not exercised with shortened waits
            e = cudaLaunchKernelEx(&cfg, kern, ma, mb2, N, m, norms, q0, nq, kc, nsplit, include_self, cand_d, cand_i,
                                   WAIT_LIMIT, ctr, (const KnnSet *)nullptr, 0, (int64_t)0);
            if (e != cudaSuccess) return e;
            return cudaGetLastError();
        }
        // no pair fits: single CTAs
    }
    auto kern = buf ? knn_tc_kernel<false, false, true> : knn_tc_kernel<false, false, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = ((nq + TBM - 1) / TBM) * nsplit;
    dim3 grid((unsigned)(items < sms ? items : sms));  // persistent: one CTA per SM
    kern<<<grid, TC_THREADS, smem, s>>>(ma, mb, N, m, norms, q0, nq, kc, nsplit, include_self, cand_d, cand_i,
                                        wait_limit, ctr, nullptr, 0, 0);
    return cudaGetLastError();
}

bool knn_tc_make_maps(KnnSet *d, int pair) {
    const void *qa = d->xb ? d->xb : d->X;
    const void *cb = d->xb2 ? d->xb2 : qa;
    return make_map(&d->map_a, qa, d->N, d->mk, d->ldb, TBM) &&
           make_map(&d->map_b, cb, d->N, d->mk, d->ldb, pair ? TBM : TBN);
}

cudaError_t launch_knn_tc_batch(const KnnSet *sets, int nsets, int64_t nitems, int kcmax, int pair,
                                long long wait_limit, DevCounters *ctr, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (kcmax > 64 || nsets < 1) return cudaErrorInvalidValue;
    if (wait_limit <= 0) wait_limit = WAIT_LIMIT;
    const size_t smem = knn_tc_smem_bytes(kcmax);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    CUtensorMap none;
    memset(&none, 0, sizeof(none));
    if (pair) {
        // items of 256 query rows (the table's item counts must be for that size)
        e = cudaFuncSetAttribute(knn_tc_kernel<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(2);
        int nclusters = 0;
        e = cudaOccupancyMaxActiveClusters(&nclusters, knn_tc_kernel<true, true, true>, &cfg);
        if (e != cudaSuccess) return e;
        if (nclusters <= 0) return cudaErrorInvalidConfiguration;
        cfg.gridDim = dim3((unsigned)(2 * (nitems < nclusters ? nitems : nclusters)));
        e = cudaLaunchKernelEx(&cfg, knn_tc_kernel<true, true, true>, none, none, (int64_t)0, (int64_t)0,
                               (const float *)nullptr, (int64_t)0, (int64_t)0, kcmax, 1, 0, (float *)nullptr,
                               (int32_t *)nullptr, WAIT_LIMIT, ctr, sets, nsets, nitems);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    e = cudaFuncSetAttribute(knn_tc_kernel<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(nitems < sms ? nitems : sms));
    knn_tc_kernel<false, true, true><<<grid, TC_THREADS, smem, s>>>(none, none, 0, 0, nullptr, 0, 0, kcmax, 1, 0, nullptr,
                                                               nullptr, wait_limit, ctr, sets, nsets, nitems);
    return cudaGetLastError();
}

// FP32 -> BF16 copy (round to nearest even) with a padded leading dimension.
__global__ void to_bf16_kernel(const float *__restrict__ X, int64_t N, int64_t m, int64_t ld,
                               __nv_bfloat16 *__restrict__ Y, int64_t ldb) {
    const int64_t row = blockIdx.x;
    for (int64_t a = threadIdx.x; a < ldb; a += blockDim.x)
        Y[row * ldb + a] = __float2bfloat16_rn(a < m ? X[row * ld + a] : 0.f);
}

// The three-term split of FP32 rows for the search: with h = bf16(x) and
// l = bf16(x - h), the query copy holds [h | h | l] and the candidate copy
// [h | l | h] along K (segments of ms columns, zero past m), so that one GEMM
// over K = 3 ms gives h.h' + h.l' + l.h', the FP32 product up to l.l' and the
// remainders past two terms.
__global__ void to_bf16_split_kernel(const float *__restrict__ X, int64_t m, int64_t ld, __nv_bfloat16 *__restrict__ Ya,
                                     __nv_bfloat16 *__restrict__ Yb, int64_t ms, int64_t ldb) {
    const int64_t row = blockIdx.x;
    const float *x = X + row * ld;
    __nv_bfloat16 *ya = Ya + row * ldb, *yb = Yb + row * ldb;
    for (int64_t a = threadIdx.x; a < ldb; a += blockDim.x) {
        const int64_t seg = a / ms, c = a - seg * ms;
        const float v = (seg < 3 && c < m) ? x[c] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        ya[a] = seg == 2 ? l : h;
        yb[a] = seg == 1 ? l : h;
    }
}

cudaError_t launch_to_bf16_split(const float *X, int64_t N, int64_t m, int64_t ld, void *Ya, void *Yb, int64_t ms,
                                 int64_t ldb, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    to_bf16_split_kernel<<<(unsigned)N, 256, 0, s>>>(X, m, ld, (__nv_bfloat16 *)Ya, (__nv_bfloat16 *)Yb, ms, ldb);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, void *Y, int64_t ldb,
                           cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    if (dt == MECUCO_BF16) {
        return cudaMemcpy2DAsync(Y, (size_t)ldb * 2, X, (size_t)ld * 2, (size_t)m * 2, (size_t)N,
                                 cudaMemcpyDeviceToDevice, s);
    }
    to_bf16_kernel<<<(unsigned)N, 256, 0, s>>>((const float *)X, N, m, ld, (__nv_bfloat16 *)Y, ldb);
    return cudaGetLastError();
}

}  // namespace mecuco
