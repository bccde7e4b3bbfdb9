// api.cu - the C ABI declared in include/mecuco.h: context, workspace,
// argument validation, stage profiling and the orchestration of the hot path
// (kNN -> gather/centre/Gram/moments -> Jacobi -> estimator).
#include <stdio.h>
#include <string.h>

#include <cstddef>

#include <algorithm>
#include <map>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace mecuco;

namespace {
thread_local char g_errmsg[512] = "";

void set_err(const char *where, cudaError_t e) {
    snprintf(g_errmsg, sizeof(g_errmsg), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
}  // namespace

void mecuco::set_error_text(const char *msg) { snprintf(g_errmsg, sizeof(g_errmsg), "%s", msg); }

namespace {

// Offsets into one device buffer, 256-byte aligned.  Sizing and carving use
// the same sequence of take() calls, first with base == nullptr.
struct Carver {
    char *base;
    size_t off;
    explicit Carver(char *b, size_t start = 0) : base(b), off(start) {}
    template <typename T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

struct EventPair {
    cudaEvent_t a, b;
    int stage;
};
}  // namespace

struct mecuco_ctx {
    int device = 0;
    int num_sms = 0;
    char *ws = nullptr;  // device workspace, grown on demand
    size_t ws_bytes = 0;
    char *io = nullptr;  // device copies of the host-buffer entry point
    size_t io_bytes = 0;
    DevCounters *ctr = nullptr;
    int32_t *m3_items[65] = {};  // per k: work items of the CUDA-core third-moment kernel
    int32_t *rowtab[65] = {};    // per k: row codes of the tensor-core moment kernel
    int32_t *tttab[65] = {};     // per k: row codes of the third-moment pass (pairs only)
    int knn_splits = 0;
    int knn_pair = -1;  // -1: CTA pairs for N >= KNN_PAIR_MIN_N
    int knn_split_bf16 = 1;  // FP32 rows: three-term BF16 split in the tensor-core search
    int chunk_share = 1;  // concurrent lanes sharing the chunk budget (batched calls)
    int tc_slots = 4;
    // third-moment pass: TMEM slots of the A operand and CTAs per SM; two CTAs
    // of 256 columns (2 tiles per pass, 9 passes at k = 64) interleave their
    // hand-over pipelines: 177 against 251 ms for one CTA of 512 columns at
    // 100k x 4096 (6 or 8 slots in one CTA: 275 / 261 ms; 2 slots in two: 289 ms)
    int tt_slots = 4;
    int tt_ctas = 2;
    // randomised low-rank SVD (mecuco_curvature_rsvd), set for the duration of a call
    struct {
        int rank = 0, cols = 0, power = 0;
        const float *omega = nullptr;
    } rsvd;
    // batched entry point: lanes (streams) and their workspace
    int batch_lanes = 8;
    char *bws = nullptr;
    size_t bws_bytes = 0;
    cudaStream_t lane_stream[32] = {};
    cudaEvent_t lane_event[32] = {};
    cudaEvent_t fork_event = nullptr;
    int batch_persistent = 1;  // BF16-mixed batches: one launch per stage (0: lanes)
    // batch signature -> tuned configuration (mecuco_autotune_batched)
    std::map<std::tuple<int, int64_t, int64_t, int64_t, int, int>, mecuco_batch_tuning> tuned;
    // device tables of the one-launch-per-stage batches, oldest first
    struct BatchTables {
        std::vector<char> host;
        char *dev = nullptr;
    };
    std::vector<BatchTables> btabs;
    // options
    int64_t knn_margin = 32;
    int jacobi_fp64 = -1;
    int jacobi_max_sweeps = 40;
    int jacobi_warp = 2;  // FP32 sweeps: warps per patch of the fused form (0: the three-pass CTA form)
    int64_t chunk_points = 0;
    int64_t knn_qchunk = 0;
    int profile = 0;
    int64_t profile_mask = -1;  // stages bracketed while profiling (bit = mecuco_stage)
    long long wait_limit = 0;   // clock cycles of the tensor-core kernels' work waits (0: default)
    size_t ws_cap = 0;          // cap on the bytes of one device allocation of the context (0: none)
    // per-call bookkeeping
    int64_t launches = 0;
    int64_t knn_rows = 0;
    // profiler
    std::vector<EventPair> events;
    size_t events_used = 0;
    double stage_ms[MECUCO_STAGE_COUNT] = {};
    int64_t stage_n[MECUCO_STAGE_COUNT] = {};
};

namespace {

#define CK(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) { set_err(#call, e_); return MECUCO_ERR_CUDA; }   \
    } while (0)

mecuco_status flush_events(mecuco_t h) {
    if (h->events_used == 0) return MECUCO_OK;
    CK(cudaEventSynchronize(h->events[h->events_used - 1].b));
    for (size_t i = 0; i < h->events_used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->events[i].a, h->events[i].b));
        h->stage_ms[h->events[i].stage] += ms;
        h->stage_n[h->events[i].stage] += 1;
    }
    h->events_used = 0;
    return MECUCO_OK;
}

mecuco_status prof_begin(mecuco_t h, int stage, cudaStream_t s, EventPair **out) {
    *out = nullptr;
    if (!h->profile || !((h->profile_mask >> stage) & 1)) return MECUCO_OK;
    if (h->events_used >= 4096) {
        mecuco_status st = flush_events(h);
        if (st != MECUCO_OK) return st;
    }
    if (h->events_used == h->events.size()) {
        EventPair ep{};
        CK(cudaEventCreate(&ep.a));
        CK(cudaEventCreate(&ep.b));
        h->events.push_back(ep);
    }
    EventPair *ep = &h->events[h->events_used++];
    ep->stage = stage;
    CK(cudaEventRecord(ep->a, s));
    *out = ep;
    return MECUCO_OK;
}

// Launch `call` (a launcher returning cudaError_t) as stage `stage` on stream s.
#define LAUNCH(h, stage, s, call)                                                \
    do {                                                                         \
        EventPair *ep_ = nullptr;                                                \
        mecuco_status ps_ = prof_begin((h), (stage), (s), &ep_);                 \
        if (ps_ != MECUCO_OK) return ps_;                                        \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) { set_err(#call, e_); return MECUCO_ERR_CUDA; }   \
        if (ep_) CK(cudaEventRecord(ep_->b, (s)));                               \
        ++(h)->launches;                                                         \
    } while (0)

// Grow a context-owned device buffer to `need` bytes.  A request above the
// context's allocation cap (MECUCO_OPT_WORKSPACE_LIMIT) fails with
// MECUCO_ERR_OOM before any allocation, as a failed cudaMalloc would.
mecuco_status ensure(char *&buf, size_t &cur, size_t need, size_t cap = 0) {
    if (need <= cur) return MECUCO_OK;
    if (cap && need > cap) {
        char msg[160];
        snprintf(msg, sizeof(msg), "workspace of %zu bytes exceeds the context's allocation limit of %zu bytes", need,
                 cap);
        set_error_text(msg);
        return MECUCO_ERR_OOM;
    }
    if (buf) {
        // earlier asynchronous work may still use the old buffer
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { set_err("cudaDeviceSynchronize", e); return MECUCO_ERR_CUDA; }
        cudaFree(buf);
        buf = nullptr;
        cur = 0;
    }
    size_t want = align_up(need + need / 8, 1 << 20);
    cudaError_t e = cudaMalloc(&buf, want);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        e = cudaMalloc(&buf, need);
        if (e != cudaSuccess) { (void)cudaGetLastError(); buf = nullptr; return MECUCO_ERR_OOM; }
        want = need;
    }
    cur = want;
    return MECUCO_OK;
}

mecuco_status check_common(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                           int k, int include_self) {
    if (!h || !X) return MECUCO_ERR_INVALID_ARG;
    if (dt != MECUCO_F32 && dt != MECUCO_BF16) return MECUCO_ERR_INVALID_ARG;
    if (N < 2 || N >= (int64_t)1 << 31 || m < 1 || ld < m) return MECUCO_ERR_INVALID_ARG;
    if (k < 2 || k > 64) return MECUCO_ERR_INVALID_ARG;
    if (include_self != 0 && include_self != 1) return MECUCO_ERR_INVALID_ARG;
    if ((int64_t)k > N - (include_self ? 0 : 1)) return MECUCO_ERR_INVALID_ARG;
    return MECUCO_OK;
}

mecuco_status check_range(int64_t N, int64_t rb, int64_t re) {
    if (rb < 0 || re > N || rb >= re) return MECUCO_ERR_INVALID_ARG;
    return MECUCO_OK;
}

int candidate_capacity(mecuco_t h, int k) {
    int64_t kc = k + h->knn_margin;
    kc = (kc + 31) / 32 * 32;
    if (kc > 128) kc = 128;
    if (kc < k) kc = k;
    return (int)kc;
}

constexpr int64_t KNN_PAIR_MIN_N = 200000;

struct KnnPlan {
    int kc, nsplit;
    int lists;      // candidate lists per query row (splits x the tensor-core kernel's column halves)
    int kcl;        // capacity of each list
    int64_t qchunk;
    bool tc;        // candidate search on the tensor cores (BF16 operands)
    bool pair;      // tensor-core search as CTA pairs sharing two-SM MMAs
    bool bf16_copy; // the tensor-core path needs a BF16 copy of X
    int quant;      // KNN_QUANT_*: how the search sees FP32 rows (the certification bounds it)
    int64_t ldb;    // leading dimension of the BF16 operand(s)
    int64_t mk;     // their K (m, or 3 ms for the three-term split)
};

// Segment width of the three-term split: m rounded up to whole 16-byte units.
inline int64_t split_segment(int64_t m) { return (m + 7) / 8 * 8; }

KnnPlan plan_knn(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int64_t nrows, int k,
                 mecuco_precision prec) {
    KnnPlan p;
    p.kc = candidate_capacity(h, k);
    p.tc = prec == MECUCO_PREC_BF16_MIXED;
    // CTA pairs (256 x 256 two-SM MMAs, half the candidate bytes per SM) pay
    // from a few hundred thousand candidates up: measured at m = 4096, k = 64,
    // 1M points 7.53 s against 7.93 s per search, 300k 0.683 against 0.716 s,
    // but 100k 88.5 against 85.4 ms
    p.pair = p.tc && (h->knn_pair > 0 || (h->knn_pair < 0 && N >= KNN_PAIR_MIN_N));
    const bool direct = dt == MECUCO_BF16 && ld % 8 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    p.bf16_copy = p.tc && !direct;
    // FP32 rows: the three-term split (a search three times as long in K whose
    // rounding bound is ~2^8 smaller, so that the certificate holds where a
    // single rounding's would send most rows to the exact scan), unless
    // MECUCO_OPT_KNN_SPLIT_BF16 = 0
    p.quant = !(p.tc && dt == MECUCO_F32) ? KNN_QUANT_NONE : (h->knn_split_bf16 ? KNN_QUANT_SPLIT : KNN_QUANT_SINGLE);
    p.mk = p.quant == KNN_QUANT_SPLIT ? 3 * split_segment(m) : m;
    p.ldb = direct ? ld : (p.mk + 7) / 8 * 8;
    p.qchunk = h->knn_qchunk > 0 ? h->knn_qchunk : (int64_t)1 << 18;
    if (p.tc && h->knn_qchunk <= 0) {
        // whole waves of the persistent search per launch: a multiple of the
        // query rows one wave of CTAs (pairs) covers, so that only the last
        // launch ends on a partial wave (1M points: 52 instead of 53 waves)
        const int64_t wave = p.pair ? (int64_t)(h->num_sms / 2) * 256 : (int64_t)h->num_sms * 128;
        if (p.qchunk > wave) p.qchunk = p.qchunk / wave * wave;
    }
    if (p.qchunk > nrows) p.qchunk = nrows;
    // keep every SM busy (tensor-core kernel: 1 CTA/SM; CUDA-core kernel: 2):
    // split the candidate range when there are few query blocks (the re-rank
    // then sees kc * nsplit candidates per row)
    const int64_t qblocks = (p.qchunk + 127) / 128;
    const int64_t want = (p.tc ? 1LL : 2LL) * h->num_sms;
    p.nsplit = 1;
    if (qblocks < want) p.nsplit = (int)std::min<int64_t>((want + qblocks - 1) / qblocks, 1024 / p.kc);
    // tensor-core search: each split leaves knn_tc_halves() lists per row, each of
    // capacity >= k (<= 64, the shared-memory budget next to three stages)
    const int halves = p.tc ? knn_tc_halves() : 1;
    p.kcl = p.tc ? std::min(p.kc, 64) : p.kc;
    const int cap = 1024 / (halves * p.kcl);
    if (p.nsplit > cap) p.nsplit = cap;
    if (h->knn_splits > 0) p.nsplit = std::min(h->knn_splits, cap);
    while (p.nsplit > 1 && (N + p.nsplit - 1) / p.nsplit < p.kc) --p.nsplit;
    p.lists = p.nsplit * halves;
    return p;
}

struct KnnBufs {
    float *norms, *cand_d;
    int32_t *cand_i, *flags;
    void *xb, *xb2;         // BF16 operand copies (query, and candidate for the split), else NULL
    float *resid, *maxima;  // BF16 rounding terms of FP32 rows (tensor-core search), else NULL
};

// Scratch of run_knn, carved after `start`.
void knn_scratch(Carver &c, const KnnPlan &p, int64_t N, KnnBufs *b) {
    b->norms = c.take<float>((size_t)N);
    b->cand_d = c.take<float>((size_t)p.qchunk * p.lists * p.kcl);
    b->cand_i = c.take<int32_t>((size_t)p.qchunk * p.lists * p.kcl);
    b->flags = c.take<int32_t>((size_t)p.qchunk);
    b->xb = p.bf16_copy ? (void *)c.take<uint16_t>((size_t)N * p.ldb) : nullptr;
    b->xb2 = p.quant == KNN_QUANT_SPLIT ? (void *)c.take<uint16_t>((size_t)N * p.ldb) : nullptr;
    b->resid = p.quant ? c.take<float>((size_t)2 * N) : nullptr;
    b->maxima = p.quant ? c.take<float>(3) : nullptr;
}

// kNN of query rows [rb, re) (outputs relative to rb); scratch at ws + start,
// the workspace already sized by the caller.
mecuco_status run_knn(mecuco_t h, char *ws, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int k,
                      int include_self, mecuco_precision prec, int64_t rb, int64_t re, int32_t *idx_out,
                      float *dist_out, cudaStream_t s, size_t start) {
    KnnPlan p = plan_knn(h, X, dt, N, m, ld, re - rb, k, prec);
    Carver c(ws, start);
    KnnBufs b;
    knn_scratch(c, p, N, &b);
    if (b.maxima) CK(cudaMemsetAsync(b.maxima, 0, 3 * sizeof(float), s));
    LAUNCH(h, MECUCO_STAGE_ROWNORM, s, launch_rownorm(X, dt, N, m, ld, b.norms, s, b.resid, b.maxima, p.quant));
    const void *Xa = X, *Xb = X;
    if (p.quant == KNN_QUANT_SPLIT) {
        CK(launch_to_bf16_split(static_cast<const float *>(X), N, m, ld, b.xb, b.xb2, split_segment(m), p.ldb, s));
        ++h->launches;
        Xa = b.xb;
        Xb = b.xb2;
    } else if (p.bf16_copy) {
        CK(launch_to_bf16(X, dt, N, m, ld, b.xb, p.ldb, s));
        ++h->launches;
        Xa = Xb = b.xb;
    }
    for (int64_t q0 = rb; q0 < re; q0 += p.qchunk) {
        int64_t nq = std::min(p.qchunk, re - q0);
        int32_t *io = idx_out + (q0 - rb) * k;
        float *dout = dist_out ? dist_out + (q0 - rb) * k : nullptr;
        if (p.tc) {
            LAUNCH(h, MECUCO_STAGE_KNN_SEARCH, s,
                   launch_knn_tc(Xa, Xb, N, p.mk, p.ldb, b.norms, q0, nq, p.kcl, p.nsplit, include_self, b.cand_d,
                                 b.cand_i, p.pair ? 1 : 0, h->wait_limit, h->ctr, s));
        } else {
            LAUNCH(h, MECUCO_STAGE_KNN_SEARCH, s,
                   launch_knn_simt(X, dt, N, m, ld, b.norms, q0, nq, p.kc, p.nsplit, include_self, b.cand_d,
                                   b.cand_i, s));
        }
        // every row's lists go to the exact re-rank together: a point that a list
        // rejected has d~ >= that list's maximum, so the smallest list maximum
        // bounds every candidate left out
        LAUNCH(h, MECUCO_STAGE_KNN_RERANK, s,
               launch_knn_rerank(X, dt, N, m, ld, b.norms, q0, nq, p.kcl, p.lists, k, b.cand_d, b.cand_i, io, dout,
                                 b.flags, h->ctr, s, b.resid, b.maxima, p.quant));
        LAUNCH(h, MECUCO_STAGE_KNN_FALLBACK, s,
               launch_knn_fallback(X, dt, N, m, ld, q0, nq, k, include_self, b.flags, io, dout, h->ctr, s));
    }
    h->knn_rows += re - rb;
    return MECUCO_OK;
}

size_t knn_bytes(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int64_t nrows, int k,
                 mecuco_precision prec, size_t start) {
    KnnPlan p = plan_knn(h, X, dt, N, m, ld, nrows, k, prec);
    Carver c(nullptr, start);
    KnnBufs b;
    knn_scratch(c, p, N, &b);
    return c.off;
}

mecuco_status begin_call(mecuco_t h, cudaStream_t s) {
    h->launches = 0;
    h->knn_rows = 0;
    CK(cudaSetDevice(h->device));
    CK(cudaMemsetAsync(h->ctr, 0, offsetof(DevCounters, status), s));
    return MECUCO_OK;
}

// Device tables built once per k and kept for the context's lifetime (the
// first use of a k copies synchronously; later calls, and stream capture, do not).
mecuco_status upload_table(int32_t **slot, const std::vector<int32_t> &host) {
    int32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(int32_t) * std::max<size_t>(host.size(), 1)) != cudaSuccess) {
        (void)cudaGetLastError();
        return MECUCO_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(d, host.data(), sizeof(int32_t) * host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); set_err("cudaMemcpy", e); return MECUCO_ERR_CUDA; }
    *slot = d;
    return MECUCO_OK;
}

mecuco_status ensure_pairs(mecuco_t h, int k) {
    if (h->rowtab[k]) return MECUCO_OK;
    std::vector<int32_t> host((size_t)moments_tc_rows(k));
    moments_tc_build_rows(k, host.data());
    return upload_table(&h->rowtab[k], host);
}

// Table of the BF16-mixed estimator in the rotated basis: the third-moment
// pass's pair rows.
mecuco_status ensure_rotated(mecuco_t h, int k) {
    mecuco_status st;
    if (!h->tttab[k]) {
        std::vector<int32_t> host((size_t)tthird_rows(k));
        tthird_build_rows(k, host.data());
        if ((st = upload_table(&h->tttab[k], host)) != MECUCO_OK) return st;
    }
    return MECUCO_OK;
}

mecuco_status ensure_items(mecuco_t h, int k) {
    if (h->m3_items[k]) return MECUCO_OK;
    std::vector<int32_t> host((size_t)mecuco::m3_items(k));
    m3_build_items(k, host.data());
    return upload_table(&h->m3_items[k], host);
}

// Leading dimension (BF16 elements) of the rotated patch Y: m rounded up to
// whole 64-column chunks.
inline int64_t rot_ld(int64_t m) { return (m + 63) / 64 * 64; }

struct EstBufs {
    float *G, *R, *Q, *M, *sig, *U, *U0;
    uint16_t *Y;  // rotated patches (BF16-mixed form): 64 rows of rot_ld(m) per point
    float *rQ, *rB, *rsig, *rV;  // randomised SVD: range basis, projected Gram and its eigenpairs
};
// ym > 0: the rotated-basis estimator (BF16-mixed form) with Y for ambient
// dimension ym in place of the third moments M.
void est_scratch(Carver &c, int64_t chunk, int k, EstBufs *b, int rsvd_cols = 0, int64_t ym = 0) {
    b->G = c.take<float>((size_t)chunk * k * k);
    b->R = c.take<float>((size_t)chunk * k);
    b->Q = c.take<float>((size_t)chunk * k * k);
    b->M = ym ? nullptr : c.take<float>((size_t)chunk * m3_pair_floats(k));
    b->Y = ym ? c.take<uint16_t>((size_t)chunk * 64 * rot_ld(ym)) : nullptr;
    b->sig = c.take<float>((size_t)chunk * k);
    b->U = c.take<float>((size_t)chunk * k * k);
    b->U0 = c.take<float>((size_t)chunk * k * k);
    const int l = rsvd_cols;
    b->rQ = l ? c.take<float>((size_t)chunk * k * l) : nullptr;
    b->rB = l ? c.take<float>((size_t)chunk * l * l) : nullptr;
    b->rsig = l ? c.take<float>((size_t)chunk * l) : nullptr;
    b->rV = l ? c.take<float>((size_t)chunk * l * l) : nullptr;
}

// Points per estimator chunk: an 8 GB scratch budget (shared by the lanes of a
// batched call) - larger chunks leave smaller partial last waves: at k = 64,
// 14k-point chunks took the per-chunk kernels 2.6% less time than 3.6k ones.
int64_t est_chunk(mecuco_t h, int64_t nrows, int k, int64_t ym = 0) {
    const int64_t per_point = (ym ? 32 * rot_ld(ym) : m3_pair_floats(k)) + 4LL * k * k + 3LL * k;
    int64_t chunk = h->chunk_points;
    if (chunk <= 0) {
        const size_t budget = ((size_t)8 << 30) / (size_t)std::max(1, h->chunk_share);
        chunk = (int64_t)(budget / (per_point * sizeof(float)));
        chunk = std::max<int64_t>(256, std::min<int64_t>(chunk, 65536));
    }
    return std::min(chunk, nrows);
}

// Workspace bytes of run_curvature for nrows query rows (idx given, or
// computed into the front of the workspace).
// The BF16-mixed form runs the rotated-basis estimator (Gram pass, eigensolve,
// rotation, third-moment pass) unless a randomised SVD replaces the eigensolve.
inline int64_t rotated_m(mecuco_t h, int64_t m, mecuco_precision prec) {
    return (prec == MECUCO_PREC_BF16_MIXED && !h->rsvd.cols) ? m : 0;
}

size_t curvature_bytes(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int k,
                       bool idx_given, int64_t nrows, mecuco_precision prec) {
    const int64_t ym = rotated_m(h, m, prec);
    const int64_t chunk = est_chunk(h, nrows, k, ym);
    const size_t idx_bytes = idx_given ? 0 : align_up((size_t)nrows * k * sizeof(int32_t), 256);
    size_t need = idx_given ? 0 : knn_bytes(h, X, dt, N, m, ld, nrows, k, prec, idx_bytes);
    Carver c(nullptr, idx_bytes);
    EstBufs b;
    est_scratch(c, chunk, k, &b, h->rsvd.cols, ym);
    return std::max(need, c.off);
}

// Curvature of query rows [rb, re): kNN (unless idx is given), then per chunk
// moments -> eigensolve -> estimator.  Scratch at ws, sized by the caller with
// curvature_bytes; the per-k tables must exist (ensure_items / ensure_pairs).
mecuco_status run_curvature(mecuco_t h, char *ws, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                            int k, const int32_t *idx, int include_self, mecuco_variant var, mecuco_precision prec,
                            int64_t rb, int64_t re, float *kappa_out, float *lambda_out, float *U_out,
                            float *s_out, cudaStream_t s) {
    mecuco_status st = MECUCO_OK;
    const bool tc_moments = prec == MECUCO_PREC_BF16_MIXED;
    const int64_t ym = rotated_m(h, m, prec);
    if (!h->m3_items[k] || (tc_moments && !h->rowtab[k]) || (ym && !h->tttab[k]))
        return MECUCO_ERR_INVALID_ARG;
    const int64_t nrows = re - rb;
    const int64_t chunk = est_chunk(h, nrows, k, ym);
    const size_t idx_bytes = idx ? 0 : align_up((size_t)nrows * k * sizeof(int32_t), 256);
    const int32_t *nbr = idx;
    if (!idx) {
        int32_t *idx_buf = reinterpret_cast<int32_t *>(ws);
        st = run_knn(h, ws, X, dt, N, m, ld, k, include_self, prec, rb, re, idx_buf, nullptr, s, idx_bytes);
        if (st != MECUCO_OK) return st;
        nbr = idx_buf;
    }
    Carver c(ws, idx_bytes);
    EstBufs b;
    est_scratch(c, chunk, k, &b, h->rsvd.cols, ym);
    const int fp64 = h->jacobi_fp64 >= 0 ? h->jacobi_fp64 : (prec == MECUCO_PREC_BF16_MIXED ? 1 : 0);
    const float *Qarg = var == MECUCO_FAST_HAAR ? b.Q : nullptr;
    for (int64_t p0 = 0; p0 < nrows; p0 += chunk) {
        const int64_t np = std::min(chunk, nrows - p0);
        const int32_t *nb = nbr + p0 * k;
        if (h->rsvd.cols) {
            // randomised low-rank SVD: moments of X_c (unrotated), the range finder
            // on its Gram, the projected Gram's eigenpairs, U = Q V_B (rank r)
            float *Ud = U_out ? U_out + p0 * (int64_t)k * k : b.U;
            const int l = h->rsvd.cols;
            if (tc_moments) {
                LAUNCH(h, MECUCO_STAGE_MOMENTS, s,
                       launch_moments_tc(X, dt, N, m, ld, nb, k, np, h->rowtab[k], b.M, b.G, b.R,
                                         var == MECUCO_FAST_HAAR ? b.Q : nullptr, h->tc_slots, h->wait_limit,
                                         h->ctr, s));
            } else {
                LAUNCH(h, MECUCO_STAGE_GRAM, s,
                       launch_patch_gram(X, dt, N, m, ld, nb, k, 0, np, nullptr, b.G, b.R,
                                         var == MECUCO_FAST_HAAR ? b.Q : nullptr, h->ctr, s));
                LAUNCH(h, MECUCO_STAGE_MOMENTS, s,
                       launch_patch_m3(X, dt, N, m, ld, nb, k, 0, np, nullptr, b.M, h->m3_items[k], h->ctr, s));
            }
            LAUNCH(h, MECUCO_STAGE_JACOBI, s,
                   launch_rsvd_range(b.G, k, np, h->rsvd.omega, l, h->rsvd.power, b.rQ, b.rB, s));
            LAUNCH(h, MECUCO_STAGE_JACOBI, s,
                   launch_jacobi(b.rB, l, np, 1, h->jacobi_max_sweeps, b.rsig, b.rV, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
            ++h->launches;
            LAUNCH(h, MECUCO_STAGE_JACOBI, s,
                   launch_rsvd_compose(b.rQ, b.rsig, b.rV, k, l, h->rsvd.rank, np, b.sig, Ud, s));
            LAUNCH(h, MECUCO_STAGE_ESTIMATOR, s,
                   launch_estimator(b.sig, Ud, b.M, b.R, Qarg, k, m, np, (int)var, rank_eps_gram32(m), kappa_out + p0,
                                    lambda_out ? lambda_out + p0 * k : nullptr, s_out ? s_out + p0 * k : nullptr,
                                    h->ctr, s, b.G));
        } else if (tc_moments) {
            // BF16-mixed, in the rotated basis: G, R (Q) of X_c on the tensor cores,
            // the eigenpairs of G, the rotated patch Y = U^T X_c, then every term of
            // the estimator from the third moments of Y (no M is stored)
            float *Ud = U_out ? U_out + p0 * (int64_t)k * k : b.U;
            PatchSeg sg{};
            sg.X = X;
            sg.N = N;
            sg.m = m;
            sg.ld = ld;
            sg.k = k;
            sg.idx = nb;
            sg.rowtab = h->tttab[k];
            sg.G = b.G;
            sg.R = b.R;
            sg.Q = b.Q;
            sg.sig = b.sig;
            sg.U = Ud;
            sg.kappa = kappa_out + p0;
            sg.lambda = lambda_out ? lambda_out + p0 * k : nullptr;
            sg.s = s_out ? s_out + p0 * k : nullptr;
            const int haar = var == MECUCO_FAST_HAAR ? 1 : 0;
            LAUNCH(h, MECUCO_STAGE_GRAM, s, launch_gram_tc(dt, sg, nullptr, 0, np, haar, h->wait_limit, h->ctr, s));
            LAUNCH(h, MECUCO_STAGE_JACOBI, s,
                   launch_jacobi_seg(sg, nullptr, 0, k, np, fp64, h->jacobi_max_sweeps, h->ctr, s, kJacobiPreLoose,
                                 h->jacobi_warp));
            if (fp64 == 1 || fp64 == 3) ++h->launches;  // the refinement is a second kernel
            LAUNCH(h, MECUCO_STAGE_ROTATE, s,
                   launch_rotate_tc(dt, sg, nullptr, 0, np, b.Y, rot_ld(m), h->wait_limit, h->ctr, s));
            LAUNCH(h, MECUCO_STAGE_MOMENTS, s,
                   launch_tthird_tc(sg, nullptr, 0, k, np, b.Y, rot_ld(m), (int)var, h->tt_slots, h->tt_ctas,
                                    h->wait_limit, h->ctr, s));
        } else {
            // plain FP32: moments of the rotated patch Z = U0^T X_c (U0 = refined
            // eigenvectors of the FP32 Gram; K is invariant under the rotation and the
            // nearly diagonal Gram of Z resolves small eigenvalues), then its eigenpairs
            LAUNCH(h, MECUCO_STAGE_GRAM, s,
                   launch_patch_gram(X, dt, N, m, ld, nb, k, 0, np, nullptr, b.G, b.R, nullptr, h->ctr, s));
            LAUNCH(h, MECUCO_STAGE_JACOBI, s, launch_jacobi(b.G, k, np, 1, h->jacobi_max_sweeps, b.sig, b.U0, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
            ++h->launches;
            LAUNCH(h, MECUCO_STAGE_GRAM, s,
                   launch_patch_gram(X, dt, N, m, ld, nb, k, 0, np, b.U0, b.G, b.R, var == MECUCO_FAST_HAAR ? b.Q : nullptr,
                                     h->ctr, s));
            LAUNCH(h, MECUCO_STAGE_MOMENTS, s,
                   launch_patch_m3(X, dt, N, m, ld, nb, k, 0, np, b.U0, b.M, h->m3_items[k], h->ctr, s));
            LAUNCH(h, MECUCO_STAGE_JACOBI, s,
                   launch_jacobi(b.G, k, np, fp64, h->jacobi_max_sweeps, b.sig, b.U, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
            if (fp64 == 1 || fp64 == 3) ++h->launches;
            LAUNCH(h, MECUCO_STAGE_ESTIMATOR, s,
                   launch_estimator(b.sig, b.U, b.M, b.R, Qarg, k, m, np, (int)var, rank_eps_rotated(k, m),
                                    kappa_out + p0, lambda_out ? lambda_out + p0 * k : nullptr,
                                    s_out ? s_out + p0 * k : nullptr, h->ctr, s));
            if (U_out) LAUNCH(h, MECUCO_STAGE_JACOBI, s,
                              launch_compose_rotation(b.U0, b.U, k, np, U_out + p0 * (int64_t)k * k, s));
        }
    }
    return MECUCO_OK;
}

// ---- batched entry point -----------------------------------------------------
mecuco_status check_set(const mecuco_dataset &d, int include_self) {
    if (!d.X || !d.kappa) return MECUCO_ERR_INVALID_ARG;
    if (d.N < 2 || d.N >= ((int64_t)1 << 31) || d.m < 1 || d.ld < d.m) return MECUCO_ERR_INVALID_ARG;
    if (d.k < 2 || d.k > 64 || (int64_t)d.k > d.N - (include_self ? 0 : 1)) return MECUCO_ERR_INVALID_ARG;
    return MECUCO_OK;
}

std::tuple<int, int64_t, int64_t, int64_t, int, int> batch_signature(const mecuco_dataset *sets, int nsets,
                                                                     mecuco_dtype dt, mecuco_precision prec) {
    int64_t sn = 0, sm = 0, sk = 0;
    for (int i = 0; i < nsets; ++i) { sn += sets[i].N; sm += sets[i].m; sk += sets[i].k; }
    return std::make_tuple(nsets, sn, sm, sk, (int)dt, (int)prec);
}

mecuco_status run_batched_lanes(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt,
                                int include_self, mecuco_variant var, mecuco_precision prec, cudaStream_t s,
                                int lanes);

// Batched calls keep 2 GB of chunk scratch per lane (a quarter of the
// single-call budget): lanes run concurrently, each with its own workspace.
mecuco_status run_batched(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt, int include_self,
                          mecuco_variant var, mecuco_precision prec, cudaStream_t s, int lanes) {
    struct Share {
        mecuco_t h;
        ~Share() { h->chunk_share = 1; }
    } guard{h};
    h->chunk_share = 4;
    return run_batched_lanes(h, sets, nsets, dt, include_self, var, prec, s, lanes);
}

mecuco_status run_batched_lanes(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt,
                                int include_self, mecuco_variant var, mecuco_precision prec, cudaStream_t s,
                                int lanes) {
    mecuco_status st;
    for (int i = 0; i < nsets; ++i) {
        if ((st = ensure_items(h, sets[i].k)) != MECUCO_OK) return st;
        if (prec == MECUCO_PREC_BF16_MIXED &&
            ((st = ensure_pairs(h, sets[i].k)) != MECUCO_OK || (st = ensure_rotated(h, sets[i].k)) != MECUCO_OK))
            return st;
    }
    lanes = std::max(1, std::min(lanes, std::min(nsets, 32)));
    // longest first onto the least-loaded lane (cost: kNN N^2 m + moments N k^2 m)
    std::vector<int> order(nsets);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(nsets);
    for (int i = 0; i < nsets; ++i) {
        const double N = (double)sets[i].N, m = (double)sets[i].m, k = (double)sets[i].k;
        cost[i] = N * N * m + N * k * k * m;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(lanes, 0.0);
    std::vector<int> lane_of(nsets);
    std::vector<size_t> lane_bytes(lanes, 0), set_idx_bytes(nsets);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost[i];
        lane_of[i] = l;
        const mecuco_dataset &d = sets[i];
        set_idx_bytes[i] = d.idx ? 0 : align_up((size_t)d.N * d.k * sizeof(int32_t), 256);
        const size_t need = set_idx_bytes[i] + std::max(knn_bytes(h, d.X, dt, d.N, d.m, d.ld, d.N, d.k, prec, 0),
                                                        curvature_bytes(h, d.X, dt, d.N, d.m, d.ld, d.k, true, d.N,
                                                                        prec));
        lane_bytes[l] = std::max(lane_bytes[l], align_up(need, 256));
    }
    std::vector<size_t> lane_off(lanes, 0);
    size_t total = 0;
    for (int l = 0; l < lanes; ++l) { lane_off[l] = total; total += lane_bytes[l]; }
    if ((st = ensure(h->bws, h->bws_bytes, total, h->ws_cap)) != MECUCO_OK) return st;
    for (int l = 0; l < lanes; ++l) {
        if (!h->lane_stream[l]) CK(cudaStreamCreateWithFlags(&h->lane_stream[l], cudaStreamNonBlocking));
        if (!h->lane_event[l]) CK(cudaEventCreateWithFlags(&h->lane_event[l], cudaEventDisableTiming));
    }
    if (!h->fork_event) CK(cudaEventCreateWithFlags(&h->fork_event, cudaEventDisableTiming));
    CK(cudaEventRecord(h->fork_event, s));
    for (int l = 0; l < lanes; ++l) CK(cudaStreamWaitEvent(h->lane_stream[l], h->fork_event, 0));
    for (int i : order) {
        const mecuco_dataset &d = sets[i];
        cudaStream_t ls = h->lane_stream[lane_of[i]];
        char *ws = h->bws + lane_off[lane_of[i]];
        int32_t *idx = d.idx ? d.idx : reinterpret_cast<int32_t *>(ws);
        const size_t ib = set_idx_bytes[i];
        if ((st = run_knn(h, ws + ib, d.X, dt, d.N, d.m, d.ld, d.k, include_self, prec, 0, d.N, idx, nullptr, ls, 0)) !=
            MECUCO_OK)
            return st;
        if ((st = run_curvature(h, ws + ib, d.X, dt, d.N, d.m, d.ld, d.k, idx, include_self, var, prec, 0, d.N,
                                d.kappa, nullptr, nullptr, nullptr, ls)) != MECUCO_OK)
            return st;
    }
    for (int l = 0; l < lanes; ++l) {
        CK(cudaEventRecord(h->lane_event[l], h->lane_stream[l]));
        CK(cudaStreamWaitEvent(s, h->lane_event[l], 0));
    }
    return MECUCO_OK;
}

// ---- batched entry point, one launch per stage (BF16-mixed) ----------------
// Every dataset's kNN work items come from one device table (KnnSet), every
// estimator launch covers the points of all datasets through a segment table
// (PatchSeg).  Datasets go in order of m, then k, then N, descending, so that
// the points of one estimator launch share the leading dimension of their
// rotated patches with little padding, and its per-patch shared memory (sized
// for the launch's largest k) fits most of its patches closely.
constexpr size_t BATCH_EST_BUDGET = (size_t)8 << 30;  // bytes of estimator chunk scratch
constexpr int BATCH_TABLES_KEPT = 64;

struct BatchChunk {
    int64_t np;    // points (blocks) of the launches
    int seg0, nseg;
    int kmax;
    int64_t ldy;   // leading dimension of the rotated patches (BF16 elements)
    uint16_t *Y;
};

struct BatchPlan {
    std::vector<int> order;       // table position -> dataset
    std::vector<KnnSet> knn;      // table order (neighbour-list pointers left out)
    std::vector<BatchChunk> chunks;
    std::vector<PatchSeg> segs;   // output pointers left out
    std::vector<SegRef> refs;     // dataset and first point of each segment
    std::vector<BatchOut> outs;   // this call's outputs, table order
    int64_t nrows = 0, nitems = 0;
    int kcmax = 0, lmax = 0, kmax = 0;
    bool any_copy = false;
    float *maxima = nullptr;      // 2 per dataset (FP32 rows), zeroed before the row norms
    size_t bytes = 0;             // workspace bytes
};

// Estimator scratch floats per point at leading dimension ldy and k.
inline int64_t batch_point_floats(int64_t ldy, int k) { return 32 * ldy + 4LL * k * k + 3LL * k; }

// Lay the batch out in the workspace at `base` (nullptr: sizes only).  The
// neighbour lists of datasets without idx come first; the kNN scratch and the
// estimator chunk scratch share what follows (the kNN stage is done before the
// first estimator launch on the same stream).
mecuco_status plan_batch(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt, int include_self,
                         int pair, char *base, BatchPlan &p) {
    p = BatchPlan();
    p.order.resize(nsets);
    std::iota(p.order.begin(), p.order.end(), 0);
    std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) {
        if (sets[a].m != sets[b].m) return sets[a].m > sets[b].m;
        if (sets[a].k != sets[b].k) return sets[a].k > sets[b].k;
        return sets[a].N > sets[b].N;
    });
    Carver c(base, 0);
    const int halves = knn_tc_halves();
    const int qrows = knn_tc_item_rows(pair);
    p.knn.resize(nsets);
    p.outs.resize(nsets);
    for (int t = 0; t < nsets; ++t) {
        const mecuco_dataset &d = sets[p.order[t]];
        p.outs[t].kappa = d.kappa;
        p.outs[t].idx = d.idx ? d.idx : c.take<int32_t>((size_t)d.N * d.k);
    }
    const size_t after_idx = c.off;
    for (int t = 0; t < nsets; ++t) {
        const mecuco_dataset &d = sets[p.order[t]];
        KnnSet &e = p.knn[t];
        memset(&e, 0, sizeof(e));
        e.X = d.X;
        e.N = d.N;
        e.m = d.m;
        e.ld = d.ld;
        e.k = d.k;
        e.include_self = include_self;
        e.kc = candidate_capacity(h, d.k);
        e.kcl = std::min(e.kc, 64);
        // one candidate split: the batch's query blocks fill the GPU.  (Two
        // splits for k > 32, where a list holds 64 < kc = 96, left 0.6% instead
        // of 1% of the 256-dataset batch's rows uncertified, but the larger
        // search and re-rank cost 205 ms more than the exact scans saved.)
        const int cap = 1024 / (halves * e.kcl);
        e.nsplit = h->knn_splits > 0 ? std::min(h->knn_splits, cap) : 1;
        while (e.nsplit > 1 && (d.N + e.nsplit - 1) / e.nsplit < e.kc) --e.nsplit;
        e.lists = e.nsplit * halves;
        const bool direct = dt == MECUCO_BF16 && d.ld % 8 == 0 && (reinterpret_cast<uintptr_t>(d.X) & 15) == 0;
        e.quant = dt != MECUCO_F32 ? KNN_QUANT_NONE : (h->knn_split_bf16 ? KNN_QUANT_SPLIT : KNN_QUANT_SINGLE);
        e.mk = e.quant == KNN_QUANT_SPLIT ? 3 * split_segment(d.m) : d.m;
        e.ldb = direct ? d.ld : (e.mk + 7) / 8 * 8;
        e.norms = c.take<float>((size_t)d.N);
        e.cand_d = c.take<float>((size_t)d.N * e.lists * e.kcl);
        e.cand_i = c.take<int32_t>((size_t)d.N * e.lists * e.kcl);
        e.flags = c.take<int32_t>((size_t)d.N);
        e.xb = direct ? nullptr : (void *)c.take<uint16_t>((size_t)d.N * e.ldb);
        e.xb2 = e.quant == KNN_QUANT_SPLIT ? (void *)c.take<uint16_t>((size_t)d.N * e.ldb) : nullptr;
        e.resid = e.quant ? c.take<float>((size_t)2 * d.N) : nullptr;
        e.item_begin = p.nitems;
        e.row_begin = p.nrows;
        p.nitems += (d.N + qrows - 1) / qrows * e.nsplit;
        p.nrows += d.N;
        p.kcmax = std::max(p.kcmax, e.kcl);
        p.lmax = std::max(p.lmax, e.kcl * e.lists);
        p.kmax = std::max(p.kmax, d.k);
        p.any_copy = p.any_copy || !direct;
    }
    // the datasets' rounding maxima, contiguous (one memset per call)
    p.maxima = dt == MECUCO_F32 ? c.take<float>((size_t)3 * nsets) : nullptr;
    for (int t = 0; t < nsets && p.maxima; ++t) p.knn[t].maxima = p.maxima + 3 * t;
    if (base) {
        for (int t = 0; t < nsets; ++t) {
            if (!knn_tc_make_maps(&p.knn[t], pair)) {
                set_error_text("batched kNN: a dataset's operand cannot be described by a tensor map");
                return MECUCO_ERR_INVALID_ARG;
            }
        }
    }
    const size_t knn_end = c.off;
    // estimator chunks: greedy over the points in table order
    const int64_t pt_cap = h->chunk_points > 0 ? h->chunk_points : ((int64_t)1 << 24);
    size_t est_end = after_idx;
    BatchChunk cur{0, 0, 0, 0, 0, nullptr};
    auto close = [&]() {
        if (cur.np == 0) return;
        Carver e(base, after_idx);
        EstBufs b;
        est_scratch(e, cur.np, cur.kmax, &b, 0, cur.ldy);
        est_end = std::max(est_end, e.off);
        cur.Y = b.Y;
        for (int i = cur.seg0; i < cur.seg0 + cur.nseg; ++i) {
            PatchSeg &g = p.segs[i];
            const size_t f = (size_t)g.first;
            const size_t kk = (size_t)cur.kmax;
            g.G = b.G + f * kk * kk;
            g.R = b.R + f * kk;
            g.Q = b.Q + f * kk * kk;
            g.sig = b.sig + f * kk;
            g.U = b.U + f * kk * kk;
        }
        p.chunks.push_back(cur);
        cur = BatchChunk{0, (int)p.segs.size(), 0, 0, 0, nullptr};
    };
    for (int t = 0; t < nsets; ++t) {
        const mecuco_dataset &d = sets[p.order[t]];
        int64_t a = 0;
        while (a < d.N) {
            const int64_t ldy = cur.np ? cur.ldy : rot_ld(d.m);
            const int kc = std::max(cur.kmax, d.k);
            int64_t cap = (int64_t)(BATCH_EST_BUDGET / (sizeof(float) * (size_t)batch_point_floats(ldy, kc)));
            cap = std::max<int64_t>(1, std::min(cap, pt_cap));
            if (cur.np >= cap) { close(); continue; }
            const int64_t take = std::min(d.N - a, cap - cur.np);
            PatchSeg g{};
            g.X = d.X;
            g.N = d.N;
            g.m = d.m;
            g.ld = d.ld;
            g.k = d.k;
            g.first = (int)cur.np;
            g.rowtab = h->tttab[d.k];
            p.segs.push_back(g);
            p.refs.push_back(SegRef{t, 0, a});
            cur.ldy = ldy;
            cur.kmax = kc;
            cur.np += take;
            ++cur.nseg;
            a += take;
        }
    }
    close();
    p.bytes = std::max(knn_end, est_end);
    return MECUCO_OK;
}

// The device copy of the plan's tables (KnnSet entries, the segments, their
// references), reused when an earlier call built the same bytes: inputs,
// workspace and sizes, not the outputs, which launch_batch_patch writes in
// every call.
mecuco_status batch_tables(mecuco_t h, const BatchPlan &p, cudaStream_t s, KnnSet **knn_dev, PatchSeg **seg_dev,
                           SegRef **ref_dev) {
    const size_t kb = align_up(sizeof(KnnSet) * p.knn.size(), 256);
    const size_t sb = align_up(sizeof(PatchSeg) * p.segs.size(), 256);
    std::vector<char> blob(kb + sb + sizeof(SegRef) * p.refs.size(), 0);
    memcpy(blob.data(), p.knn.data(), sizeof(KnnSet) * p.knn.size());
    memcpy(blob.data() + kb, p.segs.data(), sizeof(PatchSeg) * p.segs.size());
    memcpy(blob.data() + kb + sb, p.refs.data(), sizeof(SegRef) * p.refs.size());
    char *dev = nullptr;
    for (size_t i = 0; i < h->btabs.size(); ++i) {
        if (h->btabs[i].host == blob) {
            dev = h->btabs[i].dev;
            break;
        }
    }
    if (!dev) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            set_error_text("batched call under stream capture needs a new device table: make one uncaptured call "
                           "with the same datasets first");
            return MECUCO_ERR_INVALID_ARG;
        }
        if ((int)h->btabs.size() >= BATCH_TABLES_KEPT) {
            CK(cudaDeviceSynchronize());
            cudaFree(h->btabs.front().dev);
            h->btabs.erase(h->btabs.begin());
        }
        if (cudaMalloc(&dev, blob.size()) != cudaSuccess) {
            (void)cudaGetLastError();
            return MECUCO_ERR_OOM;
        }
        cudaError_t e = cudaMemcpy(dev, blob.data(), blob.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(dev); set_err("cudaMemcpy", e); return MECUCO_ERR_CUDA; }
        h->btabs.push_back({std::move(blob), dev});
    }
    *knn_dev = reinterpret_cast<KnnSet *>(dev);
    *seg_dev = reinterpret_cast<PatchSeg *>(dev + kb);
    *ref_dev = reinterpret_cast<SegRef *>(dev + kb + sb);
    return MECUCO_OK;
}

mecuco_status run_batched_persistent(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt,
                                     int include_self, mecuco_variant var, cudaStream_t s,
                                     const mecuco_batch_tuning &tn) {
    mecuco_status st;
    for (int i = 0; i < nsets; ++i)
        if ((st = ensure_rotated(h, sets[i].k)) != MECUCO_OK) return st;
    BatchPlan p;
    if ((st = plan_batch(h, sets, nsets, dt, include_self, tn.knn_pair, nullptr, p)) != MECUCO_OK) return st;
    if ((st = ensure(h->bws, h->bws_bytes, p.bytes, h->ws_cap)) != MECUCO_OK) return st;
    if ((st = plan_batch(h, sets, nsets, dt, include_self, tn.knn_pair, h->bws, p)) != MECUCO_OK) return st;
    KnnSet *kt = nullptr;
    PatchSeg *sg = nullptr;
    SegRef *refs = nullptr;
    if ((st = batch_tables(h, p, s, &kt, &sg, &refs)) != MECUCO_OK) return st;
    CK(launch_batch_patch(kt, nsets, sg, refs, (int)p.segs.size(), p.outs.data(), s));
    h->launches += (nsets + BATCH_PATCH_SETS - 1) / BATCH_PATCH_SETS;
    // kNN of every row of every dataset: one launch per stage
    if (p.maxima) CK(cudaMemsetAsync(p.maxima, 0, 3 * sizeof(float) * nsets, s));
    LAUNCH(h, MECUCO_STAGE_ROWNORM, s, launch_rownorm_batch(kt, nsets, p.nrows, dt, s));
    if (p.any_copy) {
        CK(launch_to_bf16_batch(kt, nsets, p.nrows, dt, s));
        ++h->launches;
    }
    LAUNCH(h, MECUCO_STAGE_KNN_SEARCH, s,
           launch_knn_tc_batch(kt, nsets, p.nitems, p.kcmax, tn.knn_pair, h->wait_limit, h->ctr, s));
    LAUNCH(h, MECUCO_STAGE_KNN_RERANK, s, launch_knn_rerank_batch(kt, nsets, p.nrows, p.lmax, dt, h->ctr, s));
    LAUNCH(h, MECUCO_STAGE_KNN_FALLBACK, s, launch_knn_fallback_batch(kt, nsets, p.nrows, p.kmax, dt, h->ctr, s));
    h->knn_rows += p.nrows;
    // estimator over the points of all datasets, chunk by chunk
    const int fp64 = h->jacobi_fp64 >= 0 ? h->jacobi_fp64 : 1;
    const int haar = var == MECUCO_FAST_HAAR ? 1 : 0;
    PatchSeg none{};
    for (const BatchChunk &ch : p.chunks) {
        const PatchSeg *tab = sg + ch.seg0;
        LAUNCH(h, MECUCO_STAGE_GRAM, s, launch_gram_tc(dt, none, tab, ch.nseg, ch.np, haar, h->wait_limit, h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_JACOBI, s,
               launch_jacobi_seg(none, tab, ch.nseg, ch.kmax, ch.np, fp64, h->jacobi_max_sweeps, h->ctr, s,
                                 kJacobiPreLoose, h->jacobi_warp));
        if (fp64 == 1 || fp64 == 3) ++h->launches;
        LAUNCH(h, MECUCO_STAGE_ROTATE, s,
               launch_rotate_tc(dt, none, tab, ch.nseg, ch.np, ch.Y, ch.ldy, h->wait_limit, h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_MOMENTS, s,
               launch_tthird_tc(none, tab, ch.nseg, ch.kmax, ch.np, ch.Y, ch.ldy, (int)var, tn.tt_slots, tn.tt_ctas,
                                h->wait_limit, h->ctr, s));
    }
    return MECUCO_OK;
}

// The configuration a batched call runs with: the tuned one for its
// signature, else the context's options.
mecuco_batch_tuning batch_config(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt,
                                 mecuco_precision prec) {
    auto it = h->tuned.find(batch_signature(sets, nsets, dt, prec));
    if (it != h->tuned.end()) return it->second;
    mecuco_batch_tuning t{};
    t.lanes = h->batch_lanes;
    int64_t maxn = 0;
    for (int i = 0; i < nsets; ++i) maxn = std::max(maxn, sets[i].N);
    t.knn_pair = h->knn_pair > 0 || (h->knn_pair < 0 && maxn >= KNN_PAIR_MIN_N) ? 1 : 0;
    t.tt_ctas = h->tt_ctas;
    t.tt_slots = h->tt_slots;
    return t;
}

bool batch_is_persistent(mecuco_t h, mecuco_precision prec) {
    return prec == MECUCO_PREC_BF16_MIXED && h->batch_persistent;
}

mecuco_status run_batch_call(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt, int include_self,
                             mecuco_variant var, mecuco_precision prec, cudaStream_t s,
                             const mecuco_batch_tuning &tn) {
    if (batch_is_persistent(h, prec)) return run_batched_persistent(h, sets, nsets, dt, include_self, var, s, tn);
    return run_batched(h, sets, nsets, dt, include_self, var, prec, s, tn.lanes);
}

mecuco_status check_batch(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt, int include_self,
                          mecuco_variant var, mecuco_precision prec) {
    if (!h || !sets || nsets < 1) return MECUCO_ERR_INVALID_ARG;
    if (dt != MECUCO_F32 && dt != MECUCO_BF16) return MECUCO_ERR_INVALID_ARG;
    if (include_self != 0 && include_self != 1) return MECUCO_ERR_INVALID_ARG;
    if (var != MECUCO_FAST_LITERAL && var != MECUCO_FAST_HAAR) return MECUCO_ERR_INVALID_ARG;
    if (prec != MECUCO_PREC_FP32 && prec != MECUCO_PREC_BF16_MIXED) return MECUCO_ERR_INVALID_ARG;
    for (int i = 0; i < nsets; ++i) {
        mecuco_status st = check_set(sets[i], include_self);
        if (st != MECUCO_OK) return st;
    }
    return MECUCO_OK;
}

}  // namespace

extern "C" {

const char *mecuco_status_string(mecuco_status st) {
    switch (st) {
        case MECUCO_OK: return "ok";
        case MECUCO_ERR_INVALID_ARG: return "invalid argument";
        case MECUCO_ERR_UNSUPPORTED: return "unsupported by this build";
        case MECUCO_ERR_OOM: return "out of memory";
        case MECUCO_ERR_CUDA: return "CUDA error";
        case MECUCO_ERR_NOT_CONVERGED: return "eigensolver hit its sweep cap";
        case MECUCO_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *mecuco_last_error_message(void) { return g_errmsg; }

mecuco_status mecuco_create(mecuco_t *out, int device) {
    if (!out) return MECUCO_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) { set_err("cudaGetDeviceCount", e); return MECUCO_ERR_CUDA; }
    if (device < 0 || device >= ndev) return MECUCO_ERR_INVALID_ARG;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3) return MECUCO_ERR_UNSUPPORTED;
    CK(cudaSetDevice(device));
    mecuco_ctx *h = new (std::nothrow) mecuco_ctx();
    if (!h) return MECUCO_ERR_OOM;
    h->device = device;
    h->num_sms = prop.multiProcessorCount;
    if (cudaMalloc(&h->ctr, sizeof(DevCounters)) != cudaSuccess) {
        (void)cudaGetLastError();
        delete h;
        return MECUCO_ERR_OOM;
    }
    if (cudaMemset(h->ctr, 0, sizeof(DevCounters)) != cudaSuccess) {
        cudaFree(h->ctr);
        delete h;
        return MECUCO_ERR_CUDA;
    }
    *out = h;
    return MECUCO_OK;
}

mecuco_status mecuco_destroy(mecuco_t h) {
    if (!h) return MECUCO_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &ep : h->events) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    if (h->ws) cudaFree(h->ws);
    if (h->io) cudaFree(h->io);
    if (h->ctr) cudaFree(h->ctr);
    for (int kk = 0; kk <= 64; ++kk) {
        if (h->m3_items[kk]) cudaFree(h->m3_items[kk]);
        if (h->rowtab[kk]) cudaFree(h->rowtab[kk]);
        if (h->tttab[kk]) cudaFree(h->tttab[kk]);
    }
    if (h->bws) cudaFree(h->bws);
    for (int i = 0; i < 32; ++i) {
        if (h->lane_stream[i]) cudaStreamDestroy(h->lane_stream[i]);
        if (h->lane_event[i]) cudaEventDestroy(h->lane_event[i]);
    }
    if (h->fork_event) cudaEventDestroy(h->fork_event);
    for (auto &bt : h->btabs) cudaFree(bt.dev);
    delete h;
    return MECUCO_OK;
}

mecuco_status mecuco_set_option(mecuco_t h, mecuco_option opt, int64_t v) {
    if (!h) return MECUCO_ERR_INVALID_ARG;
    switch (opt) {
        case MECUCO_OPT_KNN_MARGIN:
            if (v < 0 || v > 96) return MECUCO_ERR_INVALID_ARG;
            h->knn_margin = v;
            break;
        case MECUCO_OPT_JACOBI_FP64:
            if (v < -1 || v > 3) return MECUCO_ERR_INVALID_ARG;
            h->jacobi_fp64 = (int)v;
            break;
        case MECUCO_OPT_JACOBI_MAX_SWEEPS:
            if (v < 1 || v > 1000) return MECUCO_ERR_INVALID_ARG;
            h->jacobi_max_sweeps = (int)v;
            break;
        case MECUCO_OPT_CHUNK_POINTS:
            if (v < 0) return MECUCO_ERR_INVALID_ARG;
            h->chunk_points = v;
            break;
        case MECUCO_OPT_KNN_QUERY_CHUNK:
            if (v < 0) return MECUCO_ERR_INVALID_ARG;
            h->knn_qchunk = v;
            break;
        case MECUCO_OPT_PROFILE:
            if (v < 0 || v > 1) return MECUCO_ERR_INVALID_ARG;
            h->profile = (int)v;
            break;
        case MECUCO_OPT_KNN_SPLITS:
            if (v < 0 || v > 64) return MECUCO_ERR_INVALID_ARG;
            h->knn_splits = (int)v;
            break;
        case MECUCO_OPT_TC_SLOTS:
            if (v < 2 || v > 8 || (v & 1)) return MECUCO_ERR_INVALID_ARG;
            h->tc_slots = (int)v;
            break;
        case MECUCO_OPT_KNN_PAIR:
            if (v < -1 || v > 1) return MECUCO_ERR_INVALID_ARG;
            h->knn_pair = (int)v;
            break;
        case MECUCO_OPT_PROFILE_STAGES:
            if (v < 0 || v >= ((int64_t)1 << MECUCO_STAGE_COUNT)) return MECUCO_ERR_INVALID_ARG;
            h->profile_mask = v == 0 ? -1 : v;
            break;
        case MECUCO_OPT_TT_SLOTS:
            if (v < 2 || v > 8 || (v & 1)) return MECUCO_ERR_INVALID_ARG;
            h->tt_slots = (int)v;
            break;
        case MECUCO_OPT_TT_CTAS:
            if (v < 1 || v > 2) return MECUCO_ERR_INVALID_ARG;
            h->tt_ctas = (int)v;
            break;
        case MECUCO_OPT_WAIT_LIMIT:
            if (v < 0) return MECUCO_ERR_INVALID_ARG;
            h->wait_limit = (long long)v;
            break;
        case MECUCO_OPT_WORKSPACE_LIMIT:
            if (v < 0) return MECUCO_ERR_INVALID_ARG;
            h->ws_cap = (size_t)v;
            break;
        case MECUCO_OPT_BATCH_LANES:
            if (v < 1 || v > 32) return MECUCO_ERR_INVALID_ARG;
            h->batch_lanes = (int)v;
            break;
        case MECUCO_OPT_JACOBI_WARP:
            if (v != 0 && v != 1 && v != 2 && v != 4) return MECUCO_ERR_INVALID_ARG;
            h->jacobi_warp = (int)v;
            break;
        case MECUCO_OPT_KNN_SPLIT_BF16:
            if (v != 0 && v != 1) return MECUCO_ERR_INVALID_ARG;
            h->knn_split_bf16 = (int)v;
            break;
        case MECUCO_OPT_BATCH_PERSISTENT:
            if (v != 0 && v != 1) return MECUCO_ERR_INVALID_ARG;
            h->batch_persistent = (int)v;
            break;
        default: return MECUCO_ERR_INVALID_ARG;
    }
    return MECUCO_OK;
}

mecuco_status mecuco_knn_range(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int k,
                               int include_self, mecuco_precision prec, int64_t rb, int64_t re, int32_t *idx_out,
                               float *dist_out, void *stream) {
    mecuco_status st = check_common(h, X, dt, N, m, ld, k, include_self);
    if (st != MECUCO_OK) return st;
    if ((st = check_range(N, rb, re)) != MECUCO_OK) return st;
    if (!idx_out) return MECUCO_ERR_INVALID_ARG;
    if (prec != MECUCO_PREC_FP32 && prec != MECUCO_PREC_BF16_MIXED) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    if ((st = ensure(h->ws, h->ws_bytes, knn_bytes(h, X, dt, N, m, ld, re - rb, k, prec, 0), h->ws_cap)) !=
        MECUCO_OK)
        return st;
    return run_knn(h, h->ws, X, dt, N, m, ld, k, include_self, prec, rb, re, idx_out, dist_out, s, 0);
}

mecuco_status mecuco_knn(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int k,
                         int include_self, mecuco_precision prec, int32_t *idx_out, float *dist_out, void *stream) {
    return mecuco_knn_range(h, X, dt, N, m, ld, k, include_self, prec, 0, N, idx_out, dist_out, stream);
}

mecuco_status mecuco_curvature_range(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                     int k, const int32_t *idx, int include_self, mecuco_variant var,
                                     mecuco_precision prec, int64_t rb, int64_t re, float *kappa_out,
                                     float *lambda_out, float *U_out, float *s_out, void *stream) {
    mecuco_status st = check_common(h, X, dt, N, m, ld, k, include_self);
    if (st != MECUCO_OK) return st;
    if ((st = check_range(N, rb, re)) != MECUCO_OK) return st;
    if (!kappa_out) return MECUCO_ERR_INVALID_ARG;
    if (var != MECUCO_FAST_LITERAL && var != MECUCO_FAST_HAAR) return MECUCO_ERR_INVALID_ARG;
    if (prec != MECUCO_PREC_FP32 && prec != MECUCO_PREC_BF16_MIXED) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    if ((st = ensure_items(h, k)) != MECUCO_OK) return st;
    if (prec == MECUCO_PREC_BF16_MIXED && ((st = ensure_pairs(h, k)) != MECUCO_OK ||
                                           (st = ensure_rotated(h, k)) != MECUCO_OK))
        return st;
    if ((st = ensure(h->ws, h->ws_bytes, curvature_bytes(h, X, dt, N, m, ld, k, idx != nullptr, re - rb, prec),
                     h->ws_cap)) != MECUCO_OK)
        return st;
    return run_curvature(h, h->ws, X, dt, N, m, ld, k, idx, include_self, var, prec, rb, re, kappa_out, lambda_out,
                         U_out, s_out, s);
}

mecuco_status mecuco_curvature(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, int k,
                               const int32_t *idx, int include_self, mecuco_variant var, mecuco_precision prec,
                               float *kappa_out, float *lambda_out, float *U_out, float *s_out, void *stream) {
    return mecuco_curvature_range(h, X, dt, N, m, ld, k, idx, include_self, var, prec, 0, N, kappa_out, lambda_out,
                                  U_out, s_out, stream);
}

mecuco_status mecuco_curvature_rsvd(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                    int k, const int32_t *idx, int include_self, mecuco_variant var,
                                    mecuco_precision prec, int rank, int sketch_cols, int power_iters,
                                    const float *omega, float *kappa_out, void *stream) {
    mecuco_status st = check_common(h, X, dt, N, m, ld, k, include_self);
    if (st != MECUCO_OK) return st;
    if (!kappa_out || !omega) return MECUCO_ERR_INVALID_ARG;
    if (var != MECUCO_FAST_LITERAL && var != MECUCO_FAST_HAAR) return MECUCO_ERR_INVALID_ARG;
    if (prec != MECUCO_PREC_FP32 && prec != MECUCO_PREC_BF16_MIXED) return MECUCO_ERR_INVALID_ARG;
    if (rank < 1 || rank > k - 1 || (int64_t)rank > m || sketch_cols < rank || sketch_cols > k || power_iters < 0 ||
        power_iters > 16)
        return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    if ((st = ensure_items(h, k)) != MECUCO_OK) return st;
    if (prec == MECUCO_PREC_BF16_MIXED && ((st = ensure_pairs(h, k)) != MECUCO_OK ||
                                           (st = ensure_rotated(h, k)) != MECUCO_OK))
        return st;
    h->rsvd.rank = rank;
    h->rsvd.cols = sketch_cols;
    h->rsvd.power = power_iters;
    h->rsvd.omega = omega;
    st = ensure(h->ws, h->ws_bytes, curvature_bytes(h, X, dt, N, m, ld, k, idx != nullptr, N, prec), h->ws_cap);
    if (st == MECUCO_OK)
        st = run_curvature(h, h->ws, X, dt, N, m, ld, k, idx, include_self, var, prec, 0, N, kappa_out, nullptr,
                           nullptr, nullptr, s);
    h->rsvd.rank = h->rsvd.cols = h->rsvd.power = 0;
    h->rsvd.omega = nullptr;
    return st;
}

mecuco_status mecuco_curvature_backward(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                        int k, const int32_t *idx, mecuco_variant var, const float *dkappa,
                                        float *dX_out, void *stream) {
    mecuco_status st = check_common(h, X, dt, N, m, ld, k, 1);  // idx is given: k <= N
    if (st != MECUCO_OK) return st;
    if (!idx || !dkappa || !dX_out) return MECUCO_ERR_INVALID_ARG;
    if (var != MECUCO_FAST_LITERAL && var != MECUCO_FAST_HAAR) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    if ((st = ensure_items(h, k)) != MECUCO_OK) return st;
    // per point: forward buffers (incl. U0) + dG, dR, dQ + C and dM (k^3 each)
    const int64_t per_point = m3_pair_floats(k) + 7LL * k * k + 4LL * k + 2LL * k * k * k;
    int64_t chunk = h->chunk_points > 0 ? h->chunk_points
                                         : std::max<int64_t>(256, std::min<int64_t>(65536, ((int64_t)2 << 30) /
                                                                                             (per_point * 4)));
    chunk = std::min(chunk, N);
    Carver t(nullptr);
    EstBufs b;
    est_scratch(t, chunk, k, &b);
    t.take<float>((size_t)chunk * k * k);
    t.take<float>((size_t)chunk * k);
    t.take<float>((size_t)chunk * k * k);
    t.take<float>((size_t)chunk * k * k * k);
    t.take<float>((size_t)chunk * k * k * k);
    if ((st = ensure(h->ws, h->ws_bytes, t.off, h->ws_cap)) != MECUCO_OK) return st;
    Carver c(h->ws);
    est_scratch(c, chunk, k, &b);
    float *U0 = b.U0;
    float *dG = c.take<float>((size_t)chunk * k * k);
    float *dR = c.take<float>((size_t)chunk * k);
    float *dQ = c.take<float>((size_t)chunk * k * k);
    float *Cb = c.take<float>((size_t)chunk * k * k * k);
    float *dM = c.take<float>((size_t)chunk * k * k * k);
    CK(cudaMemsetAsync(dX_out, 0, sizeof(float) * (size_t)N * m, s));
    const bool need_q = var == MECUCO_FAST_HAAR;
    const int rot_mode = h->jacobi_fp64 >= 0 ? h->jacobi_fp64 : 3;
    for (int64_t p0 = 0; p0 < N; p0 += chunk) {
        const int64_t np = std::min(chunk, N - p0);
        const int32_t *nb = idx + p0 * k;
        // U0: eigenvectors of the plain FP32 Gram, refined so that U0 is orthogonal to
        // FP32 rounding (a rotation that is not orthogonal acts as a perturbation of X_c,
        // which ill-conditioned patches amplify)
        LAUNCH(h, MECUCO_STAGE_GRAM, s,
               launch_patch_gram(X, dt, N, m, ld, nb, k, 0, np, nullptr, b.G, b.R, nullptr, h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_JACOBI, s, launch_jacobi(b.G, k, np, 1, h->jacobi_max_sweeps, b.sig, U0, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
        ++h->launches;  // the refinement kernel
        // moments of Z = U0^T X_c and the refined eigenpairs of its Gram
        LAUNCH(h, MECUCO_STAGE_GRAM, s,
               launch_patch_gram(X, dt, N, m, ld, nb, k, 0, np, U0, b.G, b.R, need_q ? b.Q : nullptr, h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_MOMENTS, s,
               launch_patch_m3(X, dt, N, m, ld, nb, k, 0, np, U0, b.M, h->m3_items[k], h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_JACOBI, s,
               launch_jacobi(b.G, k, np, rot_mode, h->jacobi_max_sweeps, b.sig, b.U, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
        if (rot_mode == 1 || rot_mode == 3) ++h->launches;  // the refinement kernel
        LAUNCH(h, MECUCO_STAGE_ADJOINT, s,
               launch_adjoint(X, dt, N, m, ld, nb, k, np, (int)var, rank_eps_rotated(k, m), U0, b.sig, b.U, b.M, b.R,
                              b.Q, dkappa + p0, dG, dR, dQ, Cb, dM, dX_out, m, s));
        ++h->launches;  // two kernels
    }
    return MECUCO_OK;
}

mecuco_status mecuco_tangent_basis(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                   int k, const int32_t *idx, int64_t rb, int64_t re, int d_out, float *V_out,
                                   void *stream) {
    mecuco_status st = check_common(h, X, dt, N, m, ld, k, 1);  // idx is given: k <= N
    if (st != MECUCO_OK) return st;
    if ((st = check_range(N, rb, re)) != MECUCO_OK) return st;
    if (!idx || !V_out || d_out < 1 || d_out > k - 1 || (int64_t)d_out > m) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    const int64_t chunk = std::min<int64_t>(h->chunk_points > 0 ? h->chunk_points : 65536, re - rb);
    Carver t(nullptr);
    t.take<float>((size_t)chunk * k * k);
    t.take<float>((size_t)chunk * k);
    t.take<float>((size_t)chunk * k);
    t.take<float>((size_t)chunk * k * k);
    if ((st = ensure(h->ws, h->ws_bytes, t.off, h->ws_cap)) != MECUCO_OK) return st;
    Carver c(h->ws);
    float *G = c.take<float>((size_t)chunk * k * k);
    float *R = c.take<float>((size_t)chunk * k);
    float *sig = c.take<float>((size_t)chunk * k);
    float *U = c.take<float>((size_t)chunk * k * k);
    const int mode = h->jacobi_fp64 >= 0 ? h->jacobi_fp64 : 0;
    for (int64_t p0 = rb; p0 < re; p0 += chunk) {
        const int64_t np = std::min(chunk, re - p0);
        const int32_t *nb = idx + p0 * k;
        LAUNCH(h, MECUCO_STAGE_GRAM, s,
               launch_patch_gram(X, dt, N, m, ld, nb, k, 0, np, nullptr, G, R, nullptr, h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_JACOBI, s, launch_jacobi(G, k, np, mode, h->jacobi_max_sweeps, sig, U, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
        if (mode == 1 || mode == 3) ++h->launches;
        LAUNCH(h, MECUCO_STAGE_BASIS, s,
               launch_tangent_basis(X, dt, N, m, ld, nb, k, np, sig, U, d_out, rank_eps_gram32(m),
                                    V_out + (p0 - rb) * m * (int64_t)d_out, h->ctr, s));
    }
    return MECUCO_OK;
}

mecuco_status mecuco_curvature_exact(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                     int k, const int32_t *idx, int include_self, mecuco_precision prec, int64_t rb,
                                     int64_t re, float *kappa_out, float *v_out, float *W_out, void *stream) {
    mecuco_status st = check_common(h, X, dt, N, m, ld, k, include_self);
    if (st != MECUCO_OK) return st;
    if ((st = check_range(N, rb, re)) != MECUCO_OK) return st;
    if (!kappa_out || m > 64) return MECUCO_ERR_INVALID_ARG;
    if (prec != MECUCO_PREC_FP32 && prec != MECUCO_PREC_BF16_MIXED) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    const int64_t nrows = re - rb;
    const int64_t chunk = std::min<int64_t>(h->chunk_points > 0 ? h->chunk_points : 65536, nrows);
    const size_t idx_bytes = idx ? 0 : align_up((size_t)nrows * k * sizeof(int32_t), 256);
    Carver t(nullptr, idx_bytes);
    t.take<float>((size_t)chunk * m * m);
    t.take<float>((size_t)chunk * m);
    t.take<float>((size_t)chunk * m * m);
    size_t need = t.off;
    if (!idx) need = std::max(need, knn_bytes(h, X, dt, N, m, ld, nrows, k, prec, idx_bytes));
    if ((st = ensure(h->ws, h->ws_bytes, need, h->ws_cap)) != MECUCO_OK) return st;
    const int32_t *nbr = idx ? idx + rb * k : nullptr;
    if (!idx) {
        int32_t *idx_buf = reinterpret_cast<int32_t *>(h->ws);
        if ((st = run_knn(h, h->ws, X, dt, N, m, ld, k, include_self, prec, rb, re, idx_buf, nullptr, s,
                          idx_bytes)) != MECUCO_OK)
            return st;
        nbr = idx_buf;
    }
    Carver c(h->ws, idx_bytes);
    float *S = c.take<float>((size_t)chunk * m * m);
    float *vb = c.take<float>((size_t)chunk * m);
    float *Wb = c.take<float>((size_t)chunk * m * m);
    const int mode = h->jacobi_fp64 >= 0 ? h->jacobi_fp64 : 1;
    const int mm = (int)m;
    for (int64_t p0 = 0; p0 < nrows; p0 += chunk) {
        const int64_t np = std::min(chunk, nrows - p0);
        float *vd = v_out ? v_out + p0 * m : vb;
        float *Wd = W_out ? W_out + p0 * m * m : Wb;
        LAUNCH(h, MECUCO_STAGE_EXACT, s, launch_exact_cov(X, dt, N, m, ld, nbr + p0 * k, k, np, S, h->ctr, s));
        LAUNCH(h, MECUCO_STAGE_JACOBI, s, launch_jacobi(S, mm, np, mode, h->jacobi_max_sweeps, vd, Wd, h->ctr, s,
                                 kJacobiPreTight, h->jacobi_warp));
        if (mode == 1 || mode == 3) ++h->launches;
        LAUNCH(h, MECUCO_STAGE_EXACT, s, launch_exact_kappa(vd, Wd, mm, np, kappa_out + p0, s));
    }
    return MECUCO_OK;
}

mecuco_status mecuco_exact_kappa(mecuco_t h, const float *v, const float *W, int64_t m, int64_t np, float *kappa,
                                 void *stream) {
    if (!h || !v || !W || !kappa || m < 1 || m > 64 || np < 0 || np >= ((int64_t)1 << 31))
        return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    mecuco_status st;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    LAUNCH(h, MECUCO_STAGE_EXACT, s, launch_exact_kappa(v, W, (int)m, np, kappa, s));
    return MECUCO_OK;
}

mecuco_status mecuco_fidelity(mecuco_t h, const float *kappa_ref, const float *kappa, int64_t n, int normalize,
                              double *metrics_out, void *stream) {
    if (!h || !kappa_ref || !kappa || !metrics_out || n < 2 || n >= ((int64_t)1 << 31)) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    mecuco_status st;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    if ((st = ensure(h->ws, h->ws_bytes, fidelity_scratch_bytes(n), h->ws_cap)) != MECUCO_OK) return st;
    LAUNCH(h, MECUCO_STAGE_FIDELITY, s, launch_fidelity(kappa_ref, kappa, n, normalize != 0, h->ws, metrics_out, s));
    return MECUCO_OK;
}

mecuco_status mecuco_minmax_normalize(mecuco_t h, const float *x, int64_t n, float *y, void *stream) {
    if (!h || !x || !y || n < 1) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    mecuco_status st;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    if ((st = ensure(h->ws, h->ws_bytes, 8192, h->ws_cap)) != MECUCO_OK) return st;
    LAUNCH(h, MECUCO_STAGE_FIDELITY, s, launch_minmax_normalize(x, n, y, h->ws, s));
    return MECUCO_OK;
}

mecuco_status mecuco_curvature_batched(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt,
                                       int include_self, mecuco_variant var, mecuco_precision prec, void *stream) {
    mecuco_status st = check_batch(h, sets, nsets, dt, include_self, var, prec);
    if (st != MECUCO_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    return run_batch_call(h, sets, nsets, dt, include_self, var, prec, s, batch_config(h, sets, nsets, dt, prec));
}

mecuco_status mecuco_autotune_batched(mecuco_t h, const mecuco_dataset *sets, int nsets, mecuco_dtype dt,
                                      int include_self, mecuco_variant var, mecuco_precision prec, void *stream,
                                      mecuco_batch_tuning *out) {
    mecuco_status st = check_batch(h, sets, nsets, dt, include_self, var, prec);
    if (st != MECUCO_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    bool warmed = false;
    // one timed call (after a warm-up the first time) in configuration t
    auto timed = [&](const mecuco_batch_tuning &t, float *ms) -> mecuco_status {
        mecuco_status r;
        if ((r = begin_call(h, s)) != MECUCO_OK) return r;
        if (!warmed) {
            if ((r = run_batch_call(h, sets, nsets, dt, include_self, var, prec, s, t)) != MECUCO_OK) return r;
            warmed = true;
        }
        if (cudaEventRecord(e0, s) != cudaSuccess) return MECUCO_ERR_CUDA;
        if ((r = run_batch_call(h, sets, nsets, dt, include_self, var, prec, s, t)) != MECUCO_OK) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return MECUCO_ERR_CUDA;
        if (cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) return MECUCO_ERR_CUDA;
        return MECUCO_OK;
    };
    const auto sig = batch_signature(sets, nsets, dt, prec);
    h->tuned.erase(sig);
    mecuco_batch_tuning best = batch_config(h, sets, nsets, dt, prec);
    best.ms = 0.f;
    auto consider = [&](mecuco_batch_tuning t) -> mecuco_status {
        float ms = 0.f;
        mecuco_status r = timed(t, &ms);
        if (r != MECUCO_OK) return r;
        if (best.ms == 0.f || ms < best.ms) {
            best = t;
            best.ms = ms;
        }
        return MECUCO_OK;
    };
    if (batch_is_persistent(h, prec)) {
        best.lanes = 1;
        // the kNN tile form, then the third-moment pass's patches per SM and
        // TMEM slots, each with the other stage at its best so far
        for (int pair : {0, 1}) {
            mecuco_batch_tuning t = best;
            t.knn_pair = pair;
            if ((st = consider(t)) != MECUCO_OK) break;
        }
        const int tt[4][2] = {{2, 2}, {2, 4}, {1, 4}, {1, 8}};
        for (int i = 0; i < 4 && st == MECUCO_OK; ++i) {
            mecuco_batch_tuning t = best;
            t.tt_ctas = tt[i][0];
            t.tt_slots = tt[i][1];
            if (t.tt_ctas == best.tt_ctas && t.tt_slots == best.tt_slots && best.ms > 0.f) continue;
            st = consider(t);
        }
    } else {
        for (int L : {32, 16, 8, 4, 2, 1}) {  // the largest first: it sizes the workspace once
            if (L > nsets && L != 1) continue;
            mecuco_batch_tuning t = best;
            t.lanes = L;
            if ((st = consider(t)) != MECUCO_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MECUCO_OK) return st;
    h->tuned[sig] = best;
    if (out) *out = best;
    return MECUCO_OK;
}

mecuco_status mecuco_curvature_host(mecuco_t h, const void *X_host, mecuco_dtype dt, int64_t N, int64_t m,
                                    int64_t ld, int k, int include_self, mecuco_variant var, mecuco_precision prec,
                                    float *kappa_host_out, int32_t *idx_host_out, void *stream) {
    mecuco_status st = check_common(h, X_host, dt, N, m, ld, k, include_self);
    if (st != MECUCO_OK) return st;
    if (!kappa_host_out) return MECUCO_ERR_INVALID_ARG;
    if (var != MECUCO_FAST_LITERAL && var != MECUCO_FAST_HAAR) return MECUCO_ERR_INVALID_ARG;
    if (prec != MECUCO_PREC_FP32 && prec != MECUCO_PREC_BF16_MIXED) return MECUCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = begin_call(h, s)) != MECUCO_OK) return st;
    const size_t elt = dt == MECUCO_BF16 ? 2 : 4;
    const size_t xbytes = ((size_t)(N - 1) * ld + m) * elt;
    Carver t(nullptr);
    t.take<char>(xbytes);
    t.take<float>((size_t)N);
    t.take<int32_t>((size_t)N * k);
    if ((st = ensure(h->io, h->io_bytes, t.off, h->ws_cap)) != MECUCO_OK) return st;
    Carver c(h->io);
    char *Xd = c.take<char>(xbytes);
    float *kd = c.take<float>((size_t)N);
    int32_t *id = c.take<int32_t>((size_t)N * k);
    CK(cudaMemcpyAsync(Xd, X_host, xbytes, cudaMemcpyHostToDevice, s));
    if ((st = ensure_items(h, k)) != MECUCO_OK) return st;
    if (prec == MECUCO_PREC_BF16_MIXED && ((st = ensure_pairs(h, k)) != MECUCO_OK ||
                                           (st = ensure_rotated(h, k)) != MECUCO_OK))
        return st;
    const size_t need = std::max(knn_bytes(h, Xd, dt, N, m, ld, N, k, prec, 0),
                                 curvature_bytes(h, Xd, dt, N, m, ld, k, true, N, prec));
    if ((st = ensure(h->ws, h->ws_bytes, need, h->ws_cap)) != MECUCO_OK) return st;
    if ((st = run_knn(h, h->ws, Xd, dt, N, m, ld, k, include_self, prec, 0, N, id, nullptr, s, 0)) != MECUCO_OK)
        return st;
    if ((st = run_curvature(h, h->ws, Xd, dt, N, m, ld, k, id, include_self, var, prec, 0, N, kd, nullptr, nullptr,
                            nullptr, s)) != MECUCO_OK)
        return st;
    CK(cudaMemcpyAsync(kappa_host_out, kd, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
    if (idx_host_out) CK(cudaMemcpyAsync(idx_host_out, id, sizeof(int32_t) * N * k, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MECUCO_OK;
}

mecuco_status mecuco_get_last_status(mecuco_t h, void *stream) {
    if (!h) return MECUCO_ERR_INVALID_ARG;
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    DevCounters c;
    CK(cudaMemcpyAsync(&c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemsetAsync(&h->ctr->status, 0, sizeof(unsigned), s));
    CK(cudaStreamSynchronize(s));
    if (c.status & DEV_TIMEOUT) return MECUCO_ERR_TIMEOUT;
    if (c.status & DEV_INVALID) return MECUCO_ERR_INVALID_ARG;
    if (c.status & DEV_NOT_CONVERGED) return MECUCO_ERR_NOT_CONVERGED;
    return MECUCO_OK;
}

mecuco_status mecuco_get_stats(mecuco_t h, mecuco_stats *out, void *stream) {
    if (!h || !out) return MECUCO_ERR_INVALID_ARG;
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    DevCounters c;
    CK(cudaMemcpyAsync(&c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->knn_rows = h->knn_rows;
    out->knn_uncertified = (int64_t)c.knn_uncertified;
    out->knn_fallback_rows = (int64_t)c.knn_fallback_rows;
    out->jacobi_max_sweeps = (int64_t)c.jacobi_max_sweeps;
    out->jacobi_not_converged = (int64_t)c.jacobi_not_converged;
    out->rank_deficient = (int64_t)c.rank_deficient;
    out->jacobi_rotations = (int64_t)c.jacobi_rotations;
    out->kernel_launches = h->launches;
    return MECUCO_OK;
}

mecuco_status mecuco_get_stage_times(mecuco_t h, double *ms_out, int64_t *launches_out, void *stream) {
    if (!h || !ms_out || !launches_out) return MECUCO_ERR_INVALID_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    mecuco_status st = flush_events(h);
    if (st != MECUCO_OK) return st;
    for (int i = 0; i < MECUCO_STAGE_COUNT; ++i) {
        ms_out[i] = h->stage_ms[i];
        launches_out[i] = h->stage_n[i];
        h->stage_ms[i] = 0.0;
        h->stage_n[i] = 0;
    }
    return MECUCO_OK;
}

}  // extern "C"
