// kernels.h - host launchers of the MeCuCo CUDA kernels (internal, C++ linkage).
#pragma once

#include <math.h>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mecuco.h"

namespace mecuco {

struct DevCounters;
struct PatchSeg;

// Text returned by mecuco_last_error_message() for this thread.
void set_error_text(const char *msg);

// ---- Step 1: kNN -----------------------------------------------------------
// How the tensor-core search sees FP32 rows (KNN_QUANT_*): not at all (BF16
// rows, or the CUDA-core search), as one BF16 rounding h = bf16(x), or as the
// three-term split (h, l = bf16(x - h)) of launch_to_bf16_split.
enum { KNN_QUANT_NONE = 0, KNN_QUANT_SINGLE = 1, KNN_QUANT_SPLIT = 2 };
// Squared row norms |x_i|^2 (compensated sum, rounded once), i in [0, N).
// With quant != KNN_QUANT_NONE (FP32 rows only), resid[2 i .. 2 i + 1] gets the
// row's rounding terms, rounded up: single rounding |x - h| and 0; split
// |l| and |x - h - l|; maxima[0..2] (zeroed by the caller) receives the
// dataset's largest |x|^2 and the largest of each term.
cudaError_t launch_rownorm(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                           float *norms, cudaStream_t s, float *resid = nullptr, float *maxima = nullptr,
                           int quant = KNN_QUANT_NONE);

// Candidate search, plain FP32 on the CUDA cores.  Queries [q0, q0 + nq) against
// all N rows, candidate range split in `nsplit` parts; per (query, split) the
// kc smallest approximate distances |x|^2 + |y|^2 - 2 x.y are written to
// cand_d / cand_i at [(q - q0) * nsplit + split] * kc (unused slots: +inf, -1).
cudaError_t launch_knn_simt(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                            const float *norms, int64_t q0, int64_t nq, int kc, int nsplit,
                            int include_self, float *cand_d, int32_t *cand_i, cudaStream_t s);

// Candidate search, BF16 operands on the tensor cores (tcgen05, TMEM accumulators,
// TMA-fed shared memory): the output contract of launch_knn_simt with
// knn_tc_halves() lists of capacity kc per row and split.  Xa (query operand)
// and Xb (candidate operand) are BF16 row-major with K = m columns, ldb % 8 ==
// 0 and 16-byte aligned bases: both X itself when it is stored that way, both
// the copy of launch_to_bf16, or the two copies of launch_to_bf16_split (then
// m is their K = 3 ms).  kc <= 64.
// pair != 0 (and nq >= 256): CTA pairs sharing 256 x 256 cta_group::2 MMAs;
// the lists are the same.  wait_limit: clock cycles after which a wait of the
// work loops gives up (MECUCO_ERR_TIMEOUT); <= 0 selects the default (~0.5 s).
// The drains of copies and MMAs in flight always use the default.
cudaError_t launch_knn_tc(const void *Xa, const void *Xb, int64_t N, int64_t m, int64_t ldb, const float *norms,
                          int64_t q0, int64_t nq, int kc, int nsplit, int include_self,
                          float *cand_d, int32_t *cand_i, int pair, long long wait_limit, DevCounters *ctr,
                          cudaStream_t s);
size_t knn_tc_smem_bytes(int kc);
// Candidate lists the tensor-core search leaves per row and split (the epilogue's
// column halves); list h of row r, split s starts at ((r nsplit + s) halves + h) kc.
int knn_tc_halves();
// One dataset of a batched kNN (a device table of them, sorted by first
// work item / first row).  The tensor maps describe the BF16 operands (the
// query copy xb and candidate copy xb2 of a three-term split, one copy xb, or
// X itself) with TMA boxes of the search, K = mk columns; kcl is each list's
// capacity, lists = nsplit * knn_tc_halves() lists per row.
struct KnnSet {  // aligned as CUtensorMap (the device table needs 64-byte aligned maps)
    CUtensorMap map_a, map_b;
    const void *X;     // the dataset in the call's dtype (row norms, re-rank, fallback)
    void *xb;          // BF16 (query) copy, or NULL when X is BF16 with ldb = ld
    void *xb2;         // candidate copy of the three-term split, else NULL
    int64_t N, m, ld, ldb, mk;
    float *norms;      // N
    float *cand_d;     // N x lists x kcl
    int32_t *cand_i;
    int32_t *flags;    // N
    int32_t *idx;      // N x k, the neighbour lists
    float *resid;      // 2 N: the rows' rounding terms (launch_rownorm), or NULL
    float *maxima;     // 3: their maxima and the largest |x|^2 (with resid)
    int k, kc, kcl, nsplit, lists, include_self;
    int quant;         // KNN_QUANT_*
    int64_t item_begin;  // first search work item (one query block x one candidate split)
    int64_t row_begin;   // first row in the batch's row order
};
// Fill the two tensor maps of a table entry for the search form (host).
bool knn_tc_make_maps(KnnSet *d, int pair);
// The tensor-core search over every dataset of a batch in one persistent launch:
// nitems work items in all (the sum of each set's query blocks x splits, query
// blocks of knn_tc_item_rows(pair) rows), kcmax the largest list capacity.
// pair != 0: CTA pairs (256 x 256 two-SM MMAs), else one CTA per SM.
int knn_tc_item_rows(int pair);
cudaError_t launch_knn_tc_batch(const KnnSet *sets, int nsets, int64_t nitems, int kcmax, int pair,
                                long long wait_limit, DevCounters *ctr, cudaStream_t s);
// Per-call output pointers of one dataset of a batch (table order), and the
// dataset and first point of each estimator segment.  launch_batch_patch
// writes them into the device tables (KnnSet.idx; PatchSeg.kappa and .idx at
// the segment's first point) through kernel parameters, BATCH_PATCH_SETS
// datasets per launch, so a captured call carries its own outputs.
struct BatchOut {
    float *kappa;
    int32_t *idx;
};
struct SegRef {
    int32_t set;
    int32_t pad;
    int64_t a;
};
constexpr int BATCH_PATCH_SETS = 1024;
cudaError_t launch_batch_patch(KnnSet *sets, int nsets, PatchSeg *segs, const SegRef *refs, int nsegs,
                               const BatchOut *outs, cudaStream_t s);
// Row norms, BF16 copies, exact re-rank and fallback over every row of a
// batch (table rows sorted by row_begin, nrows rows in all); the re-rank's
// shared memory is sized for lmax = the largest kcl * lists.
cudaError_t launch_rownorm_batch(const KnnSet *sets, int nsets, int64_t nrows, mecuco_dtype dt, cudaStream_t s);
cudaError_t launch_to_bf16_batch(const KnnSet *sets, int nsets, int64_t nrows, mecuco_dtype dt, cudaStream_t s);
cudaError_t launch_knn_rerank_batch(const KnnSet *sets, int nsets, int64_t nrows, int lmax, mecuco_dtype dt,
                                    DevCounters *ctr, cudaStream_t s);
cudaError_t launch_knn_fallback_batch(const KnnSet *sets, int nsets, int64_t nrows, int kmax, mecuco_dtype dt,
                                      DevCounters *ctr, cudaStream_t s);

// The three-term split of FP32 rows: query copy Ya = [h | h | l], candidate
// copy Yb = [h | l | h] in segments of ms >= m columns (ms % 8 == 0, zero past
// m), leading dimension ldb >= 3 ms.
cudaError_t launch_to_bf16_split(const float *X, int64_t N, int64_t m, int64_t ld, void *Ya, void *Yb, int64_t ms,
                                 int64_t ldb, cudaStream_t s);
// BF16 copy of X (round to nearest even) with leading dimension ldb >= m.
cudaError_t launch_to_bf16(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, void *Y,
                           int64_t ldb, cudaStream_t s);

// Exact re-rank of the L = kc * nsplit candidates of each query by a
// compensated (float-float) sum of (x_a - y_a)^2, top-k by (distance, index),
// and the certification test; uncertified rows get flags[q - q0] = 1.
// idx_out / dist_out point at query q0's row (row q - q0 is written).
// resid / maxima (from launch_rownorm): the search ran on BF16 roundings of
// FP32 rows; the certification then also covers the rounding's a-priori
// bound on every candidate's distance error.
cudaError_t launch_knn_rerank(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                              const float *norms, int64_t q0, int64_t nq, int kc, int nsplit, int k,
                              const float *cand_d, const int32_t *cand_i, int32_t *idx_out,
                              float *dist_out, int32_t *flags, DevCounters *ctr, cudaStream_t s,
                              const float *resid = nullptr, const float *maxima = nullptr,
                              int quant = KNN_QUANT_NONE);

// Exact full scan for the flagged rows of [q0, q0 + nq) (outputs as above).
cudaError_t launch_knn_fallback(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                int64_t q0, int64_t nq, int k, int include_self, const int32_t *flags,
                                int32_t *idx_out, float *dist_out, DevCounters *ctr, cudaStream_t s);

// ---- Steps 2-3: patch moments -------------------------------------------
// For points [p0, p0 + np) (idx row p, outputs at p - p0); callers pass idx
// already offset to the chunk and p0 = 0.  Centred patch X_c from idx; writes
//   G   np x k x k   X_c X_c^T (full symmetric)
//   R   np x k       X_c 1_m
//   Q   np x k x k   X_c diag(c) X_c^T, c_a = sum_j X_c[j,a]^2   (nullable)
// Neighbour indices outside [0, N) are read as row 0 and raise
// MECUCO_ERR_INVALID_ARG in the device status word.  With rot (np x k x k,
// orthogonal U0 per point, nullable) the moments are those of U0^T X_c.
cudaError_t launch_patch_gram(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                              const int32_t *idx, int k, int64_t p0, int64_t np, const float *rot,
                              float *G, float *R, float *Q, DevCounters *ctr, cudaStream_t s);

// Third moments M[j,r,t] = sum_a X_c[j,a] X_c[r,a] X_c[t,a], stored pair-major:
// D[pair(a,b)][c] = M[a][b][c] for a <= b, every c; np x m3_pair_floats(k) floats.
// `items` is the work-item list built by m3_build_items.
cudaError_t launch_patch_m3(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                            const int32_t *idx, int k, int64_t p0, int64_t np, const float *rot,
                            float *M, const int32_t *items, DevCounters *ctr, cudaStream_t s);

__host__ __device__ inline int pair_index(int a, int b, int k) { return a * k - (a * (a - 1)) / 2 + (b - a); }
inline int64_t m3_pair_floats(int k) { return (int64_t)k * (k + 1) / 2 * k; }
#ifdef __CUDACC__
__device__ inline int64_t m3_pair_floats_d(int k) { return (int64_t)k * (k + 1) / 2 * k; }
#endif
// Work items (j, Rb, Tb) with Rb >= j / 8 and Tb >= Rb over nb = ceil(k / 8)
// blocks of 8, packed j | Rb << 8 | Tb << 16.
int m3_items(int k);
void m3_build_items(int k, int32_t *items /* m3_items(k) */);

// BF16-mixed form: G, R, Q and the pair-major M of each patch from
// tensor-core GEMMs over 128-row tiles of row products (BF16 operands, FP32
// accumulation), nslots TMEM slots for the A operand; wait_limit as for
// launch_knn_tc.  rowtab holds moments_tc_rows(k) row codes built by
// moments_tc_build_rows; idx points at the chunk's first neighbour row; Q may
// be NULL.
cudaError_t launch_moments_tc(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                              int k, int64_t np, const int32_t *rowtab, float *M, float *G, float *R, float *Q,
                              int nslots, long long wait_limit, DevCounters *ctr, cudaStream_t s);
int moments_tc_rows(int k);
void moments_tc_build_rows(int k, int32_t *codes /* moments_tc_rows(k) */);
size_t moments_tc_smem_bytes(int k);
// BF16-mixed estimator in the rotated basis, over the points of a launch
// described by a segment table (PatchSeg, common.cuh: one segment by value for
// a single dataset, or a device table for several).  launch_gram_tc: G, R and
// (with_q) Q of each patch, as launch_patch_gram's outputs, from BF16 operands
// on the tensor cores.  launch_rotate_tc: Y = U^T X_c per point (U from
// launch_jacobi, k x k), BF16; launch point p's row l at Y + (p * 64 + l) * ldy
// (rows k..63 zero), ldy >= every segment's m rounded up to 64, ldy % 8 == 0.
// launch_tthird_tc: the Fast estimator from Y, sig, U, R and Q (Haar) -
// kappa, and lambda / s when not NULL; rowtab from tthird_build_rows for the
// segment's k; kmax bounds every segment's k; ctas = 1 or 2 CTAs per SM (512 or
// 256 TMEM columns each, nslots of them the A operand's slots).
cudaError_t launch_gram_tc(mecuco_dtype dt, const PatchSeg &one, const PatchSeg *tab, int ntab, int64_t np,
                           int with_q, long long wait_limit, DevCounters *ctr, cudaStream_t s);
cudaError_t launch_rotate_tc(mecuco_dtype dt, const PatchSeg &one, const PatchSeg *tab, int ntab, int64_t np, void *Y,
                             int64_t ldy, long long wait_limit, DevCounters *ctr, cudaStream_t s);
__host__ __device__ int tthird_rows(int k);
void tthird_build_rows(int k, int32_t *codes /* tthird_rows(k) */);
cudaError_t launch_tthird_tc(const PatchSeg &one, const PatchSeg *tab, int ntab, int kmax, int64_t np, const void *Y,
                             int64_t ldy, int variant, int nslots, int ctas, long long wait_limit, DevCounters *ctr,
                             cudaStream_t s);

// ---- Step 3: k x k eigensolve -----------------------------------------------
// Parallel-order two-sided Jacobi, one CTA per patch.  G: np x k x k.
// Outputs sigma (np x k, descending) and U (np x k x k, column l = eigenvector).
// fp64: 0 = FP32 sweeps; 1 = FP32 sweeps then one refinement step (products
// in two-term FP32, ~2^-48 relative);
// 2 = every sweep in FP64; 3 = as 1 with the refinement's cluster test
// relative to each eigenvalue pair (for nearly diagonal Grams).
// pre_eps is the rotation threshold of the FP32 sweeps of modes 1 and 3: the
// refinement squares the eigenvector error, so kJacobiPreLoose suffices where
// the eigenpairs feed the estimator directly (on 100k curved patches, m = 4096,
// k = 64, kappa moved by <= 3.6e-7 relative and the stage took 8% less time;
// 2^-11 moved it by 1.4e-4).  Eigenvectors that later rotate a patch, whose
// rotated Gram must come out nearly diagonal, take kJacobiPreTight.
constexpr float kJacobiPreTight = 2.384185791015625e-07f;  // 2^-22
constexpr float kJacobiPreLoose = 6.103515625e-05f;        // 2^-14
// warp_form != 0: the FP32 sweeps run one warp per patch (fused 2 x 2 block
// updates, no block barriers); 0: one CTA of 128 threads per patch.  FP64
// sweeps (fp64 = 2) always take the CTA form.
cudaError_t launch_jacobi(const float *G, int k, int64_t np, int fp64, int max_sweeps,
                          float *sigma, float *U, DevCounters *ctr, cudaStream_t s,
                          float pre_eps = kJacobiPreTight, int warp_form = 1);
// The same over a segment table (PatchSeg: G, k, sig, U of each segment);
// kmax bounds every segment's k.
cudaError_t launch_jacobi_seg(const PatchSeg &one, const PatchSeg *tab, int ntab, int kmax, int64_t np, int fp64,
                              int max_sweeps, DevCounters *ctr, cudaStream_t s, float pre_eps, int warp_form = 1);

// ---- Step 4: k-space estimator ----------------------------------------------
// sigma/U from launch_jacobi, M pair-major from launch_patch_m3, R and Q from
// launch_patch_gram (Q only for the Haar variant).  Writes kappa (np) and,
// when not NULL, lambda_out (np x k) and the singular values s_out (np x k).
// G (np x k x k, nullable): the patch Grams, given when U holds Ritz vectors
// rather than eigenvectors of G (|X_c V_r|_F^2 is then computed as |G W|_F^2).
cudaError_t launch_estimator(const float *sigma, const float *U, const float *M, const float *R,
                             const float *Q, int k, int64_t m, int64_t np, int variant, float rank_eps,
                             float *kappa, float *lambda_out, float *s_out, DevCounters *ctr,
                             cudaStream_t s, const float *G = nullptr);

// Numerical-rank thresholds (eigenvalues kept above eps * s_0):
//  - a Gram accumulated in FP32 (or from BF16 products) carries rounding of
//    ~sqrt(m) 2^-24 s_0, so eigenvalues below 8x that are not resolved;
//  - the Gram of a rotated patch (U0^T X_c, nearly diagonal) resolves small
//    eigenvalues to relative accuracy ~2^-24 s_max/s_l, so it takes the FP64
//    oracle's k m 2^-52, floored at 2^-40 above the rotation's own noise.
inline float rank_eps_gram32(int64_t m) { return 8.f * sqrtf((float)m) * 5.9604644775390625e-08f; }
inline float rank_eps_rotated(int k, int64_t m) {
    const double e = (double)k * (double)m * 2.220446049250313e-16;
    return (float)(e > 9.094947017729282e-13 ? e : 9.094947017729282e-13);
}

// U_out (np x k x k) = U0 V per point (the eigenvectors of a rotated Gram back
// in the patch's own basis).
cudaError_t launch_compose_rotation(const float *U0, const float *V, int k, int64_t np, float *U_out,
                                    cudaStream_t s);

// ---- Exact mode ---------------------------------------------------------------
// S (np x m x m) = X_c^T X_c / (k - 1) of each point's patch (m <= 64); then
// kappa (np) from the eigenpairs (v np x m descending, W np x m x m) of S.
cudaError_t launch_exact_cov(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                             int k, int64_t np, float *S, DevCounters *ctr, cudaStream_t s);
cudaError_t launch_exact_kappa(const float *v, const float *W, int m, int64_t np, float *kappa, cudaStream_t s);

// ---- agreement metrics ----------------------------------------------------------
// out[0..2] (device) = MAE, Spearman rho_S, Chatterjee xi between a (reference)
// and b, after min-max normalisation of each when normalize != 0; scratch of
// fidelity_scratch_bytes(n).  launch_minmax_normalize: y = (x - min) / (max - min)
// with 8 KB of scratch.
size_t fidelity_scratch_bytes(int64_t n);
cudaError_t launch_fidelity(const float *a, const float *b, int64_t n, int normalize, void *scratch, double *out,
                            cudaStream_t s);
cudaError_t launch_minmax_normalize(const float *x, int64_t n, float *y, void *scratch, cudaStream_t s);

// ---- randomised low-rank SVD --------------------------------------------------
// Range finder on each patch Gram (np x k x k) with the shared k x l test
// matrix omega and `power` power iterations: Q (np x k x l, orthonormal
// columns, collapsed ones 0) and B = Q^T G Q (np x l x l).  Then, from the
// eigenpairs of B (launch_jacobi, descending), U (np x k x k, first r columns
// Q V_B, the rest 0) and sigma (np x k, the r largest then 0).
cudaError_t launch_rsvd_range(const float *G, int k, int64_t np, const float *omega, int l, int power, float *Q,
                              float *B, cudaStream_t s);
cudaError_t launch_rsvd_compose(const float *Q, const float *sigB, const float *VB, int k, int l, int r, int64_t np,
                                float *sigma, float *U, cudaStream_t s);

// ---- tangent bases ------------------------------------------------------------
// V (np x m x d_out, l fastest) = X_c^T U_p S^-1 for the points of one chunk
// (idx offset to the chunk), sigma/U from launch_jacobi.
cudaError_t launch_tangent_basis(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                 const int32_t *idx, int k, int64_t np, const float *sigma, const float *U,
                                 int d_out, float rank_eps, float *V, DevCounters *ctr, cudaStream_t s);

// ---- adjoint ---------------------------------------------------------------
// d(sum_i gk_i K_i)/dX for the points of one chunk (idx offset to the chunk),
// accumulated into dX (row stride ldd) with atomics.  Inputs are sigma/U (the
// eigenpairs of the rotated Gram) and M/R/Q of the rotated patch Z = U0^T X_c
// (rot = U0 per point, np x k x k); dG, dR, dQ (np x k x k, k, k x k), C and
// dMbuf (np x k^3 each) are scratch.
cudaError_t launch_adjoint(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                           int k, int64_t np, int variant, float rank_eps, const float *rot, const float *sigma,
                           const float *U, const float *M, const float *R, const float *Q, const float *gk, float *dG,
                           float *dR, float *dQ, float *C, float *dMbuf, float *dX, int64_t ldd, cudaStream_t s);

}  // namespace mecuco
