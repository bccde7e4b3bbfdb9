/*
 * mecuco.h - C ABI of the GB300 (sm_103a) MeCuCo local mean-curvature library.
 *
 * The library computes, for every point x_i of a dataset X (N x m), the
 * paper's Fast-mode mean-curvature score K_i (arXiv 2606.06329, Sec. 4,
 * Algorithm 1, Fast branch):
 *   1. the k nearest other points of x_i under squared Euclidean distance
 *      (Sec. 3 Step 1, eq. knn; Alg. 1 kNN-Graph),
 *   2. the centred k x m patch X_c (Sec. 3 Step 2; Alg. 1 Fast branch),
 *   3. its truncated SVD with p = k-1 through the k x k Gram X_c X_c^T
 *      (eq. svd_cov; Alg. 1 SVD_p),
 *   4. tau, t_range, t_A, t_B, t_null and K_i = |(t_range + t_null)/2 + tau/2|
 *      (eqs. tnull, tA, tB, fast_curv; Alg. 1 Fast branch).
 *
 * Conventions shared by every entry point
 *   - X is row-major with leading dimension ld >= m (elements, not bytes);
 *     element type F32 or BF16.  Unless an entry point says "host", every
 *     pointer is a DEVICE pointer on the context's device, owned by the
 *     caller; the library never frees or retains it past the call.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device-pointer entry points are asynchronous on that stream: they
 *     enqueue work and return; results are valid once the stream reaches
 *     that point.  Host entry points synchronise the stream before return.
 *   - Neighbour lists idx are int32, N x k row-major, each row sorted by
 *     (distance, index) ascending; a point is not its own neighbour unless
 *     include_self = 1.  Requirements: 2 <= k <= 64, k <= N - 1 (k <= N with
 *     include_self), 1 <= m, N < 2^31.
 *   - The truncation rank is p = min(k - 1, m, numerical rank of X_c), the
 *     numerical rank counting eigenvalues of X_c X_c^T above 8 sqrt(m) 2^-24
 *     times the largest (the FP32 Gram's rounding scale); q = m - p and
 *     t_null = 0 when q = 0.
 *   - Return value: MECUCO_OK, or an error code; on an argument error nothing
 *     is enqueued.  Errors detected on the device (an eigensolver sweep cap,
 *     a bounded wait that ran out) never trap: they are OR-ed into a device
 *     status word read back by mecuco_get_last_status() after the stream has
 *     been synchronised.  No entry point throws across the ABI.
 *   - A context may be used from one host thread at a time.
 */
#ifndef MECUCO_H
#define MECUCO_H

#include <stdint.h>

#if defined(__GNUC__)
#define MECUCO_API __attribute__((visibility("default")))
#else
#define MECUCO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mecuco_ctx *mecuco_t;

typedef enum {
    MECUCO_OK = 0,
    MECUCO_ERR_INVALID_ARG = 1,   /* a size, pointer, alignment or enum is out of range */
    MECUCO_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement */
    MECUCO_ERR_OOM = 3,           /* device or pinned-host allocation failed */
    MECUCO_ERR_CUDA = 4,          /* a CUDA runtime call failed (message: mecuco_last_error_message) */
    MECUCO_ERR_NOT_CONVERGED = 5, /* device: an eigensolve hit its sweep cap (result still written) */
    MECUCO_ERR_TIMEOUT = 6        /* device: a bounded wait ran out (result of that launch invalid) */
} mecuco_status;

typedef enum { MECUCO_F32 = 0, MECUCO_BF16 = 1 } mecuco_dtype;

/* Fast-mode null-space term.
 *   LITERAL: t_B = tau - 2 |X_c V_r|_F^2/(k-1) + |G_tens|_F^2/(k-1) and
 *            t_null = (t_A + 2 t_B)/(m - p), exactly as Alg. 1 prints them.
 *   HAAR:    the Haar expectation of eq. gnull_exp written out:
 *            t_B = tau - 2 sum_{j,a} X_c[j,a]^2 (1 - d_P[a])/(k-1)
 *                  + |G_tens|_F^2/(k-1), t_null = (t_A + 2 t_B)/(m - p + 2). */
typedef enum { MECUCO_FAST_LITERAL = 0, MECUCO_FAST_HAAR = 1 } mecuco_variant;

/* Arithmetic of the hot path.
 *   FP32:       distances, Gram, third moments and the k-space estimator in
 *               FP32 on the CUDA cores; FP32 Jacobi.  (the plain form)
 *   BF16_MIXED: distance GEMM in BF16 on the tensor cores with FP32
 *               accumulation and an FP32 exact re-rank of the candidates;
 *               the patch Gram (and Q) from BF16 operands on the tensor cores
 *               with FP32 accumulation; Jacobi sweeps in FP32 followed by one
 *               refinement step of the eigenpairs whose products are carried
 *               beyond FP32 (two-term FP32, ~2^-48 relative); the rotated
 *               patch Y = U^T X_c on the tensor cores (U in two BF16 terms),
 *               rounded to BF16; the estimator's sums from the third moments
 *               of Y, BF16 products with FP32 accumulation, on the tensor
 *               cores.  (the chosen form; with a randomised SVD the third
 *               moments of X_c and the k-space estimator of the plain form) */
typedef enum { MECUCO_PREC_FP32 = 0, MECUCO_PREC_BF16_MIXED = 1 } mecuco_precision;

/* Tunable options (mecuco_set_option).  Values are int64. */
typedef enum {
    MECUCO_OPT_KNN_MARGIN = 0,       /* extra candidates kept per row before the exact re-rank (default 32) */
    MECUCO_OPT_JACOBI_FP64 = 1,      /* -1: by precision (default: 0 for FP32, 1 for BF16_MIXED);
                                        0: FP32 sweeps; 1: FP32 sweeps + one refinement step in
                                        two-term FP32 (FP64-class products);
                                        2: every sweep in FP64; 3: as 1, eigenvalue clusters judged
                                        relative to each pair.  The adjoint's rotated Gram uses 3
                                        unless this option is set */
    MECUCO_OPT_JACOBI_MAX_SWEEPS = 2,/* sweep cap of the eigensolver (default 40) */
    MECUCO_OPT_CHUNK_POINTS = 3,     /* points per estimator chunk (0 = automatic) */
    MECUCO_OPT_KNN_QUERY_CHUNK = 4,  /* query rows per kNN launch (0 = automatic) */
    MECUCO_OPT_PROFILE = 5,          /* 1: bracket every kernel with CUDA events (mecuco_get_stage_times) */
    MECUCO_OPT_KNN_SPLITS = 6,       /* candidate-range splits of the kNN search (0 = automatic, else 1..64;
                                        capped so that splits * candidate capacity <= 1024) */
    MECUCO_OPT_BATCH_LANES = 7,      /* concurrent streams of mecuco_curvature_batched (1..32, default 8;
                                        a batch signature tuned by mecuco_autotune_batched uses its own) */
    MECUCO_OPT_TC_SLOTS = 8,         /* TMEM slots for the row-product operand of the tensor-core moment
                                        kernel (2, 4, 6 or 8, default 4; slots are handed between warps in
                                        pairs; more slots leave fewer accumulator tiles per pass over the
                                        patch) */
    MECUCO_OPT_KNN_PAIR = 9,         /* 1: the tensor-core kNN search runs as CTA pairs sharing 256 x 256
                                        two-SM MMAs (tcgen05 cta_group::2); 0: one CTA per SM; -1 (default):
                                        pairs for N >= 200,000 points, where they are faster.  The candidate
                                        lists are identical */
    MECUCO_OPT_WAIT_LIMIT = 10,      /* SM clock cycles after which a bounded wait in the work loops of the
                                        tensor-core kernels (kNN search on single CTAs, patch moments) gives
                                        up: the launch sets MECUCO_ERR_TIMEOUT in the status word, waits for
                                        the copies and MMAs it has in flight (always with the default limit),
                                        frees its tensor memory and returns; its outputs are then invalid.
                                        0 (default): 1e9 cycles (~0.5 s at 2 GHz) */
    MECUCO_OPT_WORKSPACE_LIMIT = 11, /* cap in bytes on each device buffer the context grows (workspace,
                                        host-call copies, batched-call lanes); a call that needs more returns
                                        MECUCO_ERR_OOM before allocating, leaving the context usable.
                                        0 (default): no cap */
    MECUCO_OPT_PROFILE_STAGES = 12,  /* bit mask of the mecuco_stage values that MECUCO_OPT_PROFILE brackets
                                        with events (1 << stage); 0 (default): every stage */
    MECUCO_OPT_TT_SLOTS = 13,        /* BF16-mixed third-moment pass: TMEM slots of its row-product operand
                                        (2, 4, 6 or 8, default 4; as MECUCO_OPT_TC_SLOTS) */
    MECUCO_OPT_TT_CTAS = 14,         /* BF16-mixed third-moment pass: CTAs per SM, 1 (512 TMEM columns each)
                                        or 2 (default; 256 each: fewer accumulators per pass over the patch,
                                        two hand-over pipelines interleaved).  Results identical */
    MECUCO_OPT_BATCH_PERSISTENT = 15,/* 1 (default): mecuco_curvature_batched with MECUCO_PREC_BF16_MIXED runs
                                        every dataset of the batch in one launch per stage (persistent kNN
                                        over a device table of all datasets' work items, estimator launches
                                        over segment tables of all datasets' points); 0: one stream lane per
                                        dataset group, as the FP32 form always does.  Results identical */
    MECUCO_OPT_JACOBI_WARP = 16,     /* FP32 Jacobi sweeps: 1, 2 (default) or 4 warps per patch in the fused
                                        form (a round's rotations applied in one pass over 2 x 2 blocks of A
                                        and U, two barriers per round, none with 1 warp); 0: one CTA of 128
                                        threads per patch in three passes (row, column and eigenvector
                                        updates, three barriers per round).  Same rotations and thresholds;
                                        the results differ only by rounding order.  Measured on 100k patches
                                        (k = 64): 230 ms (0), 221 (1), 192 (2), 192 (4) */
    MECUCO_OPT_KNN_SPLIT_BF16 = 17   /* BF16-mixed kNN of FP32 rows: 1 (default) the tensor-core search runs on
                                        the three-term split of each row (h = bf16(x), l = bf16(x - h); one GEMM
                                        over [h|h|l] . [h|l|h], three times the K of one rounding) and the
                                        certificate bounds its rounding error a priori at ~2^-16 relative;
                                        0: one BF16 rounding, a third of the search but a ~2^-8 bound, which
                                        sends most rows of clustered FP32 data to the exact scan.  The lists
                                        are identical either way */
} mecuco_option;

/* Kernel stages, for mecuco_get_stage_times. */
typedef enum {
    MECUCO_STAGE_ROWNORM = 0,    /* squared row norms (kNN) */
    MECUCO_STAGE_KNN_SEARCH = 1, /* distance tiles + per-row candidate lists */
    MECUCO_STAGE_KNN_RERANK = 2, /* exact re-rank + certification */
    MECUCO_STAGE_KNN_FALLBACK = 3,/* exact full scan of uncertified rows */
    MECUCO_STAGE_GRAM = 4,       /* gather, centre, G = X_c X_c^T, R, Q */
    MECUCO_STAGE_MOMENTS = 5,    /* third moments: of X_c (plain form, M stored), or of the rotated patch
                                    reduced on the fly to the estimator's sums (BF16-mixed form) */
    MECUCO_STAGE_JACOBI = 6,     /* k x k eigensolve */
    MECUCO_STAGE_ESTIMATOR = 7,  /* k-space Fast estimator */
    MECUCO_STAGE_ADJOINT = 8,    /* k-space adjoint + patch adjoint and scatter */
    MECUCO_STAGE_BASIS = 9,      /* tangent-basis expansion V_r = X_c^T U_p S^-1 */
    MECUCO_STAGE_EXACT = 10,     /* Exact mode: m x m covariance and K from its eigenbasis */
    MECUCO_STAGE_FIDELITY = 11,  /* agreement metrics: sorts, ranks, sums */
    MECUCO_STAGE_ROTATE = 12,    /* BF16-mixed form: gather, centre, rotated patch Y = U^T X_c */
    MECUCO_STAGE_COUNT = 13
} mecuco_stage;

/* Counters of the last completed call (valid after the stream is synchronised). */
typedef struct {
    int64_t knn_rows;            /* query rows searched */
    int64_t knn_uncertified;     /* rows whose candidate margin could not be certified */
    int64_t knn_fallback_rows;   /* rows re-solved by the exact full-scan path */
    int64_t jacobi_max_sweeps;   /* largest sweep count used by any patch */
    int64_t jacobi_not_converged;/* patches that hit the sweep cap */
    int64_t rank_deficient;      /* patches with numerical rank < min(k-1, m) */
    int64_t kernel_launches;     /* kernels launched by the call */
    int64_t jacobi_rotations;    /* plane rotations applied by the Jacobi sweeps (all patches) */
} mecuco_stats;

/* Create a context on CUDA device `device`.  It owns a device workspace that
 * grows on demand (cudaMalloc) and a device status word.  Returns
 * MECUCO_ERR_INVALID_ARG for a bad device, MECUCO_ERR_UNSUPPORTED if the
 * device is not compute capability 10.3, MECUCO_ERR_OOM on allocation
 * failure. */
MECUCO_API mecuco_status mecuco_create(mecuco_t *h, int device);

/* Release everything the context owns.  Synchronises the device first.
 * NULL is accepted and ignored. */
MECUCO_API mecuco_status mecuco_destroy(mecuco_t h);

/* Set a tuning option (see mecuco_option); out-of-range values are rejected. */
MECUCO_API mecuco_status mecuco_set_option(mecuco_t h, mecuco_option opt, int64_t value);

/* Step 1 (Sec. 3 Step 1, eq. knn): the k nearest neighbours of every point.
 *   X        device, N x m (ld) of dtype dt
 *   idx_out  device, N x k int32, overwritten; rows sorted by (d, index)
 *   dist_out device, N x k float (nullable): squared distances of idx_out,
 *            from the exact re-rank (FP32 rounding of a compensated sum)
 * prec selects the candidate search (FP32 SIMT, or BF16 tensor-core GEMM);
 * both finish with the same exact re-rank, so both return the same lists up
 * to ties closer than the re-rank's rounding. */
MECUCO_API mecuco_status mecuco_knn(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                         int64_t ld, int k, int include_self, mecuco_precision prec,
                         int32_t *idx_out, float *dist_out, void *stream);

/* Steps 2-4 (Sec. 3 Step 2; eq. svd_cov; eqs. tnull, tA, tB, fast_curv;
 * Alg. 1 Fast branch): the Fast-mode curvature of every point.
 *   X          device, N x m (ld) of dtype dt
 *   idx        device, N x k int32 neighbour lists, or NULL to run
 *              mecuco_knn first (with include_self and prec)
 *   kappa_out  device, N floats, overwritten with K_i >= 0
 *   lambda_out device, N x k floats (nullable): lambda_r = s_l^2/(k-1) in
 *              descending order, zero past p
 *   U_out      device, N x k x k floats (nullable): the k x k eigenvector
 *              matrix U of X_c X_c^T (row r, column l), columns in the order
 *              of lambda; the tangent basis is V_r = X_c^T U_p diag(s)^-1
 *   s_out      device, N x k floats (nullable): singular values s_l of X_c */
MECUCO_API mecuco_status mecuco_curvature(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                               int64_t ld, int k, const int32_t *idx, int include_self,
                               mecuco_variant var, mecuco_precision prec, float *kappa_out,
                               float *lambda_out, float *U_out, float *s_out, void *stream);

/* Row-range forms (resumable chunked runs, sampled timing, per-rank shards):
 * only query rows [row_begin, row_end) are processed; every point of X is still
 * a candidate neighbour.  Outputs hold (row_end - row_begin) rows: row r of
 * idx_out / kappa_out / ... belongs to point row_begin + r, and idx (if given)
 * holds the neighbour lists of those rows only.  Same contracts otherwise. */
MECUCO_API mecuco_status mecuco_knn_range(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N,
                                          int64_t m, int64_t ld, int k, int include_self,
                                          mecuco_precision prec, int64_t row_begin, int64_t row_end,
                                          int32_t *idx_out, float *dist_out, void *stream);
MECUCO_API mecuco_status mecuco_curvature_range(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N,
                                                int64_t m, int64_t ld, int k, const int32_t *idx,
                                                int include_self, mecuco_variant var,
                                                mecuco_precision prec, int64_t row_begin,
                                                int64_t row_end, float *kappa_out, float *lambda_out,
                                                float *U_out, float *s_out, void *stream);

/* Adjoint of the Fast-mode curvature (Alg. 1; eqs. tnull, tA, tB, fast_curv)
 * with the neighbour lists frozen: dX_out = d(sum_i dkappa_i K_i) / dX, where
 * K_i is the curvature of mecuco_curvature for the same (X, idx, var).
 * K = |f| is differentiated as sign(f) df (0 at f = 0).  Every patch's moments
 * and eigenpairs are recomputed (nothing is kept from the forward call) in
 * FP32 on a rotated copy of the patch (U0^T X_c, U0 the eigenvectors of a
 * first Gram, which leaves K unchanged and keeps the small eigenvalues
 * accurate), with refined eigenpairs (two-term FP32); the per-point adjoint
 * runs in k-space (through the derivative of the symmetric eigendecomposition,
 * which is unbounded for coinciding eigenvalues) and is scattered onto the
 * neighbour rows with atomic adds (summation order, hence the last bits, vary
 * between runs).
 *   X       device, N x m (ld) of dtype dt
 *   idx     device, N x k int32 neighbour lists (required)
 *   dkappa  device, N floats
 *   dX_out  device, N x m floats (row stride m), overwritten */
MECUCO_API mecuco_status mecuco_curvature_backward(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                                                   int64_t ld, int k, const int32_t *idx, mecuco_variant var,
                                                   const float *dkappa, float *dX_out, void *stream);

/* Tangent bases of the points [row_begin, row_end) (Alg. 1 SVD_p; eq. svd_cov):
 * the first d_out right singular vectors V_r = X_c^T U_p S^-1 of each patch,
 * from the plain FP32 Gram and eigensolve (MECUCO_OPT_JACOBI_FP64 applies).
 * Columns l >= p (the numerical rank rule of the estimator) are zero; column
 * signs are fixed so that the largest-magnitude entry of U_p's column l
 * (lowest row on ties) is positive.
 *   X      device, N x m (ld) of dtype dt
 *   idx    device, N x k int32 neighbour lists (required)
 *   d_out  1 <= d_out <= min(k - 1, m)
 *   V_out  device, (row_end - row_begin) x m x d_out floats, l fastest */
MECUCO_API mecuco_status mecuco_tangent_basis(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                                              int64_t ld, int k, const int32_t *idx, int64_t row_begin,
                                              int64_t row_end, int d_out, float *V_out, void *stream);

/* Exact mode (Theorem 1; eq. exact_curv) for the points [row_begin, row_end):
 * Sigma = X_c^T X_c / (k - 1) (m x m), Sigma = W diag(v) W^T (FP32 Jacobi
 * sweeps + refinement step, v descending), C = W^T W^{o2} and
 * K = | 1/2 v^T (C^{o2} 1) + 1/2 sum v |.  The paper's automatic mode uses it
 * for m < 50.  Requires m <= 64.  When m > k - 1, Sigma has a null space and K
 * depends on the eigenbasis returned for it (the identity sums over every
 * column of W); W_out exposes that basis.
 *   idx      device N x k neighbour lists, or NULL to compute them (prec)
 *   kappa_out device, (row_end - row_begin) floats
 *   v_out    device, (row_end - row_begin) x m floats, or NULL
 *   W_out    device, (row_end - row_begin) x m x m floats (row i, column s), or NULL */
MECUCO_API mecuco_status mecuco_curvature_exact(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                                                int64_t ld, int k, const int32_t *idx, int include_self,
                                                mecuco_precision prec, int64_t row_begin, int64_t row_end,
                                                float *kappa_out, float *v_out, float *W_out, void *stream);

/* Fast mode with the truncated SVD replaced by a randomised low-rank
 * approximation (the paper's future work, Sec. Conclusions), following the
 * range finder of Halko, Martinsson & Tropp (2011, Alg. 4.3/4.4) on each
 * patch's Gram G = X_c X_c^T: Y = G Omega, power_iters times Q = orth(Y),
 * Y = G Q; Q = orth(Y); B = Q^T G Q = V_B diag(sigma_B) V_B^T; U = Q V_B.  The
 * estimator (Alg. 1 Fast branch) then uses the r = rank largest eigenpairs,
 * i.e. p = r and a null space of dimension m - r.  Results differ from
 * mecuco_curvature unless rank = k - 1 and the sketch spans G's range.
 *   omega        device, k x sketch_cols floats row-major: one Gaussian test
 *                matrix for every point (drawn by the caller, independent of X)
 *   rank         1 <= rank <= min(k - 1, m);  rank <= sketch_cols <= k
 *   power_iters  0..16
 * Other arguments as for mecuco_curvature; neighbours computed when idx is NULL. */
MECUCO_API mecuco_status mecuco_curvature_rsvd(mecuco_t h, const void *X, mecuco_dtype dt, int64_t N, int64_t m,
                                               int64_t ld, int k, const int32_t *idx, int include_self,
                                               mecuco_variant variant, mecuco_precision prec, int rank,
                                               int sketch_cols, int power_iters, const float *omega,
                                               float *kappa_out, void *stream);

/* Theorem 1 (eq. exact_curv) evaluated on caller-supplied eigenpairs of each
 * point's covariance: C = W^T W^{o2} and K = |1/2 sum_s v_s sum_l C_sl^2 + 1/2 sum_s v_s|.
 * With the range eigenvectors fixed and the null-space columns of W drawn from
 * the Haar measure, the mean of K over draws is what eq. gnull_exp's
 * expectation (the Fast mode's null-space term) stands for.
 *   v        device, np x m floats (eigenvalues; any order matching W's columns)
 *   W        device, np x m x m floats, row-major, column s = eigenvector s
 *   kappa    device, np floats (written)
 * 1 <= m <= 64; no workspace. */
MECUCO_API mecuco_status mecuco_exact_kappa(mecuco_t h, const float *v, const float *W, int64_t m, int64_t np,
                                            float *kappa, void *stream);

/* The paper's agreement metrics between a reference curvature vector and
 * another (the curvature-fidelity experiments): mean absolute error, Spearman's
 * rank correlation rho_S (Pearson correlation of average ranks) and
 * Chatterjee's xi with the pairs ordered by the reference (ties by index) in
 * the form that allows ties, 1 - n sum |r_{i+1} - r_i| / (2 sum l_i (n - l_i)).
 * With normalize != 0 each vector is first min-max normalised to [0, 1] (the
 * normalisation experiments); rho_S and xi do not change under it.
 *   kappa_ref, kappa  device, n floats (2 <= n < 2^31)
 *   metrics_out       device, 3 doubles: MAE, rho_S, xi */
MECUCO_API mecuco_status mecuco_fidelity(mecuco_t h, const float *kappa_ref, const float *kappa, int64_t n,
                                         int normalize, double *metrics_out, void *stream);

/* y = (x - min x) / (max x - min x), 0 where max = min; x, y device, n floats. */
MECUCO_API mecuco_status mecuco_minmax_normalize(mecuco_t h, const float *x, int64_t n, float *y, void *stream);

/* One dataset of a batched call. */
typedef struct {
    const void *X;  /* device, N x m, row stride ld, of the call's dtype */
    int64_t N, m, ld;
    int k;          /* 2 <= k <= 64, k <= N - 1 (N with include_self) */
    int32_t *idx;   /* device N x k: the neighbour lists are written here (NULL: kept in scratch only) */
    float *kappa;   /* device N: the curvature of every point */
} mecuco_dataset;

/* kNN + Fast-mode curvature (Alg. 1) of many independent datasets of uneven
 * sizes in one call, each exactly as mecuco_curvature computes it (the same
 * neighbour lists and curvatures, bit for bit).
 *
 * MECUCO_PREC_BF16_MIXED (with MECUCO_OPT_BATCH_PERSISTENT = 1, the default):
 * one launch per stage for the whole batch.  The datasets are ordered by m,
 * then k, then N, descending; a device table describes each (its operand's tensor
 * maps, its first search work item and first row) and the persistent kNN
 * search takes the work items (query block x candidate split) of every
 * dataset from it, one CTA (or CTA pair) per SM; row norms, BF16 copies,
 * re-rank and fallback take every row of the batch in one launch each.  The
 * estimator stages (Gram, eigensolve, rotation, third moments) run over
 * segment tables that cover the points of all datasets; they are cut into as
 * few launches as the rotated patches fit the 8 GB chunk scratch (the points
 * of one launch share one leading dimension, that of their largest m).  The
 * kNN tile form (single-CTA 128 x 256 or CTA-pair 256 x 256 tiles) and the
 * third-moment pass's patches per SM and TMEM slots come from
 * mecuco_autotune_batched when it has tuned this batch signature, else from
 * the context's options.
 *
 * MECUCO_PREC_FP32 (or MECUCO_OPT_BATCH_PERSISTENT = 0): the datasets are
 * spread over concurrent streams ("lanes", longest first onto the least-loaded
 * lane; the caller's stream forks to them and joins them back), each lane with
 * its own slice of a batch workspace.
 *
 * `sets` is a host array read during the call.  The context keeps the device
 * tables of the last 64 distinct batches (matched byte for byte on the inputs,
 * sizes and workspace addresses; the outputs' addresses are written into the
 * table by a kernel at the start of every call, so calls with the same inputs
 * reuse one table and must not run concurrently on different streams).  A call that needs no new workspace, no
 * new per-k table (every k already seen by this context) and no new batch table
 * makes no allocation and no host synchronisation, so it can be captured into
 * a CUDA graph; make one uncaptured call with the same datasets first, and
 * replay the graph only while its batch is among the 64 kept (a captured call
 * that would need a new table fails with MECUCO_ERR_INVALID_ARG instead). */
MECUCO_API mecuco_status mecuco_curvature_batched(mecuco_t h, const mecuco_dataset *sets, int nsets,
                                                  mecuco_dtype dt, int include_self, mecuco_variant var,
                                                  mecuco_precision prec, void *stream);

/* The configuration mecuco_autotune_batched picked for a batch signature. */
typedef struct mecuco_batch_tuning {
    int lanes;            /* concurrent streams (lanes form); 1 for the one-launch-per-stage form */
    int knn_pair;         /* kNN tiles: 1 = CTA pairs, 256 x 256 per two-SM MMA; 0 = 128 x 256 per CTA */
    int tt_ctas;          /* third-moment pass: patches (CTAs) resident per SM, 1 or 2 */
    int tt_slots;         /* third-moment pass: TMEM slots of the row-product operand */
    float ms;             /* device time of one batched call in that configuration */
} mecuco_batch_tuning;

/* Times mecuco_curvature_batched on these datasets (CUDA events on `stream`,
 * after one warm-up call) over a small search space and keeps the fastest
 * configuration for this batch signature (number of sets, total N, m and k,
 * dtype, precision) in the context.  One-launch-per-stage form: the kNN tile
 * form (CTA pairs or single CTAs), then the third-moment pass's (CTAs per SM,
 * TMEM slots) in {(2, 2), (2, 4), (1, 4), (1, 8)}, each stage tuned with the
 * other at its best so far.  Lanes form: 1, 2, 4, 8, 16 and 32 lanes.
 * Synchronous; the results of the last timed call are left in the datasets'
 * outputs; `out` (may be NULL) receives the configuration kept. */
MECUCO_API mecuco_status mecuco_autotune_batched(mecuco_t h, const mecuco_dataset *sets, int nsets,
                                                 mecuco_dtype dt, int include_self, mecuco_variant var,
                                                 mecuco_precision prec, void *stream, mecuco_batch_tuning *out);

/* The same computation with HOST buffers (pageable or pinned): X_host is
 * copied to the device, the path runs, kappa (and idx if idx_host_out is not
 * NULL) are copied back.  Synchronous.  Device buffers come from the
 * context's workspace. */
MECUCO_API mecuco_status mecuco_curvature_host(mecuco_t h, const void *X_host, mecuco_dtype dt, int64_t N,
                                    int64_t m, int64_t ld, int k, int include_self,
                                    mecuco_variant var, mecuco_precision prec,
                                    float *kappa_host_out, int32_t *idx_host_out, void *stream);

/* Allocation-free k-nearest-neighbour search (the paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory -
 * code under a framework that owns all device memory through its own pool,
 * services with a fixed device-memory budget, and code that must not incur
 * the implicit synchronisation of cudaMalloc/cudaFree).  It takes no context,
 * calls no cudaMalloc/cudaFree and uses a fixed 32 MiB scratch array compiled
 * into the library, which every GPU holding this library's module keeps until
 * the process exits.  Runs on the calling thread's current device; X, idx_out
 * and dist_out as for mecuco_knn with MECUCO_PREC_FP32, and the lists are the
 * same as that call returns.  N above 4,194,304 rows is rejected with
 * MECUCO_ERR_INVALID_ARG (mecuco_last_error_message says why).  The first call
 * on a device looks up the scratch array's device address (it may load the
 * module); make that call before any stream capture.  The address is cached per
 * device and CUDA context, so a call after cudaDeviceReset looks it up again in
 * the new context.  All calls share the scratch and it keeps the last call's
 * contents; calls whose GPU work overlaps (other streams, other host threads
 * on the same device) race on it and must be serialised by the caller.
 * Device-side counters of this entry point are not reported. */
MECUCO_API mecuco_status mecuco_knn_noalloc(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                            int k, int include_self, int32_t *idx_out, float *dist_out,
                                            void *stream);

/* Status OR-ed on the device by the calls since the previous query, then
 * cleared.  Synchronises `stream` first. */
MECUCO_API mecuco_status mecuco_get_last_status(mecuco_t h, void *stream);

/* Counters of the last call (synchronises `stream` first). */
MECUCO_API mecuco_status mecuco_get_stats(mecuco_t h, mecuco_stats *out, void *stream);

/* Per-stage device time (ms) and launch counts accumulated since the previous
 * query while MECUCO_OPT_PROFILE is on; both arrays hold MECUCO_STAGE_COUNT
 * entries.  Synchronises `stream`, then resets the totals. */
MECUCO_API mecuco_status mecuco_get_stage_times(mecuco_t h, double *ms_out, int64_t *launches_out,
                                                void *stream);

/* Static description of a status code. */
MECUCO_API const char *mecuco_status_string(mecuco_status st);

/* Text of the last CUDA error seen by this thread ("" if none). */
MECUCO_API const char *mecuco_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* MECUCO_H */
