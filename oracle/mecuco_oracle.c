/*
 * mecuco_oracle.c - plain, slow FP64 CPU oracle for the MeCuCo local
 * mean-curvature estimator (arXiv 2606.06329).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers; the CUDA library never links, loads
 * or calls it, and this file includes nothing from the CUDA library.  Every
 * routine is written for readability against the paper, in double precision,
 * with no blocking, fusion or reordering beyond what the cited passage states.
 *
 * What it computes (paper sections in brackets):
 *   orc_knn            k nearest other points, squared Euclidean distance,
 *                      ties by lower index [Sec. 3 Step 1, eq. knn; Alg. 1].
 *   orc_center_patch   centroid and centred k x m patch X_c [Sec. 3 Step 2;
 *                      Alg. 1 Fast branch].
 *   orc_jacobi_eigh    own cyclic Jacobi eigensolver (Golub & Van Loan's
 *                      two-sided Jacobi rotation), eigenvalues descending.
 *   orc_svd_hestenes   own one-sided (Hestenes) Jacobi SVD of X_c.
 *   orc_fast_patch     Fast mode exactly as Alg. 1 prints it (truncated SVD,
 *                      tau, t_range, d_P, t_A, t_B2, G_tens, t_B, t_null, K),
 *                      plus the Haar-consistent variant of eq. gnull_exp.
 *   orc_exact_patch    Exact mode, Theorem 1 (eq. kappa_final / exact_curv).
 *   orc_naive_patch    the original estimator |tr(-H H^T Sigma)| with the
 *                      feature matrix H built explicitly (eq. curvature, eq. H).
 *   orc_hht            H H^T from the explicit H (for the eq. HHt_final pin).
 *   orc_curvature      the per-point loop of Alg. 1 over a whole dataset.
 *   orc_grad_fd        FP64 central finite differences of sum_i K_i with the
 *                      neighbour lists frozen (reference gradient).
 *
 * Readings of the paper taken here, where it is silent: a point is not its
 * own neighbour unless include_self (a kNN graph has no self loops); ties in
 * distance go to the lower index (a deterministic order the GPU can match);
 * the truncation rank is p = min(k-1, m, numerical rank) with numerical rank
 * #{ s_l^2 > k*m*2^-52 * s_1^2 } (Alg. 1 fixes p = k - 1, which a
 * rank-deficient patch cannot support: its extra singular values are FP64
 * rounding noise); with no null space (q = m - p = 0) the null-space term is
 * 0 (Alg. 1 would divide by m - p = 0; Fast then equals Exact).
 *
 * Parity pins: see the tests (special cases, invariants, Haar Monte Carlo,
 * library SVD cross-checks, closed-form golden patches, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_VARIANT_LITERAL 0
#define ORC_VARIANT_HAAR 1

/* terms[] layout returned by orc_fast_patch */
enum { T_TAU = 0, T_RANGE, T_A, T_B2, T_GT2, T_B, T_NULL, T_KAPPA, T_NTERMS };

static void *xmalloc(size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    return p;
}

/* Input element types of the dataset-level entry points; each element is
 * widened exactly to double before any arithmetic. */
enum { ORC_F64 = 0, ORC_F32 = 1, ORC_BF16 = 2 };

static double elem(const void *X, int elt, int64_t i) {
    if (elt == ORC_F32) return (double)((const float *)X)[i];
    if (elt == ORC_BF16) {
        uint32_t bits = (uint32_t)((const uint16_t *)X)[i] << 16;
        float f;
        memcpy(&f, &bits, sizeof f);
        return (double)f;
    }
    return ((const double *)X)[i];
}

/* ------------------------------------------------------------------------- */
/* Step 1: brute-force kNN.  d(i,j) = sum_a (x_ia - x_ja)^2, k smallest by     */
/* (d, j).  rows == NULL means every row is a query.                           */
/* ------------------------------------------------------------------------- */
int orc_knn(const void *X, int elt, int64_t n, int64_t m, const int64_t *rows, int64_t nrows,
            int k, int include_self, int32_t *idx_out, double *dist_out, int nthreads) {
    if (k < 1 || (int64_t)k > n - (include_self ? 0 : 1)) return 1;
    int64_t nq = rows ? nrows : n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < nq; ++r) {
        int64_t q = rows ? rows[r] : r;
        double *xq = (double *)xmalloc(sizeof(double) * (size_t)m);
        for (int64_t a = 0; a < m; ++a) xq[a] = elem(X, elt, q * m + a);
        double *bd = dist_out + r * k;
        int32_t *bi = idx_out + r * k;
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == q && !include_self) continue;
            double d = 0.0;
            for (int64_t a = 0; a < m; ++a) {
                double t = xq[a] - elem(X, elt, j * m + a);
                d += t * t;
            }
            if (cnt == k) {
                if (d > bd[k - 1] || (d == bd[k - 1] && j > bi[k - 1])) continue;
                --cnt; /* drop the current worst */
            }
            int pos = cnt;
            while (pos > 0 && (bd[pos - 1] > d || (bd[pos - 1] == d && bi[pos - 1] > j))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = d;
            bi[pos] = (int32_t)j;
            ++cnt;
        }
        free(xq);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Step 2: centroid xbar = k^-1 sum_j x_j and X_c = [x_j - xbar] (k x m).       */
/* ------------------------------------------------------------------------- */
static void center_patch_typed(const void *X, int elt, int64_t m, const int32_t *nb, int k, double *Xc) {
    for (int64_t a = 0; a < m; ++a) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += elem(X, elt, (int64_t)nb[j] * m + a);
        double mean = s / (double)k;
        for (int j = 0; j < k; ++j) Xc[(int64_t)j * m + a] = elem(X, elt, (int64_t)nb[j] * m + a) - mean;
    }
}

void orc_center_patch(const double *X, int64_t m, const int32_t *nb, int k, double *Xc) {
    center_patch_typed(X, ORC_F64, m, nb, k, Xc);
}

/* ------------------------------------------------------------------------- */
/* Cyclic two-sided Jacobi for a symmetric n x n matrix A (row-major, it is    */
/* overwritten).  Rotation J(p,q) with J_pp = J_qq = c, J_pq = s, J_qp = -s,    */
/* tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),   */
/* c = 1/sqrt(1+t^2), s = t c, so (J^T A J)_pq = 0.  V accumulates J (columns  */
/* of V are eigenvectors).  On return w is sorted descending with V's columns. */
/* Returns the number of sweeps used, or -1 if max_sweeps was reached.          */
/* ------------------------------------------------------------------------- */
int orc_jacobi_eigh(int n, double *A, double *w, double *V, int max_sweeps) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    int sweep = 0, converged = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v = A[i * n + j] * A[i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off == 0.0 || off <= 1e-32 * tot) { converged = 1; break; }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                /* an entry below the underflow range carries no information */
                if (fabs(apq) < 1e-300) {
                    A[p * n + q] = A[q * n + p] = 0.0;
                    continue;
                }
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- A J (columns p, q) */
                for (int r = 0; r < n; ++r) {
                    double arp = A[r * n + p], arq = A[r * n + q];
                    A[r * n + p] = c * arp - s * arq;
                    A[r * n + q] = s * arp + c * arq;
                }
                /* A <- J^T A (rows p, q) */
                for (int r = 0; r < n; ++r) {
                    double apr = A[p * n + r], aqr = A[q * n + r];
                    A[p * n + r] = c * apr - s * aqr;
                    A[q * n + r] = s * apr + c * aqr;
                }
                A[p * n + q] = A[q * n + p] = 0.0;
                /* V <- V J */
                for (int r = 0; r < n; ++r) {
                    double vrp = V[r * n + p], vrq = V[r * n + q];
                    V[r * n + p] = c * vrp - s * vrq;
                    V[r * n + q] = s * vrp + c * vrq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
    /* selection sort, descending, carrying eigenvector columns */
    for (int i = 0; i < n - 1; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (w[j] > w[best]) best = j;
        if (best != i) {
            double tw = w[i]; w[i] = w[best]; w[best] = tw;
            for (int r = 0; r < n; ++r) {
                double tv = V[r * n + i]; V[r * n + i] = V[r * n + best]; V[r * n + best] = tv;
            }
        }
    }
    return converged ? sweep : -1;
}

/* ------------------------------------------------------------------------- */
/* One-sided (Hestenes) Jacobi SVD of the k x m matrix Xc.  The k rows b_i are */
/* rotated pairwise until mutually orthogonal: with alpha = b_i.b_i,           */
/* beta = b_j.b_j, gamma = b_i.b_j the same (c, s) as above diagonalises the    */
/* 2 x 2 Gram [alpha gamma; gamma beta].  Afterwards b_l = s_l v_l^T, so        */
/* s_l = |b_l| and V[:, l] = b_l / s_l.  Outputs sorted by s descending:        */
/* s (k), V (m x k, row-major, column l = right singular vector l).             */
/* ------------------------------------------------------------------------- */
int orc_svd_hestenes(int k, int64_t m, const double *Xc, double *s, double *V, int max_sweeps) {
    double *B = (double *)xmalloc(sizeof(double) * (size_t)k * (size_t)m);
    memcpy(B, Xc, sizeof(double) * (size_t)k * (size_t)m);
    double fro = 0.0;
    for (int64_t t = 0; t < (int64_t)k * m; ++t) fro += Xc[t] * Xc[t];
    const double negligible = 1e-30 * fro; /* rows this small are numerically zero */
    int sweep = 0, converged = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int i = 0; i < k - 1; ++i) {
            for (int j = i + 1; j < k; ++j) {
                double *bi = B + (int64_t)i * m, *bj = B + (int64_t)j * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t a = 0; a < m; ++a) {
                    alpha += bi[a] * bi[a];
                    beta += bj[a] * bj[a];
                    gamma += bi[a] * bj[a];
                }
                if (alpha <= negligible || beta <= negligible) continue;
                if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
                rotated = 1;
                double tau = (beta - alpha) / (2.0 * gamma);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = t * c;
                for (int64_t a = 0; a < m; ++a) {
                    double x = bi[a], y = bj[a];
                    bi[a] = c * x - sn * y;
                    bj[a] = sn * x + c * y;
                }
            }
        }
        if (!rotated) { converged = 1; break; }
    }
    int *order = (int *)xmalloc(sizeof(int) * (size_t)k);
    double *nrm = (double *)xmalloc(sizeof(double) * (size_t)k);
    for (int l = 0; l < k; ++l) {
        double t = 0.0;
        for (int64_t a = 0; a < m; ++a) t += B[(int64_t)l * m + a] * B[(int64_t)l * m + a];
        nrm[l] = sqrt(t);
        order[l] = l;
    }
    for (int i = 0; i < k - 1; ++i) {
        int best = i;
        for (int j = i + 1; j < k; ++j)
            if (nrm[order[j]] > nrm[order[best]]) best = j;
        int tmp = order[i]; order[i] = order[best]; order[best] = tmp;
    }
    for (int l = 0; l < k; ++l) {
        int src = order[l];
        s[l] = nrm[src];
        for (int64_t a = 0; a < m; ++a)
            V[a * k + l] = (nrm[src] > 0.0) ? B[(int64_t)src * m + a] / nrm[src] : 0.0;
    }
    free(order); free(nrm); free(B);
    return converged ? sweep : -1;
}

/* ------------------------------------------------------------------------- */
/* Fast mode for one centred patch, following Alg. 1's Fast branch line by    */
/* line (and eqs. tA, tB, tnull, fast_curv).                                    */
/*   route 0: truncated SVD through the k x k Gram X_c X_c^T and orc_jacobi_eigh*/
/*   route 1: truncated SVD through orc_svd_hestenes                           */
/*   variant 0 (literal): t_B = tau - 2 t_B2 + |G_tens|^2/(k-1),               */
/*                        t_null = (t_A + 2 t_B)/(m - p)       [as printed]    */
/*   variant 1 (Haar):    the expectation that eq. gnull_exp gives,            */
/*        t_B^H = tau - 2 sum_{j,a} X_c[j,a]^2 (1 - d_P[a])/(k-1)               */
/*                + |G_tens|^2/(k-1),  t_null^H = (t_A + 2 t_B^H)/(m - p + 2)   */
/* terms[T_NTERMS] receives tau, t_range, t_A, t_B2, |G_tens|^2, t_B, t_null,   */
/* K.  lam (k entries) receives lambda_r (zeros past p), Vr (m x k, optional)   */
/* the truncated right singular vectors.  Returns p.                           */
/* ------------------------------------------------------------------------- */
int orc_fast_patch(int k, int64_t m, const double *Xc, int variant, int route,
                   double *terms, double *lam, double *Vr_out) {
    const double km1 = (double)(k - 1);
    double *s = (double *)xmalloc(sizeof(double) * (size_t)k);
    double *Vfull = (double *)xmalloc(sizeof(double) * (size_t)m * (size_t)k); /* m x k */
    if (route == 0) {
        double *G = (double *)xmalloc(sizeof(double) * (size_t)k * (size_t)k);
        double *U = (double *)xmalloc(sizeof(double) * (size_t)k * (size_t)k);
        double *sig = (double *)xmalloc(sizeof(double) * (size_t)k);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                double t = 0.0;
                for (int64_t a = 0; a < m; ++a) t += Xc[(int64_t)i * m + a] * Xc[(int64_t)j * m + a];
                G[i * k + j] = t;
            }
        orc_jacobi_eigh(k, G, sig, U, 100);
        for (int l = 0; l < k; ++l) {
            s[l] = sig[l] > 0.0 ? sqrt(sig[l]) : 0.0;
            for (int64_t a = 0; a < m; ++a) {
                double t = 0.0;
                for (int j = 0; j < k; ++j) t += Xc[(int64_t)j * m + a] * U[j * k + l];
                Vfull[a * k + l] = s[l] > 0.0 ? t / s[l] : 0.0;
            }
        }
        free(G); free(U); free(sig);
    } else {
        orc_svd_hestenes(k, m, Xc, s, Vfull, 100);
    }
    /* truncation rank: p = min(k-1, m, numerical rank) */
    int rank = 0;
    double eps_rank = (double)k * (double)m * ldexp(1.0, -52);
    for (int l = 0; l < k; ++l)
        if (s[l] * s[l] > eps_rank * s[0] * s[0] && s[l] > 0.0) ++rank;
    int p = k - 1;
    if ((int64_t)p > m) p = (int)m;
    if (rank < p) p = rank;
    /* V_r (m x p) and lambda_r = s^2/(k-1) */
    double *Vr = (double *)xmalloc(sizeof(double) * (size_t)m * (size_t)(p > 0 ? p : 1));
    for (int64_t a = 0; a < m; ++a)
        for (int l = 0; l < p; ++l) Vr[a * p + l] = Vfull[a * k + l];
    for (int l = 0; l < k; ++l) lam[l] = (l < p) ? s[l] * s[l] / km1 : 0.0;
    if (Vr_out)
        for (int64_t a = 0; a < m; ++a)
            for (int l = 0; l < k; ++l) Vr_out[a * k + l] = (l < p) ? Vr[a * p + l] : 0.0;

    /* tau = lambda_r^T 1_p */
    double tau = 0.0;
    for (int l = 0; l < p; ++l) tau += lam[l];
    /* t_range = |X_c V_r^{o2}|_F^2 / (k-1) */
    double t_range = 0.0;
    for (int j = 0; j < k; ++j)
        for (int l = 0; l < p; ++l) {
            double t = 0.0;
            for (int64_t a = 0; a < m; ++a) t += Xc[(int64_t)j * m + a] * Vr[a * p + l] * Vr[a * p + l];
            t_range += t * t;
        }
    t_range /= km1;
    /* d_P = 1_m - V_r^{o2} 1_p */
    double *dP = (double *)xmalloc(sizeof(double) * (size_t)m);
    for (int64_t a = 0; a < m; ++a) {
        double t = 0.0;
        for (int l = 0; l < p; ++l) t += Vr[a * p + l] * Vr[a * p + l];
        dP[a] = 1.0 - t;
    }
    /* t_A = |X_c d_P|^2 / (k-1) */
    double t_A = 0.0;
    for (int j = 0; j < k; ++j) {
        double t = 0.0;
        for (int64_t a = 0; a < m; ++a) t += Xc[(int64_t)j * m + a] * dP[a];
        t_A += t * t;
    }
    t_A /= km1;
    /* t_B2 = |X_c V_r|_F^2 / (k-1) */
    double t_B2 = 0.0;
    for (int j = 0; j < k; ++j)
        for (int l = 0; l < p; ++l) {
            double t = 0.0;
            for (int64_t a = 0; a < m; ++a) t += Xc[(int64_t)j * m + a] * Vr[a * p + l];
            t_B2 += t * t;
        }
    t_B2 /= km1;
    /* G_tens[j, l1, l2] = sum_a X_c[j,a] V_r[a,l1] V_r[a,l2];  |G_tens|_F^2 */
    double gt2 = 0.0;
    for (int j = 0; j < k; ++j)
        for (int l1 = 0; l1 < p; ++l1)
            for (int l2 = 0; l2 < p; ++l2) {
                double t = 0.0;
                for (int64_t a = 0; a < m; ++a)
                    t += Xc[(int64_t)j * m + a] * Vr[a * p + l1] * Vr[a * p + l2];
                gt2 += t * t;
            }
    double t_B, t_null;
    int64_t q = m - p;
    if (variant == ORC_VARIANT_HAAR) {
        double h = 0.0;
        for (int j = 0; j < k; ++j)
            for (int64_t a = 0; a < m; ++a)
                h += Xc[(int64_t)j * m + a] * Xc[(int64_t)j * m + a] * (1.0 - dP[a]);
        t_B = tau - 2.0 * h / km1 + gt2 / km1;
        t_null = (q > 0) ? (t_A + 2.0 * t_B) / (double)(q + 2) : 0.0;
    } else {
        t_B = tau - 2.0 * t_B2 + gt2 / km1;
        t_null = (q > 0) ? (t_A + 2.0 * t_B) / (double)q : 0.0;
    }
    double kappa = fabs(0.5 * (t_range + t_null) + 0.5 * tau);
    terms[T_TAU] = tau; terms[T_RANGE] = t_range; terms[T_A] = t_A; terms[T_B2] = t_B2;
    terms[T_GT2] = gt2; terms[T_B] = t_B; terms[T_NULL] = t_null; terms[T_KAPPA] = kappa;
    free(dP); free(Vr); free(Vfull); free(s);
    return p;
}

/* ------------------------------------------------------------------------- */
/* Exact mode (Theorem 1): Sigma = X_c^T X_c/(k-1) (m x m); Sigma = W diag(v)  */
/* W^T with v descending; C = W^T W^{o2}; K = |1/2 v^T (C^{o2} 1) + 1/2 sum v|. */
/* W (m x m) and v (m) are returned when non-NULL so the naive form can reuse  */
/* the very same eigenbasis.                                                   */
/* ------------------------------------------------------------------------- */
double orc_exact_patch(int k, int64_t m, const double *Xc, double *W_out, double *v_out) {
    double *S = (double *)xmalloc(sizeof(double) * (size_t)(m * m));
    double *W = (double *)xmalloc(sizeof(double) * (size_t)(m * m));
    double *v = (double *)xmalloc(sizeof(double) * (size_t)m);
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = 0; b < m; ++b) {
            double t = 0.0;
            for (int j = 0; j < k; ++j) t += Xc[(int64_t)j * m + a] * Xc[(int64_t)j * m + b];
            S[a * m + b] = t / (double)(k - 1);
        }
    orc_jacobi_eigh((int)m, S, v, W, 200);
    double acc = 0.0, trace = 0.0;
    for (int64_t s = 0; s < m; ++s) {
        double rowsum = 0.0;
        for (int64_t l = 0; l < m; ++l) {
            double c = 0.0; /* C[s,l] = sum_i W[i,s] W[i,l]^2 */
            for (int64_t i = 0; i < m; ++i) c += W[i * m + s] * W[i * m + l] * W[i * m + l];
            rowsum += c * c;
        }
        acc += v[s] * rowsum;
        trace += v[s];
    }
    if (W_out) memcpy(W_out, W, sizeof(double) * (size_t)(m * m));
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)m);
    free(S); free(W); free(v);
    return fabs(0.5 * acc + 0.5 * trace);
}

/* H H^T with H = [W^{(2)} | W^{(x)}] built column by column (eq. H): the m   */
/* squared columns w_l o w_l, then w_j o w_l for every pair j < l.            */
void orc_hht(int64_t m, const double *W, double *HHt) {
    int64_t ncols = m + m * (m - 1) / 2;
    double *H = (double *)xmalloc(sizeof(double) * (size_t)(m * ncols));
    int64_t col = 0;
    for (int64_t l = 0; l < m; ++l, ++col)
        for (int64_t i = 0; i < m; ++i) H[i * ncols + col] = W[i * m + l] * W[i * m + l];
    for (int64_t j = 0; j < m; ++j)
        for (int64_t l = j + 1; l < m; ++l, ++col)
            for (int64_t i = 0; i < m; ++i) H[i * ncols + col] = W[i * m + j] * W[i * m + l];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) {
            double t = 0.0;
            for (int64_t c = 0; c < ncols; ++c) t += H[i * ncols + c] * H[j * ncols + c];
            HHt[i * m + j] = t;
        }
    free(H);
}

/* The original estimator K = |tr(-H H^T Sigma)| (eq. curvature) with H built */
/* explicitly from the eigenbasis W of Sigma (the O(m^4) route).              */
double orc_naive_patch(int k, int64_t m, const double *Xc, const double *W) {
    double *S = (double *)xmalloc(sizeof(double) * (size_t)(m * m));
    double *HHt = (double *)xmalloc(sizeof(double) * (size_t)(m * m));
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = 0; b < m; ++b) {
            double t = 0.0;
            for (int j = 0; j < k; ++j) t += Xc[(int64_t)j * m + a] * Xc[(int64_t)j * m + b];
            S[a * m + b] = t / (double)(k - 1);
        }
    orc_hht(m, W, HHt);
    double tr = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) tr += -HHt[i * m + j] * S[j * m + i];
    free(S); free(HHt);
    return fabs(tr);
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 per-point loop.  mode 0 = Fast (variant/route as orc_fast_patch),   */
/* mode 1 = Exact (Theorem 1).  idx: n x k neighbour lists.  terms (optional) */
/* n x T_NTERMS (Fast only), lam (optional) n x k.                            */
/* ------------------------------------------------------------------------- */
int orc_curvature(const void *X, int elt, int64_t n, int64_t m, int k, const int32_t *idx,
                  const int64_t *rows, int64_t nrows, int mode, int variant, int route,
                  double *kappa, double *terms, double *lam, int nthreads) {
    int64_t nq = rows ? nrows : n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < nq; ++r) {
        int64_t i = rows ? rows[r] : r;
        double *Xc = (double *)xmalloc(sizeof(double) * (size_t)k * (size_t)m);
        center_patch_typed(X, elt, m, idx + i * k, k, Xc);
        (void)n;
        if (mode == 1) {
            kappa[r] = orc_exact_patch(k, m, Xc, NULL, NULL);
        } else {
            double t[T_NTERMS];
            double *lm = (double *)xmalloc(sizeof(double) * (size_t)k);
            orc_fast_patch(k, m, Xc, variant, route, t, lm, NULL);
            kappa[r] = t[T_KAPPA];
            if (terms) memcpy(terms + r * T_NTERMS, t, sizeof(t));
            if (lam) memcpy(lam + r * k, lm, sizeof(double) * (size_t)k);
            free(lm);
        }
        free(Xc);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Reference gradient by FP64 central differences of F(X) = sum_i K_i with    */
/* the neighbour lists frozen: dF/dX[ci,ca] ~ (F(X + h e) - F(X - h e)) / 2h. */
/* Only points whose patch contains row ci change, so only they are re-run.   */
/* ------------------------------------------------------------------------- */
int orc_grad_fd(const double *X, int64_t n, int64_t m, int k, const int32_t *idx,
                int variant, int route, const int64_t *ci, const int64_t *ca, int64_t ncoords,
                const double *h, double *out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t c = 0; c < ncoords; ++c) {
        int64_t row = ci[c], col = ca[c];
        double *Xc = (double *)xmalloc(sizeof(double) * (size_t)k * (size_t)m);
        double *Xrows = (double *)xmalloc(sizeof(double) * (size_t)k * (size_t)m);
        int32_t *loc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)k);
        double *lm = (double *)xmalloc(sizeof(double) * (size_t)k);
        double fsum[2] = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            int hit = -1;
            for (int j = 0; j < k; ++j)
                if (idx[i * k + j] == row) { hit = j; break; }
            if (hit < 0) continue;
            /* gather the patch rows into a private buffer, then perturb */
            for (int j = 0; j < k; ++j) {
                memcpy(Xrows + (int64_t)j * m, X + (int64_t)idx[i * k + j] * m, sizeof(double) * (size_t)m);
                loc[j] = j;
            }
            for (int sgn = 0; sgn < 2; ++sgn) {
                double delta = (sgn == 0) ? h[c] : -h[c];
                for (int j = 0; j < k; ++j)
                    if (idx[i * k + j] == row) Xrows[(int64_t)j * m + col] = X[row * m + col] + delta;
                orc_center_patch(Xrows, m, loc, k, Xc);
                double t[T_NTERMS];
                orc_fast_patch(k, m, Xc, variant, route, t, lm, NULL);
                fsum[sgn] += t[T_KAPPA];
            }
        }
        out[c] = (fsum[0] - fsum[1]) / (2.0 * h[c]);
        free(Xc); free(Xrows); free(loc); free(lm);
    }
    return 0;
}
