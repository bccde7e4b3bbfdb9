// jacobi.cu - Step 3 (eq. svd_cov; Alg. 1 SVD_p): eigendecomposition of the
// k x k patch Gram G = X_c X_c^T = U diag(s^2) U^T, whose top p eigenpairs give
// the truncated SVD X_c = U_p diag(s) V_r^T (V_r = X_c^T U_p diag(s)^-1).
//
// Parallel-order (round-robin) two-sided Jacobi.  A round pairs every index
// once (the circle method: index kp-1 fixed, the others rotating), so its kp/2
// plane rotations touch disjoint row/column pairs and commute.  Per round:
//   1. the table threads compute each pair's rotation from the current 2 x 2
//      block: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
//      sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c (the rotation zeroing
//      a_pq); pairs with |a_pq| <= eps sqrt(|a_pp a_qq|) are skipped (eps =
//      2^-22 in FP32, 2^-50 in FP64; before an FP64 refinement the caller's
//      pre_eps), and the
//      rotating pairs are compacted into the round's table (late sweeps are
//      cheap because few pairs still rotate);
//   2. A <- A J (each thread walks one row over its share of the pairs),
//   3. A <- J^T A (one column per thread), a_pq := 0 for rotated pairs,
//   4. U <- U J.
// kp - 1 rounds form a sweep; a sweep without any rotation ends the solve.
// One CTA of JT threads per patch keeps 4x more warps resident than one warp
// per patch at the same shared-memory footprint (A and U with row stride
// kp + 1 so column walks are bank-conflict free), which the latency-bound
// updates need.  The sweep count is capped; the cap sets
// MECUCO_ERR_NOT_CONVERGED in the device status word and keeps the current
// eigenpairs - it never traps.  Real = float (plain form) or double.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

template <typename Real>
struct JacobiEps;
template <>
struct JacobiEps<float> {
    static __host__ __device__ __forceinline__ float rel() { return 2.384185791015625e-07f; }  // 2^-22
};
template <>
struct JacobiEps<double> {
    static __host__ __device__ __forceinline__ double rel() { return 8.8817841970012523e-16; }  // 2^-50
};

constexpr int JT = 128;  // threads per patch

template <typename Real>
__global__ void __launch_bounds__(JT)
jacobi_kernel(const float *__restrict__ G, int k, int64_t np, int max_sweeps, Real eps, float *__restrict__ sigma,
              float *__restrict__ U, DevCounters *ctr) {
    extern __shared__ __align__(16) unsigned char jsm[];
    const int kp = (k + 1) & ~1;
    const int h = kp / 2;
    const int ld = kp + 1;
    Real *A = reinterpret_cast<Real *>(jsm);
    Real *V = A + (size_t)kp * ld;
    Real *tc = V + (size_t)kp * ld;  // [h] cosines
    Real *ts = tc + h;               // [h] sines
    int *tp = reinterpret_cast<int *>(ts + h);  // [h] p
    int *tq = tp + h;                           // [h] q
    __shared__ int s_rot;
    __shared__ int s_act;  // rotations in the current round (compacted table length)

    const int tid = threadIdx.x;
    const int64_t patch = blockIdx.x;
    const float *g = G + patch * (int64_t)k * k;
    for (int e = tid; e < kp * kp; e += JT) {
        int r = e / kp, c = e % kp;
        A[r * ld + c] = (r < k && c < k) ? (Real)g[r * k + c] : (Real)0;
        V[r * ld + c] = (r == c) ? (Real)1 : (Real)0;
    }
    if (tid == 0) { s_rot = 0; s_act = 0; }
    __syncthreads();
    // thread -> (line, pair group) for the row/column/U walks: kp lines, JT/kp groups
    const int groups = JT / kp > 0 ? JT / kp : 1;
    const int line = tid % kp;
    const int grp = tid / kp;
    const bool walker = tid < kp * groups;

    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps; ++sweep) {
        for (int round = 0; round < kp - 1; ++round) {
            if (tid < h) {
                int a, b;
                if (tid == 0) { a = kp - 1; b = round; }
                else { a = (round + tid) % (kp - 1); b = (round + kp - 1 - tid) % (kp - 1); }
                const int p = a < b ? a : b, q = a < b ? b : a;
                const Real app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
                if (fabs(apq) > eps * sqrt(fabs(app * aqq)) && apq != (Real)0) {
                    const Real tau = (aqq - app) / (2 * apq);
                    const Real t = (tau >= 0 ? (Real)1 : (Real)-1) / (fabs(tau) + sqrt((Real)1 + tau * tau));
                    const Real c = (Real)1 / sqrt((Real)1 + t * t);
                    // rotations of one round commute: keep only those that rotate, in any order
                    const int slot = atomicAdd(&s_act, 1);
                    tc[slot] = c; ts[slot] = t * c; tp[slot] = p; tq[slot] = q;
                }
            }
            __syncthreads();
            const int nact = s_act;
            const int per = (nact + groups - 1) / groups;
            const int i0 = grp * per, i1 = min(nact, i0 + per);
            // A <- A J (thread walks row `line`)
            if (walker && line < kp) {
                Real *row = A + line * ld;
#pragma unroll 4
                for (int i = i0; i < i1; ++i) {
                    const int p = tp[i], q = tq[i];
                    const Real c = tc[i], s = ts[i];
                    const Real x = row[p], y = row[q];
                    row[p] = c * x - s * y;
                    row[q] = s * x + c * y;
                }
            }
            __syncthreads();
            // A <- J^T A (thread walks column `line`), U <- U J (row `line`)
            if (walker && line < kp) {
                Real *urow = V + line * ld;
#pragma unroll 4
                for (int i = i0; i < i1; ++i) {
                    const int p = tp[i], q = tq[i];
                    const Real c = tc[i], s = ts[i];
                    const Real x = A[p * ld + line], y = A[q * ld + line];
                    A[p * ld + line] = c * x - s * y;
                    A[q * ld + line] = s * x + c * y;
                    const Real u = urow[p], w = urow[q];
                    urow[p] = c * u - s * w;
                    urow[q] = s * u + c * w;
                }
            }
            __syncthreads();
            if (tid < nact) {
                A[tp[tid] * ld + tq[tid]] = 0;
                A[tq[tid] * ld + tp[tid]] = 0;
            }
            if (tid == 0) { s_rot += nact; s_act = 0; }
            __syncthreads();
        }
        const int rot = s_rot;
        __syncthreads();
        if (tid == 0) s_rot = 0;
        __syncthreads();
        if (rot == 0) { converged = true; break; }
    }
    // sort eigenpairs (indices < k) descending by rank counting
    float *sg = sigma + patch * (int64_t)k;
    float *u = U + patch * (int64_t)k * k;
    for (int i = tid; i < k; i += JT) {
        const Real di = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const Real dj = A[j * ld + j];
            rank += (dj > di) || (dj == di && j < i);
        }
        sg[rank] = (float)di;
        for (int r = 0; r < k; ++r) u[r * k + rank] = (float)V[r * ld + i];
    }
    if (tid == 0) {
        atomicMax(&ctr->jacobi_max_sweeps, (unsigned long long)(converged ? sweep : max_sweeps));
        if (!converged) {
            atomicAdd(&ctr->jacobi_not_converged, 1ull);
            atomicOr(&ctr->status, (unsigned)DEV_NOT_CONVERGED);
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 refinement of an FP32 eigendecomposition (one step of the iterative
// refinement for symmetric eigenproblems of Ogita & Aishima, Japan J. Indust.
// Appl. Math. 35 (2018)), every product and sum in FP64.  With X the k x k
// eigenvector estimate from the FP32 sweeps and A = G in FP64:
//   R = I - X^T X,   S = X^T A X,   lam_i = S_ii / (1 - R_ii),
//   E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta,
//   E_ij = R_ij / 2 otherwise (and on the diagonal),   X' = X + X E.
// From FP32-accurate X (~2^-23) one step gives eigenvectors accurate to the
// square of that, i.e. to FP64 level, and re-orthogonalises them.  The
// products X^T X and X^T A X are symmetric (upper triangles only), and the
// correction X E, of relative size ~2^-23, is formed in FP32: 2k^3 FP64 FMA per
// patch.  delta =
// 2^-18 max|lam| treats eigenvalues closer than the FP32 estimate can resolve
// as a cluster (only orthogonalised).  With rel != 0 the cluster test is
// relative to the pair itself, |lam_i - lam_j| <= 2^-18 max(|lam_i|, |lam_j|):
// for a Gram whose FP32 eigenpairs are accurate to a few ulps relative to
// each eigenvalue (a nearly diagonal Gram, as in the adjoint's rotated basis),
// where the absolute test would lump all small eigenvalues into one cluster.  One CTA (RT threads) per patch; results
// re-sorted descending.
// ---------------------------------------------------------------------------
constexpr int RT = 256;

__global__ void __launch_bounds__(RT)
jacobi_refine64_kernel(const float *__restrict__ G, int k, int rel, float *__restrict__ sigma, float *__restrict__ U) {
    extern __shared__ __align__(16) unsigned char rsm[];
    const int ld = k + 1;
    double *A = reinterpret_cast<double *>(rsm);  // [k][ld]
    double *X = A + (size_t)k * ld;                 // [k][ld]
    double *T = X + (size_t)k * ld;                 // A X, then X E
    double *S = T + (size_t)k * ld;                 // X^T A X
    double *Rm = S + (size_t)k * ld;                // I - X^T X, then E
    double *lam = Rm + (size_t)k * ld;              // [k]
    __shared__ double s_lmax;
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const float *g = G + pt * (int64_t)k * k;
    float *u = U + pt * (int64_t)k * k;
    const int kk = k * k;
    for (int e = tid; e < kk; e += RT) {
        const int r = e / k, c = e % k;
        A[r * ld + c] = (double)g[e];
        X[r * ld + c] = (double)u[e];
    }
    __syncthreads();
    // T = A X (every entry)
    for (int e = tid; e < kk; e += RT) {
        const int r = e / k, c = e % k;
        double t = 0.0;
        for (int j = 0; j < k; ++j) t = fma(A[r * ld + j], X[j * ld + c], t);
        T[r * ld + c] = t;
    }
    // Rm = I - X^T X (upper triangle: both products are symmetric)
    for (int e = tid; e < kk; e += RT) {
        const int r = e / k, c = e % k;
        if (c < r) continue;
        double q = 0.0;
        for (int j = 0; j < k; ++j) q = fma(X[j * ld + r], X[j * ld + c], q);
        Rm[r * ld + c] = (r == c ? 1.0 : 0.0) - q;
    }
    __syncthreads();
    // S = X^T T (upper triangle)
    for (int e = tid; e < kk; e += RT) {
        const int r = e / k, c = e % k;
        if (c < r) continue;
        double t = 0.0;
        for (int j = 0; j < k; ++j) t = fma(X[j * ld + r], T[j * ld + c], t);
        S[r * ld + c] = t;
    }
    __syncthreads();
    if (tid < k) lam[tid] = S[tid * ld + tid] / (1.0 - Rm[tid * ld + tid]);
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(lam[i]));
        s_lmax = mx;
    }
    __syncthreads();
    const double delta = 3.814697265625e-06 * s_lmax;  // 2^-18 max|lam|
    // E (FP32: |E| ~ the FP32 eigenvector error, so X E rounded in FP32 is far below
    // FP64-level error in X + X E); X as FP32 (exact: it came from FP32)
    float *Ef = reinterpret_cast<float *>(T);       // [k][ld]
    float *Xf = Ef + (size_t)k * ld;                 // [k][ld]
    __syncthreads();
    for (int e = tid; e < kk; e += RT) {
        const int i = e / k, j = e % k;
        const int a = i < j ? i : j, b = i < j ? j : i;
        const double rij = Rm[a * ld + b];
        const double sij = S[a * ld + b];
        double v;
        const double dij = rel ? 3.814697265625e-06 * fmax(fabs(lam[i]), fabs(lam[j])) : delta;
        if (i == j || fabs(lam[i] - lam[j]) <= dij) v = 0.5 * rij;
        else v = (sij + lam[j] * rij) / (lam[j] - lam[i]);
        Ef[i * ld + j] = (float)v;
        Xf[i * ld + j] = (float)X[i * ld + j];
    }
    __syncthreads();
    // X' = X + X E (FP32), into X (as double) for the write-back
    for (int e = tid; e < kk; e += RT) {
        const int r = e / k, c = e % k;
        float t = 0.f;
        for (int j = 0; j < k; ++j) t = fmaf(Xf[r * ld + j], Ef[j * ld + c], t);
        X[r * ld + c] = (double)Xf[r * ld + c] + (double)t;
    }
    __syncthreads();
    // write back, columns re-sorted by lam descending
    float *sg = sigma + pt * (int64_t)k;
    for (int i = tid; i < k; i += RT) {
        int rank = 0;
        for (int j = 0; j < k; ++j) rank += (lam[j] > lam[i]) || (lam[j] == lam[i] && j < i);
        sg[rank] = (float)lam[i];
        for (int r = 0; r < k; ++r) u[r * k + rank] = (float)X[r * ld + i];
    }
}

size_t refine64_smem_bytes(int k) { return (size_t)5 * k * (k + 1) * sizeof(double) + (size_t)k * sizeof(double); }

size_t jacobi_smem_bytes(int k, int fp64) {
    const int kp = (k + 1) & ~1;
    const size_t real = fp64 ? sizeof(double) : sizeof(float);
    return (size_t)2 * kp * (kp + 1) * real + (size_t)kp * real + (size_t)kp * sizeof(int);
}

cudaError_t launch_jacobi(const float *G, int k, int64_t np, int fp64, int max_sweeps, float *sigma, float *U,
                          DevCounters *ctr, cudaStream_t s, float pre_eps) {
    if (np <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    cudaError_t e;
    if (fp64 == 1 || fp64 == 3) {
        // FP32 sweeps, then one FP64 refinement step (3: relative cluster test)
        const size_t smem = jacobi_smem_bytes(k, 0);
        e = cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<float><<<(unsigned)np, JT, smem, s>>>(G, k, np, max_sweeps, pre_eps, sigma, U, ctr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const size_t rs = refine64_smem_bytes(k);
        e = cudaFuncSetAttribute(jacobi_refine64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
        if (e != cudaSuccess) return e;
        jacobi_refine64_kernel<<<(unsigned)np, RT, rs, s>>>(G, k, fp64 == 3, sigma, U);
        return cudaGetLastError();
    }
    const size_t smem = jacobi_smem_bytes(k, fp64);
    if (fp64 == 2) {
        e = cudaFuncSetAttribute(jacobi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<double><<<(unsigned)np, JT, smem, s>>>(G, k, np, max_sweeps, JacobiEps<double>::rel(), sigma,
                                                             U, ctr);
    } else {
        e = cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<float><<<(unsigned)np, JT, smem, s>>>(G, k, np, max_sweeps, JacobiEps<float>::rel(), sigma, U,
                                                            ctr);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
