// jacobi.cu - Step 3 (eq. svd_cov; Alg. 1 SVD_p): eigendecomposition of the
// k x k patch Gram G = X_c X_c^T = U diag(s^2) U^T, whose top p eigenpairs give
// the truncated SVD X_c = U_p diag(s) V_r^T (V_r = X_c^T U_p diag(s)^-1).
//
// One warp per patch, parallel-order (round-robin) two-sided Jacobi.  A round
// pairs every index once (the circle method: index kp-1 fixed, the others
// rotating), so its kp/2 plane rotations touch disjoint row/column pairs and
// commute; each lane computes one rotation from the current 2 x 2 block
// (tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1 + t^2), s = t c, the rotation that zeroes a_pq), then the warp
// applies A <- A J (lanes over rows), A <- J^T A (lanes over columns) and
// U <- U J.  kp - 1 rounds form a sweep in which every pair is visited once.
// A rotation is skipped when |a_pq| <= eps sqrt(|a_pp a_qq|) (relative
// criterion); a sweep with no rotation ends the solve.  The sweep count is
// capped; hitting the cap sets MECUCO_ERR_NOT_CONVERGED in the device status
// word and keeps the current (approximate) eigenpairs - it never traps.
// Matrices live in shared memory with row stride kp + 1 so column walks are
// bank-conflict free.  Real = float (plain form) or double (chosen form).
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

template <typename Real>
struct JacobiEps;
template <>
struct JacobiEps<float> {
    static __device__ __forceinline__ float rel() { return 2.384185791015625e-07f; }  // 2^-22
};
template <>
struct JacobiEps<double> {
    static __device__ __forceinline__ double rel() { return 8.8817841970012523e-16; }  // 2^-50
};

template <typename Real>
__global__ void jacobi_kernel(const float *__restrict__ G, int k, int64_t np, int max_sweeps,
                              float *__restrict__ sigma, float *__restrict__ U, DevCounters *ctr,
                              int warps_per_block) {
    extern __shared__ __align__(16) unsigned char jsm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kp = (k + 1) & ~1;
    const int ld = kp + 1;
    Real *A = reinterpret_cast<Real *>(jsm) + (size_t)w * 2 * kp * ld;
    Real *V = A + (size_t)kp * ld;
    const int64_t patch = (int64_t)blockIdx.x * warps_per_block + w;
    if (patch >= np) return;
    const float *g = G + patch * (int64_t)k * k;
    for (int e = lane; e < kp * kp; e += 32) {
        int r = e / kp, c = e % kp;
        A[r * ld + c] = (r < k && c < k) ? (Real)g[r * k + c] : (Real)0;
        V[r * ld + c] = (r == c) ? (Real)1 : (Real)0;
    }
    __syncwarp();
    const Real eps = JacobiEps<Real>::rel();
    const unsigned full = 0xffffffffu;
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps; ++sweep) {
        int rotations = 0;
        for (int round = 0; round < kp - 1; ++round) {
            int pi = 0, qi = 0;
            Real c = 1, s = 0;
            if (lane < kp / 2) {
                int a, b;
                if (lane == 0) { a = kp - 1; b = round; }
                else { a = (round + lane) % (kp - 1); b = (round + kp - 1 - lane) % (kp - 1); }
                pi = a < b ? a : b;
                qi = a < b ? b : a;
                Real app = A[pi * ld + pi], aqq = A[qi * ld + qi], apq = A[pi * ld + qi];
                Real thr = eps * sqrt(fabs(app * aqq));
                if (fabs(apq) > thr && apq != (Real)0) {
                    Real tau = (aqq - app) / (2 * apq);
                    Real t = (tau >= 0 ? (Real)1 : (Real)-1) / (fabs(tau) + sqrt((Real)1 + tau * tau));
                    c = (Real)1 / sqrt((Real)1 + t * t);
                    s = t * c;
                    ++rotations;
                }
            }
            __syncwarp();
            // A <- A J : lanes walk rows
            for (int i = 0; i < kp / 2; ++i) {
                Real cc = __shfl_sync(full, c, i), ss = __shfl_sync(full, s, i);
                if (ss == (Real)0) continue;
                int P = __shfl_sync(full, pi, i), Q = __shfl_sync(full, qi, i);
                for (int r = lane; r < kp; r += 32) {
                    Real arp = A[r * ld + P], arq = A[r * ld + Q];
                    A[r * ld + P] = cc * arp - ss * arq;
                    A[r * ld + Q] = ss * arp + cc * arq;
                }
            }
            __syncwarp();
            // A <- J^T A : lanes walk columns
            for (int i = 0; i < kp / 2; ++i) {
                Real cc = __shfl_sync(full, c, i), ss = __shfl_sync(full, s, i);
                if (ss == (Real)0) continue;
                int P = __shfl_sync(full, pi, i), Q = __shfl_sync(full, qi, i);
                for (int col = lane; col < kp; col += 32) {
                    Real apc = A[P * ld + col], aqc = A[Q * ld + col];
                    A[P * ld + col] = cc * apc - ss * aqc;
                    A[Q * ld + col] = ss * apc + cc * aqc;
                }
            }
            __syncwarp();
            if (lane < kp / 2 && s != (Real)0) {
                A[pi * ld + qi] = 0;
                A[qi * ld + pi] = 0;
            }
            // U <- U J
            for (int i = 0; i < kp / 2; ++i) {
                Real cc = __shfl_sync(full, c, i), ss = __shfl_sync(full, s, i);
                if (ss == (Real)0) continue;
                int P = __shfl_sync(full, pi, i), Q = __shfl_sync(full, qi, i);
                for (int r = lane; r < kp; r += 32) {
                    Real vrp = V[r * ld + P], vrq = V[r * ld + Q];
                    V[r * ld + P] = cc * vrp - ss * vrq;
                    V[r * ld + Q] = ss * vrp + cc * vrq;
                }
            }
            __syncwarp();
        }
        rotations = __reduce_add_sync(full, rotations);
        if (rotations == 0) { converged = true; break; }
    }
    // sort eigenpairs (indices < k) descending by rank counting
    float *sg = sigma + patch * (int64_t)k;
    float *u = U + patch * (int64_t)k * k;
    for (int i = lane; i < k; i += 32) {
        Real di = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            Real dj = A[j * ld + j];
            rank += (dj > di) || (dj == di && j < i);
        }
        sg[rank] = (float)di;
        for (int r = 0; r < k; ++r) u[r * k + rank] = (float)V[r * ld + i];
    }
    if (lane == 0) {
        atomicMax(&ctr->jacobi_max_sweeps, (unsigned long long)(converged ? sweep : max_sweeps));
        if (!converged) {
            atomicAdd(&ctr->jacobi_not_converged, 1ull);
            atomicOr(&ctr->status, (unsigned)DEV_NOT_CONVERGED);
        }
    }
}

cudaError_t launch_jacobi(const float *G, int k, int64_t np, int fp64, int max_sweeps,
                          float *sigma, float *U, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    const int kp = (k + 1) & ~1;
    const size_t per_warp = (size_t)2 * kp * (kp + 1) * (fp64 ? sizeof(double) : sizeof(float));
    const size_t budget = 200 * 1024;
    int wpb = (int)(budget / per_warp);
    if (wpb > 8) wpb = 8;
    if (wpb < 1) return cudaErrorInvalidValue;
    size_t smem = per_warp * wpb;
    dim3 grid((unsigned)((np + wpb - 1) / wpb)), block(32 * wpb);
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(jacobi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<double><<<grid, block, smem, s>>>(G, k, np, max_sweeps, sigma, U, ctr, wpb);
    } else {
        e = cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<float><<<grid, block, smem, s>>>(G, k, np, max_sweeps, sigma, U, ctr, wpb);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
