// basis.cu - tangent bases: the right singular vectors V_r = X_c^T U_p S^-1
// of each patch (Alg. 1 SVD_p; eq. svd_cov), expanded from the compact k-space
// form (U_p, s) that the eigensolve of the k x k Gram produces.
//
// One CTA (256 threads) per point.  The patch is re-gathered and centred in
// 32-column chunks; thread (column c, output column group) forms
// V[a, l] = sum_j X_c[j, a] U[j, l] / s_l for its columns and stores the chunk
// (m x d_out per point, l fastest) with consecutive threads on consecutive
// addresses.  Columns l >= p (numerical rank, as in the estimator) are zero.
// Column signs are fixed so that the largest-magnitude entry of U's column l
// (lowest j on ties) is positive.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

constexpr int TB_CH = 32;

template <typename T>
__global__ void __launch_bounds__(256)
tangent_basis_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx,
                     int k, const float *__restrict__ sigma, const float *__restrict__ U, int d_out,
                     float rank_eps, float *__restrict__ V, DevCounters *ctr) {
    __shared__ float Xs[64][TB_CH + 1];
    __shared__ float Us[64][65];  // U[j][l] * sign_l / s_l for l < d_out (0 for l >= p)
    __shared__ float scale[64];
    __shared__ int rows[64];
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const float *sg = sigma + pt * k;
    const float *u = U + pt * (int64_t)k * k;
    if (tid < k) {
        int r = idx[pt * k + tid];
        if (r < 0 || (int64_t)r >= N) { atomicOr(&ctr->status, (unsigned)DEV_INVALID); r = 0; }
        rows[tid] = r;
    }
    if (tid < 64) {
        float sc = 0.f;
        if (tid < d_out) {
            int pmax = k - 1;
            if ((int64_t)pmax > m) pmax = (int)m;
            const float s0 = fmaxf(sg[0], 0.f);
            int rank = 0;
            for (int l = 0; l < k; ++l) rank += (sg[l] > rank_eps * s0) && (sg[l] > 0.f);
            const int p = rank < pmax ? rank : pmax;
            if (tid < p) {
                float best = -1.f, sgn = 1.f;
                for (int j = 0; j < k; ++j) {
                    const float v = u[j * k + tid];
                    if (fabsf(v) > best) { best = fabsf(v); sgn = v < 0.f ? -1.f : 1.f; }
                }
                sc = sgn * rsqrtf(sg[tid]);
            }
        }
        scale[tid] = sc;
    }
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += 256) {
        const int j = e >> 6, l = e & 63;
        Us[j][l] = (j < k && l < d_out) ? u[j * k + l] * scale[l] : 0.f;
    }
    float *Vp = V + pt * m * (int64_t)d_out;
    for (int64_t a0 = 0; a0 < m; a0 += TB_CH) {
        __syncthreads();
        for (int e = tid; e < 64 * TB_CH; e += 256) {
            const int j = e / TB_CH, cc = e % TB_CH;
            Xs[j][cc] = (j < k && a0 + cc < m) ? load_elem(X + (int64_t)rows[j] * ld + a0 + cc) : 0.f;
        }
        __syncthreads();
        if (tid < TB_CH) {
            float s = 0.f;
            for (int j = 0; j < k; ++j) s += Xs[j][tid];
            const float mean = s / (float)k;
            for (int j = 0; j < k; ++j) Xs[j][tid] -= mean;
        }
        __syncthreads();
        const int ncol = (int)((m - a0) < TB_CH ? (m - a0) : TB_CH);
        const int nout = ncol * d_out;
        for (int e = tid; e < nout; e += 256) {
            const int cc = e / d_out, l = e % d_out;
            float v = 0.f;
            for (int j = 0; j < k; ++j) v = fmaf(Xs[j][cc], Us[j][l], v);
            Vp[(a0 + cc) * d_out + l] = v;
        }
    }
}

cudaError_t launch_tangent_basis(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                 const int32_t *idx, int k, int64_t np, const float *sigma, const float *U,
                                 int d_out, float rank_eps, float *V, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64 || d_out < 1 || d_out > k) return cudaErrorInvalidValue;
    if (dt == MECUCO_BF16)
        tangent_basis_kernel<<<(unsigned)np, 256, 0, s>>>((const __nv_bfloat16 *)X, N, m, ld, idx, k, sigma, U, d_out,
                                                          rank_eps, V, ctr);
    else
        tangent_basis_kernel<<<(unsigned)np, 256, 0, s>>>((const float *)X, N, m, ld, idx, k, sigma, U, d_out,
                                                          rank_eps, V, ctr);
    return cudaGetLastError();
}

// U_out = U0 V per point: one CTA (256 threads) per point.
__global__ void __launch_bounds__(256)
compose_rotation_kernel(const float *__restrict__ U0, const float *__restrict__ V, int k, float *__restrict__ U_out) {
    __shared__ float A[64][65], B[64][65];
    const int64_t pt = blockIdx.x;
    const int kk = k * k;
    for (int e = threadIdx.x; e < kk; e += 256) {
        A[e / k][e % k] = U0[pt * kk + e];
        B[e / k][e % k] = V[pt * kk + e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kk; e += 256) {
        const int r = e / k, l = e % k;
        float t = 0.f;
        for (int c = 0; c < k; ++c) t = fmaf(A[r][c], B[c][l], t);
        U_out[pt * kk + e] = t;
    }
}

cudaError_t launch_compose_rotation(const float *U0, const float *V, int k, int64_t np, float *U_out,
                                    cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    compose_rotation_kernel<<<(unsigned)np, 256, 0, s>>>(U0, V, k, U_out);
    return cudaGetLastError();
}

}  // namespace mecuco
