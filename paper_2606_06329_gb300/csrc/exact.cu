// exact.cu - Exact mode (Theorem 1; eq. exact_curv): per point, the m x m
// covariance of the centred patch Sigma = X_c^T X_c / (k - 1), its
// eigendecomposition Sigma = W diag(v) W^T (v descending), C = W^T W^{o2}
// (C[s][l] = sum_i W[i][s] W[i][l]^2) and
//   K = | 1/2 sum_s v_s sum_l C[s][l]^2 + 1/2 sum_s v_s |.
// For m > k - 1, Sigma has a null space whose eigenbasis is not unique and K
// depends on the basis the eigensolver returns (the printed identity sums over
// every column of W); the entry point exports W for that reason.  m <= 64.
//
// Kernels: exact_cov_kernel (one CTA per point: gather + FP64 centring of the
// k x m patch in shared memory, Sigma in FP32 with FP64 accumulation of each
// entry) and exact_kappa_kernel (one CTA per point: C, its squared row sums
// and K from W and v); the eigensolve between them is launch_jacobi.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

template <typename T>
__global__ void __launch_bounds__(256)
exact_cov_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx, int k,
                 float *__restrict__ S, DevCounters *ctr) {
    __shared__ float Xs[64][65];  // [row j][column a]
    __shared__ int rows[64];
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const int mm = (int)m;
    if (tid < k) {
        int r = idx[pt * k + tid];
        if (r < 0 || (int64_t)r >= N) { atomicOr(&ctr->status, (unsigned)DEV_INVALID); r = 0; }
        rows[tid] = r;
    }
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += 256) {
        const int j = e >> 6, a = e & 63;
        Xs[j][a] = (j < k && a < mm) ? load_elem(X + (int64_t)rows[j] * ld + a) : 0.f;
    }
    __syncthreads();
    if (tid < mm) {
        double sd = 0.0;
        for (int j = 0; j < k; ++j) sd += (double)Xs[j][tid];
        const double md = sd / (double)k;
        for (int j = 0; j < k; ++j) Xs[j][tid] = (float)((double)Xs[j][tid] - md);
    }
    __syncthreads();
    const double inv = 1.0 / (double)(k - 1);
    float *Sp = S + pt * (int64_t)mm * mm;
    for (int e = tid; e < mm * mm; e += 256) {
        const int a = e / mm, b = e % mm;
        if (b < a) continue;
        double t = 0.0;
        for (int j = 0; j < k; ++j) t = fma((double)Xs[j][a], (double)Xs[j][b], t);
        const float v = (float)(t * inv);
        Sp[a * mm + b] = v;
        Sp[b * mm + a] = v;
    }
}

__global__ void __launch_bounds__(256)
exact_kappa_kernel(const float *__restrict__ v, const float *__restrict__ W, int m, float *__restrict__ kappa) {
    __shared__ float Ws[64][65];   // W[i][s]
    __shared__ float W2[64][65];   // W[i][l]^2
    __shared__ double part[256];
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const float *wp = W + pt * (int64_t)m * m;
    for (int e = tid; e < m * m; e += 256) {
        const float w = wp[e];
        Ws[e / m][e % m] = w;
        W2[e / m][e % m] = w * w;
    }
    __syncthreads();
    // thread -> entries (s, l) of C; accumulate v_s C[s][l]^2
    double acc = 0.0;
    for (int e = tid; e < m * m; e += 256) {
        const int s = e / m, l = e % m;
        float c = 0.f;
        for (int i = 0; i < m; ++i) c = fmaf(Ws[i][s], W2[i][l], c);
        acc += (double)v[pt * m + s] * (double)c * (double)c;
    }
    part[tid] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) part[tid] += part[tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        double tr = 0.0;
        for (int s = 0; s < m; ++s) tr += (double)v[pt * m + s];
        kappa[pt] = (float)fabs(0.5 * part[0] + 0.5 * tr);
    }
}

cudaError_t launch_exact_cov(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                             int k, int64_t np, float *S, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64 || m > 64) return cudaErrorInvalidValue;
    if (dt == MECUCO_BF16)
        exact_cov_kernel<<<(unsigned)np, 256, 0, s>>>((const __nv_bfloat16 *)X, N, m, ld, idx, k, S, ctr);
    else
        exact_cov_kernel<<<(unsigned)np, 256, 0, s>>>((const float *)X, N, m, ld, idx, k, S, ctr);
    return cudaGetLastError();
}

cudaError_t launch_exact_kappa(const float *v, const float *W, int m, int64_t np, float *kappa, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (m > 64) return cudaErrorInvalidValue;
    exact_kappa_kernel<<<(unsigned)np, 256, 0, s>>>(v, W, m, kappa);
    return cudaGetLastError();
}

}  // namespace mecuco
