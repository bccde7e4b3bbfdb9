// rsvd.cu - randomised low-rank variant of the Fast mode's truncated SVD (the
// paper's future work, Sec. Conclusions: replace the truncated SVD by a
// randomised low-rank approximation).  In k-space the truncated SVD of a
// patch is the eigendecomposition of its Gram G = X_c X_c^T, so the range
// finder of Halko, Martinsson & Tropp (SIAM Rev. 53, 2011; Alg. 4.3 / 4.4)
// acts on G with a k x l Gaussian test matrix Omega (one matrix shared by all
// points, drawn by the caller, independent of the data):
//   Y = G Omega;  q times: Q = orth(Y), Y = G Q;  Q = orth(Y)   (k x l)
//   B = Q^T G Q (l x l) = V_B diag(sigma_B) V_B^T   (the existing Jacobi kernels)
//   U = Q V_B, keep the r largest: U_r (k x r), sigma_r.
// The estimator then runs unchanged with p = r: the eigenvalues past r are
// written as 0, below every rank threshold.  orth() is modified Gram-Schmidt
// applied twice; a column whose norm drops below 2^-20 of its norm before
// orthogonalisation (G has rank <= k - 1: its rows sum to zero) is set to 0
// and gives a zero eigenvalue in B.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

namespace {
constexpr int RS_T = 128;
constexpr int RS_LD = 65;

// orthonormalise the l columns of Y (k x l, row stride RS_LD) in place: two
// passes of modified Gram-Schmidt, column by column (each dot reduced over
// the four warps)
__device__ void mgs2(float (*Y)[RS_LD], int k, int l, float *red, float *nrm0) {
    const int tid = threadIdx.x;
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < l; ++j) {
            // norm before orthogonalisation (first pass only: the collapse test)
            if (pass == 0) {
                float t = 0.f;
                for (int r = tid; r < k; r += RS_T) t = fmaf(Y[r][j], Y[r][j], t);
                t = warp_sum(t);
                if ((tid & 31) == 0) red[tid >> 5] = t;
                __syncthreads();
                if (tid == 0) nrm0[j] = sqrtf(red[0] + red[1] + red[2] + red[3]);
                __syncthreads();
            }
            for (int i = 0; i < j; ++i) {
                float t = 0.f;
                for (int r = tid; r < k; r += RS_T) t = fmaf(Y[r][i], Y[r][j], t);
                t = warp_sum(t);
                if ((tid & 31) == 0) red[tid >> 5] = t;
                __syncthreads();
                const float d = red[0] + red[1] + red[2] + red[3];
                for (int r = tid; r < k; r += RS_T) Y[r][j] = fmaf(-d, Y[r][i], Y[r][j]);
                __syncthreads();
            }
            float t = 0.f;
            for (int r = tid; r < k; r += RS_T) t = fmaf(Y[r][j], Y[r][j], t);
            t = warp_sum(t);
            if ((tid & 31) == 0) red[tid >> 5] = t;
            __syncthreads();
            const float nj = sqrtf(red[0] + red[1] + red[2] + red[3]);
            const float inv = (nj > 9.5367431640625e-07f * nrm0[j] && nj > 0.f) ? 1.f / nj : 0.f;
            for (int r = tid; r < k; r += RS_T) Y[r][j] *= inv;
            if (inv == 0.f && tid == 0) nrm0[j] = 0.f;  // a collapsed column stays 0 in the second pass
            __syncthreads();
        }
    }
}

// out (k x l) = G (k x k) * In (k x l)
__device__ void gram_times(const float (*Gs)[RS_LD], const float (*In)[RS_LD], float (*Out)[RS_LD], int k, int l) {
    for (int e = threadIdx.x; e < k * l; e += RS_T) {
        const int r = e / l, c = e - r * l;
        float t = 0.f;
        for (int j = 0; j < k; ++j) t = fmaf(Gs[r][j], In[j][c], t);
        Out[r][c] = t;
    }
}
}  // namespace

__global__ void __launch_bounds__(RS_T)
rsvd_range_kernel(const float *__restrict__ G, int k, const float *__restrict__ omega, int l, int power,
                  float *__restrict__ Qout, float *__restrict__ Bout) {
    extern __shared__ float rsm[];  // three 64 x RS_LD blocks (dynamic: more than the 48 KB static limit)
    float(*Gs)[RS_LD] = reinterpret_cast<float(*)[RS_LD]>(rsm);
    float(*Y)[RS_LD] = reinterpret_cast<float(*)[RS_LD]>(rsm + 64 * RS_LD);
    float(*T)[RS_LD] = reinterpret_cast<float(*)[RS_LD]>(rsm + 2 * 64 * RS_LD);
    __shared__ float red[4], nrm0[64];
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const float *g = G + pt * (int64_t)k * k;
    for (int e = tid; e < k * k; e += RS_T) Gs[e / k][e % k] = g[e];
    for (int e = tid; e < k * l; e += RS_T) T[e / l][e % l] = omega[e];
    __syncthreads();
    gram_times(Gs, T, Y, k, l);  // Y = G Omega
    __syncthreads();
    for (int it = 0; it < power; ++it) {
        mgs2(Y, k, l, red, nrm0);
        gram_times(Gs, Y, T, k, l);  // T = G Q
        __syncthreads();
        for (int e = tid; e < k * l; e += RS_T) Y[e / l][e % l] = T[e / l][e % l];
        __syncthreads();
    }
    mgs2(Y, k, l, red, nrm0);  // Q
    gram_times(Gs, Y, T, k, l);  // T = G Q
    __syncthreads();
    float *q = Qout + pt * (int64_t)k * l;
    for (int e = tid; e < k * l; e += RS_T) q[e] = Y[e / l][e % l];
    // B = Q^T (G Q), symmetric: upper triangle mirrored
    float *b = Bout + pt * (int64_t)l * l;
    for (int e = tid; e < l * l; e += RS_T) {
        const int i = e / l, j = e - i * l;
        if (j < i) continue;
        float t = 0.f;
        for (int r = 0; r < k; ++r) t = fmaf(Y[r][i], T[r][j], t);
        b[i * l + j] = t;
        b[j * l + i] = t;
    }
}

// U (k x k per point, first r columns) = Q V_B, sigma (k) = the r largest
// eigenvalues of B then zeros
__global__ void __launch_bounds__(RS_T)
rsvd_compose_kernel(const float *__restrict__ Q, const float *__restrict__ sigB, const float *__restrict__ VB, int k,
                    int l, int r, float *__restrict__ sigma, float *__restrict__ U) {
    const int64_t pt = blockIdx.x;
    const float *q = Q + pt * (int64_t)k * l;
    const float *v = VB + pt * (int64_t)l * l;
    float *u = U + pt * (int64_t)k * k;
    for (int e = threadIdx.x; e < k * k; e += RS_T) {
        const int row = e / k, c = e - row * k;
        float t = 0.f;
        if (c < r)
            for (int j = 0; j < l; ++j) t = fmaf(q[row * l + j], v[j * l + c], t);
        u[e] = t;
    }
    for (int c = threadIdx.x; c < k; c += RS_T) sigma[pt * k + c] = c < r ? fmaxf(sigB[pt * l + c], 0.f) : 0.f;
}

cudaError_t launch_rsvd_range(const float *G, int k, int64_t np, const float *omega, int l, int power, float *Q,
                              float *B, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64 || l < 1 || l > k || power < 0) return cudaErrorInvalidValue;
    const int smem = 3 * 64 * RS_LD * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(rsvd_range_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    rsvd_range_kernel<<<(unsigned)np, RS_T, smem, s>>>(G, k, omega, l, power, Q, B);
    return cudaGetLastError();
}

cudaError_t launch_rsvd_compose(const float *Q, const float *sigB, const float *VB, int k, int l, int r, int64_t np,
                                float *sigma, float *U, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64 || l > k || r < 1 || r > l) return cudaErrorInvalidValue;
    rsvd_compose_kernel<<<(unsigned)np, RS_T, 0, s>>>(Q, sigB, VB, k, l, r, sigma, U);
    return cudaGetLastError();
}

}  // namespace mecuco
