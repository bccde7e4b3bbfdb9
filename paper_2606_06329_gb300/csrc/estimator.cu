// estimator.cu - Step 4 (eqs. tnull, tA, tB, fast_curv; Alg. 1 Fast branch):
// the Fast-mode curvature from the patch moments and the eigenpairs of G.
//
// With X_c = U_p S V_r^T (U_p the top-p eigenvectors of G = X_c X_c^T, S the
// singular values) put W = U_p S^-1 (k x p), so V_r = X_c^T W.  Every term of
// Alg. 1 then lives in k-space:
//   tau     = sum_{l<p} s_l^2 / (k-1)
//   A_jl    = (X_c V_r^{o2})_jl = w_l^T M_j w_l,         M_j[r,t] = M[j,r,t]
//   t_range = sum_{j,l} A_jl^2 / (k-1)
//   X_c d_P = R - A 1_p                                   (d_P = 1 - V_r^{o2} 1)
//   t_A     = |R - A 1_p|^2 / (k-1)
//   G_tens[j] = W^T M_j W  (p x p),  |G_tens|_F^2 = sum_j |W^T M_j W|_F^2
//   |X_c V_r|_F^2 = |G W|_F^2, which is sum_{l<p} s_l^2 = (k-1) tau when U_p
//   holds eigenvectors of G, so the printed
//   t_B = tau - 2 tau + |G_tens|^2/(k-1);  t_null = (t_A + 2 t_B)/(m - p).
//   Given G (Ritz pairs of a randomised range finder, whose residuals G u_l -
//   s_l^2 u_l are not 0) |G W|_F^2 is computed instead.
//   Haar variant: sum_{j,a} X_c[j,a]^2 (1 - d_P[a]) = sum_l w_l^T Q w_l,
//   t_B^H = tau - 2 (that)/(k-1) + |G_tens|^2/(k-1), t_null^H = (t_A + 2 t_B^H)/(m - p + 2)
//   K = |(t_range + t_null)/2 + tau/2|.
// The diagonal of W^T M_j W is A_j., so one p x p product per j gives both.
// One CTA (256 threads) per point; for each j the slice M_j is read as k
// contiguous rows of the pair-major moment buffer, B = M_j W and
// S_j = W^T B are formed with 4 x 4 register blocks, and the scalar sums are
// reduced in double precision at the end.  M_j is symmetric (M[j][r][t] =
// M[j][t][r]), so the block's four rows of M_j at column c are read as row c,
// and every operand of the register blocks comes as one 16-byte shared load
// (rows padded to 68 floats): 3 shared wavefronts per warp and 16 FMAs instead
// of 8, which leaves the loops FMA-bound.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

constexpr int EST_LD = 68;  // row stride (floats): 16-byte rows for the vector loads
constexpr int EST_SMEM = 3 * 64 * EST_LD * (int)sizeof(float);

__global__ void __launch_bounds__(256)
estimator_kernel(const float *__restrict__ sigma, const float *__restrict__ U, const float *__restrict__ M,
                 const float *__restrict__ R, const float *__restrict__ Q, const float *__restrict__ Gm, int k,
                 int64_t m, int variant, float rank_eps, float *__restrict__ kappa, float *__restrict__ lambda_out,
                 float *__restrict__ s_out, DevCounters *ctr) {
    extern __shared__ __align__(16) float esm[];
    float(*Ws)[EST_LD] = reinterpret_cast<float(*)[EST_LD]>(esm);  // W[r][l], zero for l >= p
    float(*Mj)[EST_LD] = reinterpret_cast<float(*)[EST_LD]>(esm + 64 * EST_LD);
    float(*Bs)[EST_LD] = reinterpret_cast<float(*)[EST_LD]>(esm + 2 * 64 * EST_LD);
    __shared__ float Adiag[64];
    __shared__ int s_p;
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const float *sg = sigma + pt * k;
    const float *u = U + pt * (int64_t)k * k;
    if (tid == 0) {
        int pmax = k - 1;
        if ((int64_t)pmax > m) pmax = (int)m;
        float s0 = fmaxf(sg[0], 0.f);
        // numerical rank: eigenvalues above rank_eps * s_0 (the caller's threshold
        // for the accuracy of the Gram it solved)
        int rank = 0;
        for (int l = 0; l < k; ++l) rank += (sg[l] > rank_eps * s0) && (sg[l] > 0.f);
        s_p = rank < pmax ? rank : pmax;
        if (s_p < pmax) atomicAdd(&ctr->rank_deficient, 1ull);
    }
    __syncthreads();
    const int p = s_p;
    for (int e = tid; e < 64 * 64; e += 256) {
        int r = e >> 6, l = e & 63;
        float v = 0.f;
        if (r < k && l < p) v = u[r * k + l] * rsqrtf(sg[l]);
        Ws[r][l] = v;
    }
    const int bi = tid >> 4, bj = tid & 15;  // 4 x 4 block coordinates
    const float *D = M + pt * m3_pair_floats_d(k);
    // rows of M_j as 16-byte loads when k % 4 == 0: a warp takes rpw rows at a
    // time, lane = (row within the warp's rows, float4 within the row); the
    // split is fixed, so the loop over j does no index division
    const bool vec = (k & 3) == 0;
    const int q4 = k >> 2, rpw = vec ? 32 / q4 : 0;
    const int rr = vec ? (tid & 31) / q4 : 0, c4 = vec ? (tid & 31) - rr * q4 : 0;
    double acc_range = 0.0, acc_gt2 = 0.0, acc_A = 0.0;
    for (int j = 0; j < k; ++j) {
        // M_j[r][t] = D[pair(min(j,r), max(j,r))][t]
        if (vec) {
            if (rr < rpw)
                for (int r = (tid >> 5) * rpw + rr; r < k; r += 8 * rpw) {
                    const int a = j < r ? j : r, b = j < r ? r : j;
                    *reinterpret_cast<float4 *>(&Mj[r][4 * c4]) =
                        __ldg(reinterpret_cast<const float4 *>(D + (int64_t)pair_index(a, b, k) * k) + c4);
                }
        } else {
            for (int e = tid; e < k * k; e += 256) {
                int r = e / k, t = e % k;
                int a = j < r ? j : r, b = j < r ? r : j;
                Mj[r][t] = D[(int64_t)pair_index(a, b, k) * k + t];
            }
        }
        __syncthreads();
        // B = M_j W  (k x p); M_j[4 bi + i][c] = M_j[c][4 bi + i]
        if (4 * bi < k && 4 * bj < p) {
            float acc[4][4] = {};
            for (int c = 0; c < k; ++c) {
                const float4 m4 = *reinterpret_cast<const float4 *>(&Mj[c][4 * bi]);
                const float4 w4 = *reinterpret_cast<const float4 *>(&Ws[c][4 * bj]);
                const float mr[4] = {m4.x, m4.y, m4.z, m4.w}, wl[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(mr[i], wl[q], acc[i][q]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) Bs[4 * bi + i][4 * bj + q] = acc[i][q];
        }
        __syncthreads();
        // S_j = W^T B (p x p), blocks bi <= bj; diagonal entries -> Adiag
        if (bi <= bj && 4 * bi < p && 4 * bj < p) {
            float acc[4][4] = {};
            for (int r = 0; r < k; ++r) {
                const float4 w4 = *reinterpret_cast<const float4 *>(&Ws[r][4 * bi]);
                const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[r][4 * bj]);
                const float wl[4] = {w4.x, w4.y, w4.z, w4.w}, br[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(wl[i], br[q], acc[i][q]);
            }
            float part = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int l1 = 4 * bi + i, l2 = 4 * bj + q;
                    if (l1 >= p || l2 >= p || l1 > l2) continue;
                    float v = acc[i][q];
                    part += (l1 == l2 ? 1.f : 2.f) * v * v;
                    if (l1 == l2) Adiag[l1] = v;
                }
            acc_gt2 += part;
        }
        __syncthreads();
        if (tid < 32) {
            float sa = 0.f, s2 = 0.f;
            for (int l = tid; l < p; l += 32) { float a = Adiag[l]; sa += a; s2 += a * a; }
            sa = warp_sum(sa);
            s2 = warp_sum(s2);
            if (tid == 0) {
                acc_range += s2;
                float xd = R[pt * k + j] - sa;
                acc_A += (double)xd * xd;
            }
        }
        __syncthreads();
    }
    // Haar: h = sum_l w_l^T Q w_l
    double acc_h = 0.0;
    if (variant == MECUCO_FAST_HAAR) {
        const float *qm = Q + pt * (int64_t)k * k;
        for (int e = tid; e < k * p; e += 256) {
            int r = e / p, l = e % p;
            float t = 0.f;
            for (int c = 0; c < k; ++c) t = fmaf(qm[r * k + c], Ws[c][l], t);
            acc_h += (double)Ws[r][l] * t;
        }
    }
    // |G W|_F^2 (only with G given)
    double acc_b2 = 0.0;
    if (Gm) {
        const float *gm = Gm + pt * (int64_t)k * k;
        for (int e = tid; e < k * p; e += 256) {
            const int r = e / p, l = e % p;
            float t = 0.f;
            for (int c = 0; c < k; ++c) t = fmaf(gm[r * k + c], Ws[c][l], t);
            acc_b2 += (double)t * t;
        }
    }
    // block reduction of (acc_gt2, acc_h, acc_b2) and thread 0's (acc_range, acc_A)
    double v0 = acc_gt2, v1 = acc_h, v2 = acc_b2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    __shared__ double wred[8][3];
    if ((tid & 31) == 0) { wred[tid >> 5][0] = v0; wred[tid >> 5][1] = v1; wred[tid >> 5][2] = v2; }
    __syncthreads();
    if (tid == 0) {
        double gt2 = 0.0, h = 0.0, b2 = 0.0;
        for (int w = 0; w < 8; ++w) { gt2 += wred[w][0]; h += wred[w][1]; b2 += wred[w][2]; }
        const double km1 = (double)(k - 1);
        double tau = 0.0;
        for (int l = 0; l < p; ++l) tau += (double)sg[l];
        tau /= km1;
        const double t_range = acc_range / km1;
        const double t_A = acc_A / km1;
        const int64_t q = m - p;
        double t_null = 0.0;
        if (q > 0) {
            if (variant == MECUCO_FAST_HAAR) {
                double tB = tau - 2.0 * h / km1 + gt2 / km1;
                t_null = (t_A + 2.0 * tB) / (double)(q + 2);
            } else {
                const double t_B2 = Gm ? b2 / km1 : tau;  // |X_c V_r|_F^2 / (k-1)
                double tB = tau - 2.0 * t_B2 + gt2 / km1;
                t_null = (t_A + 2.0 * tB) / (double)q;
            }
        }
        kappa[pt] = (float)fabs(0.5 * (t_range + t_null) + 0.5 * tau);
    }
    if (lambda_out)
        for (int l = tid; l < k; l += 256)
            lambda_out[pt * k + l] = (l < p) ? fmaxf(sg[l], 0.f) / (float)(k - 1) : 0.f;
    if (s_out)
        for (int l = tid; l < k; l += 256) s_out[pt * k + l] = sqrtf(fmaxf(sg[l], 0.f));
}

cudaError_t launch_estimator(const float *sigma, const float *U, const float *M, const float *R,
                             const float *Q, int k, int64_t m, int64_t np, int variant, float rank_eps,
                             float *kappa, float *lambda_out, float *s_out, DevCounters *ctr,
                             cudaStream_t s, const float *G) {
    if (np <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(estimator_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EST_SMEM);
    if (e != cudaSuccess) return e;
    estimator_kernel<<<(unsigned)np, 256, EST_SMEM, s>>>(sigma, U, M, R, Q, G, k, m, variant, rank_eps, kappa,
                                                         lambda_out, s_out, ctr);
    return cudaGetLastError();
}

}  // namespace mecuco
