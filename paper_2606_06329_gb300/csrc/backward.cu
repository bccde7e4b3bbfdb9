// backward.cu - adjoint of the Fast-mode estimator: d(sum_i g_i K_i)/dX with the
// neighbour lists frozen (K_i from eqs. tnull, tA, tB, fast_curv; Alg. 1).
//
// Per point the forward is a function of the patch moments G = X_c X_c^T,
// R = X_c 1, M (third moments), Q (Haar) and of the eigenpairs (s_l^2, u_l) of
// G (see the estimator kernel).  With W = U_p diag(s)^-1, S_j = W^T M_j W,
// A_jl = (S_j)_ll, xd_j = R_j - sum_l A_jl, gt2 = sum_j |S_j|_F^2,
// h = sum_l w_l^T Q w_l, c = 1/q (printed) or 1/(q+2) (Haar), km1 = k - 1 and
// f = (t_range + t_null)/2 + tau/2, K = |f|, g~ = g sign(f):
//   dA_jl   = g~ (A_jl - c xd_j) / km1          dR_j = g~ c xd_j / km1
//   dgt2    = g~ c / km1                        dh   = -2 g~ c / km1     (Haar)
//   dtau    = g~ (1/2 - c) (printed) or g~ (1/2 + c) (Haar)
//   dS_j    = 2 dgt2 S_j + diag(dA_j.)
//   dM_j    = W dS_j W^T,   dW += 2 M_j W dS_j,   dQ = dh W W^T,  dW += 2 dh Q W
//   ds2_l   = dtau/km1 - (1/2) s_l^-3 u_l^T dw_l,  du_l = dw_l / s_l   (l < p)
//   dG      = U (diag(ds2) + F o (U^T dU)) U^T (symmetrised), F_ij = 1/(s_j^2 - s_i^2)
// (the derivative of a symmetric eigendecomposition).  Back to the patch:
//   dX_c[i,a] = 2 (dG x_a)_i + dR_i + x_a^T C_i x_a
//               + 2 w_a (dQ x_a)_i + 2 X_c[i,a] x_a^T dQ x_a            (Haar)
// with x_a = X_c[:, a], w_a = sum_j X_c[j,a]^2 and C_i[r][t] = dM[i,r,t] +
// dM[r,i,t] + dM[t,i,r] (the fully symmetric use of M), then the centring
// adjoint dX_p = dX_c - 1 (1^T dX_c)/k and a scatter-add into dX rows idx[i,:].
// Degenerate eigenvalue pairs make F unbounded; the difference is clamped at
// 2^-40 max|s^2| in magnitude (the derivative there is not defined).
//
// Conditioning.  With s_min/s_max = 1e-3 the small eigenpairs of an FP32 Gram
// carry relative errors near eps (s_max/s_min)^2 = 1e-1 and the s^-3 terms of
// the adjoint amplify them.  K is invariant under any orthogonal rotation
// Z = U0^T X_c of the point axis (tau, t_range, t_A, |G_tens|^2 and the Haar
// sum are sums of squares over j), so the adjoint works on the rotated patch:
// U0 = eigenvectors of the plain FP32 Gram (held fixed: K does not depend on
// it; refined (Ogita-Aishima step), since a U0 that is not orthogonal to FP32 rounding
// perturbs the patch), the moments of Z (whose Gram is nearly diagonal, error
// near eps s_max/s_min) and the eigenpairs of that Gram; the formulas above
// give dZ, and dX_c = U0 dZ.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

constexpr int BW_SMEM_FLOATS = 5 * 64 * 65;

// k-space adjoint: one CTA (256 threads) per point.  Outputs per point:
// dG (k x k), dR (k), dQ (k x k, Haar only), C (k x k x k) as described above.
__global__ void __launch_bounds__(256)
adjoint_kspace_kernel(const float *__restrict__ sigma, const float *__restrict__ U, const float *__restrict__ M,
                      const float *__restrict__ R, const float *__restrict__ Q, const float *__restrict__ gk, int k,
                      int64_t m, int variant, float rank_eps, float *__restrict__ dG, float *__restrict__ dR, float *__restrict__ dQ,
                      float *__restrict__ Cout, float *__restrict__ dMbuf) {
    extern __shared__ float bsm[];
    float(*Ws)[65] = reinterpret_cast<float(*)[65]>(bsm);             // W[r][l]
    float(*Mj)[65] = reinterpret_cast<float(*)[65]>(bsm + 64 * 65);   // M_j, later scratch
    float(*Bs)[65] = reinterpret_cast<float(*)[65]>(bsm + 2 * 64 * 65);  // M_j W
    float(*Sb)[65] = reinterpret_cast<float(*)[65]>(bsm + 3 * 64 * 65);  // S_j, then dS_j
    float(*dW)[65] = reinterpret_cast<float(*)[65]>(bsm + 4 * 64 * 65);  // accumulated dW
    __shared__ float Adiag[64], xd[64], sg[64];
    __shared__ double red[8][3];
    __shared__ float s_scal[8];
    __shared__ int s_p;
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const float *u = U + pt * (int64_t)k * k;
    const float *D = M + pt * m3_pair_floats_d(k);
    if (tid < k) sg[tid] = sigma[pt * k + tid];
    __syncthreads();
    if (tid == 0) {
        int pmax = k - 1;
        if ((int64_t)pmax > m) pmax = (int)m;
        const float s0 = fmaxf(sg[0], 0.f);
        int rank = 0;
        for (int l = 0; l < k; ++l) rank += (sg[l] > rank_eps * s0) && (sg[l] > 0.f);
        s_p = rank < pmax ? rank : pmax;
    }
    __syncthreads();
    const int p = s_p;
    for (int e = tid; e < 64 * 64; e += 256) {
        const int r = e >> 6, l = e & 63;
        Ws[r][l] = (r < k && l < p) ? u[r * k + l] * rsqrtf(sg[l]) : 0.f;
        dW[r][l] = 0.f;
    }
    __syncthreads();
    const double km1 = (double)(k - 1);
    const int64_t q = m - p;
    const double cnull = q > 0 ? 1.0 / (double)(variant == MECUCO_FAST_HAAR ? q + 2 : q) : 0.0;
    // ---- forward recompute: A, xd, gt2, h, tau -> f
    double acc_range = 0.0, acc_gt2 = 0.0, acc_A = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < k; ++j) {
            for (int e = tid; e < k * k; e += 256) {
                const int r = e / k, t = e % k;
                const int a = j < r ? j : r, b = j < r ? r : j;
                Mj[r][t] = D[(int64_t)pair_index(a, b, k) * k + t];
            }
            __syncthreads();
            // Bs = M_j W (k x p)
            for (int e = tid; e < k * p; e += 256) {
                const int r = e / p, l = e % p;
                float t = 0.f;
                for (int c = 0; c < k; ++c) t = fmaf(Mj[r][c], Ws[c][l], t);
                Bs[r][l] = t;
            }
            __syncthreads();
            // Sb = W^T Bs (p x p)
            for (int e = tid; e < p * p; e += 256) {
                const int l1 = e / p, l2 = e % p;
                float t = 0.f;
                for (int r = 0; r < k; ++r) t = fmaf(Ws[r][l1], Bs[r][l2], t);
                Sb[l1][l2] = t;
            }
            __syncthreads();
            if (pass == 0) {
                float part = 0.f;
                for (int e = tid; e < p * p; e += 256) { const float v = Sb[e / p][e % p]; part += v * v; }
                acc_gt2 += part;
                if (tid < 32) {
                    float sa = 0.f, s2 = 0.f;
                    for (int l = tid; l < p; l += 32) { const float a = Sb[l][l]; sa += a; s2 += a * a; }
                    sa = warp_sum(sa);
                    s2 = warp_sum(s2);
                    if (tid == 0) {
                        acc_range += s2;
                        const float x = R[pt * k + j] - sa;
                        xd[j] = x;
                        acc_A += (double)x * x;
                    }
                }
                __syncthreads();
            } else {
                // dS_j = 2 dgt2 S_j + diag(dA_j.)  (in place)
                const float dg2 = s_scal[0], ga = s_scal[1], gc = s_scal[2];
                for (int e = tid; e < p * p; e += 256) {
                    const int l1 = e / p, l2 = e % p;
                    float v = 2.f * dg2 * Sb[l1][l2];
                    if (l1 == l2) v += ga * (Sb[l1][l1] - gc * xd[j]);
                    Sb[l1][l2] = v;
                }
                __syncthreads();
                // dW += 2 Bs dS_j   (k x p)
                for (int e = tid; e < k * p; e += 256) {
                    const int r = e / p, l = e % p;
                    float t = 0.f;
                    for (int c = 0; c < p; ++c) t = fmaf(Bs[r][c], Sb[c][l], t);
                    dW[r][l] += 2.f * t;
                }
                // Mj <- W dS_j  (k x p), then dM_j = (W dS_j) W^T (k x k) to global
                for (int e = tid; e < k * p; e += 256) {
                    const int r = e / p, l = e % p;
                    float t = 0.f;
                    for (int c = 0; c < p; ++c) t = fmaf(Ws[r][c], Sb[c][l], t);
                    Mj[r][l] = t;
                }
                __syncthreads();
                float *dMj = dMbuf + (pt * (int64_t)k + j) * k * k;
                for (int e = tid; e < k * k; e += 256) {
                    const int r = e / k, t = e % k;
                    float v = 0.f;
                    for (int l = 0; l < p; ++l) v = fmaf(Mj[r][l], Ws[t][l], v);
                    dMj[e] = v;
                }
                __syncthreads();
            }
        }
        if (pass == 0) {
            // reduce gt2; h (Haar); f and the scalar adjoints
            double v0 = acc_gt2;
            for (int o = 16; o > 0; o >>= 1) v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            if ((tid & 31) == 0) red[tid >> 5][0] = v0;
            __syncthreads();
            double hsum = 0.0;
            if (variant == MECUCO_FAST_HAAR) {
                const float *qm = Q + pt * (int64_t)k * k;
                double part = 0.0;
                for (int e = tid; e < k * p; e += 256) {
                    const int r = e / p, l = e % p;
                    float t = 0.f;
                    for (int c = 0; c < k; ++c) t = fmaf(qm[r * k + c], Ws[c][l], t);
                    part += (double)Ws[r][l] * t;
                }
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if ((tid & 31) == 0) red[tid >> 5][1] = part;
                __syncthreads();
                for (int w = 0; w < 8; ++w) hsum += red[w][1];
            }
            if (tid == 0) {
                double gt2 = 0.0;
                for (int w = 0; w < 8; ++w) gt2 += red[w][0];
                double tau = 0.0;
                for (int l = 0; l < p; ++l) tau += (double)sg[l];
                tau /= km1;
                const double t_range = acc_range / km1, t_A = acc_A / km1;
                double t_null = 0.0;
                if (q > 0) {
                    const double tB = (variant == MECUCO_FAST_HAAR) ? tau - 2.0 * hsum / km1 + gt2 / km1
                                                                     : -tau + gt2 / km1;
                    t_null = (t_A + 2.0 * tB) * cnull;
                }
                const double f = 0.5 * (t_range + t_null) + 0.5 * tau;
                const double g = (double)gk[pt] * (f > 0.0 ? 1.0 : (f < 0.0 ? -1.0 : 0.0));
                s_scal[0] = (float)(g * cnull / km1);                        // dgt2
                s_scal[1] = (float)(g / km1);                                // scale of dA
                s_scal[2] = (float)cnull;                                    // c
                s_scal[3] = (float)(g * (variant == MECUCO_FAST_HAAR ? 0.5 + cnull : 0.5 - cnull));  // dtau
                s_scal[4] = (float)(variant == MECUCO_FAST_HAAR ? -2.0 * g * cnull / km1 : 0.0);    // dh
                s_scal[5] = (float)(g * cnull / km1);                        // dR scale
            }
            __syncthreads();
            if (tid < k) dR[pt * k + tid] = s_scal[5] * xd[tid];
        }
    }
    // ---- Haar: dQ = dh W W^T, dW += 2 dh Q W
    const float dh = s_scal[4];
    if (variant == MECUCO_FAST_HAAR) {
        const float *qm = Q + pt * (int64_t)k * k;
        for (int e = tid; e < k * k; e += 256) {
            const int r = e / k, t = e % k;
            float v = 0.f;
            for (int l = 0; l < p; ++l) v = fmaf(Ws[r][l], Ws[t][l], v);
            dQ[pt * (int64_t)k * k + e] = dh * v;
        }
        for (int e = tid; e < k * p; e += 256) {
            const int r = e / p, l = e % p;
            float v = 0.f;
            for (int c = 0; c < k; ++c) v = fmaf(qm[r * k + c], Ws[c][l], v);
            dW[r][l] += 2.f * dh * v;
        }
    }
    __syncthreads();
    // ---- eigen adjoint.  dU (k x k) in Bs, ds2 (k) in xd
    const float dtau = s_scal[3];
    for (int e = tid; e < k * k; e += 256) {
        const int r = e / k, l = e % k;
        Bs[r][l] = (l < p) ? dW[r][l] * rsqrtf(sg[l]) : 0.f;
    }
    if (tid < k) {
        const int l = tid;
        float v = 0.f;
        if (l < p) {
            float uw = 0.f;
            for (int r = 0; r < k; ++r) uw = fmaf(u[r * k + l], dW[r][l], uw);
            const float s = sqrtf(sg[l]);
            v = dtau / (float)km1 - 0.5f * uw / (sg[l] * s);
        }
        Adiag[l] = v;
    }
    __syncthreads();
    // Sb = U^T dU (k x k); then K = diag(ds2) + F o Sb (in Sb)
    float smax = 0.f;
    for (int l = 0; l < k; ++l) smax = fmaxf(smax, fabsf(sg[l]));
    const float floor_gap = smax * 9.094947017729282e-13f;  // 2^-40 max|s^2|
    for (int e = tid; e < k * k; e += 256) {
        const int i = e / k, j = e % k;
        float t = 0.f;
        for (int r = 0; r < k; ++r) t = fmaf(u[r * k + i], Bs[r][j], t);
        float v;
        if (i == j) {
            v = Adiag[i];
        } else {
            float dif = sg[j] - sg[i];
            if (fabsf(dif) < floor_gap) dif = dif < 0.f ? -floor_gap : floor_gap;
            v = t / dif;
        }
        Mj[i][j] = v;
    }
    __syncthreads();
    // dG = U K U^T (symmetrised): Bs = U K, then dG = Bs U^T
    for (int e = tid; e < k * k; e += 256) {
        const int r = e / k, j = e % k;
        float t = 0.f;
        for (int c = 0; c < k; ++c) t = fmaf(u[r * k + c], Mj[c][j], t);
        Bs[r][j] = t;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += 256) {
        const int r = e / k, t = e % k;
        float a = 0.f, b = 0.f;
        for (int c = 0; c < k; ++c) {
            a = fmaf(Bs[r][c], u[t * k + c], a);
            b = fmaf(Bs[t][c], u[r * k + c], b);
        }
        dG[pt * (int64_t)k * k + e] = 0.5f * (a + b);
    }
    // ---- C_i[r][t] = dM[i,r,t] + dM[r,i,t] + dM[t,i,r]
    __syncthreads();
    const float *dMp = dMbuf + pt * (int64_t)k * k * k;
    float *Cp = Cout + pt * (int64_t)k * k * k;
    for (int e = tid; e < k * k * k; e += 256) {
        const int i = e / (k * k), r = (e / k) % k, t = e % k;
        Cp[e] = dMp[(i * k + r) * k + t] + dMp[(r * k + i) * k + t] + dMp[(t * k + i) * k + r];
    }
}

// Patch-space adjoint and scatter: one CTA (256 threads) per point; the patch
// is re-gathered, centred and rotated (Z = U0^T X_c) in 32-column chunks;
// thread (column c, row group) forms dZ for its rows, dX_c = U0 dZ, the
// centring adjoint subtracts the column mean, and the result is atomically
// added to dX rows idx[pt, :].
template <typename T>
__global__ void __launch_bounds__(256)
adjoint_patch_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx, int k,
                     int variant, const float *__restrict__ rot, const float *__restrict__ dG,
                     const float *__restrict__ dR,
                     const float *__restrict__ dQ, const float *__restrict__ C, float *__restrict__ dX, int64_t ldd) {
    constexpr int CH = 32;
    extern __shared__ float psm[];
    float(*Xs)[CH + 1] = reinterpret_cast<float(*)[CH + 1]>(psm);
    float(*Ys)[CH + 1] = reinterpret_cast<float(*)[CH + 1]>(psm + 64 * (CH + 1));
    float *sdG = psm + 2 * 64 * (CH + 1);
    float *sdQ = sdG + 64 * 64;
    float(*Us)[65] = reinterpret_cast<float(*)[65]>(sdQ + 64 * 64);
    __shared__ int rows[64];
    const int tid = threadIdx.x;
    const int64_t pt = blockIdx.x;
    const int kk = k * k;
    if (tid < k) {
        int r = idx[pt * k + tid];
        rows[tid] = (r < 0 || (int64_t)r >= N) ? 0 : r;
    }
    for (int e = tid; e < kk; e += 256) {
        sdG[e] = dG[pt * (int64_t)kk + e];
        sdQ[e] = (variant == MECUCO_FAST_HAAR) ? dQ[pt * (int64_t)kk + e] : 0.f;
    }
    load_rotation(rot + pt * (int64_t)kk, k, Us);
    __syncthreads();
    const float *Cp = C + pt * (int64_t)kk * k;
    const float *dRp = dR + pt * k;
    const int c = tid % CH, grp = tid / CH;  // 8 row groups
    for (int64_t a0 = 0; a0 < m; a0 += CH) {
        for (int e = tid; e < 64 * CH; e += 256) {
            const int j = e / CH, cc = e % CH;
            Xs[j][cc] = (j < k && a0 + cc < m) ? load_elem(X + (int64_t)rows[j] * ld + a0 + cc) : 0.f;
        }
        __syncthreads();
        if (tid < CH) {
            double sd = 0.0;  // centred values rounded once from FP64, as in the rotated moments
            for (int j = 0; j < k; ++j) sd += (double)Xs[j][tid];
            const double md = sd / (double)k;
            for (int j = 0; j < k; ++j) Xs[j][tid] = (float)((double)Xs[j][tid] - md);
        }
        __syncthreads();
        rotate_rows<CH / 4>(Xs, Us, k, tid >> 6, tid & 63);
        float wa = 0.f, xqx = 0.f;
        if (variant == MECUCO_FAST_HAAR) {
            for (int j = 0; j < k; ++j) wa = fmaf(Xs[j][c], Xs[j][c], wa);
            for (int r = 0; r < k; ++r) {
                float t = 0.f;
                for (int s2 = 0; s2 < k; ++s2) t = fmaf(sdQ[r * k + s2], Xs[s2][c], t);
                xqx = fmaf(Xs[r][c], t, xqx);
            }
        }
        for (int i = grp; i < k; i += 8) {
            float v = dRp[i];
            float g = 0.f, qv = 0.f;
            for (int r = 0; r < k; ++r) {
                g = fmaf(sdG[i * k + r], Xs[r][c], g);
                qv = fmaf(sdQ[i * k + r], Xs[r][c], qv);
            }
            v += 2.f * g;
            if (variant == MECUCO_FAST_HAAR) v += 2.f * wa * qv + 2.f * Xs[i][c] * xqx;
            const float *Ci = Cp + (int64_t)i * kk;
            float cq = 0.f;
            for (int r = 0; r < k; ++r) {
                float t = 0.f;
                for (int s2 = 0; s2 < k; ++s2) t = fmaf(__ldg(Ci + r * k + s2), Xs[s2][c], t);
                cq = fmaf(Xs[r][c], t, cq);
            }
            Ys[i][c] = v + cq;
        }
        __syncthreads();
        unrotate_rows<CH / 4>(Ys, Us, k, tid >> 6, tid & 63);
        if (tid < CH && a0 + tid < m) {
            float s = 0.f;
            for (int j = 0; j < k; ++j) s += Ys[j][tid];
            const float mean = s / (float)k;
            for (int j = 0; j < k; ++j) atomicAdd(dX + (int64_t)rows[j] * ldd + a0 + tid, Ys[j][tid] - mean);
        }
        __syncthreads();
    }
}

cudaError_t launch_adjoint(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld, const int32_t *idx,
                           int k, int64_t np, int variant, float rank_eps, const float *rot, const float *sigma,
                           const float *U, const float *M, const float *R, const float *Q, const float *gk, float *dG,
                           float *dR, float *dQ, float *C, float *dMbuf, float *dX, int64_t ldd, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    const size_t smem = BW_SMEM_FLOATS * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(adjoint_kspace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adjoint_kspace_kernel<<<(unsigned)np, 256, smem, s>>>(sigma, U, M, R, Q, gk, k, m, variant, rank_eps, dG, dR, dQ, C,
                                                          dMbuf);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t psmem = (size_t)(2 * 64 * 33 + 2 * 64 * 64 + 64 * 65) * sizeof(float);
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(adjoint_patch_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)psmem);
        if (e != cudaSuccess) return e;
        adjoint_patch_kernel<<<(unsigned)np, 256, psmem, s>>>((const __nv_bfloat16 *)X, N, m, ld, idx, k, variant, rot,
                                                              dG, dR, dQ, C, dX, ldd);
    } else {
        e = cudaFuncSetAttribute(adjoint_patch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
        if (e != cudaSuccess) return e;
        adjoint_patch_kernel<<<(unsigned)np, 256, psmem, s>>>((const float *)X, N, m, ld, idx, k, variant, rot, dG, dR,
                                                              dQ, C, dX, ldd);
    }
    return cudaGetLastError();
}

}  // namespace mecuco
