// moments.cu - Steps 2-3 (Sec. 3 Step 2; Alg. 1 Fast branch: centring, and the
// k x k Gram that replaces SVD_p(X_c), eq. svd_cov) plus the patch moments the
// one-pass estimator needs.  Plain FP32 on the CUDA cores.
//
// Every estimator term of Alg. 1 is a k-space function of three moments of
// the centred patch X_c (derivation in the estimator kernel):
//   G = X_c X_c^T,  R = X_c 1_m,  M[j,r,t] = sum_a X_c[j,a] X_c[r,a] X_c[t,a],
// and, for the Haar-consistent variant, Q = X_c diag(c) X_c^T with
// c_a = sum_j X_c[j,a]^2.  Centring is per column (x_ja - mean_j x_ja), so both
// kernels stream the patch through shared memory in column chunks, centre each
// chunk and accumulate, reading every neighbour row once per kernel.
//
// Both kernels optionally take a per-point orthogonal k x k matrix U0 (row r,
// column l) and then accumulate the moments of Z = U0^T X_c instead of X_c.
// Every estimator term is invariant under such a rotation of the point axis
// (tau, t_range, t_A, |G_tens|^2 and the Haar sum are sums of squares over j),
// and with U0 the eigenvectors of a first Gram the rotated Gram is nearly
// diagonal, so its small eigenvalues come out with small relative error in
// FP32 (error of order eps s_max/s_min instead of eps (s_max/s_min)^2).  The
// adjoint uses this.
#include "common.cuh"
#include "kernels.h"

namespace mecuco {

// A neighbour index outside [0, N) is read as row 0 and flagged, never followed.
__device__ __forceinline__ int checked_row(int r, int64_t N, DevCounters *ctr) {
    if (r < 0 || (int64_t)r >= N) {
        atomicOr(&ctr->status, (unsigned)DEV_INVALID);
        return 0;
    }
    return r;
}

// ---------------------------------------------------------------------------
// Gram kernel: one CTA (256 threads) per point, chunks of GCH columns.  Thread
// (bi, bj) of a 16 x 16 grid owns the 4 x 4 block rows 4bi.., cols 4bj.. of G
// and of Q (full blocks; k <= 64).
// ---------------------------------------------------------------------------
constexpr int GCH = 64;

template <typename T, bool ROT>
__global__ void __launch_bounds__(256)
patch_gram_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx,
                  int k, int64_t p0, const float *__restrict__ rot, float *__restrict__ G, float *__restrict__ R,
                  float *__restrict__ Q, DevCounters *ctr) {
    __shared__ float Xs[64][GCH + 1];
    __shared__ float Us[ROT ? 64 : 1][65];
    __shared__ float cw[GCH];
    __shared__ int rows[64];
    const int tid = threadIdx.x;
    const int64_t p = p0 + blockIdx.x;
    if (tid < k) rows[tid] = checked_row(idx[p * k + tid], N, ctr);
    if (tid >= k && tid < 64) rows[tid] = -1;
    if (ROT) load_rotation(rot + (p - p0) * (int64_t)k * k, k, Us);
    const int bi = tid >> 4, bj = tid & 15;
    const bool active = (4 * bi < k) && (4 * bj < k);
    float g[4][4], qq[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { g[i][j] = 0.f; qq[i][j] = 0.f; }
    float rsum = 0.f;
    __syncthreads();
    for (int64_t a0 = 0; a0 < m; a0 += GCH) {
        for (int lin = tid; lin < 64 * GCH; lin += 256) {
            int j = lin / GCH, c = lin % GCH;
            float v = 0.f;
            if (j < k && a0 + c < m) v = load_elem(X + (int64_t)rows[j] * ld + a0 + c);
            Xs[j][c] = v;
        }
        __syncthreads();
        if (tid < GCH) {
            float w = 0.f;
            if (ROT) {
                // centred values rounded once from FP64 (the rotated form feeds the adjoint)
                double sd = 0.0;
                for (int j = 0; j < k; ++j) sd += (double)Xs[j][tid];
                const double md = sd / (double)k;
                for (int j = 0; j < k; ++j) {
                    const float v = (float)((double)Xs[j][tid] - md);
                    Xs[j][tid] = v;
                    w = fmaf(v, v, w);
                }
            } else {
                float s = 0.f;
                for (int j = 0; j < k; ++j) s += Xs[j][tid];
                float mean = s / (float)k;
                for (int j = 0; j < k; ++j) {
                    float v = Xs[j][tid] - mean;
                    Xs[j][tid] = v;
                    w = fmaf(v, v, w);
                }
            }
            cw[tid] = w;
        }
        __syncthreads();
        if (ROT) rotate_rows<GCH / 4>(Xs, Us, k, tid >> 6, tid & 63);
        if (active) {
#pragma unroll 4
            for (int c = 0; c < GCH; ++c) {
                float xr[4], xt[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { xr[i] = Xs[4 * bi + i][c]; xt[i] = Xs[4 * bj + i][c]; }
                float w = cw[c];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float z = xr[i] * w;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        g[i][j] = fmaf(xr[i], xt[j], g[i][j]);
                        qq[i][j] = fmaf(z, xt[j], qq[i][j]);
                    }
                }
            }
        }
        if (tid < k)
            for (int c = 0; c < GCH; ++c) rsum += Xs[tid][c];
        __syncthreads();
    }
    const int64_t kk = (int64_t)k * k;
    if (active) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int r = 4 * bi + i, t = 4 * bj + j;
                if (r < k && t < k) {
                    G[(p - p0) * kk + (int64_t)r * k + t] = g[i][j];
                    if (Q) Q[(p - p0) * kk + (int64_t)r * k + t] = qq[i][j];
                }
            }
    }
    if (tid < k) R[(p - p0) * k + tid] = rsum;
}

cudaError_t launch_patch_gram(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                              const int32_t *idx, int k, int64_t p0, int64_t np, const float *rot,
                              float *G, float *R, float *Q, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    const bool bf = dt == MECUCO_BF16;
    const __nv_bfloat16 *Xb = (const __nv_bfloat16 *)X;
    const float *Xf = (const float *)X;
    if (bf && rot)
        patch_gram_kernel<__nv_bfloat16, true><<<(unsigned)np, 256, 0, s>>>(Xb, N, m, ld, idx, k, p0, rot, G, R, Q, ctr);
    else if (bf)
        patch_gram_kernel<__nv_bfloat16, false><<<(unsigned)np, 256, 0, s>>>(Xb, N, m, ld, idx, k, p0, rot, G, R, Q, ctr);
    else if (rot)
        patch_gram_kernel<float, true><<<(unsigned)np, 256, 0, s>>>(Xf, N, m, ld, idx, k, p0, rot, G, R, Q, ctr);
    else
        patch_gram_kernel<float, false><<<(unsigned)np, 256, 0, s>>>(Xf, N, m, ld, idx, k, p0, rot, G, R, Q, ctr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Third moments.  Work items (j, Rb, Tb), Rb >= j/8, Tb >= Rb, over
// nb = ceil(k/8) blocks of 8 cover every sorted triple j <= r <= t; an item
// accumulates acc[r][t] = M[j][8Rb + r][8Tb + t].  Grid (points, item groups of
// 256); each thread owns one item (64 accumulators) and streams the patch in
// MCH-column chunks stored column-major (rows of a column contiguous,
// zero-padded to a multiple of 8) so the eight r and eight t values load as two
// float4 each.
//
// Storage is pair-major: D[pair(a, b)][c] = M[a][b][c] for a <= b and every c,
// pair(a, b) = a k - a (a - 1)/2 + (b - a), so the slice M_j (k x k) is the k
// contiguous rows pair(min(j, r), max(j, r)), r = 0..k-1.  Each sorted triple
// a <= b <= c is written to its three images D[pair(a,b)][c], D[pair(a,c)][b]
// and D[pair(b,c)][a] (the same value; coinciding images rewrite it).
// ---------------------------------------------------------------------------
int m3_items(int k) {
    int nb = (k + 7) / 8, n = 0;
    for (int j = 0; j < k; ++j) {
        int r0 = j / 8;
        n += (nb - r0) * (nb - r0 + 1) / 2;
    }
    return n;
}

void m3_build_items(int k, int32_t *items) {
    int nb = (k + 7) / 8, n = 0;
    for (int j = 0; j < k; ++j)
        for (int rb = j / 8; rb < nb; ++rb)
            for (int tb = rb; tb < nb; ++tb) items[n++] = j | (rb << 8) | (tb << 16);
}

constexpr int MCH = 32;

template <typename T, bool ROT>
__global__ void __launch_bounds__(256)
patch_m3_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, const int32_t *__restrict__ idx,
                int k, int64_t p0, const float *__restrict__ rot, float *__restrict__ M,
                const int32_t *__restrict__ items, int nitems, DevCounters *ctr) {
    __shared__ __align__(16) float Xs[MCH][64];
    __shared__ float Us[ROT ? 64 : 1][65];
    __shared__ int rows[64];
    const int tid = threadIdx.x;
    const int64_t p = p0 + blockIdx.x;
    const int item = blockIdx.y * 256 + tid;
    const int kp = ((k + 7) / 8) * 8;
    if (tid < 64) rows[tid] = (tid < k) ? checked_row(idx[p * k + tid], N, ctr) : -1;
    if (ROT) load_rotation(rot + (p - p0) * (int64_t)k * k, k, Us);
    int j = 0, rb = 0, tb = 0;
    const bool active = item < nitems;
    if (active) {
        int code = items[item];
        j = code & 0xff; rb = (code >> 8) & 0xff; tb = (code >> 16) & 0xff;
    }
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[r][t] = 0.f;
    __syncthreads();
    for (int64_t a0 = 0; a0 < m; a0 += MCH) {
        // load rows into column-major chunk: element (row jj, column c) -> Xs[c][jj]
        for (int lin = tid; lin < kp * MCH; lin += 256) {
            int jj = lin / MCH, c = lin % MCH;
            float v = 0.f;
            if (jj < k && a0 + c < m) v = load_elem(X + (int64_t)rows[jj] * ld + a0 + c);
            Xs[c][jj] = v;
        }
        __syncthreads();
        if (tid < MCH) {
            if (ROT) {
                double sd = 0.0;
                for (int jj = 0; jj < k; ++jj) sd += (double)Xs[tid][jj];
                const double md = sd / (double)k;
                for (int jj = 0; jj < k; ++jj) Xs[tid][jj] = (float)((double)Xs[tid][jj] - md);
            } else {
                float s = 0.f;
                for (int jj = 0; jj < k; ++jj) s += Xs[tid][jj];
                float mean = s / (float)k;
                for (int jj = 0; jj < k; ++jj) Xs[tid][jj] -= mean;
            }
        }
        __syncthreads();
        if (ROT) rotate_cols<MCH / 4>(Xs, Us, k, tid >> 6, tid & 63);
        if (active) {
            for (int c = 0; c < MCH; ++c) {
                const float4 *col = reinterpret_cast<const float4 *>(&Xs[c][0]);
                float4 r0 = col[2 * rb], r1 = col[2 * rb + 1];
                float4 t0 = col[2 * tb], t1 = col[2 * tb + 1];
                float xj = Xs[c][j];
                float z[8] = {xj * r0.x, xj * r0.y, xj * r0.z, xj * r0.w,
                              xj * r1.x, xj * r1.y, xj * r1.z, xj * r1.w};
                float xt[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int t = 0; t < 8; ++t) acc[r][t] = fmaf(z[r], xt[t], acc[r][t]);
            }
        }
        __syncthreads();
    }
    if (active) {
        float *D = M + (p - p0) * m3_pair_floats_d(k);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int rr = 8 * rb + r;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int tt = 8 * tb + t;
                if (rr < j || tt < rr || tt >= k) continue;  // sorted triples j <= rr <= tt < k
                float v = acc[r][t];
                D[(int64_t)pair_index(j, rr, k) * k + tt] = v;
                D[(int64_t)pair_index(j, tt, k) * k + rr] = v;
                D[(int64_t)pair_index(rr, tt, k) * k + j] = v;
            }
        }
    }
}

cudaError_t launch_patch_m3(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                            const int32_t *idx, int k, int64_t p0, int64_t np, const float *rot,
                            float *M, const int32_t *items, DevCounters *ctr, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (k > 64) return cudaErrorInvalidValue;
    int nitems = m3_items(k);
    dim3 grid((unsigned)np, (unsigned)((nitems + 255) / 256));  // (point, item group)
    const bool bf = dt == MECUCO_BF16;
    const __nv_bfloat16 *Xb = (const __nv_bfloat16 *)X;
    const float *Xf = (const float *)X;
    if (bf && rot)
        patch_m3_kernel<__nv_bfloat16, true><<<grid, 256, 0, s>>>(Xb, N, m, ld, idx, k, p0, rot, M, items, nitems, ctr);
    else if (bf)
        patch_m3_kernel<__nv_bfloat16, false><<<grid, 256, 0, s>>>(Xb, N, m, ld, idx, k, p0, rot, M, items, nitems, ctr);
    else if (rot)
        patch_m3_kernel<float, true><<<grid, 256, 0, s>>>(Xf, N, m, ld, idx, k, p0, rot, M, items, nitems, ctr);
    else
        patch_m3_kernel<float, false><<<grid, 256, 0, s>>>(Xf, N, m, ld, idx, k, p0, rot, M, items, nitems, ctr);
    return cudaGetLastError();
}

}  // namespace mecuco
