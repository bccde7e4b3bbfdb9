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
//      2^-22 in FP32, 2^-50 in FP64; before a refinement step the caller's
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

// One rotation of a round's table, read by every walker as one 16-byte (FP32)
// or 32-byte (FP64) shared load: the kernel is bound by shared-memory
// wavefronts, and four separate table loads per rotation cost as many as its
// data accesses.
template <typename Real>
struct alignas(2 * sizeof(Real) + 2 * sizeof(int) > 16 ? 32 : 16) JRot {
    Real c, s;
    int p, q;
};

template <typename Real>
__global__ void __launch_bounds__(JT)
jacobi_kernel(const __grid_constant__ PatchSeg one, const PatchSeg *__restrict__ tab, int ntab, int max_sweeps,
              Real eps, DevCounters *ctr) {
    extern __shared__ __align__(16) unsigned char jsm[];
    int local;
    const PatchSeg &seg = find_seg(one, tab, ntab, (int)blockIdx.x, local);
    const int k = seg.k;
    const float *G = seg.G;
    float *sigma = seg.sig, *U = seg.U;
    const int kp = (k + 1) & ~1;
    const int h = kp / 2;
    const int ld = kp + 1;
    Real *A = reinterpret_cast<Real *>(jsm);
    Real *V = A + (size_t)kp * ld;
    // [h] rotations of the round, after A and V (rounded up to the entry alignment)
    JRot<Real> *rtab = reinterpret_cast<JRot<Real> *>(
        (reinterpret_cast<uintptr_t>(V + (size_t)kp * ld) + alignof(JRot<Real>) - 1) & ~(uintptr_t)(alignof(JRot<Real>) - 1));
    __shared__ int s_rot;
    __shared__ int s_act;  // rotations in the current round (compacted table length)

    const int tid = threadIdx.x;
    const int64_t patch = local;
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
    unsigned long long rotations = 0;  // tid 0's running total (counters only)
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
                    rtab[slot] = JRot<Real>{c, t * c, p, q};
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
                    const JRot<Real> rt = rtab[i];
                    const int p = rt.p, q = rt.q;
                    const Real c = rt.c, s = rt.s;
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
                    const JRot<Real> rt = rtab[i];
                    const int p = rt.p, q = rt.q;
                    const Real c = rt.c, s = rt.s;
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
                const JRot<Real> rt = rtab[tid];
                A[rt.p * ld + rt.q] = 0;
                A[rt.q * ld + rt.p] = 0;
            }
            if (tid == 0) { s_rot += nact; s_act = 0; }
            __syncthreads();
        }
        const int rot = s_rot;
        rotations += (unsigned long long)rot;
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
        atomicAdd(&ctr->jacobi_rotations, rotations);
        if (!converged) {
            atomicAdd(&ctr->jacobi_not_converged, 1ull);
            atomicOr(&ctr->status, (unsigned)DEV_NOT_CONVERGED);
        }
    }
}

// ---------------------------------------------------------------------------
// The same parallel-order Jacobi (same pairing, thresholds, rotations and
// sweep cap) with a round's updates fused into one pass over 2 x 2 blocks.
// Per round, lanes i < kp/2 of warp 0 compute pair i's rotation J_i and
// publish (c, s, p, q) in a table; then every rotating pair j is taken by one
// of the NW warps of the patch (round-robin over the ballot of rotating pairs,
// JW_UNROLL pairs in flight per warp), whose lane i replaces the block
// A[{p_i,q_i}, {p_j,q_j}] by J_i^T (A_ij J_j) (J_i = I when pair i does not
// rotate; for i = j the off-diagonal pair is set to 0) and, when pair i does
// not rotate, also writes the transposed result into A[{p_j,q_j}, {p_i,q_i}],
// the block whose column pair is not visited in this round; the same warp
// applies J_j to columns p_j, q_j of U (kept transposed: rows of U^T
// contiguous, two entries per lane, 8-byte accesses).  Every block is read and
// written by one lane in one iteration and no iteration reads a block another
// one writes, so a round needs two barriers (table published; updates done)
// and none inside.  Per rotation of a full round this moves 8 words of A (plus
// 4 transposed for pairs that do not rotate) and 8 of U, against 16 plus 3
// table reads in the one-CTA form's three passes with three barriers.
// ---------------------------------------------------------------------------
namespace {
constexpr int JW_UNROLL = 4;  // rotating pairs whose block updates are in flight together per warp
// Threshold strategy (Rutishauser's, for the cyclic Jacobi method): in the
// first JW_THR_SWEEPS sweeps a pair rotates only if |a_pq| also exceeds
// JW_THR_FACTOR S / kp^2, S the sum of |a_pq| over p < q at the sweep's start.
// 100k patches at k = 64: 21-22% fewer rotations, 192 -> 182 ms; the
// 256-dataset batch 2094 -> 1918 ms (factor 0.2: 1969 ms)
constexpr int JW_THR_SWEEPS = 3;
constexpr float JW_THR_FACTOR = 0.5f;
__host__ __device__ inline size_t jw_smem_bytes(int kmax) {
    const int kp = (kmax + 1) & ~1;
    // A (row stride kp + 1), U^T (row stride kp), 8-byte pad, 16-byte pad, table
    return ((size_t)kp * (kp + 1) + (size_t)kp * kp + 2 + 4) * sizeof(float) + 32 * sizeof(float4);
}
template <int NW>
__device__ __forceinline__ void jw_sync() {
    if constexpr (NW == 1) __syncwarp();
    else __syncthreads();
}
}  // namespace

template <int NW>
__global__ void __launch_bounds__(NW * 32)
jacobi_warp_kernel(const __grid_constant__ PatchSeg one, const PatchSeg *__restrict__ tab, int ntab, int max_sweeps,
                   float eps, DevCounters *ctr) {
    extern __shared__ __align__(16) float jw_sm[];
    __shared__ unsigned ctl_mask;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int local;
    const PatchSeg &seg = find_seg(one, tab, ntab, (int)blockIdx.x, local);
    const int k = seg.k;
    const int kp = (k + 1) & ~1;
    const int h = kp / 2;
    const int ld = kp + 1;
    const int n1 = kp - 1;
    float *A = jw_sm;
    float *Ut = A + (size_t)kp * ld;
    Ut += (reinterpret_cast<uintptr_t>(Ut) & 7) ? 1 : 0;  // 8-byte aligned rows (kp is even)
    float4 *T = reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(Ut + (size_t)kp * kp) + 15) & ~(uintptr_t)15);
    const int64_t patch = local;
    const float *g = seg.G + patch * (int64_t)k * k;
    for (int e = threadIdx.x; e < kp * kp; e += NW * 32) {
        const int r = e / kp, c = e % kp;
        A[r * ld + c] = (r < k && c < k) ? g[r * k + c] : 0.f;
        Ut[e] = (r == c) ? 1.f : 0.f;
    }
    jw_sync<NW>();
    const unsigned FULL = 0xffffffffu;
    int sweep = 0;
    bool converged = false;
    unsigned long long rotations = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rot = 0;
        // threshold strategy in the first sweeps: small off-diagonal entries are
        // left for later sweeps, whose rotations would disturb them anyway
        float thr = 0.f;
        if (sweep < JW_THR_SWEEPS && warp == 0) {
            float part = 0.f;
            for (int e = lane; e < kp * kp; e += 32) {
                const int r = e / kp, c = e % kp;
                if (r < c) part += fabsf(A[r * ld + c]);
            }
            thr = JW_THR_FACTOR * warp_sum(part) / (float)(kp * kp);
        }
        // circle method (warp 0): index kp - 1 fixed (lane 0's a), the others rotate
        int a = lane == 0 ? n1 : lane % n1, b = lane == 0 ? 0 : (n1 - lane) % n1;
        for (int round = 0; round < n1; ++round) {
            if (warp == 0) {
                bool act = false;
                if (lane < h) {
                    const int p = a < b ? a : b, q = a < b ? b : a;
                    float c = 1.f, sn = 0.f;
                    const float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
                    if (fabsf(apq) > eps * sqrtf(fabsf(app * aqq)) && fabsf(apq) > thr && apq != 0.f) {
                        const float tau = (aqq - app) / (2 * apq);
                        const float t = (tau >= 0 ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
                        c = 1.f / sqrtf(1.f + t * t);
                        sn = t * c;
                        act = true;
                    }
                    T[lane] = make_float4(c, sn, __int_as_float(p), __int_as_float(q));
                }
                const unsigned m = __ballot_sync(FULL, act);
                if (lane == 0) ctl_mask = m;
                // next round's pair
                if (lane == 0) b = b + 1;
                else { a = a + 1 == n1 ? 0 : a + 1; b = b + 1 == n1 ? 0 : b + 1; }
            }
            jw_sync<NW>();  // the round's table
            unsigned mask = ctl_mask;
            rot += __popc(mask);
            if (mask != 0u && lane < h) {
                const float4 ti = T[lane];
                const float c = ti.x, sn = ti.y;
                const int p = __float_as_int(ti.z), q = __float_as_int(ti.w);
                const bool act = (mask >> lane) & 1u;
                float *rp = A + p * ld, *rq = A + q * ld;
                // this warp's share: every NW-th rotating pair, starting at the warp's index
                for (int w = 0; w < warp && mask; ++w) mask &= mask - 1;
                while (mask) {
                    int js[JW_UNROLL];
                    float4 tj[JW_UNROLL];
                    float av[JW_UNROLL][4];
                    float2 uv[JW_UNROLL], wv[JW_UNROLL];
#pragma unroll
                    for (int u = 0; u < JW_UNROLL; ++u) {
                        js[u] = mask ? __ffs(mask) - 1 : -1;
#pragma unroll
                        for (int w = 0; w < NW; ++w) mask &= mask - 1;
                    }
                    // every load of the group before its first store (no element
                    // loaded in a round is stored by another pair's update)
#pragma unroll
                    for (int u = 0; u < JW_UNROLL; ++u) {
                        if (js[u] < 0) continue;
                        tj[u] = T[js[u]];
                        const int pj = __float_as_int(tj[u].z), qj = __float_as_int(tj[u].w);
                        av[u][0] = rp[pj];
                        av[u][1] = rp[qj];
                        av[u][2] = rq[pj];
                        av[u][3] = rq[qj];
                        uv[u] = reinterpret_cast<const float2 *>(Ut + pj * kp)[lane];
                        wv[u] = reinterpret_cast<const float2 *>(Ut + qj * kp)[lane];
                    }
#pragma unroll
                    for (int u = 0; u < JW_UNROLL; ++u) {
                        if (js[u] < 0) continue;
                        const float c1 = tj[u].x, s1 = tj[u].y;
                        const int pj = __float_as_int(tj[u].z), qj = __float_as_int(tj[u].w);
                        // A J_j on the block's columns, then J_i^T on its rows
                        const float t00 = c1 * av[u][0] - s1 * av[u][1], t01 = s1 * av[u][0] + c1 * av[u][1];
                        const float t10 = c1 * av[u][2] - s1 * av[u][3], t11 = s1 * av[u][2] + c1 * av[u][3];
                        float r00 = t00, r01 = t01, r10 = t10, r11 = t11;
                        if (act) {
                            r00 = c * t00 - sn * t10;
                            r10 = sn * t00 + c * t10;
                            r01 = c * t01 - sn * t11;
                            r11 = sn * t01 + c * t11;
                        }
                        if (lane == js[u]) { r01 = 0.f; r10 = 0.f; }
                        rp[pj] = r00;
                        rp[qj] = r01;
                        rq[pj] = r10;
                        rq[qj] = r11;
                        if (!act) {
                            A[pj * ld + p] = r00;
                            A[qj * ld + p] = r01;
                            A[pj * ld + q] = r10;
                            A[qj * ld + q] = r11;
                        }
                        // U J_j: rows p_j, q_j of U^T
                        reinterpret_cast<float2 *>(Ut + pj * kp)[lane] =
                            make_float2(c1 * uv[u].x - s1 * wv[u].x, c1 * uv[u].y - s1 * wv[u].y);
                        reinterpret_cast<float2 *>(Ut + qj * kp)[lane] =
                            make_float2(s1 * uv[u].x + c1 * wv[u].x, s1 * uv[u].y + c1 * wv[u].y);
                    }
                }
            }
            jw_sync<NW>();  // the round's updates
        }
        rotations += (unsigned long long)rot;
        if (rot == 0) { converged = true; break; }
    }
    // eigenpairs (indices < k) sorted descending by rank counting
    float *sg = seg.sig + patch * (int64_t)k;
    float *u = seg.U + patch * (int64_t)k * k;
    for (int i = threadIdx.x; i < k; i += NW * 32) {
        const float di = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const float dj = A[j * ld + j];
            rank += (dj > di) || (dj == di && j < i);
        }
        sg[rank] = di;
        for (int r = 0; r < k; ++r) u[r * k + rank] = Ut[i * kp + r];
    }
    if (threadIdx.x == 0) {
        atomicMax(&ctr->jacobi_max_sweeps, (unsigned long long)(converged ? sweep : max_sweeps));
        atomicAdd(&ctr->jacobi_rotations, rotations);
        if (!converged) {
            atomicAdd(&ctr->jacobi_not_converged, 1ull);
            atomicOr(&ctr->status, (unsigned)DEV_NOT_CONVERGED);
        }
    }
}

namespace {
template <int NW>
cudaError_t launch_jw(const PatchSeg &one, const PatchSeg *tab, int ntab, int kmax, int64_t np, int max_sweeps,
                      float eps, DevCounters *ctr, cudaStream_t s) {
    const size_t smem = jw_smem_bytes(kmax);
    cudaError_t e = cudaFuncSetAttribute(jacobi_warp_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    jacobi_warp_kernel<NW><<<(unsigned)np, NW * 32, smem, s>>>(one, tab, ntab, max_sweeps, eps, ctr);
    return cudaGetLastError();
}

// warps per patch of the fused form (1, 2 or 4)
cudaError_t launch_jacobi_warp(const PatchSeg &one, const PatchSeg *tab, int ntab, int kmax, int64_t np,
                               int max_sweeps, float eps, DevCounters *ctr, cudaStream_t s, int nw) {
    if (nw == 4) return launch_jw<4>(one, tab, ntab, kmax, np, max_sweeps, eps, ctr, s);
    if (nw == 2) return launch_jw<2>(one, tab, ntab, kmax, np, max_sweeps, eps, ctr, s);
    return launch_jw<1>(one, tab, ntab, kmax, np, max_sweeps, eps, ctr, s);
}
}  // namespace

// ---------------------------------------------------------------------------
// Refinement of an FP32 eigendecomposition: one step of the iterative
// refinement for symmetric eigenproblems of Ogita & Aishima (Japan J. Indust.
// Appl. Math. 35, 2018).  With X the k x k eigenvector estimate from the FP32
// sweeps and A = G:
//   R = I - X^T X,   S = X^T A X,   lam_i = S_ii / (1 - R_ii),
//   E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta,
//   E_ij = R_ij / 2 otherwise (and on the diagonal),   X' = X + X E.
// From FP32-accurate X one step squares the eigenvector error and
// re-orthogonalises X.  delta = 2^-18 max|lam| treats eigenvalues closer than
// the FP32 estimate resolves as a cluster (only orthogonalised); with rel != 0
// the test is relative to the pair, |lam_i - lam_j| <= 2^-18 max(|lam_i|,
// |lam_j|), for Grams whose FP32 eigenpairs are accurate relative to each
// eigenvalue (a nearly diagonal Gram, as in the adjoint's rotated basis).
// The O(k^3) products R, S and T = A X need more than FP32.  They are carried
// in two-term FP32 arithmetic ("double-float": a value is hi + lo, |lo| <=
// ulp(hi) / 2) because GB300 issues FP32 at ~60x its FP64 rate: A and X are
// FP32 values, so each product a x is exact as p + e (TwoProd: p = a x
// rounded, e = fma(a, x, -p)); the running sum takes p with Knuth's TwoSum
// (exact error term, no ordering assumption) and gathers e and the TwoSum
// errors in lo.  The accumulated error is ~n 2^-48 of the sum of |terms|
// (FP64: ~n 2^-53), far below what the FP32 eigenvectors written back can
// show: on 100k curved patches (m = 4096, k = 64) kappa came out bit-identical
// to an FP64 refinement, in 32% less stage time.  T is kept as hi + lo; S
// uses both parts (X T_lo as a plain FP32 product: it is 2^-24 of the term).
// The O(k^2) part (lambda, E) runs in FP64 from hi + lo, the correction X E
// (relative size ~2^-23) in FP32.  Every EFT step uses the _rn intrinsics,
// which the compiler never contracts into an FMA.  One CTA (256 threads,
// ~100 KB of shared memory, two per SM) per patch; results re-sorted
// descending.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ void ff_mac(float &hi, float &lo, float a, float x) {
    const float p = __fmul_rn(a, x);
    const float e = __fmaf_rn(a, x, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}
// upper-triangle packed index of (a, b), a <= b < k
__device__ __forceinline__ int tri(int a, int b, int k) { return a * k - (a * (a - 1)) / 2 + (b - a); }
}  // namespace

constexpr int FT_REFINE = 256;

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
jacobi_refine_ff_kernel(const __grid_constant__ PatchSeg one, const PatchSeg *__restrict__ tab, int ntab, int rel) {
    extern __shared__ __align__(16) unsigned char fsm[];
    int local;
    const PatchSeg &seg = find_seg(one, tab, ntab, (int)blockIdx.x, local);
    const int k = seg.k;
    const float *G = seg.G;
    float *sigma = seg.sig, *U = seg.U;
    const int ld = k + 1;
    const int ntri = k * (k + 1) / 2;
    float *A = reinterpret_cast<float *>(fsm);  // [k][ld], later E
    float *X = A + k * ld;                      // [k][ld]
    float *Th = X + k * ld;                     // [k][ld]  T = A X, high part; later X'
    float *Tl = Th + k * ld;                    // [k][ld]  low part
    float *Sh = Tl + k * ld;                    // [ntri] S = X^T A X (upper)
    float *Sl = Sh + ntri;
    float *Rh = Sl + ntri;                      // [ntri] X^T X (upper)
    float *Rl = Rh + ntri;
    double *lam = reinterpret_cast<double *>(reinterpret_cast<uintptr_t>(Rl + ntri + 1) & ~(uintptr_t)7);  // [k]
    __shared__ double s_lmax;
    const int tid = threadIdx.x;
    const int64_t pt = local;
    const float *g = G + pt * (int64_t)k * k;
    float *u = U + pt * (int64_t)k * k;
    const int kk = k * k;
    for (int e = tid; e < kk; e += NT) {
        const int r = e / k, c = e - r * k;
        A[r * ld + c] = g[e];
        X[r * ld + c] = u[e];
    }
    __syncthreads();
    // T = A X: four outputs of one row per thread pass (independent chains)
    for (int q = tid; q * 4 < kk; q += NT) {
        const int e0 = q * 4;
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        int rr[4], cc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = e0 + i < kk ? e0 + i : kk - 1;
            rr[i] = e / k;
            cc[i] = e - rr[i] * k;
        }
        for (int j = 0; j < k; ++j) {
#pragma unroll
            for (int i = 0; i < 4; ++i) ff_mac(hi[i], lo[i], A[rr[i] * ld + j], X[j * ld + cc[i]]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (e0 + i < kk) {
                Th[rr[i] * ld + cc[i]] = hi[i];
                Tl[rr[i] * ld + cc[i]] = lo[i];
            }
    }
    __syncthreads();
    // S = X^T T and R = X^T X on the upper triangle, two outputs per thread pass
    for (int q = tid; q * 2 < ntri; q += NT) {
        int ra[2], ca[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            int t = q * 2 + i < ntri ? q * 2 + i : ntri - 1;
            int a = 0;
            while (t >= k - a) { t -= k - a; ++a; }
            ra[i] = a;
            ca[i] = a + t;
        }
        float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f}, rh[2] = {0.f, 0.f}, rl[2] = {0.f, 0.f};
        for (int j = 0; j < k; ++j) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float xr = X[j * ld + ra[i]];
                ff_mac(sh[i], sl[i], xr, Th[j * ld + ca[i]]);
                sl[i] = __fmaf_rn(xr, Tl[j * ld + ca[i]], sl[i]);
                ff_mac(rh[i], rl[i], xr, X[j * ld + ca[i]]);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
            if (q * 2 + i < ntri) {
                const int t = q * 2 + i;
                Sh[t] = sh[i];
                Sl[t] = sl[i];
                Rh[t] = rh[i];
                Rl[t] = rl[i];
            }
    }
    __syncthreads();
    auto Sd = [&](int a, int b) { const int t = tri(a, b, k); return (double)Sh[t] + (double)Sl[t]; };
    // I - X^T X: the identity minus hi, then minus lo, in FP64
    auto Rd = [&](int a, int b) {
        const int t = tri(a, b, k);
        return ((a == b ? 1.0 : 0.0) - (double)Rh[t]) - (double)Rl[t];
    };
    if (tid < k) lam[tid] = Sd(tid, tid) / (1.0 - Rd(tid, tid));
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(lam[i]));
        s_lmax = mx;
    }
    __syncthreads();
    const double delta = 3.814697265625e-06 * s_lmax;  // 2^-18 max|lam|
    float *Ef = A;  // A is no longer needed
    for (int e = tid; e < kk; e += NT) {
        const int i = e / k, j = e - i * k;
        const int a = i < j ? i : j, b = i < j ? j : i;
        const double rij = Rd(a, b);
        const double sij = Sd(a, b);
        const double dij = rel ? 3.814697265625e-06 * fmax(fabs(lam[i]), fabs(lam[j])) : delta;
        double v;
        if (i == j || fabs(lam[i] - lam[j]) <= dij) v = 0.5 * rij;
        else v = (sij + lam[j] * rij) / (lam[j] - lam[i]);
        Ef[i * ld + j] = (float)v;
    }
    __syncthreads();
    // X' = X + X E (FP32), into Th
    float *Xn = Th;
    for (int e = tid; e < kk; e += NT) {
        const int r = e / k, c = e - r * k;
        float t = 0.f;
        for (int j = 0; j < k; ++j) t = fmaf(X[r * ld + j], Ef[j * ld + c], t);
        Xn[r * ld + c] = X[r * ld + c] + t;
    }
    __syncthreads();
    float *sg = sigma + pt * (int64_t)k;
    for (int i = tid; i < k; i += NT) {
        int rank = 0;
        for (int j = 0; j < k; ++j) rank += (lam[j] > lam[i]) || (lam[j] == lam[i] && j < i);
        sg[rank] = (float)lam[i];
        for (int r = 0; r < k; ++r) u[r * k + rank] = Xn[r * ld + i];
    }
}

size_t refine_ff_smem_bytes(int k) {
    return (size_t)4 * k * (k + 1) * sizeof(float) + (size_t)2 * k * (k + 1) * sizeof(float) + 16 +
           (size_t)k * sizeof(double);
}


size_t jacobi_smem_bytes(int k, int fp64) {
    const int kp = (k + 1) & ~1;
    const size_t real = fp64 ? sizeof(double) : sizeof(float);
    const size_t ent = fp64 ? sizeof(JRot<double>) : sizeof(JRot<float>);
    return (size_t)2 * kp * (kp + 1) * real + ent + (size_t)(kp / 2) * ent;
}

cudaError_t launch_jacobi_seg(const PatchSeg &one, const PatchSeg *tab, int ntab, int kmax, int64_t np, int fp64,
                              int max_sweeps, DevCounters *ctr, cudaStream_t s, float pre_eps, int warp_form) {
    if (np <= 0) return cudaSuccess;
    if (kmax > 64 || kmax < 1) return cudaErrorInvalidValue;
    cudaError_t e;
    // FP32 sweeps: one warp per patch, or one CTA per patch
    auto sweeps32 = [&](float eps) -> cudaError_t {
        if (warp_form) return launch_jacobi_warp(one, tab, ntab, kmax, np, max_sweeps, eps, ctr, s, warp_form);
        const size_t smem = jacobi_smem_bytes(kmax, 0);
        cudaError_t r = cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (r != cudaSuccess) return r;
        jacobi_kernel<float><<<(unsigned)np, JT, smem, s>>>(one, tab, ntab, max_sweeps, eps, ctr);
        return cudaGetLastError();
    };
    if (fp64 == 1 || fp64 == 3) {
        // FP32 sweeps, then one refinement step (3: relative cluster test)
        e = sweeps32(pre_eps);
        if (e != cudaSuccess) return e;
        // threads per patch: 64 (k <= 16), 128 (k <= 32) or 256, so that small
        // patches are not limited to 8 per SM by idle threads
        const size_t rs = refine_ff_smem_bytes(kmax);
        auto refine = [&](auto kern, int nt) -> cudaError_t {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
            if (r != cudaSuccess) return r;
            kern<<<(unsigned)np, nt, rs, s>>>(one, tab, ntab, fp64 == 3);
            return cudaGetLastError();
        };
        if (kmax <= 16) return refine(jacobi_refine_ff_kernel<64>, 64);
        if (kmax <= 32) return refine(jacobi_refine_ff_kernel<128>, 128);
        return refine(jacobi_refine_ff_kernel<FT_REFINE>, FT_REFINE);
    }
    if (fp64 == 2) {
        const size_t smem = jacobi_smem_bytes(kmax, fp64);
        e = cudaFuncSetAttribute(jacobi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<double><<<(unsigned)np, JT, smem, s>>>(one, tab, ntab, max_sweeps, JacobiEps<double>::rel(), ctr);
        return cudaGetLastError();
    }
    return sweeps32(JacobiEps<float>::rel());
}

cudaError_t launch_jacobi(const float *G, int k, int64_t np, int fp64, int max_sweeps, float *sigma, float *U,
                          DevCounters *ctr, cudaStream_t s, float pre_eps, int warp_form) {
    PatchSeg one{};
    one.k = k;
    one.G = const_cast<float *>(G);
    one.sig = sigma;
    one.U = U;
    return launch_jacobi_seg(one, nullptr, 0, k, np, fp64, max_sweeps, ctr, s, pre_eps, warp_form);
}

}  // namespace mecuco
