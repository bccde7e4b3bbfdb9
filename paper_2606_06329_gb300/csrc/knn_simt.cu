// knn_simt.cu - Step 1 (Sec. 3 Step 1, eq. knn; Alg. 1 kNN-Graph): candidate
// search with FP32 arithmetic on the CUDA cores, the exact re-rank with its
// certification test, and the exact full-scan fallback.
//
// Candidate search: a CTA owns BM = 128 query rows and sweeps the candidate
// rows of its split in BN = 128 tiles.  Each of 256 threads accumulates an
// 8 x 8 block of dot products x_i . y_j over BK = 8 wide K slices staged in
// shared memory; the epilogue forms d~ = |x|^2 + |y|^2 - 2 x.y and one thread
// per query row folds the tile into that row's list of the kc smallest d~
// (unsorted, with its current maximum tracked as the admission threshold).
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

// The table entry of batch row `row` (entries sorted by row_begin).
__device__ __forceinline__ const KnnSet &find_set_row(const KnnSet *sets, int nsets, int64_t row) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sets[mid].row_begin <= row) lo = mid;
        else hi = mid - 1;
    }
    return sets[lo];
}

// One warp: |x|^2 of a row as a compensated sum (hi + lo rounded once, so
// within a few FP32 units of the exact value) and, for quant != NONE, the
// norms of the row's BF16 rounding terms (rounded up) into resid[0..1]:
// single rounding h = bf16(x): |x - h| and 0; three-term split, l = bf16(x - h):
// |l| and |x - h - l| (both differences exact in FP32).  The dataset's largest
// |x|^2 and terms go to maxima[0..2] (non-negative floats, so their bit
// patterns order as integers).
template <typename T>
__device__ __forceinline__ void row_norm_warp(const T *__restrict__ x, int64_t m, int lane, float *norm_out,
                                              float *resid_out, float *maxima, int quant) {
    ff acc{0.f, 0.f};
    float a1 = 0.f, a2 = 0.f;
    for (int64_t a = lane; a < m; a += 32) {
        const float v = load_elem(x + a);
        ff_acc_sqdiff(acc, v, 0.f);
        if (quant != KNN_QUANT_NONE) {
            const float r = v - __bfloat162float(__float2bfloat16_rn(v));
            if (quant == KNN_QUANT_SINGLE) {
                a1 = fmaf(r, r, a1);
            } else {
                const float l = __bfloat162float(__float2bfloat16_rn(r));
                const float r2 = r - l;
                a1 = fmaf(l, l, a1);
                a2 = fmaf(r2, r2, a2);
            }
        }
    }
    acc = ff_warp_sum(acc);
    const float n = acc.hi + acc.lo;
    if (quant != KNN_QUANT_NONE) {
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
    }
    if (lane == 0) {
        *norm_out = n;
        if (quant != KNN_QUANT_NONE) {
            // the FP32 sums of m squares are within m 2^-24 of their values: 2^-10 covers it
            const float t1 = sqrtf(a1) * (1.f + 9.765625e-04f), t2 = sqrtf(a2) * (1.f + 9.765625e-04f);
            resid_out[0] = t1;
            resid_out[1] = t2;
            atomicMax(reinterpret_cast<int *>(maxima), __float_as_int(n));
            atomicMax(reinterpret_cast<int *>(maxima) + 1, __float_as_int(t1));
            atomicMax(reinterpret_cast<int *>(maxima) + 2, __float_as_int(t2));
        }
    }
}

template <typename T>
__global__ void rownorm_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld, float *__restrict__ out,
                               float *__restrict__ resid, float *__restrict__ maxima, int quant) {
    int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= N) return;
    row_norm_warp(X + row * ld, m, lane, out + row, quant ? resid + 2 * row : nullptr, maxima, quant);
}

cudaError_t launch_rownorm(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                           float *norms, cudaStream_t s, float *resid, float *maxima, int quant) {
    if (N <= 0) return cudaSuccess;
    if (dt == MECUCO_BF16 || !resid || !maxima) quant = KNN_QUANT_NONE;
    dim3 block(256), grid((unsigned)((N + 7) / 8));
    if (dt == MECUCO_BF16)
        rownorm_kernel<<<grid, block, 0, s>>>((const __nv_bfloat16 *)X, N, m, ld, norms, nullptr, nullptr, quant);
    else
        rownorm_kernel<<<grid, block, 0, s>>>((const float *)X, N, m, ld, norms, resid, maxima, quant);
    return cudaGetLastError();
}

// Row norms of every row of a batch: one warp per row, each row's dataset from
// the table.
template <typename T>
__global__ void rownorm_batch_kernel(const KnnSet *__restrict__ sets, int nsets, int64_t nrows) {
    const int64_t gr = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (gr >= nrows) return;
    const KnnSet &d = find_set_row(sets, nsets, gr);
    const int64_t row = gr - d.row_begin;
    row_norm_warp(static_cast<const T *>(d.X) + row * d.ld, d.m, lane, d.norms + row,
                  d.quant ? d.resid + 2 * row : nullptr, d.maxima, d.quant);
}

cudaError_t launch_rownorm_batch(const KnnSet *sets, int nsets, int64_t nrows, mecuco_dtype dt, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    dim3 block(256), grid((unsigned)((nrows + 7) / 8));
    if (dt == MECUCO_BF16) rownorm_batch_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(sets, nsets, nrows);
    else rownorm_batch_kernel<float><<<grid, block, 0, s>>>(sets, nsets, nrows);
    return cudaGetLastError();
}

// BF16 copies (round to nearest even, zero past m) of the rows of every
// dataset that has one (xb): one warp per row, coalesced along the row.
template <typename T>
__global__ void to_bf16_batch_kernel(const KnnSet *__restrict__ sets, int nsets, int64_t nrows) {
    const int64_t gr = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (gr >= nrows) return;
    const KnnSet &d = find_set_row(sets, nsets, gr);
    if (!d.xb) return;
    const int64_t row = gr - d.row_begin;
    const T *x = static_cast<const T *>(d.X) + row * d.ld;
    __nv_bfloat16 *y = static_cast<__nv_bfloat16 *>(d.xb) + row * d.ldb;
    if (!d.xb2) {
        for (int64_t a = lane; a < d.ldb; a += 32) y[a] = __float2bfloat16_rn(a < d.m ? load_elem(x + a) : 0.f);
        return;
    }
    // three-term split (as launch_to_bf16_split): query [h | h | l], candidate [h | l | h]
    __nv_bfloat16 *yb = static_cast<__nv_bfloat16 *>(d.xb2) + row * d.ldb;
    const int64_t ms = d.mk / 3;
    for (int64_t a = lane; a < d.ldb; a += 32) {
        const int64_t seg = a / ms, c = a - seg * ms;
        const float v = (seg < 3 && c < d.m) ? load_elem(x + c) : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        y[a] = seg == 2 ? l : h;
        yb[a] = seg == 1 ? l : h;
    }
}

cudaError_t launch_to_bf16_batch(const KnnSet *sets, int nsets, int64_t nrows, mecuco_dtype dt, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    dim3 block(256), grid((unsigned)((nrows + 7) / 8));
    if (dt == MECUCO_BF16) to_bf16_batch_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(sets, nsets, nrows);
    else to_bf16_batch_kernel<float><<<grid, block, 0, s>>>(sets, nsets, nrows);
    return cudaGetLastError();
}

namespace {
constexpr int SBM = 128, SBN = 128, SBK = 8, STHREADS = 256;

__device__ __forceinline__ void list_rescan(const float *Ld, int kc, int stride, int row, float &thr,
                                            int &slot) {
    float mx = -INFINITY;
    int sl = 0;
    for (int s = 0; s < kc; ++s) {
        float v = Ld[s * stride + row];
        if (v > mx) { mx = v; sl = s; }
    }
    thr = mx;
    slot = sl;
}
}  // namespace

template <typename T>
__global__ void __launch_bounds__(STHREADS, 1)
knn_simt_kernel(const T *__restrict__ X, int64_t N, int64_t m, int64_t ld,
                const float *__restrict__ norms, int64_t q0, int64_t nq, int kc, int nsplit,
                int include_self, float *__restrict__ cand_d, int32_t *__restrict__ cand_i) {
    extern __shared__ float smem[];
    float *As = smem;                     // [SBK][SBM]
    float *Bs = As + SBK * SBM;           // [SBK][SBN]
    float *Ds = Bs + SBK * SBN;           // [SBM][SBN + 1]
    float *qns = Ds + SBM * (SBN + 1);    // [SBM]
    float *cns = qns + SBM;               // [SBN]
    float *Ld = cns + SBN;                // [kc][SBM]
    int *Li = reinterpret_cast<int *>(Ld + kc * SBM);  // [kc][SBM]

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t qb = q0 + (int64_t)blockIdx.x * SBM;
    const int64_t qend = q0 + nq;
    const int split = blockIdx.y;
    const int64_t per = (N + nsplit - 1) / nsplit;
    const int64_t cbeg = (int64_t)split * per;
    const int64_t cend = min(N, cbeg + per);

    for (int r = tid; r < SBM; r += STHREADS) qns[r] = (qb + r < qend) ? norms[qb + r] : 0.f;
    int cnt = 0, slot = 0;
    float thr = INFINITY;

    for (int64_t c0 = cbeg; c0 < cend; c0 += SBN) {
        for (int c = tid; c < SBN; c += STHREADS) cns[c] = (c0 + c < cend) ? norms[c0 + c] : 0.f;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        for (int64_t k0 = 0; k0 < m; k0 += SBK) {
            // stage the BM x BK query slice and BN x BK candidate slice (transposed)
#pragma unroll
            for (int e = 0; e < (SBM * SBK) / STHREADS; ++e) {
                int lin = tid + e * STHREADS;
                int r = lin / SBK, kk = lin % SBK;
                int64_t gq = qb + r, ga = k0 + kk;
                As[kk * SBM + r] = (gq < qend && ga < m) ? load_elem(X + gq * ld + ga) : 0.f;
                int64_t gc = c0 + r;
                Bs[kk * SBN + r] = (gc < cend && ga < m) ? load_elem(X + gc * ld + ga) : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < SBK; ++kk) {
                float a[8], b[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = As[kk * SBM + ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 8; ++j) b[j] = Bs[kk * SBN + tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
        // epilogue: approximate distances into Ds
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int r = ty + 16 * i;
            int64_t gq = qb + r;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int c = tx + 16 * j;
                int64_t gc = c0 + c;
                float d = qns[r] + cns[c] - 2.f * acc[i][j];
                if (gq >= qend || gc >= cend || (!include_self && gc == gq)) d = INFINITY;
                Ds[r * (SBN + 1) + c] = d;
            }
        }
        __syncthreads();
        if (tid < SBM) {
            const int row = tid;
            for (int c = 0; c < SBN; ++c) {
                float d = Ds[row * (SBN + 1) + c];
                if (!(d < thr)) continue;
                int j = (int)(c0 + c);
                if (cnt < kc) {
                    Ld[cnt * SBM + row] = d;
                    Li[cnt * SBM + row] = j;
                    ++cnt;
                    if (cnt == kc) list_rescan(Ld, kc, SBM, row, thr, slot);
                } else {
                    Ld[slot * SBM + row] = d;
                    Li[slot * SBM + row] = j;
                    list_rescan(Ld, kc, SBM, row, thr, slot);
                }
            }
        }
        __syncthreads();
    }
    if (tid < SBM && qb + tid < qend) {
        int64_t base = ((qb + tid - q0) * nsplit + split) * (int64_t)kc;
        for (int s = 0; s < kc; ++s) {
            bool used = s < cnt;
            cand_d[base + s] = used ? Ld[s * SBM + tid] : INFINITY;
            cand_i[base + s] = used ? Li[s * SBM + tid] : -1;
        }
    }
}

cudaError_t launch_knn_simt(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                            const float *norms, int64_t q0, int64_t nq, int kc, int nsplit,
                            int include_self, float *cand_d, int32_t *cand_i, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    size_t smem = sizeof(float) * (size_t)(2 * SBK * SBM + SBM * (SBN + 1) + SBM + SBN) +
                  (size_t)kc * SBM * (sizeof(float) + sizeof(int));
    dim3 grid((unsigned)((nq + SBM - 1) / SBM), (unsigned)nsplit), block(STHREADS);
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(knn_simt_kernel<__nv_bfloat16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        knn_simt_kernel<<<grid, block, smem, s>>>((const __nv_bfloat16 *)X, N, m, ld, norms, q0, nq,
                                                  kc, nsplit, include_self, cand_d, cand_i);
    } else {
        e = cudaFuncSetAttribute(knn_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        knn_simt_kernel<<<grid, block, smem, s>>>((const float *)X, N, m, ld, norms, q0, nq, kc,
                                                  nsplit, include_self, cand_d, cand_i);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact re-rank + certification.  One warp per query row.  Each candidate's
// squared distance sum_a (x_a - y_a)^2 is accumulated as a float-float pair
// (TwoSum of the difference, FMA TwoProd of the square), so it carries ~2^-44
// relative error: ranks agree with an FP64 brute force except at ties closer
// than that.  Certification: every row left out of the candidate set has
// d~ >= thr (the smallest admission threshold of the full splits), so its true
// distance is >= thr - e_hi, e_hi bounding the overestimate d~ - d; the row is
// certified when thr - e_hi exceeds the exact k-th distance.  The search's
// accumulation error has no documented worst-case bound on the tensor-core
// path and is dominated by a per-row bias (the FP32 accumulator's rounding of
// partial sums of similar size), so e_hi is estimated a posteriori from the
// row's own candidates: the largest observed d~ - d plus 3x the observed spread
// of d~ - d, plus 2^-21 (|x|^2 + max |y|^2) (a few units in the last place of
// the norms).  Rows failing the test are re-solved exactly by the full scan.
// ---------------------------------------------------------------------------
constexpr int RR_WARPS = 4;
constexpr int RR_MAXL = 1024;

template <typename T, bool BATCH>
__global__ void __launch_bounds__(RR_WARPS * 32)
knn_rerank_kernel(const T *__restrict__ X_, int64_t N_, int64_t m_, int64_t ld_,
                  const float *__restrict__ norms_, int64_t q0_, int64_t nq, int kc_, int nsplit_, int k_,
                  const float *__restrict__ cand_d_, const int32_t *__restrict__ cand_i_,
                  int32_t *__restrict__ idx_out_, float *__restrict__ dist_out_,
                  int32_t *__restrict__ flags_, DevCounters *ctr, const KnnSet *__restrict__ sets, int nsets,
                  int lmax, const float *__restrict__ resid_, const float *__restrict__ maxima_, int quant_) {
    extern __shared__ float rsm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t qi = (int64_t)blockIdx.x * RR_WARPS + w;  // the launch's row (the batch's row when batched)
    if (qi >= nq) return;
    // the row's dataset: the arguments, or its entry of a batch's table
    const T *X = X_;
    int64_t N = N_, m = m_, ld = ld_, q0 = q0_;
    const float *norms = norms_, *cand_d = cand_d_;
    const int32_t *cand_i = cand_i_;
    int32_t *idx_out = idx_out_, *flags = flags_;
    float *dist_out = dist_out_;
    const float *resid = resid_, *maxima = maxima_;
    int quant = quant_;
    int kc = kc_, nsplit = nsplit_, k = k_;
    if constexpr (BATCH) {
        const KnnSet &d = find_set_row(sets, nsets, qi);
        qi -= d.row_begin;
        X = static_cast<const T *>(d.X);
        N = d.N;
        m = d.m;
        ld = d.ld;
        q0 = 0;
        norms = d.norms;
        cand_d = d.cand_d;
        cand_i = d.cand_i;
        idx_out = d.idx;
        flags = d.flags;
        dist_out = nullptr;
        kc = d.kcl;
        nsplit = d.lists;
        k = d.k;
        resid = d.resid;
        maxima = d.maxima;
        quant = d.quant;
    }
    const int L = kc * nsplit;
    const int LS = BATCH ? lmax : L;  // per-warp shared-memory stride
    float *hi = rsm + (size_t)w * LS * 3;
    float *lo = hi + L;
    int *ci = reinterpret_cast<int *>(lo + L);
    const int64_t q = q0 + qi;
    const float *cd = cand_d + qi * (int64_t)L;
    const int32_t *cidx = cand_i + qi * (int64_t)L;
    const T *xq = X + q * ld;

    float err_max = -INFINITY, err_min = INFINITY, nmax = 0.f;
    bool bad = false;
    // a complete search leaves -1 or a row of X in every slot; anything else
    // (slots a search that timed out never wrote) is skipped, never read
    auto cand = [&](int c) {
        int j = cidx[c];
        if (j >= N) { bad = true; j = -1; }
        return j;
    };
    auto record = [&](int c, int j, ff acc) {
        if (j >= 0) {
            const float e = cd[c] - acc.hi;  // overestimate of the search's distance
            err_max = fmaxf(err_max, e);
            err_min = fminf(err_min, e);
            nmax = fmaxf(nmax, norms[j]);
        } else {
            acc.hi = INFINITY;
        }
        if (lane == 0) { hi[c] = acc.hi; lo[c] = acc.lo; ci[c] = j; }
    };
    // Rows as 16-byte vectors when every row starts 16-byte aligned: four
    // candidates at a time, each lane summing its share of the four rows with
    // independent compensated accumulators, so that 4 x (m / 32 / VEC) loads
    // are in flight per lane instead of one 2- or 4-byte load per step.  The
    // terms are the same; only the summation order differs from the scalar form.
    constexpr int VEC = 16 / (int)sizeof(T);
    const bool vec = (ld % VEC == 0) && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    int c = 0;
    if (vec) {
        const int64_t mv = m / VEC * VEC;  // vector part of the row; the tail is scalar
        for (; c + 4 <= L; c += 4) {
            int j[4];
            const T *xr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                j[u] = cand(c + u);
                xr[u] = X + (int64_t)(j[u] >= 0 ? j[u] : q) * ld;  // an empty slot reads the query row, discarded
            }
            ff acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int64_t a = (int64_t)lane * VEC; a < mv; a += 32 * VEC) {
                const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(xq + a));
                uint4 yv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) yv[u] = __ldg(reinterpret_cast<const uint4 *>(xr[u] + a));
                const T *qe = reinterpret_cast<const T *>(&qv);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T *ye = reinterpret_cast<const T *>(&yv[u]);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) ff_acc_sqdiff(acc[u], to_f32(qe[e]), to_f32(ye[e]));
                }
            }
            for (int64_t a = mv + lane; a < m; a += 32)
#pragma unroll
                for (int u = 0; u < 4; ++u) ff_acc_sqdiff(acc[u], load_elem(xq + a), load_elem(xr[u] + a));
#pragma unroll
            for (int u = 0; u < 4; ++u) record(c + u, j[u], ff_warp_sum(acc[u]));
        }
    }
    for (; c < L; ++c) {
        const int j = cand(c);
        ff acc{0.f, 0.f};
        if (j >= 0) {
            const T *xj = X + (int64_t)j * ld;
            for (int64_t a = lane; a < m; a += 32) ff_acc_sqdiff(acc, load_elem(xq + a), load_elem(xj + a));
            acc = ff_warp_sum(acc);
        }
        record(c, j, acc);
    }
    __syncwarp();
    // thresholds: a split whose list is full admitted only d~ < its max
    float thr = INFINITY;
    for (int sp = 0; sp < nsplit; ++sp) {
        float mx = -INFINITY;
        bool full = true;
        for (int c = lane; c < kc; c += 32) {
            float v = cd[sp * kc + c];
            full = full && (ci[sp * kc + c] >= 0);
            mx = fmaxf(mx, v);
        }
        mx = warp_max(mx);
        full = __all_sync(0xffffffffu, full);
        if (full) thr = fminf(thr, mx);
    }
    // rank each candidate by (hi, lo, index); write the k best in order
    float theta = 0.f;
    for (int c = lane; c < L; c += 32) {
        int j = ci[c];
        if (j < 0) continue;
        ff me{hi[c], lo[c]};
        int rank = 0;
        for (int o = 0; o < L; ++o) {
            if (ci[o] < 0) continue;
            if (ff_less(ff{hi[o], lo[o]}, ci[o], me, j)) ++rank;
        }
        if (rank < k) {
            idx_out[qi * k + rank] = j;
            if (dist_out) dist_out[qi * k + rank] = me.hi + me.lo;
        }
        if (rank == k - 1) theta = me.hi;
    }
    theta = warp_max(theta);
    if (lane == 0 && bad) atomicOr(&ctr->status, (unsigned)DEV_INVALID);
    if (lane == 0) {
        const float spread = err_max - err_min;
        float e_hi = fmaxf(err_max, 0.f) + 3.f * spread + ldexpf(norms[q] + nmax, -21);
        if (quant != KNN_QUANT_NONE) {
            // BF16 operands from FP32 rows: an a-priori bound (not estimated from
            // the candidates) on |x.y - (the search's product)| for any
            // candidate y, with the dataset's largest |y| and rounding terms.
            //   single (x = h + d):      |h||d_y| + |d||h_y| + |d||d_y|
            //   split (x = h + l + r):   |l||l_y| + |h + l||r_y| + |r||h_y + l_y| + |r||r_y|
            // The tensor core's FP32 accumulation stays with the estimate.
            const float t1 = resid[2 * q], t2 = resid[2 * q + 1], xq = sqrtf(norms[q]);
            const float ym = sqrtf(maxima[0]), m1 = maxima[1], m2 = maxima[2];
            const float b = quant == KNN_QUANT_SINGLE ? (xq + t1) * m1 + t1 * (ym + m1) + t1 * m1
                                                      : t1 * m1 + (xq + t2) * m2 + t2 * (ym + m2) + t2 * m2;
            const float eq = 2.f * b * (1.f + 9.765625e-04f) + ldexpf(norms[q] + maxima[0], -21);
            e_hi = fmaxf(e_hi, eq);
        }
        int ok = (thr == INFINITY) || (thr - e_hi > theta);
        flags[qi] = ok ? 0 : 1;
        if (!ok) atomicAdd(&ctr->knn_uncertified, 1ull);
    }
}

cudaError_t launch_knn_rerank(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                              const float *norms, int64_t q0, int64_t nq, int kc, int nsplit, int k,
                              const float *cand_d, const int32_t *cand_i, int32_t *idx_out,
                              float *dist_out, int32_t *flags, DevCounters *ctr, cudaStream_t s,
                              const float *resid, const float *maxima, int quant) {
    if (!resid || !maxima) quant = KNN_QUANT_NONE;
    if (nq <= 0) return cudaSuccess;
    int L = kc * nsplit;
    if (L > RR_MAXL) return cudaErrorInvalidValue;
    size_t smem = (size_t)RR_WARPS * L * 3 * sizeof(float);
    dim3 grid((unsigned)((nq + RR_WARPS - 1) / RR_WARPS)), block(RR_WARPS * 32);
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(knn_rerank_kernel<__nv_bfloat16, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        knn_rerank_kernel<__nv_bfloat16, false><<<grid, block, smem, s>>>((const __nv_bfloat16 *)X, N, m, ld, norms,
                                                                          q0, nq, kc, nsplit, k, cand_d, cand_i,
                                                                          idx_out, dist_out, flags, ctr, nullptr, 0, 0,
                                                                          resid, maxima, quant);
    } else {
        e = cudaFuncSetAttribute(knn_rerank_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        knn_rerank_kernel<float, false><<<grid, block, smem, s>>>((const float *)X, N, m, ld, norms, q0, nq, kc,
                                                                  nsplit, k, cand_d, cand_i, idx_out, dist_out, flags,
                                                                  ctr, nullptr, 0, 0, resid, maxima, quant);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact full scan for flagged rows: one CTA of 8 warps per query; warp w takes
// candidates j = w, w + 8, ...; each distance is a warp-cooperative compensated
// sum; lane 0 keeps the warp's k best in shared memory (sorted insertion);
// finally the 8 lists are merged by rank.
// ---------------------------------------------------------------------------
constexpr int FB_WARPS = 8;

template <typename T, bool BATCH>
__global__ void __launch_bounds__(FB_WARPS * 32)
knn_fallback_kernel(const T *__restrict__ X_, int64_t N_, int64_t m_, int64_t ld_, int64_t q0_,
                    int64_t nq, int k_, int include_self_, const int32_t *__restrict__ flags_,
                    int32_t *__restrict__ idx_out_, float *__restrict__ dist_out_, DevCounters *ctr,
                    const KnnSet *__restrict__ sets, int nsets, int kmax) {
    extern __shared__ float fsm[];
    const int KS = BATCH ? kmax : k_;      // shared-memory stride of one warp's list
    float *bh = fsm;                       // [FB_WARPS][KS]
    float *bl = bh + FB_WARPS * KS;        // [FB_WARPS][KS]
    int *bi = reinterpret_cast<int *>(bl + FB_WARPS * KS);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t gi = blockIdx.x; gi < nq; gi += gridDim.x) {
        // the row's dataset: the arguments, or its entry of a batch's table
        const T *X = X_;
        int64_t N = N_, m = m_, ld = ld_, q0 = q0_, qi = gi;
        const int32_t *flags = flags_;
        int32_t *idx_out = idx_out_;
        float *dist_out = dist_out_;
        int k = k_, include_self = include_self_;
        if constexpr (BATCH) {
            const KnnSet &d = find_set_row(sets, nsets, gi);
            qi = gi - d.row_begin;
            X = static_cast<const T *>(d.X);
            N = d.N;
            m = d.m;
            ld = d.ld;
            q0 = 0;
            flags = d.flags;
            idx_out = d.idx;
            dist_out = nullptr;
            k = d.k;
            include_self = d.include_self;
        }
        if (flags[qi] == 0) continue;  // uniform across the CTA
        const int64_t q = q0 + qi;
        const T *xq = X + q * ld;
        float *mh = bh + w * KS, *ml = bl + w * KS;
        int *mi = bi + w * KS;
        if (lane == 0)
            for (int s = 0; s < k; ++s) { mh[s] = INFINITY; ml[s] = 0.f; mi[s] = 0x7fffffff; }
        __syncwarp();
        for (int64_t j = w; j < N; j += FB_WARPS) {
            if (!include_self && j == q) continue;
            const T *xj = X + j * ld;
            ff acc{0.f, 0.f};
            for (int64_t a = lane; a < m; a += 32) ff_acc_sqdiff(acc, load_elem(xq + a), load_elem(xj + a));
            acc = ff_warp_sum(acc);
            if (lane == 0 && ff_less(acc, (int)j, ff{mh[k - 1], ml[k - 1]}, mi[k - 1])) {
                int pos = k - 1;
                while (pos > 0 && ff_less(acc, (int)j, ff{mh[pos - 1], ml[pos - 1]}, mi[pos - 1])) {
                    mh[pos] = mh[pos - 1]; ml[pos] = ml[pos - 1]; mi[pos] = mi[pos - 1];
                    --pos;
                }
                mh[pos] = acc.hi; ml[pos] = acc.lo; mi[pos] = (int)j;
            }
            __syncwarp();
        }
        __syncthreads();
        // merge: rank every entry among all FB_WARPS * k entries
        for (int e = threadIdx.x; e < FB_WARPS * KS; e += blockDim.x) {
            if (e % KS >= k || bi[e] == 0x7fffffff) continue;
            ff me{bh[e], bl[e]};
            int rank = 0;
            for (int o = 0; o < FB_WARPS * KS; ++o)
                if (o % KS < k && bi[o] != 0x7fffffff && ff_less(ff{bh[o], bl[o]}, bi[o], me, bi[e])) ++rank;
            if (rank < k) {
                idx_out[qi * k + rank] = bi[e];
                if (dist_out) dist_out[qi * k + rank] = me.hi + me.lo;
            }
        }
        if (threadIdx.x == 0) atomicAdd(&ctr->knn_fallback_rows, 1ull);
        __syncthreads();
    }
}

cudaError_t launch_knn_fallback(const void *X, mecuco_dtype dt, int64_t N, int64_t m, int64_t ld,
                                int64_t q0, int64_t nq, int k, int include_self, const int32_t *flags,
                                int32_t *idx_out, float *dist_out, DevCounters *ctr, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    size_t smem = (size_t)FB_WARPS * k * 3 * sizeof(float);
    unsigned grid = (unsigned)(nq < 4096 ? nq : 4096);
    if (dt == MECUCO_BF16)
        knn_fallback_kernel<__nv_bfloat16, false><<<grid, FB_WARPS * 32, smem, s>>>(
            (const __nv_bfloat16 *)X, N, m, ld, q0, nq, k, include_self, flags, idx_out, dist_out, ctr, nullptr, 0, 0);
    else
        knn_fallback_kernel<float, false><<<grid, FB_WARPS * 32, smem, s>>>(
            (const float *)X, N, m, ld, q0, nq, k, include_self, flags, idx_out, dist_out, ctr, nullptr, 0, 0);
    return cudaGetLastError();
}

// Batched forms: the rows of every dataset of a table, one launch.
cudaError_t launch_knn_rerank_batch(const KnnSet *sets, int nsets, int64_t nrows, int lmax, mecuco_dtype dt,
                                    DevCounters *ctr, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    if (lmax > RR_MAXL) return cudaErrorInvalidValue;
    size_t smem = (size_t)RR_WARPS * lmax * 3 * sizeof(float);
    dim3 grid((unsigned)((nrows + RR_WARPS - 1) / RR_WARPS)), block(RR_WARPS * 32);
    cudaError_t e;
    if (dt == MECUCO_BF16) {
        e = cudaFuncSetAttribute(knn_rerank_kernel<__nv_bfloat16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        knn_rerank_kernel<__nv_bfloat16, true><<<grid, block, smem, s>>>(nullptr, 0, 0, 0, nullptr, 0, nrows, 0, 0, 0,
                                                                         nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                         ctr, sets, nsets, lmax, nullptr, nullptr, 0);
    } else {
        e = cudaFuncSetAttribute(knn_rerank_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        knn_rerank_kernel<float, true><<<grid, block, smem, s>>>(nullptr, 0, 0, 0, nullptr, 0, nrows, 0, 0, 0, nullptr,
                                                                 nullptr, nullptr, nullptr, nullptr, ctr, sets, nsets,
                                                                 lmax, nullptr, nullptr, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_knn_fallback_batch(const KnnSet *sets, int nsets, int64_t nrows, int kmax, mecuco_dtype dt,
                                      DevCounters *ctr, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    size_t smem = (size_t)FB_WARPS * kmax * 3 * sizeof(float);
    unsigned grid = (unsigned)(nrows < 4096 ? nrows : 4096);
    if (dt == MECUCO_BF16)
        knn_fallback_kernel<__nv_bfloat16, true><<<grid, FB_WARPS * 32, smem, s>>>(
            nullptr, 0, 0, 0, 0, nrows, 0, 0, nullptr, nullptr, nullptr, ctr, sets, nsets, kmax);
    else
        knn_fallback_kernel<float, true><<<grid, FB_WARPS * 32, smem, s>>>(
            nullptr, 0, 0, 0, 0, nrows, 0, 0, nullptr, nullptr, nullptr, ctr, sets, nsets, kmax);
    return cudaGetLastError();
}

}  // namespace mecuco
