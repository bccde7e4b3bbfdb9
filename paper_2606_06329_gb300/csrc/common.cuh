// common.cuh - device helpers shared by the MeCuCo CUDA kernels (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mecuco.h"

namespace mecuco {

// Bits OR-ed into the device status word (mirrors mecuco_status codes).
enum : unsigned {
    DEV_NOT_CONVERGED = 1u << MECUCO_ERR_NOT_CONVERGED,
    DEV_TIMEOUT = 1u << MECUCO_ERR_TIMEOUT,
    DEV_INVALID = 1u << MECUCO_ERR_INVALID_ARG,
};

// Device-side counters, one struct per context (zeroed at the start of a call).
struct DevCounters {
    unsigned long long knn_uncertified;
    unsigned long long knn_fallback_rows;
    unsigned long long jacobi_max_sweeps;
    unsigned long long jacobi_not_converged;
    unsigned long long rank_deficient;
    unsigned long long jacobi_rotations;  // plane rotations applied by the Jacobi sweeps
    unsigned status;
    unsigned pad;
};

// One run of consecutive points of one dataset within a launch over the points
// of a chunk.  A single-dataset call passes one segment by value; a batched
// call passes a device table of segments (one per dataset part in the chunk),
// and each CTA finds the segment of its point.  Pointers are those of the
// segment's first point; per-point rows follow with the segment's own k.
struct PatchSeg {
    const void *X;            // the dataset, row-major, leading dimension ld
    int64_t N, m, ld;
    int k;
    int first;                // first point (block) of the launch in this segment
    const int32_t *idx;       // neighbour lists (k per point)
    const int32_t *rowtab;    // third-moment pass: row table for this k
    float *G, *R, *Q;         // k x k, k, k x k per point
    float *sig, *U;           // eigenpairs: k and k x k per point
    float *kappa, *lambda, *s;// outputs: 1, k, k per point (lambda, s nullable)
};

// The segment of launch point `blk` and the point's index within it.
__device__ __forceinline__ const PatchSeg &find_seg(const PatchSeg &one, const PatchSeg *tab, int ntab, int blk,
                                                    int &local) {
    if (ntab == 0) {
        local = blk;
        return one;
    }
    int lo = 0, hi = ntab - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].first <= blk) lo = mid;
        else hi = mid - 1;
    }
    local = blk - tab[lo].first;
    return tab[lo];
}

// --- element loads ---------------------------------------------------------
__device__ __forceinline__ float load_elem(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_elem(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p)));
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// --- error-free transformations (Knuth TwoSum, FMA-based TwoProd) ----------
// A value is carried as an unevaluated sum hi + lo with |lo| <= ulp(hi)/2.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    float h = s + e;
    return ff{h, e - (h - s)};
}
// (x - y)^2 accumulated exactly enough: diff by TwoSum, square by FMA TwoProd.
__device__ __forceinline__ void ff_acc_sqdiff(ff &acc, float x, float y) {
    float dh, dl;
    two_sum(x, -y, dh, dl);
    float ph = dh * dh;
    float pl = fmaf(dh, dh, -ph) + 2.0f * dh * dl + dl * dl;
    float s, e;
    two_sum(acc.hi, ph, s, e);
    e += acc.lo + pl;
    acc.hi = s + e;
    acc.lo = e - (acc.hi - s);
}
__device__ __forceinline__ ff ff_shfl_xor(ff v, int mask) {
    return ff{__shfl_xor_sync(0xffffffffu, v.hi, mask), __shfl_xor_sync(0xffffffffu, v.lo, mask)};
}
__device__ __forceinline__ ff ff_warp_sum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
    return v;
}
// lexicographic (hi, lo, index) order of compensated distances
__device__ __forceinline__ bool ff_less(ff a, int ia, ff b, int ib) {
    if (a.hi != b.hi) return a.hi < b.hi;
    if (a.lo != b.lo) return a.lo < b.lo;
    return ia < ib;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void atomic_max_u64(unsigned long long *p, unsigned long long v) {
    atomicMax(p, v);
}

// ---- rotation of a patch chunk by a per-point orthogonal k x k matrix U0 ----
// Us[r][l] = U0[r][l] for r, l < k, zero elsewhere (all 64 x 64 entries).
__device__ __forceinline__ void load_rotation(const float *__restrict__ u, int k, float (*Us)[65]) {
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int r = e >> 6, l = e & 63;
        Us[r][l] = (r < k && l < k) ? u[r * k + l] : 0.f;
    }
}

// In-place Z = U0^T Xs for a row-major chunk Xs[row][column] (rows >= k stay
// zero).  256 threads: thread (l = tid & 63, column group cg = tid >> 6) forms
// row l of Z for NC columns cg*NC.. into registers; a barrier separates the
// reads from the writes.  Called by all threads, between barriers.
template <int NC, int LDX>
__device__ __forceinline__ void rotate_rows(float (*Xs)[LDX], const float (*Us)[65], int k, int cg, int l) {
    float z[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) z[c] = 0.f;
    for (int r = 0; r < k; ++r) {
        const float u = Us[r][l];
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c] = fmaf(u, Xs[r][cg * NC + c], z[c]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) Xs[l][cg * NC + c] = z[c];
    __syncthreads();
}

// The same for a column-major chunk Xs[column][row].
template <int NC, int LDX>
__device__ __forceinline__ void rotate_cols(float (*Xs)[LDX], const float (*Us)[65], int k, int cg, int l) {
    float z[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) z[c] = 0.f;
    for (int r = 0; r < k; ++r) {
        const float u = Us[r][l];
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c] = fmaf(u, Xs[cg * NC + c][r], z[c]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) Xs[cg * NC + c][l] = z[c];
    __syncthreads();
}

// In-place Y = U0 Y for a row-major chunk (the inverse rotation): thread
// (j = tid & 63, cg = tid >> 6) forms row j for NC columns; rows >= k of Y are
// never read.
template <int NC, int LDX>
__device__ __forceinline__ void unrotate_rows(float (*Ys)[LDX], const float (*Us)[65], int k, int cg, int j) {
    float z[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) z[c] = 0.f;
    for (int l = 0; l < k; ++l) {
        const float u = Us[j][l];
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c] = fmaf(u, Ys[l][cg * NC + c], z[c]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) Ys[j][cg * NC + c] = z[c];
    __syncthreads();
}

}  // namespace mecuco
