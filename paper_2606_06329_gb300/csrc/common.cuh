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
    unsigned status;
    unsigned pad;
};

// --- element loads ---------------------------------------------------------
__device__ __forceinline__ float load_elem(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_elem(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p)));
}

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

}  // namespace mecuco
