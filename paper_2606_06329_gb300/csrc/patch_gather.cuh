// patch_gather.cuh - shared-memory staging helpers of the tensor-core patch
// kernels: the raw gather of 8-column units of neighbour rows, the
// bank-conflict-free FP32 staging stores, BF16 packing and the offset of a
// 16-byte unit in a 128-byte-swizzled K-major operand tile.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mecuco {
namespace pg {

__device__ __forceinline__ uint32_t sw128(int row, int unit16) {
    // byte offset of 16-byte unit `unit16` (0..7) of `row` in a 128B-swizzled K-major tile
    return (uint32_t)(row * 128 + ((unit16 ^ (row & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// 32 bytes (lo, hi) of a lane at dst.  Eight lanes with consecutive 32-byte
// destinations write the lower halves in one 128-bit store and the upper halves
// in another; lanes 4..7 of each eight swap the two (swap = true), so that each
// store covers all 32 banks instead of hitting 16 of them twice.
__device__ __forceinline__ void store_halves(float *dst, float4 lo, float4 hi, bool swap) {
    reinterpret_cast<float4 *>(dst)[swap ? 1 : 0] = swap ? hi : lo;
    reinterpret_cast<float4 *>(dst)[swap ? 0 : 1] = swap ? lo : hi;
}
__device__ __forceinline__ void load_halves(const float *src, float4 &lo, float4 &hi, bool swap) {
    const float4 first = reinterpret_cast<const float4 *>(src)[swap ? 1 : 0];
    const float4 second = reinterpret_cast<const float4 *>(src)[swap ? 0 : 1];
    lo = swap ? second : first;
    hi = swap ? first : second;
}

// Raw gather of one 8-column unit of one row (zero past m).
template <typename T>
struct Unit8;
template <>
struct Unit8<__nv_bfloat16> {
    uint4 v;
    __device__ __forceinline__ void load(const __nv_bfloat16 *row, int64_t a, int64_t m, bool vec) {
        if (vec && a + 8 <= m) {
            v = __ldg(reinterpret_cast<const uint4 *>(row + a));
        } else {
            uint32_t h[8];
            for (int e = 0; e < 8; ++e)
                h[e] = (a + e < m) ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(row) + a + e) : 0u;
            v = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
    }
    __device__ __forceinline__ void zero() { v = make_uint4(0, 0, 0, 0); }
    // swap: write the upper 16 bytes first (see store_halves)
    __device__ __forceinline__ void store(float *dst, bool swap) const {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        float f[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            f[2 * e] = __uint_as_float(w[e] << 16);
            f[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
        }
        store_halves(dst, make_float4(f[0], f[1], f[2], f[3]), make_float4(f[4], f[5], f[6], f[7]), swap);
    }
};
template <>
struct Unit8<float> {
    float4 lo, hi;
    __device__ __forceinline__ void load(const float *row, int64_t a, int64_t m, bool vec) {
        if (vec && a + 8 <= m) {
            lo = __ldg(reinterpret_cast<const float4 *>(row + a));
            hi = __ldg(reinterpret_cast<const float4 *>(row + a) + 1);
        } else {
            float f[8];
            for (int e = 0; e < 8; ++e) f[e] = (a + e < m) ? __ldg(row + a + e) : 0.f;
            lo = make_float4(f[0], f[1], f[2], f[3]);
            hi = make_float4(f[4], f[5], f[6], f[7]);
        }
    }
    __device__ __forceinline__ void zero() { lo = hi = make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ void store(float *dst, bool swap) const { store_halves(dst, lo, hi, swap); }
};
// Centre the staged chunk Xs (64 rows of row stride LD, rows past k zero) in
// place: thread (column cc, rows 16 rg .. 16 rg + 15) sums its 16 values,
// the four partial sums of a column (Part[rg * 64 + cc]) give its mean over the
// k rows, and x = v - mean (0 past k) goes to x[] and back to Xs.  Called by
// the 256 threads of named barrier 1 right after the chunk was staged; the
// same operations in the same order wherever the patch is centred, so every
// pass sees the same values.
template <int LD>
__device__ __forceinline__ void centre_chunk(float *Xs, float *Part, int cc, int rg, int k, float inv_k,
                                             float (&x)[16]) {
    asm volatile("bar.sync 1, 256;" ::: "memory");
    float v[16], sum = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        v[e] = Xs[(rg * 16 + e) * LD + cc];
        sum += v[e];
    }
    Part[rg * 64 + cc] = sum;
    asm volatile("bar.sync 1, 256;" ::: "memory");
    const float mean = (Part[cc] + Part[64 + cc] + Part[128 + cc] + Part[192 + cc]) * inv_k;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        x[e] = (rg * 16 + e < k) ? v[e] - mean : 0.f;
        Xs[(rg * 16 + e) * LD + cc] = x[e];
    }
}

}  // namespace pg
}  // namespace mecuco
