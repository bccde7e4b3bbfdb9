// patch_gather.cuh - shared-memory staging helpers of the tensor-core patch
// kernels: the raw gather of 8-column units of neighbour rows (into registers,
// or into a multi-stage ring by cp.async), the bank-conflict-free FP32 staging
// stores, BF16 packing and the offset of a 16-byte unit in a
// 128-byte-swizzled K-major operand tile.
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
    // unit g of row r in a gather ring stage (see raw_off)
    __device__ __forceinline__ void store_raw(uint8_t *stage, int r, int g) const;
    __device__ __forceinline__ void load_raw(const uint8_t *stage, int r, int g);
    __device__ __forceinline__ void to_float(float (&f)[8]) const {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            f[2 * e] = __uint_as_float(w[e] << 16);
            f[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
        }
    }
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
    __device__ __forceinline__ void store_raw(uint8_t *stage, int r, int g) const;
    __device__ __forceinline__ void load_raw(const uint8_t *stage, int r, int g);
    __device__ __forceinline__ void to_float(float (&f)[8]) const {
        f[0] = lo.x, f[1] = lo.y, f[2] = lo.z, f[3] = lo.w, f[4] = hi.x, f[5] = hi.y, f[6] = hi.z, f[7] = hi.w;
    }
    __device__ __forceinline__ void store(float *dst, bool swap) const { store_halves(dst, lo, hi, swap); }
};

// Gather ring: stages of raw copies of a chunk (64 rows x 64 columns of T)
// filled by 16-byte cp.async copies, which go through L2 only and hold no
// registers, so that several chunks of a patch are in flight.  Thread (row r,
// unit g) of the 256 producers issues unit g (8 columns) of rows r and r + 32,
// eight threads covering a row's 128 (BF16) or 256 (FP32) contiguous bytes;
// lane l of warp u later reads unit u of rows l and l + 32 (centre_lane).  The
// 16-byte pieces of a row are stored XOR-swizzled by the row index, so both
// the copies and the column reads hit every bank once.  Units that are not
// whole, aligned and live (rows past k, the ragged end of m, unaligned rows)
// are written with plain stores, zero past m.  The caller orders copies, reads
// and reuse of a stage with cp.async.wait_group and a CTA barrier.
template <typename T>
__host__ __device__ constexpr int raw_stage_bytes() {
    return 64 * 64 * (int)sizeof(T);
}
template <typename T>
__device__ __forceinline__ uint32_t raw_off(int r, int piece) {
    constexpr int PR = 4 * (int)sizeof(T);  // 16-byte pieces per row: 8 (BF16), 16 (FP32)
    return (uint32_t)(r * PR * 16 + ((piece ^ (r & (PR - 1))) << 4));
}
__device__ __forceinline__ void Unit8<__nv_bfloat16>::store_raw(uint8_t *stage, int r, int g) const {
    *reinterpret_cast<uint4 *>(stage + raw_off<__nv_bfloat16>(r, g)) = v;
}
__device__ __forceinline__ void Unit8<__nv_bfloat16>::load_raw(const uint8_t *stage, int r, int g) {
    v = *reinterpret_cast<const uint4 *>(stage + raw_off<__nv_bfloat16>(r, g));
}
__device__ __forceinline__ void Unit8<float>::store_raw(uint8_t *stage, int r, int g) const {
    *reinterpret_cast<float4 *>(stage + raw_off<float>(r, 2 * g)) = lo;
    *reinterpret_cast<float4 *>(stage + raw_off<float>(r, 2 * g + 1)) = hi;
}
__device__ __forceinline__ void Unit8<float>::load_raw(const uint8_t *stage, int r, int g) {
    lo = *reinterpret_cast<const float4 *>(stage + raw_off<float>(r, 2 * g));
    hi = *reinterpret_cast<const float4 *>(stage + raw_off<float>(r, 2 * g + 1));
}
template <typename T>
__device__ __forceinline__ void raw_issue(uint8_t *stage, int r, int g, const T *row, bool live, int64_t a, int64_t m,
                                          bool vec) {
    constexpr int PP = (int)sizeof(T) / 2;  // 16-byte pieces per unit
    if (live && vec && a + 8 <= m) {
        const uint32_t s = (uint32_t)__cvta_generic_to_shared(stage);
        const char *src = reinterpret_cast<const char *>(row + a);
#pragma unroll
        for (int h = 0; h < PP; ++h)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s + raw_off<T>(r, g * PP + h)),
                         "l"(src + 16 * h)
                         : "memory");
    } else {
        Unit8<T> u;
        if (live) u.load(row, a, m, vec);
        else u.zero();
        u.store_raw(stage, r, g);
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Sum over the 32 lanes of a warp, for each of 8 columns held by every lane
// (s[e], column e): three reduce-scatter steps leave lane l with the sum over
// the eight lanes that share l's bits 0-1 of column c(l) = 4 b4 + 2 b3 + b2 (b
// the bits of l), two butterfly steps complete it over all 32 lanes (the four
// lanes of a column add the same two terms in swapped order, so they hold the
// same value), and eight broadcasts return all 8 column sums to every lane.
// 17 shuffles instead of 40 for eight full butterflies; a fixed order, so
// every caller gets identical sums from identical inputs.
__device__ __forceinline__ void warp_colsum8(float (&s)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float t[4], u[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? s[i] : s[i + 4], keep = b4 ? s[i + 4] : s[i];
        t[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? t[i] : t[i + 2], keep = b3 ? t[i + 2] : t[i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c;
    {
        const float send = b2 ? u[0] : u[1], keep = b2 ? u[1] : u[0];
        c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
#pragma unroll
    for (int e = 0; e < 8; ++e) s[e] = __shfl_sync(0xffffffffu, c, ((e & 4) << 2) | ((e & 2) << 2) | ((e & 1) << 2));
}

// Centre one chunk of a patch from a gather ring stage: lane l of the calling
// warp takes rows l and l + 32 of unit u (columns 8u .. 8u + 7); the column
// means over the k rows come from warp_colsum8 (rows past k are zero in the
// stage), and x = v - mean for rows below k, 0 past k (and past m, where the
// stage holds zeros).  Every pass that centres a patch calls this, so all of
// them see the same values.
template <typename T>
__device__ __forceinline__ void centre_lane(const uint8_t *stage, int lane, int u, int k, float inv_k,
                                            float (&x0)[8], float (&x1)[8]) {
    Unit8<T> w0, w1;
    w0.load_raw(stage, lane, u);
    w1.load_raw(stage, lane + 32, u);
    float v0[8], v1[8], mean[8];
    w0.to_float(v0);
    w1.to_float(v1);
#pragma unroll
    for (int e = 0; e < 8; ++e) mean[e] = v0[e] + v1[e];
    warp_colsum8(mean, lane);
    const bool live0 = lane < k, live1 = lane + 32 < k;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float mu = mean[e] * inv_k;
        x0[e] = live0 ? v0[e] - mu : 0.f;
        x1[e] = live1 ? v1[e] - mu : 0.f;
    }
}

}  // namespace pg
}  // namespace mecuco
