// fidelity.cu - the paper's agreement metrics between two curvature vectors a
// (reference, e.g. the original method) and b (e.g. MeCuCo): the mean absolute
// error, Spearman's rank correlation rho_S and Chatterjee's xi, optionally
// after min-max normalisation of each vector to [0, 1] (Sec. experiments,
// "curvature fidelity"; "The Effect of Normalization").
//
//   min-max:   x' = (x - min x) / (max x - min x)   (0 when max = min)
//   MAE:       sum |a_i - b_i| / n
//   rho_S:     Pearson correlation of the average ranks of a and of b
//   xi:        with the pairs ordered by a (ties by index), r_i = #{j: b_j <= b_(i)}
//              and l_i = #{j: b_j >= b_(i)}:
//              xi = 1 - n sum_{i<n} |r_{i+1} - r_i| / (2 sum_i l_i (n - l_i))
//              (Chatterjee 2021, the form that allows ties; it reduces to
//              1 - 3 sum |r_{i+1} - r_i| / (n^2 - 1) without ties in b).
//
// Min-max normalisation is strictly increasing, so rho_S and xi are taken on
// the ranks of the raw vectors (FP32 rounding of the normalised values could
// merge distinct values into ties); only the MAE uses the normalised values.
// Inputs are finite.  rho_S = 0 when either vector is constant, xi = 0 when b is.
//
// Ranks come from a stable LSD radix sort (four 8-bit passes of histogram,
// scan and stable scatter) of an order-preserving unsigned image of the float
// keys; tie groups are found by binary search in the sorted keys.  Sums are
// taken in FP64 as fixed-order block partials (deterministic).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mecuco {

namespace {
constexpr int FT = 256;                 // threads per block
constexpr int FITEMS = 8;               // keys per thread in the sort
constexpr int FTILE = FT * FITEMS;      // keys per sort block

__device__ __forceinline__ uint32_t key_of(float f) {
    uint32_t u = f == 0.f ? 0u : __float_as_uint(f);  // -0 and +0 are one value
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void keys_kernel(const float *__restrict__ x, int64_t n, uint32_t *__restrict__ key, int32_t *__restrict__ id) {
    const int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x;
    if (i < n) { key[i] = key_of(x[i]); id[i] = (int32_t)i; }
}

// per-block digit histogram: counts[digit * nblocks + block]
__global__ void hist_kernel(const uint32_t *__restrict__ key, int64_t n, int shift, int nblocks,
                            uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * FTILE;
    for (int r = 0; r < FITEMS; ++r) {
        const int64_t i = base + r * FT + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of cnt entries in place (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t *__restrict__ c, int64_t cnt) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < cnt; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < cnt ? c[i] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const uint32_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < cnt) c[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

// stable scatter: elements in round-major order r * FT + tid; rank among equal
// digits = earlier rounds + earlier warps of this round + earlier lanes
__global__ void scatter_kernel(const uint32_t *__restrict__ key, const int32_t *__restrict__ id, int64_t n, int shift,
                               int nblocks, const uint32_t *__restrict__ offs, uint32_t *__restrict__ key_out,
                               int32_t *__restrict__ id_out) {
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcnt[FT / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    running[tid] = 0;
    const int64_t base = (int64_t)blockIdx.x * FTILE;
    for (int r = 0; r < FITEMS; ++r) {
        for (int w = 0; w < FT / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t i = base + r * FT + tid;
        const bool live = i < n;
        const uint32_t k = live ? key[i] : 0u;
        const int d = live ? (int)((k >> shift) & 255) : 256 + lane;  // dead lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = __popc(peers & ((1u << lane) - 1u));
        if (live && before == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (live) {
            uint32_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + running[d] + (uint32_t)before;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            key_out[pos] = k;
            id_out[pos] = id[i];
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < FT / 32; ++w) add += wcnt[w][tid];
        running[tid] += add;
        __syncthreads();
    }
}

// tie groups of the sorted keys by binary search: first / last position of
// each position's key; scattered back to the original index
__global__ void ranks_kernel(const uint32_t *__restrict__ skey, const int32_t *__restrict__ sid, int64_t n,
                             double *__restrict__ avg_rank, int64_t *__restrict__ le_count,
                             int64_t *__restrict__ ge_count) {
    const int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = skey[i];
    int64_t lo = 0, hi = i;  // first position with key == k
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (skey[mid] < k) lo = mid + 1; else hi = mid;
    }
    const int64_t first = lo;
    lo = i; hi = n - 1;      // last position with key == k
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (skey[mid] > k) hi = mid - 1; else lo = mid;
    }
    const int64_t last = lo;
    const int32_t j = sid[i];
    if (avg_rank) avg_rank[j] = 0.5 * (double)(first + last) + 1.0;
    if (le_count) le_count[j] = last + 1;
    if (ge_count) ge_count[j] = n - first;
}

__global__ void minmax_kernel(const float *__restrict__ x, int64_t n, float *__restrict__ part) {
    __shared__ float smin[FT], smax[FT];
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        mn = fminf(mn, x[i]);
        mx = fmaxf(mx, x[i]);
    }
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int o = FT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = smin[0]; part[2 * blockIdx.x + 1] = smax[0]; }
}

__global__ void normalize_kernel(const float *__restrict__ x, int64_t n, const float *__restrict__ part, int nparts,
                                 float *__restrict__ y) {
    __shared__ float s_mn, s_mx;
    if (threadIdx.x == 0) {
        float mn = INFINITY, mx = -INFINITY;
        for (int p = 0; p < nparts; ++p) { mn = fminf(mn, part[2 * p]); mx = fmaxf(mx, part[2 * p + 1]); }
        s_mn = mn;
        s_mx = mx;
    }
    __syncthreads();
    const float range = s_mx - s_mn;
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        y[i] = range > 0.f ? (x[i] - s_mn) / range : 0.f;
}

// block partials (fixed order): 0 sum|a-b|, 1 sum ra, 2 sum rb, 3 sum ra^2, 4 sum rb^2,
// 5 sum ra rb, 6 sum |r_{i+1} - r_i| (order of a), 7 sum l (n - l)
constexpr int NSUMS = 8;

__global__ void sums_kernel(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                            const double *__restrict__ ra, const double *__restrict__ rb,
                            const int32_t *__restrict__ perm_a, const int64_t *__restrict__ le_b,
                            const int64_t *__restrict__ ge_b, double *__restrict__ part) {
    __shared__ double s[NSUMS][FT];
    double acc[NSUMS] = {};
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        acc[0] += fabs((double)a[i] - (double)b[i]);
        acc[1] += ra[i];
        acc[2] += rb[i];
        acc[3] += ra[i] * ra[i];
        acc[4] += rb[i] * rb[i];
        acc[5] += ra[i] * rb[i];
        const int32_t p = perm_a[i];
        if (i + 1 < n) acc[6] += fabs((double)(le_b[perm_a[i + 1]] - le_b[p]));
        const double l = (double)ge_b[p];
        acc[7] += l * ((double)n - l);
    }
    for (int q = 0; q < NSUMS; ++q) s[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int o = FT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < NSUMS; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < NSUMS) part[(int64_t)blockIdx.x * NSUMS + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void finish_kernel(const double *__restrict__ part, int nparts, int64_t n, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t[NSUMS] = {};
    for (int p = 0; p < nparts; ++p)
        for (int q = 0; q < NSUMS; ++q) t[q] += part[(int64_t)p * NSUMS + q];
    const double nn = (double)n;
    out[0] = t[0] / nn;
    const double cov = t[5] - t[1] * t[2] / nn;
    const double va = t[3] - t[1] * t[1] / nn, vb = t[4] - t[2] * t[2] / nn;
    out[1] = (va > 0.0 && vb > 0.0) ? cov / sqrt(va * vb) : 0.0;
    out[2] = t[7] > 0.0 ? 1.0 - nn * t[6] / (2.0 * t[7]) : 0.0;
}
}  // namespace

size_t fidelity_scratch_bytes(int64_t n) {
    const int64_t nb = (n + FTILE - 1) / FTILE;
    // keys x2, indices x2, ranks of a and b, <= and >= counts of b, order of a, normalised a and b
    return (size_t)n * (2 * sizeof(uint32_t) + 2 * sizeof(int32_t) + 2 * sizeof(double) + 2 * sizeof(int64_t) +
                        sizeof(int32_t) + 2 * sizeof(float)) +
           (size_t)256 * nb * sizeof(uint32_t) + (size_t)1024 * NSUMS * sizeof(double) + 4096 * sizeof(float) +
           16 * 256;
}

namespace {
// stable sort of x's keys; sorted keys in *skey, original indices in *sid
cudaError_t sort_keys(const float *x, int64_t n, uint32_t *k0, int32_t *i0, uint32_t *k1, int32_t *i1,
                      uint32_t *counts, uint32_t **skey, int32_t **sid, cudaStream_t s) {
    const unsigned gb = (unsigned)((n + FT - 1) / FT);
    const int nb = (int)((n + FTILE - 1) / FTILE);
    keys_kernel<<<gb, FT, 0, s>>>(x, n, k0, i0);
    for (int pass = 0; pass < 4; ++pass) {
        hist_kernel<<<nb, FT, 0, s>>>(k0, n, 8 * pass, nb, counts);
        scan_kernel<<<1, 1024, 0, s>>>(counts, (int64_t)256 * nb);
        scatter_kernel<<<nb, FT, 0, s>>>(k0, i0, n, 8 * pass, nb, counts, k1, i1);
        uint32_t *tk = k0; k0 = k1; k1 = tk;
        int32_t *ti = i0; i0 = i1; i1 = ti;
    }
    *skey = k0;
    *sid = i0;
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fidelity(const float *a, const float *b, int64_t n, int normalize, void *scratch, double *out,
                            cudaStream_t s) {
    if (n < 2) return cudaErrorInvalidValue;
    char *p = static_cast<char *>(scratch);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += (bytes + 255) / 256 * 256;
        return r;
    };
    const int nb = (int)((n + FTILE - 1) / FTILE);
    uint32_t *k0 = reinterpret_cast<uint32_t *>(take(n * sizeof(uint32_t)));
    uint32_t *k1 = reinterpret_cast<uint32_t *>(take(n * sizeof(uint32_t)));
    int32_t *i0 = reinterpret_cast<int32_t *>(take(n * sizeof(int32_t)));
    int32_t *i1 = reinterpret_cast<int32_t *>(take(n * sizeof(int32_t)));
    uint32_t *counts = reinterpret_cast<uint32_t *>(take((size_t)256 * nb * sizeof(uint32_t)));
    double *ra = reinterpret_cast<double *>(take(n * sizeof(double)));
    double *rb = reinterpret_cast<double *>(take(n * sizeof(double)));
    int64_t *le_b = reinterpret_cast<int64_t *>(take(n * sizeof(int64_t)));
    int64_t *ge_b = reinterpret_cast<int64_t *>(take(n * sizeof(int64_t)));
    int32_t *perm_a = reinterpret_cast<int32_t *>(take(n * sizeof(int32_t)));
    float *na = reinterpret_cast<float *>(take(n * sizeof(float)));
    float *nbv = reinterpret_cast<float *>(take(n * sizeof(float)));
    float *mm = reinterpret_cast<float *>(take(4096 * sizeof(float)));  // min/max partials of a, then b
    double *part = reinterpret_cast<double *>(take((size_t)1024 * NSUMS * sizeof(double)));
    const unsigned g = (unsigned)std::min<int64_t>(1024, (n + FT - 1) / FT);
    const float *ea = a, *eb = b;  // the values the MAE is taken on
    if (normalize) {
        minmax_kernel<<<g, FT, 0, s>>>(a, n, mm);
        normalize_kernel<<<g, FT, 0, s>>>(a, n, mm, (int)g, na);
        minmax_kernel<<<g, FT, 0, s>>>(b, n, mm + 2048);
        normalize_kernel<<<g, FT, 0, s>>>(b, n, mm + 2048, (int)g, nbv);
        ea = na;
        eb = nbv;
    }
    const unsigned gb = (unsigned)((n + FT - 1) / FT);
    uint32_t *skey;
    int32_t *sid;
    // a: average ranks and the order of a (ties by index: the sort is stable)
    cudaError_t e = sort_keys(a, n, k0, i0, k1, i1, counts, &skey, &sid, s);
    if (e != cudaSuccess) return e;
    ranks_kernel<<<gb, FT, 0, s>>>(skey, sid, n, ra, nullptr, nullptr);
    e = cudaMemcpyAsync(perm_a, sid, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // b: average ranks, #{b_j <= b_i} and #{b_j >= b_i}
    e = sort_keys(b, n, k0, i0, k1, i1, counts, &skey, &sid, s);
    if (e != cudaSuccess) return e;
    ranks_kernel<<<gb, FT, 0, s>>>(skey, sid, n, rb, le_b, ge_b);
    sums_kernel<<<g, FT, 0, s>>>(ea, eb, n, ra, rb, perm_a, le_b, ge_b, part);
    finish_kernel<<<1, 32, 0, s>>>(part, (int)g, n, out);
    return cudaGetLastError();
}

cudaError_t launch_minmax_normalize(const float *x, int64_t n, float *y, void *scratch, cudaStream_t s) {
    if (n < 1) return cudaErrorInvalidValue;
    float *mm = static_cast<float *>(scratch);
    const unsigned g = (unsigned)std::min<int64_t>(1024, (n + FT - 1) / FT);
    minmax_kernel<<<g, FT, 0, s>>>(x, n, mm);
    normalize_kernel<<<g, FT, 0, s>>>(x, n, mm, (int)g, y);
    return cudaGetLastError();
}

}  // namespace mecuco
