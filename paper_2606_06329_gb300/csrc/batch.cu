// batch.cu - per-call output pointers of a batched call, written into its
// device tables.  The tables (one KnnSet per dataset, one PatchSeg per
// estimator segment) are cached by content across calls; only the outputs
// (neighbour lists and curvatures) change from call to call, and they reach
// the tables through this kernel's parameters, so that a call captured into a
// CUDA graph replays with its own outputs and without any host copy.
#include "common.cuh"
#include "kernels.h"

namespace mecuco {

namespace {
struct PatchArgs {
    BatchOut out[BATCH_PATCH_SETS];  // datasets t0 .. t0 + count - 1 (table order)
};
}  // namespace

__global__ void batch_patch_kernel(KnnSet *__restrict__ sets, PatchSeg *__restrict__ segs,
                                   const SegRef *__restrict__ refs, int nsegs, int t0, int count,
                                   const __grid_constant__ PatchArgs args) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) sets[t0 + i].idx = args.out[i].idx;
    for (int g = i; g < nsegs; g += gridDim.x * blockDim.x) {
        const int t = refs[g].set - t0;
        if (t < 0 || t >= count) continue;
        PatchSeg &sg = segs[g];
        sg.kappa = args.out[t].kappa + refs[g].a;
        sg.idx = args.out[t].idx + refs[g].a * sg.k;
    }
}

cudaError_t launch_batch_patch(KnnSet *sets, int nsets, PatchSeg *segs, const SegRef *refs, int nsegs,
                               const BatchOut *outs, cudaStream_t s) {
    for (int t0 = 0; t0 < nsets; t0 += BATCH_PATCH_SETS) {
        const int count = nsets - t0 < BATCH_PATCH_SETS ? nsets - t0 : BATCH_PATCH_SETS;
        PatchArgs a;
        for (int i = 0; i < count; ++i) a.out[i] = outs[t0 + i];
        const int work = count > nsegs ? count : nsegs;
        const unsigned grid = (unsigned)((work + 255) / 256 < 1024 ? (work + 255) / 256 : 1024);
        batch_patch_kernel<<<grid, 256, 0, s>>>(sets, segs, refs, nsegs, t0, count, a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mecuco
