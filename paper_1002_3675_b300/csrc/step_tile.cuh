// Device-side block of the step norm |f_k+1 - f_k| of Algorithm A1 (shared by the
// single-request and batched kernels, so both give the same partials bit for bit).
#pragma once
#include "cbct_internal.h"

namespace cbct {

constexpr int STEP_THREADS = 256;

// Block blk (256 voxels): f = v and partial[blk] = sum of (v - f_old)^2, float32
// within a warp (shuffle tree), float64 across the 8 warps in order.
__device__ __forceinline__ void step_block(const float *__restrict__ v, float *__restrict__ f, size_t n,
                                           double *__restrict__ partial, size_t blk) {
    __shared__ double sh[STEP_THREADS / 32];
    const size_t o = blk * STEP_THREADS + threadIdx.x;
    float d2 = 0.f;
    if (o < n) {
        const float nv = v[o];
        const float dv = __fsub_rn(nv, f[o]);
        d2 = __fmul_rn(dv, dv);
        f[o] = nv;
    }
    for (int off = 16; off > 0; off >>= 1) d2 = __fadd_rn(d2, __shfl_down_sync(0xffffffffu, d2, off));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < STEP_THREADS / 32; ++w) s += sh[w];
        partial[blk] = s;
    }
    __syncthreads();
}

}  // namespace cbct
