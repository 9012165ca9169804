// Device-side blocks of the step norm |f_k+1 - f_k| of Algorithm A1 and of the power
// iteration's dot products and scaling (shared by the single-request and batched
// kernels, so both give the same partials bit for bit).
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

// Energy finalisation: the three float64 sums of a trace entry at once, one group of
// 256 threads per array (block of ENERGY_THREADS): group g sums its array strided by
// 256 (thread q: p[q], p[q + 256], ...), then by a fixed tree, so each sum is that of a
// single 256-thread block.  out[g] (shared) receives sum g; n = 0 gives 0.
constexpr int ENERGY_THREADS = 768;
__device__ __forceinline__ void sum3_fixed(const double *p0, int n0, const double *p1, int n1, const double *p2,
                                           int n2, double *out) {
    __shared__ double sh[ENERGY_THREADS];
    const int grp = threadIdx.x >> 8, q0 = threadIdx.x & 255;
    const double *p = grp == 0 ? p0 : grp == 1 ? p1 : p2;
    const int n = grp == 0 ? n0 : grp == 1 ? n1 : n2;
    double s = 0.0;
    for (int q = q0; q < n; q += 256) s += p[q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (q0 < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (q0 == 0) out[grp] = sh[threadIdx.x];
    __syncthreads();
}

// Power iteration: tiles of VEC_TILE elements, 4 per thread of a 256-thread block.
constexpr int VEC_THREADS = 256;
constexpr int VEC_TILE = 4 * VEC_THREADS;
__host__ __device__ __forceinline__ long vec_tiles(long n) { return (n + VEC_TILE - 1) / VEC_TILE; }

// partial[2 t] = <x, y>, partial[2 t + 1] = <y, y> over tile t: float32 per thread (4
// elements in order) and within a warp (pairwise tree), float64 across the 8 warps.
__device__ __forceinline__ void dot2_tile(const float *__restrict__ x, const float *__restrict__ y, long n,
                                          long t, double *__restrict__ partial) {
    __shared__ double a[VEC_THREADS / 32], b[VEC_THREADS / 32];
    float sxy = 0.f, syy = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long o = t * VEC_TILE + q * VEC_THREADS + threadIdx.x;
        if (o < n) {
            const float xv = x[o], yv = y[o];
            sxy = __fmaf_rn(xv, yv, sxy);
            syy = __fmaf_rn(yv, yv, syy);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sxy = __fadd_rn(sxy, __shfl_down_sync(0xffffffffu, sxy, off));
        syy = __fadd_rn(syy, __shfl_down_sync(0xffffffffu, syy, off));
    }
    if ((threadIdx.x & 31) == 0) {
        a[threadIdx.x >> 5] = (double)sxy;
        b[threadIdx.x >> 5] = (double)syy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < VEC_THREADS / 32; ++w) {
            s1 += a[w];
            s2 += b[w];
        }
        partial[2 * t] = s1;
        partial[2 * t + 1] = s2;
    }
    __syncthreads();
}

// x = y * scale over tile t
__device__ __forceinline__ void scale_tile(const float *y, const float *scale, float *x, long n, long t) {
    const float sc = *scale;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long o = t * VEC_TILE + q * VEC_THREADS + threadIdx.x;
        if (o < n) x[o] = __fmul_rn(y[o], sc);
    }
}

}  // namespace cbct
