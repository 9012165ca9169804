// Device-side block of the TV prox sweep (shared by the single-request and batched
// kernels).
#pragma once

// Step 2 (and 3) of Algorithm A1 (Jia et al. 2010): one projected-gradient step on
//   Phi(f) = TV_eps(f) + beta/2 |f - g|^2,   f >= 0,
// where TV_eps is E1 of Eq. 1 read as the forward-difference total variation with
// Neumann boundary.  Isotropic (A.aniso == 0): sum_j sqrt(|grad f|_j^2 + eps^2), whose
// gradient sum_d D_d^T (D_d f / |grad f|_eps) is a 13-point stencil per voxel.
// Anisotropic (A.aniso == 1): sum_j sum_d sqrt((D_d f)_j^2 + eps^2), gradient
// sum_d D_d^T (D_d f / sqrt((D_d f)^2 + eps^2)), a 7-point stencil.  In both,
//   (D_d^T p)_i = (p_{i-1} [i > 0] - p_i [i < n-1]) / h_d.
// The sweep also emits the partial sums of |grad f|_eps of its input (the
// E1 energy of the entering iterate when the input is f_k).
//
// Layout [nx][ny][nz] (z fastest); one thread per voxel, consecutive lanes along z.
#include "cbct_internal.h"

namespace cbct {

constexpr int TV_THREADS = 256;

// grad TV_eps at voxel idx (internal layout) and, if E1, the voxel's term of TV_eps
// itself (|grad f|_eps, or the sum over the axes in the anisotropic reading).  Shared
// by the prox sweep and the energy gradient of the multigrid cycle.
template <bool E1>
__device__ __forceinline__ float tv_div(const TvArgs &A, const float *__restrict__ fin, const size_t idx, float &e1) {
    const int k = (int)(idx % A.nz);
    const size_t t = idx / A.nz;
    const int j = (int)(t % A.ny);
    const int i = (int)(t / A.ny);
    const size_t sx = (size_t)A.ny * A.nz, sy = A.nz;
    const bool xp = i < A.nx - 1, yp = j < A.ny - 1, zp = k < A.nz - 1;
    const float f0 = __ldg(fin + idx);
    // every rounding spelled out (no compiler contraction), so the result does not
    // depend on the kernel this body is inlined into
    // own gradient (zero difference at the last index)
    const float gx = __fmul_rn(__fsub_rn(xp ? __ldg(fin + idx + sx) : f0, f0), A.ihx);
    const float gy = __fmul_rn(__fsub_rn(yp ? __ldg(fin + idx + sy) : f0, f0), A.ihy);
    const float gz = __fmul_rn(__fsub_rn(zp ? __ldg(fin + idx + 1) : f0, f0), A.ihz);
    float div;
    if (A.aniso) {
        // each axis smoothed on its own: p_d = D_d f / sqrt((D_d f)^2 + eps^2)
        const float qx = __fmaf_rn(gx, gx, A.eps2), qy = __fmaf_rn(gy, gy, A.eps2), qz = __fmaf_rn(gz, gz, A.eps2);
        const float rx = rsqrtf(qx), ry = rsqrtf(qy), rz = rsqrtf(qz);
        div = -__fmaf_rn(__fmul_rn(gx, rx), A.ihx,
                         __fmaf_rn(__fmul_rn(gy, ry), A.ihy, __fmul_rn(__fmul_rn(gz, rz), A.ihz)));
        if (E1) e1 = __fadd_rn(__fadd_rn(__fmul_rn(qx, rx), __fmul_rn(qy, ry)), __fmul_rn(qz, rz));
        if (i > 0) {
            const float a = __fmul_rn(__fsub_rn(f0, __ldg(fin + idx - sx)), A.ihx);
            div = __fmaf_rn(__fmul_rn(a, rsqrtf(__fmaf_rn(a, a, A.eps2))), A.ihx, div);
        }
        if (j > 0) {
            const float a = __fmul_rn(__fsub_rn(f0, __ldg(fin + idx - sy)), A.ihy);
            div = __fmaf_rn(__fmul_rn(a, rsqrtf(__fmaf_rn(a, a, A.eps2))), A.ihy, div);
        }
        if (k > 0) {
            const float a = __fmul_rn(__fsub_rn(f0, __ldg(fin + idx - 1)), A.ihz);
            div = __fmaf_rn(__fmul_rn(a, rsqrtf(__fmaf_rn(a, a, A.eps2))), A.ihz, div);
        }
    } else {
        const float q0 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmaf_rn(gz, gz, A.eps2)));
        const float n0 = rsqrtf(q0);
        div = -__fmul_rn(__fmaf_rn(gx, A.ihx, __fmaf_rn(gy, A.ihy, __fmul_rn(gz, A.ihz))), n0);
        if (E1) e1 = __fmul_rn(q0, n0);
        // p_x at i-1
        if (i > 0) {
            const float fm = __ldg(fin + idx - sx);
            const float ax = __fmul_rn(__fsub_rn(f0, fm), A.ihx);
            const float ay = __fmul_rn(__fsub_rn(yp ? __ldg(fin + idx - sx + sy) : fm, fm), A.ihy);
            const float az = __fmul_rn(__fsub_rn(zp ? __ldg(fin + idx - sx + 1) : fm, fm), A.ihz);
            const float n = rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2))));
            div = __fmaf_rn(__fmul_rn(ax, n), A.ihx, div);
        }
        // p_y at j-1
        if (j > 0) {
            const float fm = __ldg(fin + idx - sy);
            const float ax = __fmul_rn(__fsub_rn(xp ? __ldg(fin + idx - sy + sx) : fm, fm), A.ihx);
            const float ay = __fmul_rn(__fsub_rn(f0, fm), A.ihy);
            const float az = __fmul_rn(__fsub_rn(zp ? __ldg(fin + idx - sy + 1) : fm, fm), A.ihz);
            const float n = rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2))));
            div = __fmaf_rn(__fmul_rn(ay, n), A.ihy, div);
        }
        // p_z at k-1
        if (k > 0) {
            const float fm = __ldg(fin + idx - 1);
            const float ax = __fmul_rn(__fsub_rn(xp ? __ldg(fin + idx - 1 + sx) : fm, fm), A.ihx);
            const float ay = __fmul_rn(__fsub_rn(yp ? __ldg(fin + idx - 1 + sy) : fm, fm), A.ihy);
            const float az = __fmul_rn(__fsub_rn(f0, fm), A.ihz);
            const float n = rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2))));
            div = __fmaf_rn(__fmul_rn(az, n), A.ihz, div);
        }
    }
    return div;
}

// One block of TV_THREADS voxels (block index blk).  Shared by the single-request
// and batched kernels.
template <bool CLAMP, bool E1>
__device__ __forceinline__ void tv_block(const TvArgs &A, const float *__restrict__ fin, const float *__restrict__ g,
                                         float *__restrict__ fout, double *__restrict__ partial, const long blk) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    const size_t idx = (size_t)blk * TV_THREADS + threadIdx.x;
    float e1 = 0.f;
    if (idx < n) {
        const float f0 = __ldg(fin + idx);
        const float div = tv_div<E1>(A, fin, idx, e1);
        const float x = __fmaf_rn(-A.s, __fmaf_rn(A.beta, __fsub_rn(f0, __ldg(g + idx)), div), f0);
        fout[idx] = CLAMP ? fmaxf(x, 0.f) : x;
    }
    if (E1) {
        // float32 within a warp (pairwise tree), float64 across warps and blocks
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e1 += __shfl_down_sync(0xffffffffu, e1, off);
        __shared__ double red[TV_THREADS / 32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)e1;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < TV_THREADS / 32; ++w) s += red[w];
            partial[blk] = s;
        }
    }
}


}  // namespace cbct
