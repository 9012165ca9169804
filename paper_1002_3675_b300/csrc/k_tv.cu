// Step 2 (and 3) of Algorithm A1 (Jia et al. 2010): one projected-gradient step on
//   Phi(f) = TV_eps(f) + beta/2 |f - g|^2,   f >= 0,
// where TV_eps is E1 of Eq. 1 read as the isotropic forward-difference total
// variation with Neumann boundary, sum_j sqrt(|grad f|_j^2 + eps^2).  Its gradient
// is sum_d D_d^T (D_d f / |grad f|_eps), a 13-point stencil per voxel:
//   (D_d^T p)_i = (p_{i-1} [i > 0] - p_i [i < n-1]) / h_d.
// The sweep also emits the partial sums of |grad f|_eps of its input (the
// E1 energy of the entering iterate when the input is f_k).
//
// Layout [nx][ny][nz] (z fastest); one thread per voxel, consecutive lanes along z.
#include "cbct_internal.h"

namespace cbct {

static constexpr int TV_THREADS = 256;

template <bool CLAMP, bool E1>
__global__ void __launch_bounds__(TV_THREADS)
k_tv_sweep(TvArgs A, const float *__restrict__ fin, const float *__restrict__ g, float *__restrict__ fout,
           double *__restrict__ partial) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    const size_t idx = (size_t)blockIdx.x * TV_THREADS + threadIdx.x;
    float e1 = 0.f;
    if (idx < n) {
        const int k = (int)(idx % A.nz);
        const size_t t = idx / A.nz;
        const int j = (int)(t % A.ny);
        const int i = (int)(t / A.ny);
        const size_t sx = (size_t)A.ny * A.nz, sy = A.nz;
        const bool xp = i < A.nx - 1, yp = j < A.ny - 1, zp = k < A.nz - 1;
        const float f0 = __ldg(fin + idx);
        // own gradient (zero difference at the last index)
        const float gx = ((xp ? __ldg(fin + idx + sx) : f0) - f0) * A.ihx;
        const float gy = ((yp ? __ldg(fin + idx + sy) : f0) - f0) * A.ihy;
        const float gz = ((zp ? __ldg(fin + idx + 1) : f0) - f0) * A.ihz;
        const float q0 = gx * gx + gy * gy + gz * gz + A.eps2;
        const float n0 = rsqrtf(q0);
        float div = -(gx * A.ihx + gy * A.ihy + gz * A.ihz) * n0;
        if (E1) e1 = q0 * n0;
        // p_x at i-1
        if (i > 0) {
            const float fm = __ldg(fin + idx - sx);
            const float ax = (f0 - fm) * A.ihx;
            const float ay = ((yp ? __ldg(fin + idx - sx + sy) : fm) - fm) * A.ihy;
            const float az = ((zp ? __ldg(fin + idx - sx + 1) : fm) - fm) * A.ihz;
            div += ax * rsqrtf(ax * ax + ay * ay + az * az + A.eps2) * A.ihx;
        }
        // p_y at j-1
        if (j > 0) {
            const float fm = __ldg(fin + idx - sy);
            const float ax = ((xp ? __ldg(fin + idx - sy + sx) : fm) - fm) * A.ihx;
            const float ay = (f0 - fm) * A.ihy;
            const float az = ((zp ? __ldg(fin + idx - sy + 1) : fm) - fm) * A.ihz;
            div += ay * rsqrtf(ax * ax + ay * ay + az * az + A.eps2) * A.ihy;
        }
        // p_z at k-1
        if (k > 0) {
            const float fm = __ldg(fin + idx - 1);
            const float ax = ((xp ? __ldg(fin + idx - 1 + sx) : fm) - fm) * A.ihx;
            const float ay = ((yp ? __ldg(fin + idx - 1 + sy) : fm) - fm) * A.ihy;
            const float az = (f0 - fm) * A.ihz;
            div += az * rsqrtf(ax * ax + ay * ay + az * az + A.eps2) * A.ihz;
        }
        const float x = f0 - A.s * (div + A.beta * (f0 - __ldg(g + idx)));
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
            partial[blockIdx.x] = s;
        }
    }
}

// E1 alone: float64 partial sums of |grad f|_eps.
__global__ void __launch_bounds__(TV_THREADS)
k_tv_energy(TvArgs A, const float *__restrict__ fin, double *__restrict__ partial) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    const size_t idx = (size_t)blockIdx.x * TV_THREADS + threadIdx.x;
    double e1 = 0.0;
    if (idx < n) {
        const int k = (int)(idx % A.nz);
        const size_t t = idx / A.nz;
        const int j = (int)(t % A.ny);
        const int i = (int)(t / A.ny);
        const size_t sx = (size_t)A.ny * A.nz, sy = A.nz;
        const float f0 = fin[idx];
        const float gx = ((i < A.nx - 1 ? fin[idx + sx] : f0) - f0) * A.ihx;
        const float gy = ((j < A.ny - 1 ? fin[idx + sy] : f0) - f0) * A.ihy;
        const float gz = ((k < A.nz - 1 ? fin[idx + 1] : f0) - f0) * A.ihz;
        e1 = sqrt((double)gx * gx + (double)gy * gy + (double)gz * gz + (double)A.eps2);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e1 += __shfl_down_sync(0xffffffffu, e1, off);
    __shared__ double red[TV_THREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e1;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < TV_THREADS / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

size_t tv_partials(int nx, int ny, int nz) { return ((size_t)nx * ny * nz + TV_THREADS - 1) / TV_THREADS; }

cudaError_t launch_tv_sweep(const TvArgs &a, const float *fin, const float *g, float *fout, bool clamp,
                            double *partial_e1, cudaStream_t s, int *nblocks_out) {
    const size_t nb = tv_partials(a.nx, a.ny, a.nz);
    if (nblocks_out) *nblocks_out = (int)nb;
    dim3 grid((unsigned)nb), block(TV_THREADS);
    if (clamp) {
        if (partial_e1) k_tv_sweep<true, true><<<grid, block, 0, s>>>(a, fin, g, fout, partial_e1);
        else k_tv_sweep<true, false><<<grid, block, 0, s>>>(a, fin, g, fout, nullptr);
    } else {
        if (partial_e1) k_tv_sweep<false, true><<<grid, block, 0, s>>>(a, fin, g, fout, partial_e1);
        else k_tv_sweep<false, false><<<grid, block, 0, s>>>(a, fin, g, fout, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_tv_energy(const TvArgs &a, const float *f, double *partial, cudaStream_t s,
                             int *nblocks_out) {
    const size_t nb = tv_partials(a.nx, a.ny, a.nz);
    if (nblocks_out) *nblocks_out = (int)nb;
    k_tv_energy<<<(unsigned)nb, TV_THREADS, 0, s>>>(a, f, partial);
    return cudaGetLastError();
}

}  // namespace cbct
