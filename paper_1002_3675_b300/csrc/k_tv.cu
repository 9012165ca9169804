// TV prox sweep launchers (single request).  The arithmetic is in tv_tile.cuh.
#include "tv_tile.cuh"

namespace cbct {

// Full columns of 2 or 3 voxels per lane: at most 64 registers, 4 blocks per SM.  Uncapped,
// 3 voxels per lane took 80 registers and was slower; 2 per lane with the E1 or step
// accumulator took 72 (3 blocks per SM), and the cap (no spills) made the medium
// level's TV class 1.7 % faster.
template <bool CLAMP, int ACC, bool ANISO, int FORM>
__global__ void __launch_bounds__(TV_THREADS, FORM >= 3 ? 4 : 1)
k_tv_sweep(TvArgs A, const float *__restrict__ fin, const float *__restrict__ g, float *__restrict__ fout,
           double *__restrict__ partial) {
    tv_block_t<CLAMP, ACC, ANISO, FORM>(A, fin, g, fout, partial, blockIdx.x);
}

template <bool CLAMP, int ACC, bool ANISO>
static void launch_form(const TvArgs &a, dim3 grid, const float *fin, const float *g, float *fout, double *p,
                        cudaStream_t s) {
    switch (tv_form(a)) {
        case 0: k_tv_sweep<CLAMP, ACC, ANISO, 0><<<grid, TV_THREADS, 0, s>>>(a, fin, g, fout, p); break;
        case 1: k_tv_sweep<CLAMP, ACC, ANISO, 1><<<grid, TV_THREADS, 0, s>>>(a, fin, g, fout, p); break;
        case 2: k_tv_sweep<CLAMP, ACC, ANISO, 2><<<grid, TV_THREADS, 0, s>>>(a, fin, g, fout, p); break;
        case 3: k_tv_sweep<CLAMP, ACC, ANISO, 3><<<grid, TV_THREADS, 0, s>>>(a, fin, g, fout, p); break;
        default: k_tv_sweep<CLAMP, ACC, ANISO, 4><<<grid, TV_THREADS, 0, s>>>(a, fin, g, fout, p); break;
    }
    count_launch();
}

template <bool CLAMP, int ACC>
static void launch_sweep(const TvArgs &a, dim3 grid, const float *fin, const float *g, float *fout, double *p,
                         cudaStream_t s) {
    if (a.aniso) launch_form<CLAMP, ACC, true>(a, grid, fin, g, fout, p, s);
    else launch_form<CLAMP, ACC, false>(a, grid, fin, g, fout, p, s);
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
        if (A.aniso)
            e1 = sqrt((double)gx * gx + (double)A.eps2) + sqrt((double)gy * gy + (double)A.eps2) +
                 sqrt((double)gz * gz + (double)A.eps2);
        else
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

size_t tv_partials(int nx, int ny, int nz) {
    const long wt = tv_warp_tiles(nx, ny, nz);
    return (size_t)(tv_rows_per_tile(nx, ny, nz) == 0 ? wt / TV_WARPS : wt);
}
size_t tv_blocks(int nx, int ny, int nz) { return (size_t)((tv_warp_tiles(nx, ny, nz) + TV_WARPS - 1) / TV_WARPS); }
size_t tv_energy_partials(int nx, int ny, int nz) { return ((size_t)nx * ny * nz + TV_THREADS - 1) / TV_THREADS; }

cudaError_t launch_tv_sweep(const TvArgs &a, const float *fin, const float *g, float *fout, bool clamp,
                            double *partial_e1, cudaStream_t s, int *nblocks_out, double *partial_step) {
    if (nblocks_out) *nblocks_out = (int)tv_partials(a.nx, a.ny, a.nz);
    if (partial_e1 && partial_step) return cudaErrorInvalidValue;  // one accumulator per sweep
    dim3 grid((unsigned)tv_blocks(a.nx, a.ny, a.nz));
    if (clamp) {
        if (partial_e1) launch_sweep<true, TV_ACC_E1>(a, grid, fin, g, fout, partial_e1, s);
        else if (partial_step) launch_sweep<true, TV_ACC_STEP>(a, grid, fin, g, fout, partial_step, s);
        else launch_sweep<true, TV_ACC_NONE>(a, grid, fin, g, fout, nullptr, s);
    } else {
        if (partial_e1) launch_sweep<false, TV_ACC_E1>(a, grid, fin, g, fout, partial_e1, s);
        else if (partial_step) launch_sweep<false, TV_ACC_STEP>(a, grid, fin, g, fout, partial_step, s);
        else launch_sweep<false, TV_ACC_NONE>(a, grid, fin, g, fout, nullptr, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_tv_energy(const TvArgs &a, const float *f, double *partial, cudaStream_t s,
                             int *nblocks_out) {
    const size_t nb = tv_energy_partials(a.nx, a.ny, a.nz);
    if (nblocks_out) *nblocks_out = (int)nb;
    k_tv_energy<<<(unsigned)nb, TV_THREADS, 0, s>>>(a, f, partial);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cbct
