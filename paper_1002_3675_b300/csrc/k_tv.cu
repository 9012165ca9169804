// TV prox sweep launchers (single request).  The arithmetic is in tv_tile.cuh and,
// for the x-marching fused sweeps, tv_xmarch.cuh.
#include <float.h>

#include <algorithm>
#include <atomic>

#include "tv_xmarch.cuh"

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

// ---- x-marching fused sweeps -------------------------------------------------------
// 64 registers per thread at most (1024 threads, or two blocks of 512, per SM).
template <int T, int VZ, int W, bool ANISO>
__global__ void __launch_bounds__(32 * W, 1024 / (32 * W))
k_tv_x(TvArgs A, TvXArgs X, const float *__restrict__ fin, const float *__restrict__ g, float *__restrict__ fout,
       double *__restrict__ partial) {
    extern __shared__ float tvx_sm[];
    tv_x_tile<T, VZ, W, ANISO>(A, X, fin, g, fout, partial, tvx_sm, blockIdx.x);
}

// Warps per block (16 or 32) and output rows: W = by + 2T - 1.
static int tvx_warps(const TvArgs &a, int T) { return a.xW > 0 ? a.xW : (T == 2 ? 32 : 16); }

static TvXArgs tvx_args(const TvArgs &a, int T) {
    TvXArgs x;
    x.W = tvx_warps(a, T);
    x.by = x.W - 2 * T + 1;
    x.lx = a.xLX;
    x.nyt = (a.ny + x.by - 1) / x.by;
    x.clamp = 0;
    x.e1 = x.step = 0;
    return x;
}

size_t tv_x_partials(const TvArgs &a, int T) {
    const TvXArgs x = tvx_args(a, T);
    return (size_t)x.nyt * ((a.nx + x.lx - 1) / x.lx);
}

// Shapes: W in {16, 32} warps with T in {1, 2} (so by >= 13) and planes >= 8.
size_t tv_x_partials_max(int nx, int ny, int nz) {
    (void)nz;
    return (size_t)((ny + 12) / 13) * ((nx + 7) / 8);
}

void tv_x_shape(TvArgs &a, int sweeps, int warps, int planes) {
    a.xT = a.xW = a.xLX = 0;
    // columns of at most 96 voxels in whole lanes, enough tiles, eps^2 a normal float (the
    // tile's ftz reciprocal square root).  Down to 128x128 planes (half a wave of blocks)
    // the fused sweeps still beat ten one-sweep launches: timed on B300 for the 128x128x32
    // coarse level of 256x256x64, the TV class of a reconstruction 13.65 -> 12.74 ms
    if (!(tvx_vz(a.nz) && (long)a.nx * ((a.ny + 3) / 4) >= 2048) || sweeps < 0 || !(a.eps2 >= FLT_MIN)) return;
    a.xT = (sweeps == 1 || sweeps == 2) ? sweeps : 2;
    a.xW = (warps == 16 || warps == 32) ? warps : 0;
    // planes per block: one wave of blocks (one 1024-thread block, or two of 512, per
    // SM) with the x-range split as little as that allows (every block recomputes the
    // planes its sweeps need beyond its own: fewer, longer blocks waste less; timed on
    // B300 for 512x512x96 and 256x256x{48,64})
    int lx = planes >= 8 ? planes : 0;
    if (!lx) {
        const int W = tvx_warps(a, a.xT), by = W - 2 * a.xT + 1;
        const long nyt = (a.ny + by - 1) / by;
        const long slots = (long)device_sm_count() * (W == 16 ? 2 : 1);
        const long nxc = std::max<long>(1, slots / nyt);
        lx = (int)std::max<long>(8, (a.nx + nxc - 1) / nxc);
    }
    a.xLX = std::min(lx, a.nx);
}

template <int T, int VZ, int W, bool ANISO>
static cudaError_t launch_x4(const TvArgs &a, const TvXArgs &x, const float *fin, const float *g, float *fout,
                             double *p, cudaStream_t s, unsigned nblk) {
    const size_t smem = tvx_smem_floats(T, W, VZ) * sizeof(float);
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_tv_x<T, VZ, W, ANISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    k_tv_x<T, VZ, W, ANISO><<<nblk, 32 * W, smem, s>>>(a, x, fin, g, fout, p);
    count_launch();
    return cudaGetLastError();
}

template <int T, int VZ, bool ANISO>
static cudaError_t launch_x3(const TvArgs &a, const TvXArgs &x, const float *fin, const float *g, float *fout,
                             double *p, cudaStream_t s, unsigned nblk) {
    if (x.W == 16) return launch_x4<T, VZ, 16, ANISO>(a, x, fin, g, fout, p, s, nblk);
    return launch_x4<T, VZ, 32, ANISO>(a, x, fin, g, fout, p, s, nblk);
}

template <int T, bool ANISO>
static cudaError_t launch_x2(const TvArgs &a, const TvXArgs &x, const float *fin, const float *g, float *fout,
                             double *p, cudaStream_t s, unsigned nblk) {
    const int vz = tvx_vz(a.nz);
    if (vz == 1) return launch_x3<T, 1, ANISO>(a, x, fin, g, fout, p, s, nblk);
    if (vz == 2) return launch_x3<T, 2, ANISO>(a, x, fin, g, fout, p, s, nblk);
    return launch_x3<T, 3, ANISO>(a, x, fin, g, fout, p, s, nblk);
}

cudaError_t launch_tv_x(const TvArgs &a, int T, unsigned clamp, const float *fin, const float *g, float *fout,
                        double *partial_e1, double *partial_step, cudaStream_t s, int *nblocks_out) {
    if (a.xT == 0 || !tvx_vz(a.nz) || (T != 1 && T != 2) || fin == fout || (partial_e1 && partial_step))
        return cudaErrorInvalidValue;
    TvXArgs x = tvx_args(a, T);
    if (x.by < 1 || x.lx < 1 || (x.W != 16 && x.W != 32)) return cudaErrorInvalidValue;
    x.clamp = clamp;
    x.e1 = partial_e1 != nullptr;
    x.step = partial_step != nullptr;
    double *p = partial_e1 ? partial_e1 : partial_step;
    const unsigned nblk = (unsigned)tv_x_partials(a, T);
    if (nblocks_out) *nblocks_out = (int)nblk;
    if (T == 1) return a.aniso ? launch_x2<1, true>(a, x, fin, g, fout, p, s, nblk)
                               : launch_x2<1, false>(a, x, fin, g, fout, p, s, nblk);
    return a.aniso ? launch_x2<2, true>(a, x, fin, g, fout, p, s, nblk)
                   : launch_x2<2, false>(a, x, fin, g, fout, p, s, nblk);
}

XProxPlan xprox_plan(const TvArgs &a, int M, int clamp_mode, const float *src0, float *f, float *A, float *B,
                     bool want_e1, bool want_step, size_t nvox) {
    XProxPlan pl;
    const float *src = src0;
    for (int m0 = 0; m0 < M;) {
        XLaunch x;
        x.T = std::min(a.xT, M - m0);
        const bool last = m0 + x.T == M;
        x.fout = (last && src != f) ? f : (src == A ? B : A);
        x.fin = src;
        x.clamp = 0;
        for (int t = 0; t < x.T; ++t)
            if (clamp_mode == 0 || m0 + t == M - 1) x.clamp |= 1u << t;
        x.e1 = want_e1 && m0 == 0;
        x.step = want_step && last && x.fout == f;
        pl.launches.push_back(x);
        src = x.fout;
        m0 += x.T;
    }
    pl.result = src;
    pl.step_fused = !pl.launches.empty() && pl.launches.back().step;
    pl.n_e1 = pl.launches.empty() ? 0 : (int)tv_x_partials(a, pl.launches.front().T);
    pl.n_step = pl.step_fused ? (int)tv_x_partials(a, pl.launches.back().T) : (int)step_partials(nvox);
    return pl;
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
