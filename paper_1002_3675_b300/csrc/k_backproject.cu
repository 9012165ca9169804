// Adjoint gather launchers (single request).  The arithmetic is in bp_tile.cuh.
#include "bp_tile.cuh"

namespace cbct {

// at most 51 registers per thread (48 used): 10 blocks of 128 threads per SM (64
// registers for 4 voxels per lane); dynamic shared memory: the warps' setup records
template <int MODE, int VPL>
__global__ void __launch_bounds__(256, VPL == 4 ? 4 : 5)
k_backproject(GeoDev G, const float *__restrict__ rs, const float *__restrict__ fin,
              float *__restrict__ out, float c) {
    extern __shared__ float4 rec[];
    const long gwarp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= bp_warp_tiles<VPL>(G)) return;
    bp_warp<VPL>(G, MODE, rs, fin, out, c, gwarp, rec + (threadIdx.x >> 5) * BP_REC_PER_WARP);
}

template <int VPL>
static void launch_vpl(const GeoDev &g, const float *rs, const float *fin, float *out, float c, int mode,
                       cudaStream_t s) {
    const int T = (g.bp_threads == 64 || g.bp_threads == 256) ? g.bp_threads : BP_THREADS;
    const long nb = (bp_warp_tiles<VPL>(g) * 32 + T - 1) / T;
    const size_t smem = (size_t)(T / 32) * BP_REC_PER_WARP * sizeof(float4);
    if (mode == BP_PLAIN)
        k_backproject<BP_PLAIN, VPL><<<(unsigned)nb, T, smem, s>>>(g, rs, fin, out, c);
    else
        k_backproject<BP_STEP, VPL><<<(unsigned)nb, T, smem, s>>>(g, rs, fin, out, c);
    count_launch();
}

// Running sums of rs along every detector column (one thread per column, float64, in
// row order): rowsum[b] = sum_{b' < b} rs[b'], stored as hi = float(s), lo = float(s - hi).
__global__ void k_row_prefix(const float *__restrict__ rs, float2 *__restrict__ out, long ncol, int nv) {
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += (long)gridDim.x * blockDim.x) {
        const float *r = rs + c * nv;
        float2 *o = out + c * (nv + 1);
        double sum = 0.0;
        o[0] = make_float2(0.f, 0.f);
        for (int b = 0; b < nv; ++b) {
            sum += (double)__ldg(r + b);
            const float hi = (float)sum;
            o[b + 1] = make_float2(hi, (float)(sum - (double)hi));
        }
    }
}

cudaError_t launch_row_prefix(const GeoDev &g, const float *rs, cudaStream_t s) {
    const long ncol = (long)g.na * g.nu;
    long nb = (ncol + 127) / 128;
    if (nb > 148 * 16) nb = 148 * 16;
    k_row_prefix<<<(unsigned)nb, 128, 0, s>>>(rs, g.rowsum, ncol, g.nv);
    count_launch();
    return cudaGetLastError();
}

// voxels per lane: cover a z-column with as few warps as possible, up to 4 per lane
int bp_default_vpl(const GeoDev &g) { return min(4, max(1, (g.nz + 31) / 32)); }

cudaError_t launch_backproject(const GeoDev &g, const float *rs, const float *fin, float *out, float c,
                               int mode, cudaStream_t s) {
    const cudaError_t e = launch_row_prefix(g, rs, s);
    if (e != cudaSuccess) return e;
    const int vpl = (g.bp_vpl >= 1 && g.bp_vpl <= 4) ? g.bp_vpl : bp_default_vpl(g);
    if (vpl == 4) launch_vpl<4>(g, rs, fin, out, c, mode, s);
    else if (vpl == 3) launch_vpl<3>(g, rs, fin, out, c, mode, s);
    else if (vpl == 2) launch_vpl<2>(g, rs, fin, out, c, mode, s);
    else launch_vpl<1>(g, rs, fin, out, c, mode, s);
    return cudaGetLastError();
}

}  // namespace cbct
