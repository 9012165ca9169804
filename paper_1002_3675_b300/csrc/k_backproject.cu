// Adjoint gather launchers (single request).  The arithmetic is in bp_tile.cuh.
#include "bp_tile.cuh"

namespace cbct {

// at most 51 registers per thread (48 used): 10 blocks of 128 threads per SM
template <int MODE, int VPL>
__global__ void __launch_bounds__(256, 5)
k_backproject(GeoDev G, const float *__restrict__ rs, const float *__restrict__ fin,
              float *__restrict__ out, float c) {
    const long gwarp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= bp_warp_tiles<VPL>(G)) return;
    bp_warp<VPL>(G, MODE, rs, fin, out, c, gwarp);
}

template <int VPL>
static void launch_vpl(const GeoDev &g, const float *rs, const float *fin, float *out, float c, int mode,
                       cudaStream_t s) {
    const int T = (g.bp_threads == 64 || g.bp_threads == 256) ? g.bp_threads : BP_THREADS;
    const long nb = (bp_warp_tiles<VPL>(g) * 32 + T - 1) / T;
    if (mode == BP_PLAIN)
        k_backproject<BP_PLAIN, VPL><<<(unsigned)nb, T, 0, s>>>(g, rs, fin, out, c);
    else
        k_backproject<BP_STEP, VPL><<<(unsigned)nb, T, 0, s>>>(g, rs, fin, out, c);
}

// voxels per lane: cover a z-column with as few warps as possible, up to 4 per lane
int bp_default_vpl(const GeoDev &g) { return min(4, max(1, (g.nz + 31) / 32)); }

cudaError_t launch_backproject(const GeoDev &g, const float *rs, const float *fin, float *out, float c,
                               int mode, cudaStream_t s) {
    const int vpl = (g.bp_vpl >= 1 && g.bp_vpl <= 4) ? g.bp_vpl : bp_default_vpl(g);
    if (vpl == 4) launch_vpl<4>(g, rs, fin, out, c, mode, s);
    else if (vpl == 3) launch_vpl<3>(g, rs, fin, out, c, mode, s);
    else if (vpl == 2) launch_vpl<2>(g, rs, fin, out, c, mode, s);
    else launch_vpl<1>(g, rs, fin, out, c, mode, s);
    return cudaGetLastError();
}

}  // namespace cbct
