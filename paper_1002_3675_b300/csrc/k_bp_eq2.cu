// Eq. 2 adjoint launcher (single request).  The arithmetic is in bp_eq2_tile.cuh.
#include "bp_eq2_tile.cuh"

namespace cbct {

__global__ void __launch_bounds__(EQ2_THREADS)
k_bp_eq2(GeoDev G, const float *__restrict__ r, const float *__restrict__ fin, float *__restrict__ out,
         float cscale, int mode) {
    eq2_block(G, r, fin, out, cscale, mode, blockIdx.x);
}

cudaError_t launch_backproject_eq2(const GeoDev &g, const float *r, const float *fin, float *out, float cscale,
                                   int mode, cudaStream_t s) {
    const long nb = eq2_tiles(g);
    k_bp_eq2<<<(unsigned)nb, EQ2_THREADS, 0, s>>>(g, r, fin, out, cscale, mode);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cbct
