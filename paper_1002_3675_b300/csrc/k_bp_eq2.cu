// Eq. 2 adjoint launcher (single request).  The arithmetic is in bp_eq2_tile.cuh.
#include "bp_eq2_tile.cuh"

namespace cbct {

__global__ void __launch_bounds__(EQ2_THREADS)
k_bp_eq2(GeoDev G, const float *__restrict__ r, int pad, const float *__restrict__ fin, float *__restrict__ out,
         float cscale, int mode) {
    eq2_block(G, r, pad != 0, fin, out, cscale, mode, blockIdx.x);
}

// The interior of the zero-bordered residual: rp[ia][a + 1][b + 1] = r[ia][a][b] (rp is
// [na][nu + 2][nv + 2]; its border stays as zeroed at allocation).  Consecutive threads
// take consecutive rows, so reads and writes are coalesced.
__global__ void __launch_bounds__(256)
k_eq2_pad(const float *__restrict__ r, float *__restrict__ rp, int na, int nu, int nv) {
    const long n = (long)na * nu * nv;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int b = (int)(e % nv);
        const long col = e / nv;  // ia nu + a
        const long ia = col / nu;
        const int a = (int)(col - ia * nu);
        rp[(ia * (nu + 2) + a + 1) * (nv + 2) + b + 1] = __ldg(r + e);
    }
}

cudaError_t launch_backproject_eq2(const GeoDev &g, const float *r, float *padded, const float *fin, float *out,
                                   float cscale, int mode, cudaStream_t s) {
    if (padded) {
        const long n = (long)g.na * g.nu * g.nv;
        long nb = (n + 255) / 256;
        if (nb > 148L * 64) nb = 148L * 64;
        k_eq2_pad<<<(unsigned)nb, 256, 0, s>>>(r, padded, g.na, g.nu, g.nv);
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long nb = eq2_tiles(g);
    k_bp_eq2<<<(unsigned)nb, EQ2_THREADS, 0, s>>>(g, padded ? padded : r, padded ? 1 : 0, fin, out, cscale, mode);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cbct
