// Forward projection launchers (single request).  The arithmetic is in
// project_tile.cuh.
#include <algorithm>
#include <atomic>

#include "project_tile.cuh"

namespace cbct {

template <int MODE, bool VEC>
__global__ void __launch_bounds__(PROJ_MAX_THREADS, 2)
k_project(GeoDev G, const float *__restrict__ vol, const float *__restrict__ y32,
          const __half *__restrict__ y16, float *__restrict__ out, double *__restrict__ partial, int kr0, int kr1,
          int carry) {
    extern __shared__ float smem[];
    project_tile<VEC>(G, MODE, vol, y32, y16, out, partial, blockIdx.x, blockIdx.y, blockIdx.z, smem, kr0, kr1,
                      (carry & 1) != 0, (carry & 2) != 0);
}

// Levels per launch: G.proj_levels if set, else the whole volume in one launch while it fits comfortably in the
// 126 MB L2 next to the projection data; otherwise slabs of whole 32-level groups of at
// most 64 MB, so that the blocks of one launch (every view and column) find their slab
// in L2 instead of re-reading the volume from HBM for every view.  Timed on B300 for
// 512x512x96 (1 MB per level): 64 + 32 levels 2.63 ms per projection, 3 x 32 levels
// 2.79 ms, one launch 2.89 ms, 2 x 48 levels 3.04 ms.
int project_levels_per_launch(const GeoDev &g) {
    if (g.proj_levels >= 1 && g.proj_levels <= g.nz) return g.proj_levels;
    const size_t level_bytes = (size_t)g.nx * g.ny * sizeof(float);
    if (level_bytes * g.nz <= (size_t)48 << 20) return g.nz;
    int r = (int)(((size_t)64 << 20) / level_bytes);
    if (r >= 32) r &= ~31;
    return std::max(1, std::min(r, g.nz));
}

int project_threads(const GeoDev &g) { return proj_threads_of(g); }

static dim3 project_grid(const GeoDev &g) {
    const int T = project_threads(g);
    return dim3((unsigned)g.nu, (unsigned)g.na, (unsigned)((g.nv + T - 1) / T));
}

size_t project_partials(const GeoDev &g) {
    const dim3 d = project_grid(g);
    return (size_t)d.x * d.y * d.z;
}

cudaError_t launch_project(const GeoDev &g, const float *vol, const float *y32, const __half *y16,
                           float *out, double *partial, int mode, cudaStream_t s, int *nblocks_out) {
    if (nblocks_out) *nblocks_out = (int)project_partials(g);
    // the segment list and one level of running sums must fit
    const int smem = proj_smem_of(g);
    if (smem > PROJ_SMEM) return cudaErrorInvalidValue;
    // per device: the attribute belongs to the device's context (setting it twice is harmless)
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
#define CBCT_PROJ_ATTR(M)                                                                                    \
    cudaFuncSetAttribute(k_project<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);      \
    cudaFuncSetAttribute(k_project<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM)
        CBCT_PROJ_ATTR(PROJ_PLAIN);
        CBCT_PROJ_ATTR(PROJ_RESID32);
        CBCT_PROJ_ATTR(PROJ_RESID16);
        CBCT_PROJ_ATTR(PROJ_SCALED);
        CBCT_PROJ_ATTR(PROJ_RAW32);
        CBCT_PROJ_ATTR(PROJ_RAW16);
#undef CBCT_PROJ_ATTR
        attr_set[dev] = true;
    }
    // z-columns in 16-byte pieces (and slabs starting at multiples of 4 levels), and room
    // for 4 levels of running sums at the longest cell sequence: 4 levels per lane
    const int slots = g.nx + g.ny + 1;
    const int R = project_levels_per_launch(g);
    const bool vec = (g.nz & 3) == 0 && (R & 3) == 0 &&
                     (smem / 4 - proj_list_floats(slots)) / (slots + (slots + CHUNK - 1) / CHUNK) >= 4;
    const dim3 grid = project_grid(g), block((unsigned)project_threads(g));
    for (int k0 = 0; k0 < g.nz; k0 += R) {
        const int k1 = std::min(g.nz, k0 + R);
        const int carry = (k0 > 0 ? 1 : 0) | (k1 < g.nz ? 2 : 0);
#define CBCT_PROJ_LAUNCH(M)                                                                 \
    if (vec) k_project<M, true><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial, k0, k1, carry); \
    else k_project<M, false><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial, k0, k1, carry)
        switch (mode) {
            case PROJ_PLAIN: CBCT_PROJ_LAUNCH(PROJ_PLAIN); break;
            case PROJ_RESID32: CBCT_PROJ_LAUNCH(PROJ_RESID32); break;
            case PROJ_RESID16: CBCT_PROJ_LAUNCH(PROJ_RESID16); break;
            case PROJ_RAW32: CBCT_PROJ_LAUNCH(PROJ_RAW32); break;
            case PROJ_RAW16: CBCT_PROJ_LAUNCH(PROJ_RAW16); break;
            default: CBCT_PROJ_LAUNCH(PROJ_SCALED); break;
        }
#undef CBCT_PROJ_LAUNCH
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cbct
