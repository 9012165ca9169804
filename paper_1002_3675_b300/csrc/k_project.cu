// Forward projection launchers (single request).  The arithmetic is in
// project_tile.cuh.
#include "project_tile.cuh"

namespace cbct {

template <int MODE>
__global__ void __launch_bounds__(PROJ_MAX_THREADS, 2)
k_project(GeoDev G, const float *__restrict__ vol, const float *__restrict__ y32,
          const __half *__restrict__ y16, float *__restrict__ out, double *__restrict__ partial) {
    extern __shared__ float smem[];
    project_tile(G, MODE, vol, y32, y16, out, partial, blockIdx.x, blockIdx.y, blockIdx.z, smem);
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
    static bool attr_set[64] = {};   // per device: the attribute belongs to the device's context
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        cudaFuncSetAttribute(k_project<PROJ_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        cudaFuncSetAttribute(k_project<PROJ_RESID32>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        cudaFuncSetAttribute(k_project<PROJ_RESID16>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        cudaFuncSetAttribute(k_project<PROJ_SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        cudaFuncSetAttribute(k_project<PROJ_RAW32>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        cudaFuncSetAttribute(k_project<PROJ_RAW16>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        attr_set[dev] = true;
    }
    const dim3 grid = project_grid(g), block((unsigned)project_threads(g));
    switch (mode) {
        case PROJ_PLAIN: k_project<PROJ_PLAIN><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial); break;
        case PROJ_RESID32: k_project<PROJ_RESID32><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial); break;
        case PROJ_RESID16: k_project<PROJ_RESID16><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial); break;
        case PROJ_RAW32: k_project<PROJ_RAW32><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial); break;
        case PROJ_RAW16: k_project<PROJ_RAW16><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial); break;
        default: k_project<PROJ_SCALED><<<grid, block, smem, s>>>(g, vol, y32, y16, out, partial); break;
    }
    return cudaGetLastError();
}

}  // namespace cbct
