// E1 energy without any allocation: cbct_tv_energy_noalloc.
//
// Some callers cannot call cudaMalloc: real-time or embedded hosts that forbid
// allocation after start-up, and plug-ins that must not touch the process's device
// heap.
// They cannot create a cbct_geometry (whose workspaces are allocated), yet may
// still want the TV energy of a volume they own.  This entry point serves them: it
// is a variant of the library's E1 reduction (the per-block float64 partial sums
// of |grad f|_eps that cbct_energy computes) whose only scratch is the file-scope
// array below, reserved when the library is loaded and kept until the process
// exits on every GPU that loads it.
//
// The scratch holds one double per 256-voxel block, so a call handles at most
// CBCT_NOALLOC_MAX_VOXELS voxels.  All calls share the array: every slot a call
// reads is written earlier in the same call (stream order), so nothing needs
// clearing between calls, but calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised.
#include <math.h>

#include <mutex>

#include "cbct_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPartials = CBCT_NOALLOC_MAX_VOXELS / kThreads;  // 131072 doubles = 1 MiB

static __device__ __align__(256) double g_noalloc_partials[kMaxPartials];

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kMaxDevices = 64;
double *g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Variant of the E1 reduction on the caller's [n0][n1][n2] volume (any axis order;
// the spacings follow the axes): forward differences with zero difference at the
// last index, sqrt(|grad f|^2 + eps^2) per voxel, one float64 partial per block.
__global__ void __launch_bounds__(kThreads)
k_tv_energy_static(int n0, int n1, int n2, float ih0, float ih1, float ih2, float eps2,
                   const float *__restrict__ f, double *__restrict__ partials) {
    const size_t n = (size_t)n0 * n1 * n2;
    const size_t idx = (size_t)blockIdx.x * kThreads + threadIdx.x;
    double e = 0.0;
    if (idx < n) {
        const int q2 = (int)(idx % n2);
        const size_t t = idx / n2;
        const int q1 = (int)(t % n1);
        const int q0 = (int)(t / n1);
        const size_t s0 = (size_t)n1 * n2, s1 = n2;
        const float v = f[idx];
        const float g0 = ((q0 < n0 - 1 ? f[idx + s0] : v) - v) * ih0;
        const float g1 = ((q1 < n1 - 1 ? f[idx + s1] : v) - v) * ih1;
        const float g2 = ((q2 < n2 - 1 ? f[idx + 1] : v) - v) * ih2;
        e = sqrt((double)g0 * g0 + (double)g1 * g1 + (double)g2 * g2 + (double)eps2);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
    __shared__ double red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// Fixed-order sum of the nb partials; writes E1 = sum / Nv.
__global__ void k_tv_energy_static_final(const double *__restrict__ partials, int nb, double inv_nv,
                                         double *__restrict__ out) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int q = threadIdx.x; q < nb; q += kThreads) s += partials[q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * inv_nv;
}

// Once per device, with that device current: the device address of the scratch.  The
// address is kept for the life of the process; a device reset (cudaDeviceReset) unloads
// the library's module, after which the kept address is stale and this entry point must
// not be called again on that device.
cbct_status partials_for_current_device(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cbct::cuda_fail(e, "cbct_tv_energy_noalloc: no current device");
    if (dev < 0 || dev >= kMaxDevices) {
        cbct::set_error("cbct_tv_energy_noalloc: device ordinal %d above %d", dev, kMaxDevices - 1);
        return CBCT_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) return cbct::cuda_fail(e, "cbct_tv_energy_noalloc: cudaGetSymbolAddress");
        g_partials_addr[dev] = (double *)p;
    }
    *out = g_partials_addr[dev];
    return CBCT_OK;
}

}  // namespace

extern "C" cbct_status cbct_tv_energy_noalloc(int nx, int ny, int nz, double hx, double hy, double hz,
                                              double eps, const float *f_dev, double *e1_dev,
                                              cudaStream_t stream) {
    if (nx < 1 || ny < 1 || nz < 1) {
        cbct::set_error("cbct_tv_energy_noalloc: sizes must be >= 1");
        return CBCT_ERR_INVALID_ARG;
    }
    const double nvox = (double)nx * ny * nz;
    if (nvox > (double)CBCT_NOALLOC_MAX_VOXELS) {
        cbct::set_error("cbct_tv_energy_noalloc: %d x %d x %d = %.0f voxels exceeds the static scratch limit of "
                        "%d voxels (CBCT_NOALLOC_MAX_VOXELS); use cbct_energy for larger volumes",
                        nx, ny, nz, nvox, CBCT_NOALLOC_MAX_VOXELS);
        return CBCT_ERR_INVALID_ARG;
    }
    // eps = 0 is the unsmoothed TV (the square root is taken in float64), as in cbct_energy
    if (!(hx > 0) || !(hy > 0) || !(hz > 0) || !(eps >= 0) || !isfinite(eps)) {
        cbct::set_error("cbct_tv_energy_noalloc: spacings must be > 0 and eps finite and >= 0");
        return CBCT_ERR_INVALID_ARG;
    }
    // (the kernel reads f one float at a time: 4-byte alignment suffices)
    if (!f_dev || ((uintptr_t)f_dev & 3u) || !e1_dev || ((uintptr_t)e1_dev & 7u)) {
        cbct::set_error("cbct_tv_energy_noalloc: f_dev must be 4-byte and e1_dev 8-byte aligned device pointers");
        return CBCT_ERR_INVALID_ARG;
    }
    double *partials = nullptr;
    cbct_status st = partials_for_current_device(&partials);
    if (st != CBCT_OK) return st;
    const size_t n = (size_t)nvox;
    const int nb = (int)((n + kThreads - 1) / kThreads);
    // caller layout [nz][ny][nx]: axis 0 is z, axis 2 is x
    k_tv_energy_static<<<nb, kThreads, 0, stream>>>(nz, ny, nx, (float)(1.0 / hz), (float)(1.0 / hy),
                                                     (float)(1.0 / hx), (float)(eps * eps), f_dev, partials);
    cbct::count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cbct::cuda_fail(e, "cbct_tv_energy_noalloc: launch");
    k_tv_energy_static_final<<<1, kThreads, 0, stream>>>(partials, nb, 1.0 / nvox, e1_dev);
    cbct::count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cbct::cuda_fail(e, "cbct_tv_energy_noalloc: launch");
    return CBCT_OK;
}
