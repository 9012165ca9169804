// Kernels of the V-cycle (full-approximation multigrid cycle).  Volumes are in the
// internal layout [nx][ny][nz]; every transfer is separable, so it is written for a
// generic [n0][n1][n2] volume.
#include "tv_tile.cuh"

namespace cbct {

namespace {

__device__ __forceinline__ size_t grid_stride_start() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t grid_stride() { return (size_t)gridDim.x * blockDim.x; }

unsigned blocks_for(size_t n) {
    size_t nb = (n + 255) / 256;
    if (nb > 148u * 32u) nb = 148u * 32u;
    return (unsigned)(nb > 0 ? nb : 1);
}

// Trilinear cell-centred weights of fine index i (n fine, nc coarse): coarse i0, i1 and
// the weight w of i1 (the same expression as the prolongation kernel).
__device__ __forceinline__ void mg_prolong_w(int i, int n, int nc, int &i0, int &i1, float &w) {
    const float c = ((float)i - 0.5f * (float)(n - 1)) * 0.5f + 0.5f * (float)(nc - 1);
    const float fl = floorf(c);
    w = c - fl;
    const int a = (int)fl;
    i0 = min(max(a, 0), nc - 1);
    i1 = min(max(a + 1, 0), nc - 1);
}

// Fine indices (at most 6) whose prolongation stencil uses coarse index ic, with that
// weight.
__device__ __forceinline__ int mg_adjoint_taps(int ic, int n, int nc, int *idx, float *wt) {
    int m = 0;
    for (int i = max(2 * ic - 2, 0); i <= min(2 * ic + 3, n - 1); ++i) {
        int i0, i1;
        float w;
        mg_prolong_w(i, n, nc, i0, i1, w);
        const float v = (i0 == ic ? 1.f - w : 0.f) + (i1 == ic ? w : 0.f);
        if (v != 0.f) {
            idx[m] = i;
            wt[m] = v;
            ++m;
        }
    }
    return m;
}

}  // namespace

// Mean of the existing fine voxels of each 2x2x2 block.
__global__ void k_restrict_vol(const float *__restrict__ f, int n0, int n1, int n2, float *__restrict__ fc, int c0,
                               int c1, int c2) {
    const size_t n = (size_t)c0 * c1 * c2;
    for (size_t o = grid_stride_start(); o < n; o += grid_stride()) {
        const int q2 = (int)(o % c2);
        const size_t t = o / c2;
        const int q1 = (int)(t % c1), q0 = (int)(t / c1);
        float s = 0.f;
        int cnt = 0;
        for (int d0 = 0; d0 < 2; ++d0)
            for (int d1 = 0; d1 < 2; ++d1)
                for (int d2 = 0; d2 < 2; ++d2) {
                    const int a = 2 * q0 + d0, b = 2 * q1 + d1, c = 2 * q2 + d2;
                    if (a < n0 && b < n1 && c < n2) {
                        s += f[((size_t)a * n1 + b) * n2 + c];
                        ++cnt;
                    }
                }
        fc[o] = s / (float)cnt;
    }
}

// Transpose of the trilinear prolongation: each coarse voxel gathers the fine values
// that its weight reaches (no atomics, fixed order).
__global__ void k_prolong_adjoint(const float *__restrict__ x, int n0, int n1, int n2, float *__restrict__ out,
                                  int c0, int c1, int c2) {
    const size_t n = (size_t)c0 * c1 * c2;
    for (size_t o = grid_stride_start(); o < n; o += grid_stride()) {
        const int q2 = (int)(o % c2);
        const size_t t = o / c2;
        const int q1 = (int)(t % c1), q0 = (int)(t / c1);
        int i0[6], i1[6], i2[6];
        float w0[6], w1[6], w2[6];
        const int m0 = mg_adjoint_taps(q0, n0, c0, i0, w0);
        const int m1 = mg_adjoint_taps(q1, n1, c1, i1, w1);
        const int m2 = mg_adjoint_taps(q2, n2, c2, i2, w2);
        float s = 0.f;
        for (int a = 0; a < m0; ++a)
            for (int b = 0; b < m1; ++b) {
                const float wab = w0[a] * w1[b];
                const float *row = x + ((size_t)i0[a] * n1 + i1[b]) * n2;
                for (int c = 0; c < m2; ++c) s = fmaf(wab * w2[c], row[i2[c]], s);
            }
        out[o] = s;
    }
}

// Gradient of the grid energy of Eq. 1 minus an optional linear term:
//   out = (grad TV_eps(f) + gamma P^T r) / Nv - lin,  bp = P^T r.
__global__ void k_energy_grad(TvArgs A, const float *__restrict__ f, const float *__restrict__ bp, float gamma,
                              float inv_nv, const float *__restrict__ lin, float *__restrict__ out) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    for (size_t o = grid_stride_start(); o < n; o += grid_stride()) {
        float unused = 0.f;
        const float div = A.aniso ? tv_div<false, true>(A, f, o, unused) : tv_div<false, false>(A, f, o, unused);
        float gr = __fmul_rn(__fmaf_rn(gamma, bp[o], div), inv_nv);
        if (lin) gr = __fsub_rn(gr, lin[o]);
        out[o] = gr;
    }
}

__global__ void k_axpy(float *__restrict__ y, const float *__restrict__ x, float a, size_t n) {
    for (size_t o = grid_stride_start(); o < n; o += grid_stride()) y[o] = __fmaf_rn(a, x[o], y[o]);
}

__global__ void k_sub(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ out, size_t n) {
    for (size_t o = grid_stride_start(); o < n; o += grid_stride()) out[o] = __fsub_rn(a[o], b[o]);
}

__global__ void k_add_clamp(const float *__restrict__ f, const float *__restrict__ c, float *__restrict__ out,
                            size_t n) {
    for (size_t o = grid_stride_start(); o < n; o += grid_stride()) out[o] = fmaxf(__fadd_rn(f[o], c[o]), 0.f);
}

// <x, y>: float32 within a warp, float64 across warps, one partial per block of 256.
__global__ void k_dot(const float *__restrict__ x, const float *__restrict__ y, size_t n, double *__restrict__ partial) {
    const size_t o = (size_t)blockIdx.x * 256 + threadIdx.x;
    float v = o < n ? __fmul_rn(x[o], y[o]) : 0.f;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

// out = sum of the partials (fixed strided order, then a fixed tree).
__global__ void k_sum_partials(const double *__restrict__ p, int n, double *__restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 256) s += p[q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_restrict_vol(const float *f, int n0, int n1, int n2, float *fc, cudaStream_t s) {
    const int c0 = (n0 + 1) / 2, c1 = (n1 + 1) / 2, c2 = (n2 + 1) / 2;
    k_restrict_vol<<<blocks_for((size_t)c0 * c1 * c2), 256, 0, s>>>(f, n0, n1, n2, fc, c0, c1, c2);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_prolong_adjoint(const float *x, int n0, int n1, int n2, float *out, int c0, int c1, int c2,
                                   cudaStream_t s) {
    k_prolong_adjoint<<<blocks_for((size_t)c0 * c1 * c2), 256, 0, s>>>(x, n0, n1, n2, out, c0, c1, c2);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_energy_grad(const TvArgs &a, const float *f, const float *bp, float gamma, float inv_nv,
                               const float *lin, float *out, cudaStream_t s) {
    k_energy_grad<<<blocks_for((size_t)a.nx * a.ny * a.nz), 256, 0, s>>>(a, f, bp, gamma, inv_nv, lin, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_axpy(float *y, const float *x, float a, size_t n, cudaStream_t s) {
    k_axpy<<<blocks_for(n), 256, 0, s>>>(y, x, a, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sub(const float *a, const float *b, float *out, size_t n, cudaStream_t s) {
    k_sub<<<blocks_for(n), 256, 0, s>>>(a, b, out, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_add_clamp(const float *f, const float *c, float *out, size_t n, cudaStream_t s) {
    k_add_clamp<<<blocks_for(n), 256, 0, s>>>(f, c, out, n);
    count_launch();
    return cudaGetLastError();
}

size_t dot_partials(size_t n) { return (n + 255) / 256; }

cudaError_t launch_dot(const float *x, const float *y, size_t n, double *partial, double *out, cudaStream_t s) {
    const size_t nb = dot_partials(n);
    k_dot<<<(unsigned)nb, 256, 0, s>>>(x, y, n, partial);
    count_launch();
    k_sum_partials<<<1, 256, 0, s>>>(partial, (int)nb, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cbct
