// Layout changes at the ABI boundary, multigrid transfers (the multigrid of Jia et
// al. 2010, cited method [20], read as a coarse-to-fine cascade) and deterministic
// float64 reductions for the energies of Eq. 1 and the step-size estimate.
#include "step_tile.cuh"

namespace cbct {

// ---------------------------------------------------------------------------------
// Layout changes: tiled 32x32 transposes through shared memory.
// ---------------------------------------------------------------------------------

// api [nz][ny][nx]  <->  internal [nx][ny][nz]: for each j, transpose the (k, i) plane.
template <bool TO_INTERNAL>
__global__ void k_vol_transpose(const float *__restrict__ src, float *__restrict__ dst, int nx, int ny, int nz) {
    __shared__ float tile[32][33];
    const int j = blockIdx.z;
    // TO_INTERNAL: read rows along i (fast in src), write rows along k (fast in dst)
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int n_r = TO_INTERNAL ? nz : nx;  // slow index of src plane
    const int n_c = TO_INTERNAL ? nx : nz;  // fast index of src plane
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        if (r < n_r && c < n_c) {
            size_t o = TO_INTERNAL ? ((size_t)r * ny + j) * nx + c : ((size_t)r * ny + j) * nz + c;
            tile[dy][threadIdx.x] = src[o];
        }
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;  // dst: slow index c, fast index r
        if (r < n_r && c < n_c) {
            size_t o = TO_INTERNAL ? ((size_t)c * ny + j) * nz + r : ((size_t)c * ny + j) * nx + r;
            dst[o] = tile[threadIdx.x][dy];
        }
    }
}

cudaError_t launch_vol_to_internal(const float *api, float *in, int nx, int ny, int nz, cudaStream_t s) {
    dim3 grid((nx + 31) / 32, (nz + 31) / 32, ny), block(32, 8);
    k_vol_transpose<true><<<grid, block, 0, s>>>(api, in, nx, ny, nz);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vol_to_api(const float *in, float *api, int nx, int ny, int nz, cudaStream_t s) {
    dim3 grid((nz + 31) / 32, (nx + 31) / 32, ny), block(32, 8);
    k_vol_transpose<false><<<grid, block, 0, s>>>(in, api, nx, ny, nz);
    count_launch();
    return cudaGetLastError();
}

// sinogram api [na][nv][nu] -> internal [na][nu][nv], optionally x sec(phi), optional half copy
__global__ void k_sino_to_internal(const float *__restrict__ src, float *__restrict__ d32, __half *__restrict__ d16,
                                   const float4 *__restrict__ ray_z, int nu, int nv) {
    __shared__ float tile[32][33];
    const int ia = blockIdx.z;
    const int b0 = blockIdx.y * 32, a0 = blockIdx.x * 32;
    const float *s = src + (size_t)ia * nu * nv;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int b = b0 + dy, a = a0 + threadIdx.x;
        if (b < nv && a < nu) tile[dy][threadIdx.x] = s[(size_t)b * nu + a];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int a = a0 + dy, b = b0 + threadIdx.x;
        if (b < nv && a < nu) {
            float v = tile[threadIdx.x][dy];
            const size_t o = ((size_t)ia * nu + a) * nv + b;
            if (ray_z) v *= ray_z[(size_t)a * nv + b].z;
            if (d32) d32[o] = v;
            if (d16) d16[o] = __float2half_rn(v);
        }
    }
}

cudaError_t launch_sino_to_internal(const float *api, float *out32, __half *out16, const float4 *ray_z,
                                    int na, int nu, int nv, cudaStream_t s) {
    dim3 grid((nu + 31) / 32, (nv + 31) / 32, na), block(32, 8);
    k_sino_to_internal<<<grid, block, 0, s>>>(api, out32, out16, ray_z, nu, nv);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_sino_to_api(const float *__restrict__ src, float *__restrict__ dst, int nu, int nv) {
    __shared__ float tile[32][33];
    const int ia = blockIdx.z;
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
    const float *s = src + (size_t)ia * nu * nv;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int a = a0 + dy, b = b0 + threadIdx.x;
        if (a < nu && b < nv) tile[dy][threadIdx.x] = s[(size_t)a * nv + b];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int b = b0 + dy, a = a0 + threadIdx.x;
        if (a < nu && b < nv) dst[((size_t)ia * nv + b) * nu + a] = tile[threadIdx.x][dy];
    }
}

cudaError_t launch_sino_to_api(const float *in, float *api, int na, int nu, int nv, cudaStream_t s) {
    dim3 grid((nv + 31) / 32, (nu + 31) / 32, na), block(32, 8);
    k_sino_to_api<<<grid, block, 0, s>>>(in, api, nu, nv);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Multigrid transfers
// ---------------------------------------------------------------------------------

// [na][n1][n2] -> [na][ceil n1/2][ceil n2/2]: mean over the existing pixels of each 2x2 block
__global__ void k_restrict(const float *__restrict__ y, float *__restrict__ yc, int na, int n1, int n2) {
    const int m1 = (n1 + 1) / 2, m2 = (n2 + 1) / 2;
    const size_t n = (size_t)na * m1 * m2;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int c2 = (int)(o % m2);
        const size_t t = o / m2;
        const int c1 = (int)(t % m1);
        const int ia = (int)(t / m1);
        float s = 0.f;
        int cnt = 0;
        for (int d1 = 0; d1 < 2; ++d1)
            for (int d2 = 0; d2 < 2; ++d2) {
                const int p1 = 2 * c1 + d1, p2 = 2 * c2 + d2;
                if (p1 < n1 && p2 < n2) {
                    s += y[((size_t)ia * n1 + p1) * n2 + p2];
                    ++cnt;
                }
            }
        yc[o] = s / (float)cnt;
    }
}

cudaError_t launch_restrict(const float *y, float *yc, int na, int n1, int n2, cudaStream_t s) {
    const size_t n = (size_t)na * ((n1 + 1) / 2) * ((n2 + 1) / 2);
    unsigned nb = (unsigned)((n + 255) / 256);
    if (nb > 148u * 32u) nb = 148u * 32u;
    k_restrict<<<nb > 0 ? nb : 1, 256, 0, s>>>(y, yc, na, n1, n2);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_to_half(const float *__restrict__ x, __half *__restrict__ y, size_t n) {
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        y[o] = __float2half_rn(x[o]);
}

cudaError_t launch_to_half(const float *x, __half *y, size_t n, cudaStream_t s) {
    unsigned nb = (unsigned)((n + 255) / 256);
    if (nb > 148u * 32u) nb = 148u * 32u;
    k_to_half<<<nb > 0 ? nb : 1, 256, 0, s>>>(x, y, n);
    count_launch();
    return cudaGetLastError();
}

// coarse coordinate of fine cell-centre i (spacing ratio 2), edge-replicated weights
__device__ __forceinline__ void prolong_w(int i, int n, int nc, int &i0, int &i1, float &w) {
    const float c = ((float)i - 0.5f * (float)(n - 1)) * 0.5f + 0.5f * (float)(nc - 1);
    const float fl = floorf(c);
    w = c - fl;
    const int a = (int)fl;
    i0 = min(max(a, 0), nc - 1);
    i1 = min(max(a + 1, 0), nc - 1);
}

// [c0][c1][c2] coarse -> [n0][n1][n2] fine, trilinear (works for either axis order)
__global__ void k_prolong(const float *__restrict__ fc, int c0, int c1, int c2, float *__restrict__ f, int n0,
                          int n1, int n2) {
    const size_t n = (size_t)n0 * n1 * n2;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int q2 = (int)(o % n2);
        const size_t t = o / n2;
        const int q1 = (int)(t % n1);
        const int q0 = (int)(t / n1);
        int a0, a1, b0, b1, e0, e1;
        float wa, wb, we;
        prolong_w(q0, n0, c0, a0, a1, wa);
        prolong_w(q1, n1, c1, b0, b1, wb);
        prolong_w(q2, n2, c2, e0, e1, we);
#define FC(x, y, z) fc[((size_t)(x) * c1 + (y)) * c2 + (z)]
        const float v00 = (1.f - we) * FC(a0, b0, e0) + we * FC(a0, b0, e1);
        const float v01 = (1.f - we) * FC(a0, b1, e0) + we * FC(a0, b1, e1);
        const float v10 = (1.f - we) * FC(a1, b0, e0) + we * FC(a1, b0, e1);
        const float v11 = (1.f - we) * FC(a1, b1, e0) + we * FC(a1, b1, e1);
#undef FC
        const float v0 = (1.f - wb) * v00 + wb * v01;
        const float v1 = (1.f - wb) * v10 + wb * v11;
        f[o] = (1.f - wa) * v0 + wa * v1;
    }
}

cudaError_t launch_prolong(const float *fc, int c0, int c1, int c2, float *f, int n0, int n1, int n2,
                           cudaStream_t s) {
    const size_t n = (size_t)n0 * n1 * n2;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (nb > 148u * 32u) nb = 148u * 32u;
    k_prolong<<<nb > 0 ? nb : 1, 256, 0, s>>>(fc, c0, c1, c2, f, n0, n1, n2);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Deterministic float64 reductions (fixed partition, fixed tree)
// ---------------------------------------------------------------------------------

// E = E1 + mu E2 with E1 = sum|grad f|_eps / Nv and mu E2 = mu |r|^2 / Nr, and (when
// pstep is given) |f_k+1 - f_k|_2 from its partials; written to trace[TRACE_W * (*counter)]
// and the counter advanced (so a captured graph can be replayed).
__global__ void __launch_bounds__(ENERGY_THREADS)
k_energy_finalize(const double *pe2, int n2, const double *pe1, int n1, const double *pstep, int nstep,
                  double inv_nv, double mu_over_nr, double *trace, int *counter) {
    __shared__ double sums[3];
    sum3_fixed(pe2, n2, pe1, n1, pstep, pstep ? nstep : 0, sums);
    const double q = sums[0], t = sums[1], d = sums[2];
    if (threadIdx.x == 0) {
        const int it = *counter;
        const double e1 = t * inv_nv, e2 = q * mu_over_nr;
        trace[TRACE_W * it + 0] = e1 + e2;
        trace[TRACE_W * it + 1] = e1;
        trace[TRACE_W * it + 2] = e2;
        trace[TRACE_W * it + 3] = pstep ? sqrt(d) : 0.0;
        *counter = it + 1;
    }
}

cudaError_t launch_energy_finalize(const double *pe2, int n2, const double *pe1, int n1, double inv_nv,
                                   double mu_over_nr, double *trace, int *counter, cudaStream_t s,
                                   const double *pstep, int nstep) {
    k_energy_finalize<<<1, ENERGY_THREADS, 0, s>>>(pe2, n2, pe1, n1, pstep, nstep, inv_nv, mu_over_nr, trace,
                                                   counter);
    count_launch();
    return cudaGetLastError();
}

// f = v and per-block float64 partials of |v - f_old|^2: the step norm of Algorithm A1
// while the prox result is moved into the iterate.
__global__ void k_step_copy(const float *__restrict__ v, float *__restrict__ f, size_t n, double *__restrict__ partial) {
    step_block(v, f, n, partial, blockIdx.x);
}

size_t step_partials(size_t n) { return (n + STEP_THREADS - 1) / STEP_THREADS; }

cudaError_t launch_step_copy(const float *v, float *f, size_t n, double *partial, cudaStream_t s) {
    if (!partial) return cudaMemcpyAsync(f, v, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    k_step_copy<<<(unsigned)step_partials(n), STEP_THREADS, 0, s>>>(v, f, n, partial);
    count_launch();
    return cudaGetLastError();
}

// per-tile partials of <x, y> and <y, y> (dot2_tile)
__global__ void __launch_bounds__(VEC_THREADS)
k_dot2(const float *__restrict__ x, const float *__restrict__ y, size_t n, double *partial) {
    dot2_tile(x, y, (long)n, blockIdx.x, partial);
}

cudaError_t launch_dot2(const float *x, const float *y, size_t n, double *partial, cudaStream_t s,
                        int *nblocks_out) {
    const unsigned nb = (unsigned)vec_tiles((long)n);
    if (nblocks_out) *nblocks_out = (int)nb;
    k_dot2<<<nb, VEC_THREADS, 0, s>>>(x, y, n, partial);
    count_launch();
    return cudaGetLastError();
}

// lam = <x, y>, scale = 1/|y|
__global__ void k_power_finalize(const double *partial, int nblk, double *lam, float *scale) {
    __shared__ double sh1[256], sh2[256];
    double s1 = 0.0, s2 = 0.0;
    for (int q = threadIdx.x; q < nblk; q += 256) {
        s1 += partial[2 * q];
        s2 += partial[2 * q + 1];
    }
    sh1[threadIdx.x] = s1;
    sh2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
            sh2[threadIdx.x] += sh2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *lam = sh1[0];
        *scale = sh2[0] > 0.0 ? (float)(1.0 / sqrt(sh2[0])) : 0.f;
    }
}

cudaError_t launch_power_finalize(const double *partial, int nblk, double *lam, float *scale, cudaStream_t s) {
    k_power_finalize<<<1, 256, 0, s>>>(partial, nblk, lam, scale);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(VEC_THREADS)
k_scale(const float *__restrict__ y, const float *__restrict__ scale, float *__restrict__ x, size_t n) {
    scale_tile(y, scale, x, (long)n, blockIdx.x);
}

cudaError_t launch_scale(const float *y, const float *scale, float *x, size_t n, cudaStream_t s) {
    const unsigned nb = (unsigned)vec_tiles((long)n);
    k_scale<<<nb > 0 ? nb : 1, VEC_THREADS, 0, s>>>(y, scale, x, n);
    count_launch();
    return cudaGetLastError();
}

// Start volume of the power iteration: seeded uniform(0,1) values from the counter-based
// SplitMix64 generator (Steele, Lea and Flood 2014): value a = the 64-bit finaliser of
// seed + (a + 1) * 0x9E3779B97F4A7C15, top 24 bits over 2^24 (exact in float32), where a
// is the voxel's index in the [nz][ny][nx] order of the C ABI; written in the internal
// [nx][ny][nz] layout.
__device__ __forceinline__ unsigned long long sm64_value(unsigned long long seed, unsigned long long a) {
    unsigned long long z = seed + (a + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_fill_uniform(float *__restrict__ x, int nx, int ny, int nz, unsigned long long seed) {
    const size_t n = (size_t)nx * ny * nz;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(o % nz);
        const size_t t = o / nz;
        const int j = (int)(t % ny), i = (int)(t / ny);
        const unsigned long long a = ((unsigned long long)k * ny + j) * nx + i;
        x[o] = (float)(unsigned)(sm64_value(seed, a) >> 40) * (1.f / 16777216.f);
    }
}

cudaError_t launch_fill_uniform(float *x, int nx, int ny, int nz, unsigned long long seed, cudaStream_t s) {
    size_t nb = ((size_t)nx * ny * nz + 255) / 256;
    if (nb > 148u * 32u) nb = 148u * 32u;
    k_fill_uniform<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, s>>>(x, nx, ny, nz, seed);
    count_launch();
    return cudaGetLastError();
}

__global__ void k_fill(float *x, float v, size_t n) {
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
        x[o] = v;
}

cudaError_t launch_fill(float *x, float v, size_t n, cudaStream_t s) {
    unsigned nb = (unsigned)((n + 255) / 256);
    if (nb > 148u * 32u) nb = 148u * 32u;
    k_fill<<<nb > 0 ? nb : 1, 256, 0, s>>>(x, v, n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cbct
