// Forward projection P^theta (problem statement before Eq. 1 of Jia et al. 2010):
// exact intersection-length line integrals of the voxelised f along every
// source-to-pixel ray, with the step-1 residual r = P f - Y and the float64 partial
// sums of |r|^2 (E2 of Eq. 1) fused into the epilogue.
//
// Work decomposition.  All rays of one detector column (view ia, column a) lie in
// one vertical plane and cross the same sequence of xy-cells.  One warp takes 32
// consecutive rows b of that column: the walk through the xy-grid is computed by
// every lane identically (uniform control flow, no divergence), and each lane
// splits the current xy-cell's t-interval at its own z-plane crossings.  With the
// volume stored z-fastest the 32 lanes read neighbouring addresses of one z-column.
#include "cbct_internal.h"

namespace cbct {

static constexpr int PROJ_THREADS = 128;

template <int MODE>
__global__ void __launch_bounds__(PROJ_THREADS)
k_project(GeoDev G, const float *__restrict__ vol, const float *__restrict__ y32,
          const __half *__restrict__ y16, float *__restrict__ out, double *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const long gwarp = ((long)blockIdx.x * PROJ_THREADS + threadIdx.x) >> 5;
    const int nbc = (G.nv + 31) >> 5;
    const long nwarps = (long)G.na * G.nu * nbc;
    double r2 = 0.0;

    if (gwarp < nwarps) {
        const int bc = (int)(gwarp % nbc);
        const long rem = gwarp / nbc;
        const int a = (int)(rem % G.nu);
        const int ia = (int)(rem / G.nu);
        const int b = bc * 32 + lane;
        const bool valid = b < G.nv;
        const int bq = valid ? b : G.nv - 1;
        const float4 rxy = G.ray_xy[(size_t)ia * G.nu + a];
        const float2 re = G.ray_e[(size_t)ia * G.nu + a];
        const float4 rz = G.ray_z[(size_t)a * G.nv + bq];
        const float Ox = rxy.x, Oy = rxy.y, ix = rxy.z, iy = rxy.w;
        const float zO = rz.x, cotp = rz.y, secp = rz.z, tanp = rz.w;

        // --- entry into the xy box (identical in every lane) -------------------------
        const float xN = plane_at(G.nx, G.hx, G.x0), yN = plane_at(G.ny, G.hy, G.y0);
        float tin = -INFINITY, tout = INFINITY;
        bool hit = true;
        if (ix != 0.f) {
            float t0 = t_cross(G.x0, Ox, ix), t1 = t_cross(xN, Ox, ix);
            tin = fmaxf(tin, fminf(t0, t1));
            tout = fminf(tout, fmaxf(t0, t1));
        } else {
            hit = hit && Ox >= G.x0 && Ox < xN;
        }
        if (iy != 0.f) {
            float t0 = t_cross(G.y0, Oy, iy), t1 = t_cross(yN, Oy, iy);
            tin = fmaxf(tin, fminf(t0, t1));
            tout = fminf(tout, fmaxf(t0, t1));
        } else {
            hit = hit && Oy >= G.y0 && Oy < yN;
        }
        hit = hit && tout > tin;

        float acc = 0.f;
        if (hit) {
            // starting cell, fixed against the crossing values themselves
            int i, si;
            float txn;
            if (ix != 0.f) {
                si = ix > 0.f ? 1 : -1;
                float xin = __fmaf_rn(tin, re.x, Ox);
                i = min(max((int)floorf((xin - G.x0) * G.inv_hx), 0), G.nx - 1);
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    float ten = t_cross(plane_at(i + (si < 0), G.hx, G.x0), Ox, ix);
                    float tex = t_cross(plane_at(i + (si > 0), G.hx, G.x0), Ox, ix);
                    if (ten > tin && i - si >= 0 && i - si < G.nx) i -= si;
                    else if (tex <= tin && i + si >= 0 && i + si < G.nx) i += si;
                    else break;
                }
                txn = t_cross(plane_at(i + (si > 0), G.hx, G.x0), Ox, ix);
            } else {
                si = 0;
                i = min(max((int)floorf((Ox - G.x0) * G.inv_hx), 0), G.nx - 1);
                txn = INFINITY;
            }
            int j, sj;
            float tyn;
            if (iy != 0.f) {
                sj = iy > 0.f ? 1 : -1;
                float yin = __fmaf_rn(tin, re.y, Oy);
                j = min(max((int)floorf((yin - G.y0) * G.inv_hy), 0), G.ny - 1);
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    float ten = t_cross(plane_at(j + (sj < 0), G.hy, G.y0), Oy, iy);
                    float tex = t_cross(plane_at(j + (sj > 0), G.hy, G.y0), Oy, iy);
                    if (ten > tin && j - sj >= 0 && j - sj < G.ny) j -= sj;
                    else if (tex <= tin && j + sj >= 0 && j + sj < G.ny) j += sj;
                    else break;
                }
                tyn = t_cross(plane_at(j + (sj > 0), G.hy, G.y0), Oy, iy);
            } else {
                sj = 0;
                j = min(max((int)floorf((Oy - G.y0) * G.inv_hy), 0), G.ny - 1);
                tyn = INFINITY;
            }

            // per-lane z state at the entry; a ray leaves z = 0 monotonically, so a lane
            // outside the slab range at entry (or after leaving it) stays outside
            int k, sk;
            float tzn;
            if (cotp != 0.f) {
                sk = cotp > 0.f ? 1 : -1;
                float zin = __fmaf_rn(tin, tanp, zO);
                k = min(max((int)floorf((zin - G.z0) * G.inv_hz), -1), G.nz);
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    float ten = t_cross(plane_at(k + (sk < 0), G.hz, G.z0), zO, cotp);
                    float tex = t_cross(plane_at(k + (sk > 0), G.hz, G.z0), zO, cotp);
                    if (ten > tin && k - sk >= -1 && k - sk <= G.nz) k -= sk;
                    else if (tex <= tin && k + sk >= -1 && k + sk <= G.nz) k += sk;
                    else break;
                }
                tzn = t_cross(plane_at(k + (sk > 0), G.hz, G.z0), zO, cotp);
            } else {
                sk = 0;
                k = (int)floorf((zO - G.z0) * G.inv_hz);
                tzn = INFINITY;
            }
            bool act = valid && k >= 0 && k < G.nz;

            // --- walk ------------------------------------------------------------------
            float t = tin;
            const int maxit = G.nx + G.ny + 2;
#pragma unroll 1
            for (int it = 0; it <= maxit; ++it) {
                const float tn = fminf(fminf(txn, tyn), tout);
                if (act) {
                    const float *colp = vol + ((size_t)i * G.ny + j) * G.nz;
                    float ts = t;
                    while (tzn < tn) {
                        acc = __fmaf_rn(__fsub_rn(tzn, ts), __ldg(colp + k), acc);
                        ts = tzn;
                        k += sk;
                        if ((unsigned)k >= (unsigned)G.nz) {
                            act = false;
                            break;
                        }
                        tzn = t_cross(plane_at(k + (sk > 0), G.hz, G.z0), zO, cotp);
                    }
                    if (act) acc = __fmaf_rn(__fsub_rn(tn, ts), __ldg(colp + k), acc);
                }
                if (tn >= tout) break;
                if (!__any_sync(0xffffffffu, act)) break;
                if (txn <= tyn) {
                    i += si;
                    if ((unsigned)i >= (unsigned)G.nx) break;
                    txn = t_cross(plane_at(i + (si > 0), G.hx, G.x0), Ox, ix);
                } else {
                    j += sj;
                    if ((unsigned)j >= (unsigned)G.ny) break;
                    tyn = t_cross(plane_at(j + (sj > 0), G.hy, G.y0), Oy, iy);
                }
                t = tn;
            }
        }

        // --- epilogue ----------------------------------------------------------------
        const float p = acc * secp;  // horizontal length -> 3D length
        const size_t o = ((size_t)ia * G.nu + a) * G.nv + b;
        if (valid) {
            if (MODE == PROJ_PLAIN) {
                out[o] = p;
            } else if (MODE == PROJ_SCALED) {
                out[o] = p * secp;
            } else {
                const float yv = (MODE == PROJ_RESID32) ? __ldg(y32 + o) : __half2float(y16[o]);
                const float r = p - yv;
                r2 = (double)r * (double)r;
                out[o] = r * secp;
            }
        }
    }

    if (MODE == PROJ_RESID32 || MODE == PROJ_RESID16) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, off);
        __shared__ double red[PROJ_THREADS / 32];
        if (lane == 0) red[threadIdx.x >> 5] = r2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < PROJ_THREADS / 32; ++w) s += red[w];
            partial[blockIdx.x] = s;
        }
    }
}

static long project_blocks(const GeoDev &g) {
    const long nwarps = (long)g.na * g.nu * ((g.nv + 31) / 32);
    return (nwarps * 32 + PROJ_THREADS - 1) / PROJ_THREADS;
}

size_t project_partials(const GeoDev &g) { return (size_t)project_blocks(g); }

cudaError_t launch_project(const GeoDev &g, const float *vol, const float *y32, const __half *y16,
                           float *out, double *partial, int mode, cudaStream_t s, int *nblocks_out) {
    const long nb = project_blocks(g);
    if (nblocks_out) *nblocks_out = (int)nb;
    dim3 grid((unsigned)nb), block(PROJ_THREADS);
    switch (mode) {
        case PROJ_PLAIN: k_project<PROJ_PLAIN><<<grid, block, 0, s>>>(g, vol, y32, y16, out, partial); break;
        case PROJ_RESID32: k_project<PROJ_RESID32><<<grid, block, 0, s>>>(g, vol, y32, y16, out, partial); break;
        case PROJ_RESID16: k_project<PROJ_RESID16><<<grid, block, 0, s>>>(g, vol, y32, y16, out, partial); break;
        default: k_project<PROJ_SCALED><<<grid, block, 0, s>>>(g, vol, y32, y16, out, partial); break;
    }
    return cudaGetLastError();
}

}  // namespace cbct
