// Device body of the Eq. 2 adjoint (shared by the single-request and batched kernels).
//
// Eq. 2 (Jia et al. 2010) evaluates the variation of E2 voxel by voxel: for each view
// the residual is read at the imager point (u*, v*) where the line from the source
// through the voxel meets the imager, weighted by L^3 / (L0 l^2), with l the source
// to voxel distance, L the source to (u*, v*) distance and L0 = dsd.  Multiplied by
// Nv, with A = Np du dv, this replaces P^T r of step 1 by
//   (B r)_j = dV / (du dv) * sum_theta L^3 / (L0 l^2) * r_theta(u*, v*),
// where r_theta(u*, v*) is the bilinear interpolation of the residual between pixel
// centres (samples outside the pixel grid count as 0).  Since L = l dsd / depth
// (depth = distance along the central ray), the weight is dsd^2 l / depth^3.
//
// Layouts: volume [nx][ny][nz] (z fastest), residual [na][nu][nv] (v fastest).  A warp
// owns one z-column (i, j), its lane l holding the voxels k = l + 32 v (v < VZ), so the
// 32 VZ voxels of the column share everything that depends on the column and the view
// alone (the depth and its reciprocal, u*, the imager column pair (a0, a0 + 1) and its
// weight, the horizontal distance to the source), computed once per view; per voxel
// remain v*, the bilinear taps of two imager rows, l and the weight.  The reciprocal
// and the reciprocal square root are the hardware's approximate ones (relative error
// about 2^-22, far inside the operator's 1e-5 parity); every other rounding is spelled
// out, so the value does not depend on the kernel this body is inlined into.
#pragma once

#include "cbct_internal.h"

namespace cbct {

constexpr int EQ2_THREADS = 256;
constexpr int EQ2_COLS = EQ2_THREADS / 32;   // z-columns per block (one per warp)
constexpr int EQ2_MAX_VZ = 4;                // voxels per lane: z-blocks of 128 voxels

// blocks of one launch (tiles of the batched kernel)
__host__ __device__ __forceinline__ long eq2_tiles(const GeoDev &g) {
    return ((long)g.nx * g.ny + EQ2_COLS - 1) / EQ2_COLS;
}

// lerp with explicit roundings: a + t (b - a) as t b + (a - t a)
__device__ __forceinline__ float eq2_lerp(float a, float b, float t) { return __fmaf_rn(t, b, __fmaf_rn(-t, a, a)); }

__device__ __forceinline__ float eq2_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float eq2_rsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The voxels k = kz0 + lane + 32 v (v < VZ) of column (i, j): acc[v] = (B r)_k without the
// dV/(du dv) factor.
//
// PAD: r is the residual with a zero border, [na][nu + 2][nv + 2] with pixel (a, b) at
// (a + 1, b + 1) (eq2_pad), so that the taps of a voxel need no checks: its row index is
// clamped to [-1, nv - 1] (a voxel below or above the imager reads any row pair and is
// given the value 0), and a view whose column pair lies wholly off the imager is skipped
// (its taps are all 0, and adding w * 0 to an accumulator that started at +0 changes no
// bit).  The taps read are the same numbers, so the result is the same either way.
template <int VZ, bool PAD>
__device__ __forceinline__ void eq2_column(const GeoDev &G, const float *__restrict__ r, int i, int j, int kz0,
                                           float *acc) {
    const int lane = threadIdx.x & 31;
    const float x = __fmaf_rn((float)i + 0.5f, G.hx, G.x0);
    const float y = __fmaf_rn((float)j + 0.5f, G.hy, G.y0);
    float z[VZ], z2[VZ];
#pragma unroll
    for (int v = 0; v < VZ; ++v) {
        z[v] = __fmaf_rn((float)(kz0 + lane + 32 * v) + 0.5f, G.hz, G.z0);
        z2[v] = __fmul_rn(z[v], z[v]);
        acc[v] = 0.f;
    }
    const float dsd2 = __fmul_rn(G.dsd, G.dsd);
    const size_t plane = (size_t)G.nu * G.nv;
    // The column quantities of a view are the same for every lane: lane l computes those
    // of view vb + l for a group of 32 views (the same expressions), and the warp takes
    // each view's in turn from its lane.  The fast-path test of a view (every tap of the
    // column on the imager) needs only the column's lowest and highest voxel, since v*
    // grows with z (sv > 0: the depth is positive).
    const float zlo = __fmaf_rn((float)kz0 + 0.5f, G.hz, G.z0);
    const float zhi = __fmaf_rn((float)(kz0 + 31 + 32 * (VZ - 1)) + 0.5f, G.hz, G.z0);
    for (int vb = 0; vb < G.na; vb += 32) {
        float g_ta = 0.f, g_sv = 0.f, g_wc = 0.f, g_e2 = 0.f;
        int g_a0 = -2, g_in = 0;
        if (vb + lane < G.na) {
            const float2 cs = __ldg(G.view + vb + lane);  // cos, sin
            // depth along the central ray, u* in pixels, and the column pair
            const float depth = __fsub_rn(G.dso, __fmaf_rn(x, cs.x, __fmul_rn(y, cs.y)));
            const float inv = eq2_rcp(depth);
            const float us = __fmul_rn(__fmul_rn(G.dsd, __fmaf_rn(y, cs.x, -__fmul_rn(x, cs.y))), inv);
            const float fa = __fmaf_rn(us, G.inv_du, G.cu);
            const float a0f = floorf(fa);
            g_ta = __fsub_rn(fa, a0f);
            g_a0 = (int)a0f;
            // v* = dsd z / depth in pixels; weight L^3 / (L0 l^2) = dsd^2 l / depth^3
            g_sv = __fmul_rn(__fmul_rn(G.dsd, inv), G.inv_dv);
            g_wc = __fmul_rn(dsd2, __fmul_rn(inv, __fmul_rn(inv, inv)));
            const float ex = __fmaf_rn(-G.dso, cs.x, x), ey = __fmaf_rn(-G.dso, cs.y, y);
            g_e2 = __fmaf_rn(ex, ex, __fmul_rn(ey, ey));
            g_in = g_a0 >= 0 && g_a0 + 1 < G.nu && __fmaf_rn(zlo, g_sv, G.cv) >= 0.f &&
                   __fmaf_rn(zhi, g_sv, G.cv) < (float)(G.nv - 1) && kz0 + 32 * VZ <= G.nz;
        }
        const int nview = min(32, G.na - vb);
        for (int jv = 0; jv < nview; ++jv) {
            const int ia = vb + jv;
            const float ta = __shfl_sync(0xffffffffu, g_ta, jv);
            const float sv = __shfl_sync(0xffffffffu, g_sv, jv);
            const float wc = __shfl_sync(0xffffffffu, g_wc, jv);
            const float e2 = __shfl_sync(0xffffffffu, g_e2, jv);
            const int a0 = __shfl_sync(0xffffffffu, g_a0, jv);
            const bool all_inside = __shfl_sync(0xffffffffu, g_in, jv) != 0;
            if constexpr (PAD) {
                if (a0 < -1 || a0 > G.nu - 1) continue;  // (warp-uniform)
                const float *rv0 = r + ((size_t)ia * (G.nu + 2) + (a0 + 1)) * (G.nv + 2) + 1;
                const float *rv1 = rv0 + (G.nv + 2);
#pragma unroll
                for (int v = 0; v < VZ; ++v) {
                    const float fb = __fmaf_rn(z[v], sv, G.cv);
                    const float b0f = floorf(fb);
                    const float tb = __fsub_rn(fb, b0f);
                    const int b0 = (int)b0f;
                    const int bc = min(max(b0, -1), G.nv - 1);
                    const float r00 = __ldg(rv0 + bc), r01 = __ldg(rv0 + bc + 1);
                    const float r10 = __ldg(rv1 + bc), r11 = __ldg(rv1 + bc + 1);
                    float val = eq2_lerp(eq2_lerp(r00, r01, tb), eq2_lerp(r10, r11, tb), ta);
                    if (bc != b0) val = 0.f;
                    const float l2 = __fadd_rn(e2, z2[v]);
                    const float w = __fmul_rn(wc, __fmul_rn(l2, eq2_rsqrt(l2)));   // dsd^2 depth^-3 l
                    acc[v] = __fmaf_rn(w, val, acc[v]);
                }
                continue;
            }
            const bool a0in = a0 >= 0 && a0 < G.nu, a1in = a0 + 1 >= 0 && a0 + 1 < G.nu;
            const float *rv0 = r + (size_t)ia * plane + (size_t)(a0in ? a0 : 0) * G.nv;
            const float *rv1 = r + (size_t)ia * plane + (size_t)(a1in ? a0 + 1 : 0) * G.nv;
            if (all_inside) {
    #pragma unroll
                for (int v = 0; v < VZ; ++v) {
                    const float fb = __fmaf_rn(z[v], sv, G.cv);
                    const float b0f = floorf(fb);
                    const float tb = __fsub_rn(fb, b0f);
                    const int b0 = (int)b0f;
                    const float r00 = __ldg(rv0 + b0), r01 = __ldg(rv0 + b0 + 1);
                    const float r10 = __ldg(rv1 + b0), r11 = __ldg(rv1 + b0 + 1);
                    const float val = eq2_lerp(eq2_lerp(r00, r01, tb), eq2_lerp(r10, r11, tb), ta);
                    const float l2 = __fadd_rn(e2, z2[v]);
                    const float w = __fmul_rn(wc, __fmul_rn(l2, eq2_rsqrt(l2)));   // dsd^2 depth^-3 l
                    acc[v] = __fmaf_rn(w, val, acc[v]);
                }
            } else {
    #pragma unroll
                for (int v = 0; v < VZ; ++v) {
                    const float fb = __fmaf_rn(z[v], sv, G.cv);
                    const float b0f = floorf(fb);
                    const float tb = __fsub_rn(fb, b0f);
                    const int b0 = (int)b0f;
                    const bool b0in = b0 >= 0 && b0 < G.nv, b1in = b0 + 1 >= 0 && b0 + 1 < G.nv;
                    // bilinear interpolation, zero outside the pixel grid
                    const float r00 = (a0in && b0in) ? __ldg(rv0 + b0) : 0.f;
                    const float r01 = (a0in && b1in) ? __ldg(rv0 + b0 + 1) : 0.f;
                    const float r10 = (a1in && b0in) ? __ldg(rv1 + b0) : 0.f;
                    const float r11 = (a1in && b1in) ? __ldg(rv1 + b0 + 1) : 0.f;
                    const float val = eq2_lerp(eq2_lerp(r00, r01, tb), eq2_lerp(r10, r11, tb), ta);
                    const float l2 = __fadd_rn(e2, z2[v]);
                    const float w = __fmul_rn(wc, __fmul_rn(l2, eq2_rsqrt(l2)));   // dsd^2 depth^-3 l
                    acc[v] = __fmaf_rn(w, val, acc[v]);
                }
            }
        }
    }
}

// Block blk (EQ2_COLS z-columns, one per warp): out = cscale * B' r (plain) or
// fin - cscale * B' r (step), B' being B without its dV/(du dv) factor.
// pad: r is the zero-bordered residual (eq2_column's PAD form).
__device__ __forceinline__ void eq2_block(const GeoDev &G, const float *__restrict__ r, bool pad,
                                          const float *__restrict__ fin, float *__restrict__ out, float cscale,
                                          int mode, long blk) {
    const long col = blk * EQ2_COLS + (threadIdx.x >> 5);
    if (col >= (long)G.nx * G.ny) return;
    const int i = (int)(col / G.ny), j = (int)(col % G.ny);
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)col * G.nz;     // internal layout: (i, j, k) at (i ny + j) nz + k
    for (int kz0 = 0; kz0 < G.nz; kz0 += 32 * EQ2_MAX_VZ) {
        const int vz = min(EQ2_MAX_VZ, (G.nz - kz0 + 31) / 32);
        float acc[EQ2_MAX_VZ] = {0.f, 0.f, 0.f, 0.f};
        if (pad) {
            if (vz == 1) eq2_column<1, true>(G, r, i, j, kz0, acc);
            else if (vz == 2) eq2_column<2, true>(G, r, i, j, kz0, acc);
            else if (vz == 3) eq2_column<3, true>(G, r, i, j, kz0, acc);
            else eq2_column<4, true>(G, r, i, j, kz0, acc);
        } else {
            if (vz == 1) eq2_column<1, false>(G, r, i, j, kz0, acc);
            else if (vz == 2) eq2_column<2, false>(G, r, i, j, kz0, acc);
            else if (vz == 3) eq2_column<3, false>(G, r, i, j, kz0, acc);
            else eq2_column<4, false>(G, r, i, j, kz0, acc);
        }
#pragma unroll
        for (int v = 0; v < EQ2_MAX_VZ; ++v) {
            const int k = kz0 + lane + 32 * v;
            if (v >= vz || k >= G.nz) continue;
            const size_t idx = base + k;
            out[idx] = mode == BP_STEP ? __fmaf_rn(-cscale, acc[v], __ldg(fin + idx)) : __fmul_rn(cscale, acc[v]);
        }
    }
}

}  // namespace cbct
