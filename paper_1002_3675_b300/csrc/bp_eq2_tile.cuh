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
// Layouts: volume [nx][ny][nz] (z fastest), residual [na][nu][nv] (v fastest).  One
// thread per voxel; the 32 lanes of a warp are consecutive voxels of one z-column, so
// they share the imager column pair (a0, a0 + 1) of every view and read nearby rows.
#pragma once

#include "cbct_internal.h"

namespace cbct {

constexpr int EQ2_THREADS = 256;

// lerp with explicit roundings: a + t (b - a) as t b + (a - t a)
__device__ __forceinline__ float eq2_lerp(float a, float b, float t) { return __fmaf_rn(t, b, __fmaf_rn(-t, a, a)); }

// Voxel idx (internal layout) of B r, without the dV/(du dv) factor.  Every rounding is
// spelled out, so the value does not depend on the kernel this body is inlined into.
__device__ __forceinline__ float eq2_voxel(const GeoDev &G, const float *__restrict__ r, size_t idx) {
    const int k = (int)(idx % (size_t)G.nz);
    const size_t t = idx / (size_t)G.nz;
    const int j = (int)(t % (size_t)G.ny);
    const int i = (int)(t / (size_t)G.ny);
    // voxel centre
    const float x = __fmaf_rn((float)i + 0.5f, G.hx, G.x0);
    const float y = __fmaf_rn((float)j + 0.5f, G.hy, G.y0);
    const float z = __fmaf_rn((float)k + 0.5f, G.hz, G.z0);
    const float dsd2 = __fmul_rn(G.dsd, G.dsd);
    const float z2 = __fmul_rn(z, z);
    const float dz = __fmul_rn(G.dsd, z);
    const size_t plane = (size_t)G.nu * G.nv;
    float acc = 0.f;
    for (int ia = 0; ia < G.na; ++ia) {
        const float2 cs = __ldg(G.view + ia);  // cos, sin
        // depth along the central ray and offsets along u and v, scaled to the imager
        const float depth = __fsub_rn(G.dso, __fmaf_rn(x, cs.x, __fmul_rn(y, cs.y)));
        const float inv = __frcp_rn(depth);
        const float us = __fmul_rn(__fmul_rn(G.dsd, __fmaf_rn(y, cs.x, -__fmul_rn(x, cs.y))), inv);
        const float vs = __fmul_rn(dz, inv);
        const float fa = __fmaf_rn(us, G.inv_du, G.cu);
        const float fb = __fmaf_rn(vs, G.inv_dv, G.cv);
        // weight L^3 / (L0 l^2) = dsd^2 l / depth^3
        const float ex = __fmaf_rn(-G.dso, cs.x, x), ey = __fmaf_rn(-G.dso, cs.y, y);
        const float l = __fsqrt_rn(__fmaf_rn(ex, ex, __fmaf_rn(ey, ey, z2)));
        const float w = __fmul_rn(__fmul_rn(dsd2, l), __fmul_rn(inv, __fmul_rn(inv, inv)));
        // bilinear interpolation, zero outside the pixel grid
        const float a0f = floorf(fa), b0f = floorf(fb);
        const float ta = __fsub_rn(fa, a0f), tb = __fsub_rn(fb, b0f);
        const int a0 = (int)a0f, b0 = (int)b0f;
        const float *rv = r + (size_t)ia * plane;
        const bool a0in = a0 >= 0 && a0 < G.nu, a1in = a0 + 1 >= 0 && a0 + 1 < G.nu;
        const bool b0in = b0 >= 0 && b0 < G.nv, b1in = b0 + 1 >= 0 && b0 + 1 < G.nv;
        const float r00 = (a0in && b0in) ? __ldg(rv + (size_t)a0 * G.nv + b0) : 0.f;
        const float r01 = (a0in && b1in) ? __ldg(rv + (size_t)a0 * G.nv + b0 + 1) : 0.f;
        const float r10 = (a1in && b0in) ? __ldg(rv + (size_t)(a0 + 1) * G.nv + b0) : 0.f;
        const float r11 = (a1in && b1in) ? __ldg(rv + (size_t)(a0 + 1) * G.nv + b0 + 1) : 0.f;
        const float val = eq2_lerp(eq2_lerp(r00, r01, tb), eq2_lerp(r10, r11, tb), ta);
        acc = __fmaf_rn(w, val, acc);
    }
    return acc;
}

// One block of EQ2_THREADS voxels: out = scale * B r (plain) or fin - cscale * B r (step).
__device__ __forceinline__ void eq2_block(const GeoDev &G, const float *__restrict__ r,
                                          const float *__restrict__ fin, float *__restrict__ out, float cscale,
                                          int mode, long blk) {
    const size_t idx = (size_t)blk * EQ2_THREADS + threadIdx.x;
    if (idx >= vol_elems(G)) return;
    const float acc = eq2_voxel(G, r, idx);
    out[idx] = mode == BP_STEP ? __fmaf_rn(-cscale, acc, __ldg(fin + idx)) : __fmul_rn(cscale, acc);
}

}  // namespace cbct
