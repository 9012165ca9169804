// Adjoint of the projector, evaluated voxel by voxel (the structure of Eq. 2 of Jia
// et al. 2010: every voxel's variation of E2 is computed independently from the
// residual images), with the exact intersection lengths of P instead of Eq. 2's
// interpolated weights, so that the result is the matrix transpose P^T of the
// paragraph before Eq. 2.  Fused epilogue: step 1 of Algorithm A1,
// g = f - c P^T r with c = gamma / beta.
//
// Work decomposition.  One warp owns 32*VPL voxels of one z-column (i, j); lane l
// holds voxels k = base + l + 32 v, v < VPL.  For each view, the candidate detector
// columns are those whose ray plane meets the xy-cell: the interval spanned by the
// cell's four projected corners, widened by CAND_MARGIN pixel (the computed bounds
// are accurate to ~1e-4 pixel, and a ray outside the exact interval meets the cell
// in a zero-length set).  The xy part of the intersection interval is the same for
// the whole column, so it is computed once per warp.  Each lane then visits, for each
// of its voxels, the detector rows whose ray meets the voxel (the interval spanned by
// the four (t, z) corners, same margin) and adds length * (sec(phi) r), the residual
// having been pre-scaled by sec(phi) in the projector's epilogue.  The sum is taken
// in a fixed order (view, column, row) with no atomics, so results are deterministic.
#include "cbct_internal.h"

namespace cbct {

static constexpr int BP_THREADS = 128;
static constexpr float CAND_MARGIN = 0.01f;  // pixels

template <int MODE, int VPL>
__global__ void __launch_bounds__(BP_THREADS, 8)
k_backproject(GeoDev G, const float *__restrict__ rs, const float *__restrict__ fin,
              float *__restrict__ out, float c) {
    const int lane = threadIdx.x & 31;
    const long gwarp = ((long)blockIdx.x * BP_THREADS + threadIdx.x) >> 5;
    const int nkc = (G.nz + 32 * VPL - 1) / (32 * VPL);
    const long nwarps = (long)G.nx * G.ny * nkc;
    if (gwarp >= nwarps) return;
    const int kc = (int)(gwarp % nkc);
    const long colid = gwarp / nkc;
    const int j = (int)(colid % G.ny);
    const int i = (int)(colid / G.ny);

    float zl[VPL], zh[VPL], acc[VPL];
    bool valid[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int k = kc * 32 * VPL + lane + 32 * v;
        valid[v] = k < G.nz;
        const int kq = valid[v] ? k : G.nz - 1;
        zl[v] = plane_at(kq, G.hz, G.z0);
        zh[v] = plane_at(kq + 1, G.hz, G.z0);
        acc[v] = 0.f;
    }
    const float xl = plane_at(i, G.hx, G.x0), xh = plane_at(i + 1, G.hx, G.x0);
    const float yl = plane_at(j, G.hy, G.y0), yh = plane_at(j + 1, G.hy, G.y0);
    const float ufac = G.dsd * G.inv_du;

#pragma unroll 1
    for (int ia = 0; ia < G.na; ++ia) {
        const float2 cs = G.view[ia];
        // detector-column interval of the xy-cell: u* = dsd (p.u) / (dso - p.s)
        float amin = INFINITY, amax = -INFINITY;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float px = (q & 1) ? xh : xl, py = (q & 2) ? yh : yl;
            const float num = py * cs.x - px * cs.y;
            const float den = G.dso - (px * cs.x + py * cs.y);
            const float ac = __fdividef(num, den) * ufac + G.cu;
            amin = fminf(amin, ac);
            amax = fmaxf(amax, ac);
        }
        const int alo = max(0, (int)ceilf(amin - CAND_MARGIN));
        const int ahi = min(G.nu - 1, (int)floorf(amax + CAND_MARGIN));
        const float *rsv = rs + (size_t)ia * G.nu * G.nv;
#pragma unroll 1
        for (int a = alo; a <= ahi; ++a) {
            const float4 rxy = G.ray_xy[(size_t)ia * G.nu + a];
            float tlo = -INFINITY, thi = INFINITY;
            if (rxy.z != 0.f) {
                const float t1 = t_cross(xl, rxy.x, rxy.z), t2 = t_cross(xh, rxy.x, rxy.z);
                tlo = fminf(t1, t2);
                thi = fmaxf(t1, t2);
            } else if (!(rxy.x >= xl && rxy.x < xh)) {
                continue;
            }
            if (rxy.w != 0.f) {
                const float t1 = t_cross(yl, rxy.y, rxy.w), t2 = t_cross(yh, rxy.y, rxy.w);
                tlo = fmaxf(tlo, fminf(t1, t2));
                thi = fminf(thi, fmaxf(t1, t2));
            } else if (!(rxy.y >= yl && rxy.y < yh)) {
                continue;
            }
            if (!(thi > tlo)) continue;
            // detector-row interval of a voxel on column a: v* = z D / (tS + t); with
            // q1 = D/(tS + tlo) > q2 = D/(tS + thi) > 0 the extreme corners follow from
            // the signs of the voxel's bounding planes
            const float2 Dt = G.col[a];
            const float q1 = __fdividef(Dt.x, Dt.y + tlo) * G.inv_dv;
            const float q2 = __fdividef(Dt.x, Dt.y + thi) * G.inv_dv;
            const float2 *rzp = G.ray_zc + (size_t)a * G.nv;
            const float *rsp = rsv + (size_t)a * G.nv;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const float bmin = zl[v] * (zl[v] > 0.f ? q2 : q1) + G.cv;
                const float bmax = zh[v] * (zh[v] > 0.f ? q1 : q2) + G.cv;
                const int blo = max(0, (int)ceilf(bmin - CAND_MARGIN));
                int bhi = min(G.nv - 1, (int)floorf(bmax + CAND_MARGIN));
                if (!valid[v]) bhi = blo - 1;
                for (int b = blo; b <= bhi; ++b) {
                    const float2 rz = __ldg(rzp + b);
                    float lo = tlo, hi = thi;
                    if (rz.y != 0.f) {
                        const float z1 = t_cross(zl[v], rz.x, rz.y), z2 = t_cross(zh[v], rz.x, rz.y);
                        lo = fmaxf(lo, fminf(z1, z2));
                        hi = fminf(hi, fmaxf(z1, z2));
                    } else if (!(rz.x >= zl[v] && rz.x < zh[v])) {
                        continue;
                    }
                    if (hi > lo) acc[v] = __fmaf_rn(__fsub_rn(hi, lo), __ldg(rsp + b), acc[v]);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        if (!valid[v]) continue;
        const size_t o = ((size_t)i * G.ny + j) * G.nz + kc * 32 * VPL + lane + 32 * v;
        out[o] = (MODE == BP_PLAIN) ? acc[v] : __ldg(fin + o) - c * acc[v];
    }
}

template <int VPL>
static void launch_vpl(const GeoDev &g, const float *rs, const float *fin, float *out, float c, int mode,
                       cudaStream_t s) {
    const long nwarps = (long)g.nx * g.ny * ((g.nz + 32 * VPL - 1) / (32 * VPL));
    const long nb = (nwarps * 32 + BP_THREADS - 1) / BP_THREADS;
    if (mode == BP_PLAIN)
        k_backproject<BP_PLAIN, VPL><<<(unsigned)nb, BP_THREADS, 0, s>>>(g, rs, fin, out, c);
    else
        k_backproject<BP_STEP, VPL><<<(unsigned)nb, BP_THREADS, 0, s>>>(g, rs, fin, out, c);
}

cudaError_t launch_backproject(const GeoDev &g, const float *rs, const float *fin, float *out, float c,
                               int mode, cudaStream_t s) {
    // voxels per lane: cover a z-column with as few warps as possible, up to 4 per lane
    const int per_lane = (g.nz + 31) / 32;
    if (per_lane >= 4) launch_vpl<4>(g, rs, fin, out, c, mode, s);
    else if (per_lane == 3) launch_vpl<3>(g, rs, fin, out, c, mode, s);
    else if (per_lane == 2) launch_vpl<2>(g, rs, fin, out, c, mode, s);
    else launch_vpl<1>(g, rs, fin, out, c, mode, s);
    return cudaGetLastError();
}

}  // namespace cbct
