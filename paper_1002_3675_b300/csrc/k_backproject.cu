// Adjoint of the projector, evaluated voxel by voxel (the structure of Eq. 2 of Jia
// et al. 2010: every voxel's variation of E2 is computed independently from the
// residual images), with the exact intersection lengths of P instead of Eq. 2's
// interpolated weights, so that the result is the matrix transpose P^T of the
// paragraph before Eq. 2.  Fused epilogue: step 1 of Algorithm A1,
// g = f - c P^T r with c = gamma / beta.
//
// Work decomposition.  One warp owns 32 consecutive voxels of one z-column (i, j).
// For each view the candidate detector columns are those whose ray plane meets the
// xy-cell (the interval spanned by the cell's four projected corners, widened by
// one); the xy part of the intersection interval is the same for the whole column,
// so it is computed once per warp.  Each lane then visits the detector rows whose
// ray meets its voxel (again the interval spanned by four corners) and adds
// length * (sec(phi) r), the residual having been pre-scaled by sec(phi) in the
// projector's epilogue.  The sum is taken in a fixed order (view, column, row) with
// no atomics, so results are deterministic.
#include "cbct_internal.h"

namespace cbct {

static constexpr int BP_THREADS = 128;

template <int MODE>
__global__ void __launch_bounds__(BP_THREADS)
k_backproject(GeoDev G, const float *__restrict__ rs, const float *__restrict__ fin,
              float *__restrict__ out, float c) {
    const int lane = threadIdx.x & 31;
    const long gwarp = ((long)blockIdx.x * BP_THREADS + threadIdx.x) >> 5;
    const int nkc = (G.nz + 31) >> 5;
    const long nwarps = (long)G.nx * G.ny * nkc;
    if (gwarp >= nwarps) return;
    const int kc = (int)(gwarp % nkc);
    const long colid = gwarp / nkc;
    const int j = (int)(colid % G.ny);
    const int i = (int)(colid / G.ny);
    const int k = kc * 32 + lane;
    const bool valid = k < G.nz;
    const int kq = valid ? k : G.nz - 1;

    const float xl = plane_at(i, G.hx, G.x0), xh = plane_at(i + 1, G.hx, G.x0);
    const float yl = plane_at(j, G.hy, G.y0), yh = plane_at(j + 1, G.hy, G.y0);
    const float zl = plane_at(kq, G.hz, G.z0), zh = plane_at(kq + 1, G.hz, G.z0);
    const float ufac = G.dsd * G.inv_du;

    float acc = 0.f;
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
        const int alo = max(0, (int)floorf(amin));
        const int ahi = min(G.nu - 1, (int)ceilf(amax));
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
            // detector-row interval of this voxel on column a: v* = z D / (tS + t)
            const float2 Dt = G.col[a];
            const float q1 = __fdividef(Dt.x, Dt.y + tlo), q2 = __fdividef(Dt.x, Dt.y + thi);
            const float v1 = zl * q1, v2 = zl * q2, v3 = zh * q1, v4 = zh * q2;
            const float vmin = fminf(fminf(v1, v2), fminf(v3, v4));
            const float vmax = fmaxf(fmaxf(v1, v2), fmaxf(v3, v4));
            const int blo = max(0, (int)floorf(__fmaf_rn(vmin, G.inv_dv, G.cv)));
            int bhi = min(G.nv - 1, (int)ceilf(__fmaf_rn(vmax, G.inv_dv, G.cv)));
            if (!valid) bhi = blo - 1;
            const float4 *rzp = G.ray_z + (size_t)a * G.nv;
            const float *rsp = rsv + (size_t)a * G.nv;
            for (int b = blo; b <= bhi; ++b) {
                const float4 rz = __ldg(rzp + b);
                float lo = tlo, hi = thi;
                if (rz.y != 0.f) {
                    const float z1 = t_cross(zl, rz.x, rz.y), z2 = t_cross(zh, rz.x, rz.y);
                    lo = fmaxf(lo, fminf(z1, z2));
                    hi = fminf(hi, fmaxf(z1, z2));
                } else if (!(rz.x >= zl && rz.x < zh)) {
                    continue;
                }
                if (hi > lo) acc = __fmaf_rn(__fsub_rn(hi, lo), __ldg(rsp + b), acc);
            }
        }
    }
    if (valid) {
        const size_t o = ((size_t)i * G.ny + j) * G.nz + k;
        out[o] = (MODE == BP_PLAIN) ? acc : __ldg(fin + o) - c * acc;
    }
}

cudaError_t launch_backproject(const GeoDev &g, const float *rs, const float *fin, float *out, float c,
                               int mode, cudaStream_t s) {
    const long nwarps = (long)g.nx * g.ny * ((g.nz + 31) / 32);
    const long nb = (nwarps * 32 + BP_THREADS - 1) / BP_THREADS;
    dim3 grid((unsigned)nb), block(BP_THREADS);
    if (mode == BP_PLAIN)
        k_backproject<BP_PLAIN><<<grid, block, 0, s>>>(g, rs, fin, out, c);
    else
        k_backproject<BP_STEP><<<grid, block, 0, s>>>(g, rs, fin, out, c);
    return cudaGetLastError();
}

}  // namespace cbct
