// Device-side warp tile of the adjoint gather (shared by the single-request and
// batched kernels).
#pragma once

// Adjoint of the projector, evaluated voxel by voxel (the structure of Eq. 2 of Jia
// et al. 2010: every voxel's variation of E2 is computed independently from the
// residual images), with the exact intersection lengths of P instead of Eq. 2's
// interpolated weights, so that the result is the matrix transpose P^T of the
// paragraph before Eq. 2.  Fused epilogue: step 1 of Algorithm A1,
// g = f - c P^T r with c = gamma / beta.
//
// Work decomposition.  One warp owns 32*VPL voxels of one z-column (i, j); lane l
// holds VPL of them, in one of two layouts (IL, bitwise the same results):
// consecutive, k = base + VPL l + v, or interleaved, k = base + l + 32 v, v < VPL, where
// each gather of a detector column's running sums spans the rows of 32 planes instead
// of 32 VPL (fewer cache lines when a voxel covers several detector rows, for a few
// more shuffles).  The (view, detector
// column) pairs whose ray plane meets the xy-cell are derived by the warp from the
// cell's corners (bp_columns), in view then column order; for each, the part of the
// rays' horizontal parameter t inside the cell, [tlo, thi], is the same for the whole
// z-column.
//
// Plane sweep.  In detector-row units, a ray b sits at row b and the plane z at
// rho_z(t) = z D / ((tS + t) dv) + cv, monotone in t.  Ray b is inside voxel k at t iff
// rho_{z_k}(t) <= b < rho_{z_k+1}(t), so its length in the voxel is
// J_{z_k+1}(b) - J_{z_k}(b) with J_z(b) = |{t in [tlo, thi] : b < rho_z(t)}|: thi - tlo for
// rows below both ends of rho_z, 0 for rows above both, and the exact crossing
// t* = (z - zO_b) cot_b otherwise (at most one row per plane here).  Hence
//   sum_b r_b len = (thi - tlo) sum_{b in [N(z_k), N(z_k+1))} r_b + P(z_k+1) - P(z_k),
// with N(z) the rows below both ends and P(z) the partial rows' sum.  The sum over
// full rows is a difference of running sums along the detector column (double-float
// sums stored as a float32 pair, so the difference keeps float32 accuracy).  Each lane
// evaluates the planes below its voxels and takes the plane above from its own next
// voxel or from the next lane (the chunk's top plane for the last voxel).
// The residual is pre-scaled by sec(phi) (3D length = t-length * sec(phi)).  Sums are
// taken in a fixed order with no atomics, so results are deterministic.
#include "cbct_internal.h"

namespace cbct {

constexpr int BP_THREADS = 128;

// N(z) and P(z) of one plane for detector column rzp/rsp over [tlo, thi].  At most one
// row is partial on almost every plane, so the first one is taken without a loop.
__device__ __forceinline__ void eval_plane(float z, float q1, float q2, float cv, int nv, float tlo, float thi,
                                           const float2 *__restrict__ rzp, const float *__restrict__ rsp,
                                           int &nmin, float &part) {
    const float r1 = __fmaf_rn(z, q1, cv), r2 = __fmaf_rn(z, q2, cv);
    const float lo = fminf(r1, r2), hi = fmaxf(r1, r2);
    nmin = min(max((int)ceilf(lo), 0), nv);
    const int nmax = min(max((int)ceilf(hi), 0), nv);
    const bool dec = r1 > r2;  // rho falls with t: the row is below the plane before t*
    part = 0.f;
    if (nmax > nmin) {
        const float2 rz = __ldg(rzp + nmin);
        const float ts = fminf(fmaxf(t_cross(z, rz.x, rz.y), tlo), thi);
        part = __fmul_rn(__ldg(rsp + nmin), dec ? ts - tlo : thi - ts);
        for (int b = nmin + 1; b < nmax; ++b) {
            const float2 rz2 = __ldg(rzp + b);
            const float ts2 = fminf(fmaxf(t_cross(z, rz2.x, rz2.y), tlo), thi);
            part = __fmaf_rn(__ldg(rsp + b), dec ? ts2 - tlo : thi - ts2, part);
        }
    }
}

// Number of warp tiles of a level: z-chunks of 32*VPL voxels times xy-cells.
template <int VPL>
__host__ __device__ __forceinline__ long bp_warp_tiles(const GeoDev &G) {
    return (long)G.nx * G.ny * ((G.nz + 32 * VPL - 1) / (32 * VPL));
}

// One warp tile (warp-uniform): z-chunk kc of xy-cell colid.  Lane l holds VPL voxels
// and evaluates the planes below them.  Consecutive layout: the plane above its last
// voxel is the next lane's first plane (the chunk's top plane for lane 31).
// Interleaved: the plane above voxel base + l + 32 v is the next lane's plane of the
// same slot (for lane 31, lane 0's plane of the next slot, or the chunk's top plane).  mode: BP_PLAIN writes P^T rs, BP_STEP writes fin - c P^T rs.  Shared by the
// single-request and batched kernels, so a request's result does not depend on what
// else is in the launch.
//
// The cell's candidate (view, column) pairs are taken 32 at a time: each lane first
// sets up one pair (its t-interval inside the cell, the row slopes at both ends and
// the chunk's top plane) into the warp's record buffer rec (2 float4 per lane, shared
// memory), then the warp walks the valid pairs in pair order, reading each record as
// a broadcast.  The sums are taken in the same order as a pair-by-pair walk.  Behind
// the records, 64 entries (a group of 64 views) of first pair and column offset.
constexpr int BP_REC_PER_WARP = 64 + 32;  // float4 of one warp: 2 per lane, then 2 x 64 ints

// Order of the xy-cells over the warp tiles: super-tiles of BP_SUPER x BP_SUPER cells
// (i rows of super-tiles, j fastest inside a row; ragged at the far edges), cells j
// fastest inside a super-tile.  The warps in flight then cover a compact patch of cells,
// whose footprint on each view's imager is a narrow band of columns, instead of a strip
// across the whole volume that touches most columns of most views: the row sums and
// residuals they gather stay in L2.  The order changes no result bit (every warp's
// voxels depend on that warp alone).
constexpr int BP_SUPER = 64;
// (32-bit arithmetic: a geometry has fewer than 2^31 voxels, so fewer cells)
__host__ __device__ __forceinline__ void bp_cell_of(const GeoDev &G, int q, int &i, int &j) {
    const int row = BP_SUPER * G.ny;                // cells in one row of super-tiles
    const int R = q / row;
    const int wi = min(BP_SUPER, G.nx - R * BP_SUPER);
    const int off = q - R * row;
    const int C = off / (wi * BP_SUPER);
    const int wj = min(BP_SUPER, G.ny - C * BP_SUPER);
    const int rem = off - C * wi * BP_SUPER;
    i = R * BP_SUPER + rem / wj;
    j = C * BP_SUPER + rem % wj;
}

// Candidate detector columns of view v for the xy-cell [xl, xh) x [yl, yh): the interval
// spanned by the cell's four corners projected onto the imager (u = dsd (p . u_hat) /
// (dso - p . s_hat), in column units), widened by 0.01 column.  A ray plane outside it
// misses the cell by about a hundred ulps of its parameter t at least, so its
// intersection test below comes out empty; every column whose test is not empty is
// inside.  Gives the first column in d and the count in n (0 for v >= na).  Float32
// rounding moves a projected corner by about 1e-4 column at most, far inside the margin,
// so the pairs that contribute are those of the exact intervals.
__device__ __forceinline__ void bp_columns(const GeoDev &G, int v, float xl, float xh, float yl, float yh, int &d,
                                           int &n) {
    d = 0;
    n = 0;
    if (v >= G.na) return;
    const float2 cs = __ldg(G.view + v);
    const float k = G.dsd * G.inv_du;
    float amin = INFINITY, amax = -INFINITY;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float px = (q & 1) ? xh : xl, py = (q & 2) ? yh : yl;
        const float num = py * cs.x - px * cs.y;
        const float den = G.dso - (px * cs.x + py * cs.y);
        const float av = __fdividef(k * num, den) + G.cu;
        amin = fminf(amin, av);
        amax = fmaxf(amax, av);
    }
    const int lo = max((int)ceilf(amin - 0.01f), 0), hi = min((int)floorf(amax + 0.01f), G.nu - 1);
    d = lo;
    n = max(hi - lo + 1, 0);
}

template <int VPL, bool IL>
__device__ __forceinline__ void bp_warp(const GeoDev &G, const int mode, const float *__restrict__ rs,
                                         const float *__restrict__ fin, float *__restrict__ out, const float c,
                                         const long wtile, float4 *__restrict__ rec) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nkc = (G.nz + 32 * VPL - 1) / (32 * VPL);
    const int kc = (int)(wtile % nkc);
    int i, j;
    bp_cell_of(G, (int)(wtile / nkc), i, j);
    const int base = kc * 32 * VPL + (IL ? lane : lane * VPL);  // voxel v: base + (IL ? 32 v : v)
    constexpr int VS = IL ? 32 : 1;
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.f;
    int *ent_s = reinterpret_cast<int *>(rec + 64);  // [64] first pair of each entry
    int *ent_d = ent_s + 64;                          // [64] column minus pair index
#pragma unroll 1
    for (int vb = 0; vb < G.na; vb += 64) {
        // the candidate columns of views vb + lane (entry lane) and vb + 32 + lane (entry
        // 32 + lane), and each entry's first pair in view order (a warp scan of the counts)
        int n0, n1, d0, d1;
        {
            const float xl = plane_at(i, G.hx, G.x0), xh = plane_at(i + 1, G.hx, G.x0);
            const float yl = plane_at(j, G.hy, G.y0), yh = plane_at(j + 1, G.hy, G.y0);
            bp_columns(G, vb + lane, xl, xh, yl, yh, d0, n0);
            bp_columns(G, vb + 32 + lane, xl, xh, yl, yh, d1, n1);
        }
        int s0 = n0, s1 = n1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t0 = __shfl_up_sync(FULL, s0, d), t1 = __shfl_up_sync(FULL, s1, d);
            if (lane >= d) {
                s0 += t0;
                s1 += t1;
            }
        }
        const int tot0 = __shfl_sync(FULL, s0, 31);
        const int tot = tot0 + __shfl_sync(FULL, s1, 31);
        s0 -= n0;
        s1 += tot0 - n1;
        ent_s[lane] = s0;
        ent_s[32 + lane] = s1;
        ent_d[lane] = d0 - s0;
        ent_d[32 + lane] = d1 - s1;
        __syncwarp();
#pragma unroll 1
        for (int pb = 0; pb < tot; pb += 32) {
            // pair pb + lane: its entry is the last one whose first pair is <= it
            const int q = pb + lane;
            int e = q >= ent_s[32] ? 32 : 0;     // entry 32 starts at the first half's total
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1)
                if (ent_s[e + st] <= q) e += st;
            // setup of pair q
            bool ok = false;
            if (q < tot) {
                const float xl = plane_at(i, G.hx, G.x0), xh = plane_at(i + 1, G.hx, G.x0);
                const float yl = plane_at(j, G.hy, G.y0), yh = plane_at(j + 1, G.hy, G.y0);
                const int a = q + ent_d[e];
                const int col = (vb + e) * G.nu + a;
                const float4 rxy = __ldg(G.ray_xy + col);
                float tlo = -INFINITY, thi = INFINITY;
                ok = true;
                if (rxy.z != 0.f) {
                    const float t1 = t_cross(xl, rxy.x, rxy.z), t2 = t_cross(xh, rxy.x, rxy.z);
                    tlo = fminf(t1, t2);
                    thi = fmaxf(t1, t2);
                } else if (!(rxy.x >= xl && rxy.x < xh)) {
                    ok = false;
                }
                if (rxy.w != 0.f) {
                    const float t1 = t_cross(yl, rxy.y, rxy.w), t2 = t_cross(yh, rxy.y, rxy.w);
                    tlo = fmaxf(tlo, fminf(t1, t2));
                    thi = fminf(thi, fmaxf(t1, t2));
                } else if (!(rxy.y >= yl && rxy.y < yh)) {
                    ok = false;
                }
                ok = ok && thi > tlo;
                if (ok) {
                    const float2 Dt = __ldg(G.col + a);
                    const float q1 = __fdividef(Dt.x, Dt.y + tlo) * G.inv_dv;
                    const float q2 = __fdividef(Dt.x, Dt.y + thi) * G.inv_dv;
                    int nt;
                    float pt;
                    eval_plane(plane_at(kc * 32 * VPL + 32 * VPL, G.hz, G.z0), q1, q2, G.cv, G.nv, tlo, thi,
                               G.ray_zc + (size_t)a * G.nv, rs + (size_t)col * G.nv, nt, pt);
                    rec[2 * lane] = make_float4(tlo, thi, q1, q2);
                    rec[2 * lane + 1] = make_float4(__int_as_float(col), __int_as_float(a), __int_as_float(nt), pt);
                }
            }
            unsigned valid = __ballot_sync(FULL, ok);
            __syncwarp();
    #pragma unroll 1
            while (valid) {
                const int src = __ffs(valid) - 1;
                valid &= valid - 1;
                const float4 r0 = rec[2 * src], r1 = rec[2 * src + 1];
                const float tlo = r0.x, thi = r0.y, q1 = r0.z, q2 = r0.w;
                const int col = __float_as_int(r1.x), a = __float_as_int(r1.y);
                const float w = thi - tlo;
                const float2 *rzp = G.ray_zc + (size_t)a * G.nv;
                const float *rsp = rs + (size_t)col * G.nv;
                const float2 *cum = G.rowsum + (size_t)col * (G.nv + 1);
                int nb[VPL + 1];
                float pbv[VPL + 1];
    #pragma unroll
                for (int v = 0; v < VPL; ++v)
                    eval_plane(plane_at(base + VS * v, G.hz, G.z0), q1, q2, G.cv, G.nv, tlo, thi, rzp, rsp, nb[v],
                               pbv[v]);
                if constexpr (!IL) {
                    nb[VPL] = __shfl_down_sync(FULL, nb[0], 1);
                    pbv[VPL] = __shfl_down_sync(FULL, pbv[0], 1);
                    if (lane == 31) {
                        nb[VPL] = __float_as_int(r1.z);
                        pbv[VPL] = r1.w;
                    }
                    float2 c0 = __ldg(cum + nb[0]);
    #pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        const float2 c1 = __ldg(cum + nb[v + 1]);
                        const float full = __fadd_rn(__fsub_rn(c1.x, c0.x), __fsub_rn(c1.y, c0.y));
                        acc[v] += __fmaf_rn(w, full, pbv[v + 1] - pbv[v]);
                        c0 = c1;
                    }
                } else {
                    float2 cb[VPL];
    #pragma unroll
                    for (int v = 0; v < VPL; ++v) cb[v] = __ldg(cum + nb[v]);
                    float2 ctop = make_float2(0.f, 0.f);  // lane 31: the chunk's top plane
                    if (lane == 31) ctop = __ldg(cum + __float_as_int(r1.z));
                    // the plane above each voxel: the next lane's plane of the same slot
                    const int nxt = (lane + 1) & 31;
                    float pu[VPL];
                    float2 cu[VPL];
    #pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        pu[v] = __shfl_sync(FULL, pbv[v], nxt);
                        cu[v].x = __shfl_sync(FULL, cb[v].x, nxt);
                        cu[v].y = __shfl_sync(FULL, cb[v].y, nxt);
                    }
    #pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        float p1 = pu[v];
                        float2 c1 = cu[v];
                        if (lane == 31) {  // lane 0's next slot, or the chunk's top plane
                            p1 = v + 1 < VPL ? pu[v + 1 < VPL ? v + 1 : v] : r1.w;
                            c1 = v + 1 < VPL ? cu[v + 1 < VPL ? v + 1 : v] : ctop;
                        }
                        const float full = __fadd_rn(__fsub_rn(c1.x, cb[v].x), __fsub_rn(c1.y, cb[v].y));
                        acc[v] += __fmaf_rn(w, full, p1 - pbv[v]);
                    }
                }
            }
            __syncwarp();  // the next chunk's setup overwrites the records
        }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int k = base + VS * v;
        if (k >= G.nz) continue;
        const size_t o = ((size_t)i * G.ny + j) * G.nz + k;
        out[o] = (mode == BP_PLAIN) ? acc[v] : __fmaf_rn(-c, acc[v], __ldg(fin + o));
    }
}

}  // namespace cbct
