// Device-side block of the TV prox sweep (shared by the single-request and batched
// kernels).
#pragma once

// Step 2 (and 3) of Algorithm A1 (Jia et al. 2010): one projected-gradient step on
//   Phi(f) = TV_eps(f) + beta/2 |f - g|^2,   f >= 0,
// where TV_eps is E1 of Eq. 1 read as the forward-difference total variation with
// Neumann boundary.  Isotropic (A.aniso == 0): sum_j sqrt(|grad f|_j^2 + eps^2), whose
// gradient sum_d D_d^T (D_d f / |grad f|_eps) is a 13-point stencil per voxel.
// Anisotropic (A.aniso == 1): sum_j sum_d sqrt((D_d f)_j^2 + eps^2), gradient
// sum_d D_d^T (D_d f / sqrt((D_d f)^2 + eps^2)), a 7-point stencil.  In both,
//   (D_d^T p)_i = (p_{i-1} [i > 0] - p_i [i < n-1]) / h_d.
// A sweep also emits one of two partial sums (ACC): those of |grad f|_eps of its
// input (TV_ACC_E1: the E1 energy of the entering iterate when the input is f_k), or,
// on the last sweep of an Algorithm A1 iteration, which overwrites f_k in place with
// f_k+1, those of (f_k+1 - f_k)^2 (TV_ACC_STEP: the step norm).
//
// Layout [nx][ny][nz] (z fastest); one thread per voxel, consecutive lanes along z.
#include "cbct_internal.h"

namespace cbct {

constexpr int TV_THREADS = 256;
constexpr int TV_ACC_NONE = 0, TV_ACC_E1 = 1, TV_ACC_STEP = 2;

// grad TV_eps at voxel idx (internal layout) and, if E1, the voxel's term of TV_eps
// itself (|grad f|_eps, or the sum over the axes in the anisotropic reading).  Shared
// by the prox sweep and the energy gradient of the multigrid cycle.
template <bool E1, bool ANISO>
__device__ __forceinline__ float tv_div(const TvArgs &A, const float *__restrict__ fin, const size_t idx, float &e1) {
    const int k = (int)(idx % A.nz);
    const size_t t = idx / A.nz;
    const int j = (int)(t % A.ny);
    const int i = (int)(t / A.ny);
    const size_t sx = (size_t)A.ny * A.nz, sy = A.nz;
    const bool xp = i < A.nx - 1, yp = j < A.ny - 1, zp = k < A.nz - 1;
    const float f0 = __ldg(fin + idx);
    // every rounding spelled out (no compiler contraction), so the result does not
    // depend on the kernel this body is inlined into
    // own gradient (zero difference at the last index)
    const float gx = __fmul_rn(__fsub_rn(xp ? __ldg(fin + idx + sx) : f0, f0), A.ihx);
    const float gy = __fmul_rn(__fsub_rn(yp ? __ldg(fin + idx + sy) : f0, f0), A.ihy);
    const float gz = __fmul_rn(__fsub_rn(zp ? __ldg(fin + idx + 1) : f0, f0), A.ihz);
    float div;
    if (ANISO) {
        // each axis smoothed on its own: p_d = D_d f / sqrt((D_d f)^2 + eps^2)
        const float qx = __fmaf_rn(gx, gx, A.eps2), qy = __fmaf_rn(gy, gy, A.eps2), qz = __fmaf_rn(gz, gz, A.eps2);
        const float rx = rsqrtf(qx), ry = rsqrtf(qy), rz = rsqrtf(qz);
        div = -__fmaf_rn(__fmul_rn(gx, rx), A.ihx,
                         __fmaf_rn(__fmul_rn(gy, ry), A.ihy, __fmul_rn(__fmul_rn(gz, rz), A.ihz)));
        if (E1) e1 = __fadd_rn(__fadd_rn(__fmul_rn(qx, rx), __fmul_rn(qy, ry)), __fmul_rn(qz, rz));
        if (i > 0) {
            const float a = __fmul_rn(__fsub_rn(f0, __ldg(fin + idx - sx)), A.ihx);
            div = __fmaf_rn(__fmul_rn(a, rsqrtf(__fmaf_rn(a, a, A.eps2))), A.ihx, div);
        }
        if (j > 0) {
            const float a = __fmul_rn(__fsub_rn(f0, __ldg(fin + idx - sy)), A.ihy);
            div = __fmaf_rn(__fmul_rn(a, rsqrtf(__fmaf_rn(a, a, A.eps2))), A.ihy, div);
        }
        if (k > 0) {
            const float a = __fmul_rn(__fsub_rn(f0, __ldg(fin + idx - 1)), A.ihz);
            div = __fmaf_rn(__fmul_rn(a, rsqrtf(__fmaf_rn(a, a, A.eps2))), A.ihz, div);
        }
    } else {
        const float q0 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmaf_rn(gz, gz, A.eps2)));
        const float n0 = rsqrtf(q0);
        div = -__fmul_rn(__fmaf_rn(gx, A.ihx, __fmaf_rn(gy, A.ihy, __fmul_rn(gz, A.ihz))), n0);
        if (E1) e1 = __fmul_rn(q0, n0);
        // p_x at i-1
        if (i > 0) {
            const float fm = __ldg(fin + idx - sx);
            const float ax = __fmul_rn(__fsub_rn(f0, fm), A.ihx);
            const float ay = __fmul_rn(__fsub_rn(yp ? __ldg(fin + idx - sx + sy) : fm, fm), A.ihy);
            const float az = __fmul_rn(__fsub_rn(zp ? __ldg(fin + idx - sx + 1) : fm, fm), A.ihz);
            const float n = rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2))));
            div = __fmaf_rn(__fmul_rn(ax, n), A.ihx, div);
        }
        // p_y at j-1
        if (j > 0) {
            const float fm = __ldg(fin + idx - sy);
            const float ax = __fmul_rn(__fsub_rn(xp ? __ldg(fin + idx - sy + sx) : fm, fm), A.ihx);
            const float ay = __fmul_rn(__fsub_rn(f0, fm), A.ihy);
            const float az = __fmul_rn(__fsub_rn(zp ? __ldg(fin + idx - sy + 1) : fm, fm), A.ihz);
            const float n = rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2))));
            div = __fmaf_rn(__fmul_rn(ay, n), A.ihy, div);
        }
        // p_z at k-1
        if (k > 0) {
            const float fm = __ldg(fin + idx - 1);
            const float ax = __fmul_rn(__fsub_rn(xp ? __ldg(fin + idx - 1 + sx) : fm, fm), A.ihx);
            const float ay = __fmul_rn(__fsub_rn(yp ? __ldg(fin + idx - 1 + sy) : fm, fm), A.ihy);
            const float az = __fmul_rn(__fsub_rn(f0, fm), A.ihz);
            const float n = rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2))));
            div = __fmaf_rn(__fmul_rn(az, n), A.ihz, div);
        }
    }
    return div;
}

// Warp tile of the sweep: lanes are 32 consecutive z-voxels of the column (i, j) and
// the warp walks j over A.jc rows (tv_rows_per_tile).  Every voxel gets exactly the arithmetic above
// (same expressions, same order), but the terms shared between neighbours are not
// recomputed: the p_y term at (i, j-1) is the previous row's own term, the p_z term
// at (i, j, k-1) is the lower lane's own term (lane 0 of a tile that does not start
// at k = 0 computes it), and f(i, j, k), f(i-1, j, k) come from the previous row's
// loads.  Each tile writes one float64 partial of the E1 (or step) terms of its
// voxels (float32 along the rows, then over the lanes).
constexpr int TV_WARPS = TV_THREADS / 32;

// Warp tiles of a sweep (full columns or row walks), or, for the per-voxel form, 8 per
// block of TV_THREADS voxels; E1 partials: one per warp tile, or one per block.
__host__ __device__ __forceinline__ long tv_warp_tiles(int nx, int ny, int nz) {
    const int jc = tv_rows_per_tile(nx, ny, nz);
    if (jc == 0) return TV_WARPS * (((long)nx * ny * nz + TV_THREADS - 1) / TV_THREADS);
    if (tv_col_vz(nx, ny, nz)) return (long)nx * ((ny + jc - 1) / jc);
    return (long)nx * ((ny + jc - 1) / jc) * ((nz + 31) / 32);
}

// own term of voxel (i, j, k) from its value c and its +x, +y, +z neighbours (the
// neighbour equals c where the difference is zero): the py/pz pieces D_d f * w_d, the
// -(sum_d p_d / h_d) part of the divergence and the voxel's E1 term
struct TvOwn {
    float px, py, pz, div, e1;
};
template <bool E1, bool ANISO>
__device__ __forceinline__ TvOwn tv_own(const TvArgs &A, float c, float fxp, float fyp, float fzp) {
    TvOwn o;
    const float gx = __fmul_rn(__fsub_rn(fxp, c), A.ihx);
    const float gy = __fmul_rn(__fsub_rn(fyp, c), A.ihy);
    const float gz = __fmul_rn(__fsub_rn(fzp, c), A.ihz);
    o.e1 = 0.f;
    if (ANISO) {
        const float qx = __fmaf_rn(gx, gx, A.eps2), qy = __fmaf_rn(gy, gy, A.eps2), qz = __fmaf_rn(gz, gz, A.eps2);
        const float rx = rsqrtf(qx), ry = rsqrtf(qy), rz = rsqrtf(qz);
        o.px = __fmul_rn(gx, rx);
        o.py = __fmul_rn(gy, ry);
        o.pz = __fmul_rn(gz, rz);
        o.div = -__fmaf_rn(__fmul_rn(gx, rx), A.ihx, __fmaf_rn(o.py, A.ihy, __fmul_rn(o.pz, A.ihz)));
        if (E1) o.e1 = __fadd_rn(__fadd_rn(__fmul_rn(qx, rx), __fmul_rn(qy, ry)), __fmul_rn(qz, rz));
    } else {
        const float q0 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmaf_rn(gz, gz, A.eps2)));
        const float n0 = rsqrtf(q0);
        o.px = __fmul_rn(gx, n0);
        o.py = __fmul_rn(gy, n0);
        o.pz = __fmul_rn(gz, n0);
        o.div = -__fmul_rn(__fmaf_rn(gx, A.ihx, __fmaf_rn(gy, A.ihy, __fmul_rn(gz, A.ihz))), n0);
        if (E1) o.e1 = __fmul_rn(q0, n0);
    }
    return o;
}

// p_x piece of voxel (i-1, j, k) (value m) as the voxel (i, j, k) (value c) sees it
template <bool ANISO>
__device__ __forceinline__ float tv_px_minus(const TvArgs &A, float c, float m, float myp, float mzp) {
    const float ax = __fmul_rn(__fsub_rn(c, m), A.ihx);
    if (ANISO) return __fmul_rn(ax, rsqrtf(__fmaf_rn(ax, ax, A.eps2)));
    const float ay = __fmul_rn(__fsub_rn(myp, m), A.ihy);
    const float az = __fmul_rn(__fsub_rn(mzp, m), A.ihz);
    return __fmul_rn(ax, rsqrtf(__fmaf_rn(ax, ax, __fmaf_rn(ay, ay, __fmaf_rn(az, az, A.eps2)))));
}

template <bool CLAMP, int ACC, bool ANISO>
__device__ __forceinline__ void tv_warp(const TvArgs &A, const float *__restrict__ fin, const float *__restrict__ g,
                                        float *__restrict__ fout, double *__restrict__ partial, const long wtile) {
    constexpr bool E1 = ACC == TV_ACC_E1;
    const int lane = threadIdx.x & 31;
    const int nkb = (A.nz + 31) >> 5, njc = (A.ny + A.jc - 1) / A.jc;
    const int kb = (int)(wtile % nkb);
    const long tt = wtile / nkb;
    const int jc = (int)(tt % njc), i = (int)(tt / njc);
    const int k = kb * 32 + lane;
    const bool kin = k < A.nz;
    const int kq = kin ? k : A.nz - 1;               // idle lanes read a valid address
    const int j0 = jc * A.jc, j1 = min(j0 + A.jc, A.ny);
    const size_t sx = (size_t)A.ny * A.nz, sy = A.nz;
    const bool xp = i < A.nx - 1, xm = i > 0, zp = kq < A.nz - 1, zm = kq > 0;
    const bool halo = lane == 0 && zm;               // p_z at k-1 is not in this tile
    size_t o = ((size_t)i * A.ny + j0) * A.nz + kq;  // (i, j, k)
    float e1 = 0.f;
    float c = __ldg(fin + o);                        // f(i, j, k)
    float m = xm ? __ldg(fin + o - sx) : 0.f;        // f(i-1, j, k)
    float py_prev = 0.f;                             // p_y piece of (i, j-1, k)
    if (j0 > 0) {
        const float b = __ldg(fin + o - sy);
        const float bxp = xp ? __ldg(fin + o - sy + sx) : b;
        const float bzp = zp ? __ldg(fin + o - sy + 1) : b;
        py_prev = tv_own<false, ANISO>(A, b, bxp, c, bzp).py;
    }
    // the loads of row j (fy: +y, fx: +x, fz: +z, my/mz: the +y/+z neighbours of
    // f(i-1, j, k), gv: g, d*: the halo voxel (i, j, k-1) and its +x/+y neighbours),
    // issued one row ahead so that they are in flight during the previous row's
    // arithmetic
    // (fo: with the step accumulator, f_k where the result goes, read with the row's
    // other loads rather than at its store, which would expose its latency)
    float fy, fx, fz, my, mz, gv, d, dx, dy, fo;
    auto load_row = [&](int jr, size_t orow, float cr, float mr, float &ly, float &lx, float &lz, float &lmy,
                        float &lmz, float &lg, float &ld, float &ldx, float &ldy, float &lfo) {
        const bool ypr = jr < A.ny - 1;
        lfo = ACC == TV_ACC_STEP ? fout[orow] : 0.f;
        ly = ypr ? __ldg(fin + orow + sy) : cr;
        lx = xp ? __ldg(fin + orow + sx) : cr;
        lz = zp ? __ldg(fin + orow + 1) : cr;
        lmy = (xm && ypr) ? __ldg(fin + orow - sx + sy) : mr;
        lmz = (xm && zp) ? __ldg(fin + orow - sx + 1) : mr;
        lg = __ldg(g + orow);
        if (halo) {
            ld = __ldg(fin + orow - 1);
            ldx = xp ? __ldg(fin + orow - 1 + sx) : ld;
            ldy = ypr ? __ldg(fin + orow - 1 + sy) : ld;
        } else {
            ld = ldx = ldy = 0.f;
        }
    };
    load_row(j0, o, c, m, fy, fx, fz, my, mz, gv, d, dx, dy, fo);
#pragma unroll 1
    for (int j = j0; j < j1; ++j) {
        // next row: its own value is fy, its (i-1) value my
        float nfy = 0.f, nfx = 0.f, nfz = 0.f, nmy = 0.f, nmz = 0.f, ngv = 0.f, nd = 0.f, ndx = 0.f, ndy = 0.f,
              nfo = 0.f;
        if (j + 1 < j1) load_row(j + 1, o + sy, fy, my, nfy, nfx, nfz, nmy, nmz, ngv, nd, ndx, ndy, nfo);
        const TvOwn own = tv_own<E1, ANISO>(A, c, fx, fy, fz);
        float div = own.div;
        if (xm) div = __fmaf_rn(tv_px_minus<ANISO>(A, c, m, my, mz), A.ihx, div);
        if (j > 0) div = __fmaf_rn(py_prev, A.ihy, div);
        float pz_lo = __shfl_up_sync(0xffffffffu, own.pz, 1);
        if (halo) pz_lo = tv_own<false, ANISO>(A, d, dx, dy, c).pz;  // own term of (i, j, k-1)
        if (zm) div = __fmaf_rn(pz_lo, A.ihz, div);
        if (kin) {
            const float x = __fmaf_rn(-A.s, __fmaf_rn(A.beta, __fsub_rn(c, gv), div), c);
            const float y = CLAMP ? fmaxf(x, 0.f) : x;
            if (ACC == TV_ACC_STEP) {  // fo: f_k, read before it is overwritten
                const float dd = __fsub_rn(y, fo);
                e1 = __fmaf_rn(dd, dd, e1);
            }
            fout[o] = y;
            if (E1) e1 = __fadd_rn(e1, own.e1);
        }
        py_prev = own.py;
        c = fy;
        m = my;
        fy = nfy; fx = nfx; fz = nfz; my = nmy; mz = nmz; gv = ngv; d = nd; dx = ndx; dy = ndy; fo = nfo;
        o += sy;
    }
    if (ACC != TV_ACC_NONE) {
        // float32 along the rows, a pairwise tree over the lanes, one float64 per tile
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e1 += __shfl_down_sync(0xffffffffu, e1, off);
        if (lane == 0) partial[wtile] = (double)e1;
    }
}

// Full-column warp tile: the warp owns the whole z-column of (i, j) for A.jc rows in y
// from j0, lane l holding the voxels k = l + 32 v (v < VZ, interleaved so that every load
// is coalesced).  The same arithmetic as the row walk (same expressions, same order);
// the +z neighbours f(i, j, k+1), f(i-1, j, k+1) and the p_z term of (i, j, k-1) come from
// the neighbouring lane (lane 31 / lane 0 of the next / previous slot), so nothing in z
// is loaded twice and no lane computes a halo.  One float64 partial per tile.
template <bool CLAMP, int ACC, bool ANISO, int VZ>
__device__ __forceinline__ void tv_col(const TvArgs &A, const float *__restrict__ fin, const float *__restrict__ g,
                                       float *__restrict__ fout, double *__restrict__ partial, const long wtile) {
    constexpr bool E1 = ACC == TV_ACC_E1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int njc = (A.ny + A.jc - 1) / A.jc;
    const int jc = (int)(wtile % njc), i = (int)(wtile / njc);
    const int j0 = jc * A.jc, j1 = min(j0 + A.jc, A.ny);
    const size_t sx = (size_t)A.ny * A.nz, sy = A.nz;
    const bool xp = i < A.nx - 1, xm = i > 0;
    int kq[VZ];
    bool kin[VZ];
#pragma unroll
    for (int v = 0; v < VZ; ++v) {
        const int k = lane + 32 * v;
        kin[v] = k < A.nz;
        kq[v] = kin[v] ? k : A.nz - 1;  // idle lanes read a valid address
    }
    // value at k + 1 of a per-slot quantity q (q itself at the top of the column)
    auto zup = [&](const float (&q)[VZ], int v) {
        const float dn = __shfl_down_sync(FULL, q[v], 1);
        const float nx0 = __shfl_sync(FULL, q[v + 1 < VZ ? v + 1 : v], 0);
        const float r = lane == 31 ? nx0 : dn;
        return lane + 32 * v < A.nz - 1 ? r : q[v];
    };
    size_t o = ((size_t)i * A.ny + j0) * A.nz;   // (i, j, 0)
    float e1 = 0.f;
    float c[VZ], m[VZ], py_prev[VZ];
#pragma unroll
    for (int v = 0; v < VZ; ++v) {
        c[v] = __ldg(fin + o + kq[v]);
        m[v] = xm ? __ldg(fin + o - sx + kq[v]) : 0.f;
        py_prev[v] = 0.f;
    }
    if (j0 > 0) {  // p_y piece of (i, j0 - 1, k)
        float b[VZ], bxp[VZ];
#pragma unroll
        for (int v = 0; v < VZ; ++v) {
            b[v] = __ldg(fin + o - sy + kq[v]);
            bxp[v] = xp ? __ldg(fin + o - sy + sx + kq[v]) : b[v];
        }
#pragma unroll
        for (int v = 0; v < VZ; ++v) py_prev[v] = tv_own<false, ANISO>(A, b[v], bxp[v], c[v], zup(b, v)).py;
    }
#pragma unroll 1
    for (int j = j0; j < j1; ++j) {
        const bool yp = j < A.ny - 1;
        float fy[VZ], fx[VZ], my[VZ], gv[VZ], fo[VZ];
#pragma unroll
        for (int v = 0; v < VZ; ++v) {
            fy[v] = yp ? __ldg(fin + o + sy + kq[v]) : c[v];
            fx[v] = xp ? __ldg(fin + o + sx + kq[v]) : c[v];
            my[v] = (xm && yp) ? __ldg(fin + o - sx + sy + kq[v]) : m[v];
            gv[v] = __ldg(g + o + kq[v]);
            // f_k where the result goes, read with this row's other loads (before any of
            // the row's stores), not at the store: its latency then overlaps theirs
            fo[v] = ACC == TV_ACC_STEP ? fout[o + kq[v]] : 0.f;
        }
        float pz[VZ], div[VZ];
#pragma unroll
        for (int v = 0; v < VZ; ++v) {
            const TvOwn own = tv_own<E1, ANISO>(A, c[v], fx[v], fy[v], zup(c, v));
            pz[v] = own.pz;
            float d = own.div;
            if (xm) d = __fmaf_rn(tv_px_minus<ANISO>(A, c[v], m[v], my[v], zup(m, v)), A.ihx, d);
            if (j > 0) d = __fmaf_rn(py_prev[v], A.ihy, d);
            div[v] = d;
            py_prev[v] = own.py;
            if (E1 && kin[v]) e1 = __fadd_rn(e1, own.e1);
        }
#pragma unroll
        for (int v = 0; v < VZ; ++v) {
            // p_z piece of (i, j, k - 1): the lower lane's, lane 31 of the previous slot for lane 0
            const float up1 = __shfl_up_sync(FULL, pz[v], 1);
            const float prev = __shfl_sync(FULL, pz[v > 0 ? v - 1 : 0], 31);
            const float pz_lo = lane == 0 ? prev : up1;
            float d = div[v];
            if (lane + 32 * v > 0) d = __fmaf_rn(pz_lo, A.ihz, d);
            if (kin[v]) {
                const size_t ov = o + kq[v];
                const float x = __fmaf_rn(-A.s, __fmaf_rn(A.beta, __fsub_rn(c[v], gv[v]), d), c[v]);
                const float y = CLAMP ? fmaxf(x, 0.f) : x;
                if (ACC == TV_ACC_STEP) {  // fo: f_k, read before it is overwritten
                    const float dd = __fsub_rn(y, fo[v]);
                    e1 = __fmaf_rn(dd, dd, e1);
                }
                fout[ov] = y;
            }
            c[v] = fy[v];
            m[v] = my[v];
        }
        o += sy;
    }
    if (ACC != TV_ACC_NONE) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e1 += __shfl_down_sync(FULL, e1, off);
        if (lane == 0) partial[wtile] = (double)e1;
    }
}

// One thread per voxel (small or oddly sized volumes): the same arithmetic, one E1
// partial per block (float32 within a warp, float64 across the warps).
template <bool CLAMP, int ACC, bool ANISO>
__device__ __forceinline__ void tv_voxels(const TvArgs &A, const float *__restrict__ fin, const float *__restrict__ g,
                                          float *__restrict__ fout, double *__restrict__ partial, const long blk) {
    constexpr bool E1 = ACC == TV_ACC_E1;
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    const size_t idx = (size_t)blk * TV_THREADS + threadIdx.x;
    float e1 = 0.f;
    if (idx < n) {
        const float f0 = __ldg(fin + idx);
        const float div = tv_div<E1, ANISO>(A, fin, idx, e1);
        const float x = __fmaf_rn(-A.s, __fmaf_rn(A.beta, __fsub_rn(f0, __ldg(g + idx)), div), f0);
        const float y = CLAMP ? fmaxf(x, 0.f) : x;
        if (ACC == TV_ACC_STEP) {
            const float d = __fsub_rn(y, fout[idx]);
            e1 = __fmul_rn(d, d);
        }
        fout[idx] = y;
    }
    if (ACC != TV_ACC_NONE) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e1 += __shfl_down_sync(0xffffffffu, e1, off);
        __shared__ double red[TV_WARPS];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)e1;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < TV_WARPS; ++w) s += red[w];
            partial[blk] = s;
        }
    }
}

// One block of the sweep (block index blk): TV_WARPS warp tiles (FORM 1: row walks;
// FORM 2 + v: full columns with v + 1 voxels per lane, v < 3), or TV_THREADS voxels in
// the per-voxel form (FORM 0).  With TV_ACC_STEP, fout holds f_k on entry.
template <bool CLAMP, int ACC, bool ANISO, int FORM>
__device__ __forceinline__ void tv_block_t(const TvArgs &A, const float *__restrict__ fin, const float *__restrict__ g,
                                           float *__restrict__ fout, double *__restrict__ partial, const long blk) {
    if (FORM == 0) {
        tv_voxels<CLAMP, ACC, ANISO>(A, fin, g, fout, partial, blk);
        return;
    }
    const long wt = blk * TV_WARPS + (threadIdx.x >> 5);
    if (wt >= tv_warp_tiles(A.nx, A.ny, A.nz)) return;
    if (FORM == 1) tv_warp<CLAMP, ACC, ANISO>(A, fin, g, fout, partial, wt);
    else tv_col<CLAMP, ACC, ANISO, (FORM >= 2 ? FORM - 1 : 1)>(A, fin, g, fout, partial, wt);
}

// The form of a level's sweep (FORM of tv_block_t).
__host__ __device__ __forceinline__ int tv_form(const TvArgs &A) { return A.jc == 0 ? 0 : A.vz ? 1 + A.vz : 1; }

// The same with the reading and the form chosen at run time, for the batched kernels.
// Only the per-voxel form and the row walk: a level big enough for full-column tiles
// fills the GPU by itself, and the batch engine launches its sweeps as single-request
// launches (so the batched kernel keeps the registers of the two small forms).
template <bool CLAMP, int ACC>
__device__ __forceinline__ void tv_block(const TvArgs &A, const float *__restrict__ fin, const float *__restrict__ g,
                                         float *__restrict__ fout, double *__restrict__ partial, const long blk) {
    if (A.aniso) {
        if (A.jc) tv_block_t<CLAMP, ACC, true, 1>(A, fin, g, fout, partial, blk);
        else tv_block_t<CLAMP, ACC, true, 0>(A, fin, g, fout, partial, blk);
    } else {
        if (A.jc) tv_block_t<CLAMP, ACC, false, 1>(A, fin, g, fout, partial, blk);
        else tv_block_t<CLAMP, ACC, false, 0>(A, fin, g, fout, partial, blk);
    }
}

}  // namespace cbct
