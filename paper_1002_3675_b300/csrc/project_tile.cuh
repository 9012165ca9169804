// Device-side tile body of the forward projection (shared by the single-request
// and batched kernels).
#pragma once

// Forward projection P^theta (problem statement before Eq. 1 of Jia et al. 2010):
// exact intersection-length line integrals of the voxelised f along every
// source-to-pixel ray, with the step-1 residual r = P f - Y and the float64 partial
// sums of |r|^2 (E2 of Eq. 1) fused into the epilogue.
//
// Work decomposition.  All rays of one detector column (view ia, column a) lie in
// one vertical plane and cross the same sequence of xy-cells.  One thread block owns
// one column (and up to 512 of its rows):
//   1. it builds that cell sequence once, in shared memory, as a list of segments
//      (exit parameter t, offset of the cell's z-column).  The x- and y-plane
//      crossings are two monotone sequences; each crossing's place in the merged
//      order is its own index plus a binary search in the other sequence (ties put
//      the x crossing first), so the list is built in parallel;
//   2. for every z-level k it forms the running slice integral
//      C_k[s] = sum_{s' <= s} (t_s' - t_s'-1) f[cell_s'][k]  (warps over levels, so
//      each load is a contiguous piece of a z-column);
//   3. a ray (one per thread) stays in level k over one t-interval [ta, tb]
//      between two z-plane crossings, and C_k is piecewise linear in t, so its line
//      integral is sum_k C_k(tb) - C_k(ta), each value found by a binary search in
//      the segment list and a linear interpolation.
// The work per column is (segments x levels) plus (rays x levels crossed), instead of
// segments x rays.  Levels are processed in bands when the table would not fit.
// The plane-crossing values are the same float32 expressions the adjoint uses.
#include "cbct_internal.h"

namespace cbct {

namespace proj_detail {

struct ColumnRay {  // the xy-part of one detector column's ray plane
    float Ox, Oy, ix, iy, ex, ey;
    float tin, tout;
    bool hit;
    int i0, j0, si, sj;
};

__device__ __forceinline__ float x_crossing(const GeoDev &G, const ColumnRay &c, int m) {
    // m-th x-plane crossed after the entry cell (m >= 1)
    return t_cross(plane_at(c.i0 + (c.si > 0 ? m : 1 - m), G.hx, G.x0), c.Ox, c.ix);
}
__device__ __forceinline__ float y_crossing(const GeoDev &G, const ColumnRay &c, int m) {
    return t_cross(plane_at(c.j0 + (c.sj > 0 ? m : 1 - m), G.hy, G.y0), c.Oy, c.iy);
}

// number of m in [1, mmax] with crossing(m) < v (strict) or <= v (inclusive).  The
// crossings are evenly spaced in exact arithmetic and monotone in float32, so the
// count is a linear estimate corrected by a walk over the float32 values themselves
// (the same count as a search of the sequence).
template <bool X, bool INCL>
__device__ __forceinline__ int count_before(const GeoDev &G, const ColumnRay &c, int mmax, float v) {
    if (mmax <= 0) return 0;
    const float t1 = X ? x_crossing(G, c, 1) : y_crossing(G, c, 1);
    const float rate = X ? fabsf(c.ex) * G.inv_hx : fabsf(c.ey) * G.inv_hy;  // crossings per unit t
    const float est = (v - t1) * rate;
    int m = est >= 0.f ? min((int)fminf(est, (float)mmax) + 1, mmax) : 0;
    auto before = [&](int q) {
        const float t = X ? x_crossing(G, c, q) : y_crossing(G, c, q);
        return INCL ? (t <= v) : (t < v);
    };
    while (m < mmax && before(m + 1)) ++m;
    while (m > 0 && !before(m)) --m;
    return m;
}

__device__ __forceinline__ ColumnRay column_setup(const GeoDev &G, int ia, int a) {
    ColumnRay c;
    const float4 rxy = G.ray_xy[(size_t)ia * G.nu + a];
    const float2 re = G.ray_e[(size_t)ia * G.nu + a];
    c.Ox = rxy.x; c.Oy = rxy.y; c.ix = rxy.z; c.iy = rxy.w; c.ex = re.x; c.ey = re.y;
    const float xN = plane_at(G.nx, G.hx, G.x0), yN = plane_at(G.ny, G.hy, G.y0);
    float tin = -INFINITY, tout = INFINITY;
    bool hit = true;
    if (c.ix != 0.f) {
        const float t0 = t_cross(G.x0, c.Ox, c.ix), t1 = t_cross(xN, c.Ox, c.ix);
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
    } else {
        hit = hit && c.Ox >= G.x0 && c.Ox < xN;
    }
    if (c.iy != 0.f) {
        const float t0 = t_cross(G.y0, c.Oy, c.iy), t1 = t_cross(yN, c.Oy, c.iy);
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
    } else {
        hit = hit && c.Oy >= G.y0 && c.Oy < yN;
    }
    c.hit = hit && tout > tin;
    c.tin = tin;
    c.tout = tout;
    // entry cell, fixed against the crossing values themselves
    if (c.ix != 0.f) {
        c.si = c.ix > 0.f ? 1 : -1;
        const float xin = __fmaf_rn(tin, c.ex, c.Ox);
        int i = min(max((int)floorf((xin - G.x0) * G.inv_hx), 0), G.nx - 1);
        for (int q = 0; q < 2; ++q) {
            const float ten = t_cross(plane_at(i + (c.si < 0), G.hx, G.x0), c.Ox, c.ix);
            const float tex = t_cross(plane_at(i + (c.si > 0), G.hx, G.x0), c.Ox, c.ix);
            if (ten > tin && i - c.si >= 0 && i - c.si < G.nx) i -= c.si;
            else if (tex <= tin && i + c.si >= 0 && i + c.si < G.nx) i += c.si;
            else break;
        }
        c.i0 = i;
    } else {
        c.si = 0;
        c.i0 = min(max((int)floorf((c.Ox - G.x0) * G.inv_hx), 0), G.nx - 1);
    }
    if (c.iy != 0.f) {
        c.sj = c.iy > 0.f ? 1 : -1;
        const float yin = __fmaf_rn(tin, c.ey, c.Oy);
        int j = min(max((int)floorf((yin - G.y0) * G.inv_hy), 0), G.ny - 1);
        for (int q = 0; q < 2; ++q) {
            const float ten = t_cross(plane_at(j + (c.sj < 0), G.hy, G.y0), c.Oy, c.iy);
            const float tex = t_cross(plane_at(j + (c.sj > 0), G.hy, G.y0), c.Oy, c.iy);
            if (ten > tin && j - c.sj >= 0 && j - c.sj < G.ny) j -= c.sj;
            else if (tex <= tin && j + c.sj >= 0 && j + c.sj < G.ny) j += c.sj;
            else break;
        }
        c.j0 = j;
    } else {
        c.sj = 0;
        c.j0 = min(max((int)floorf((c.Oy - G.y0) * G.inv_hy), 0), G.ny - 1);
    }
    return c;
}

}  // namespace proj_detail
using namespace proj_detail;

// Shared memory per block: the segment list (t, offset) for nx + ny + 1 slots, the
// chunk offsets, and in the rest the running slice integrals C of a band of z-levels.
// The size is a launch shape: it sets how many levels a band holds, and no result bit
// depends on it (every ray adds its levels in ascending order whatever the bands).
constexpr int PROJ_SMEM = 110 * 1024;   // largest size used
constexpr int PROJ_SMEM_MIN = 16 * 1024;
constexpr int PROJ_MAX_THREADS = 512;
// prefix chunks of 16 segments: the running sums of a chunk are a chain of dependent
// additions whose loads go out 4 (float4) or 8 at a time, and the chunk offsets are a
// chain over the chunks, so short chunks keep both chains short while every warp of the
// block gets chunks (timed on B300 for 512x512x96: 8, 12, 16, 24 segments 2.51, 2.32,
// 2.28, 2.33 ms per projection; 48 segments with one level per lane took 2.57 ms)
constexpr int CHUNK = 16;
constexpr int PROJ_BATCH = 8;           // voxel loads in flight per thread
constexpr int PROJ_VBATCH = 4;          // 16-byte voxel loads in flight per thread (4 levels each)

// Projector block size (rows per tile): G.proj_threads if valid, else the default: one
// thread per row up to 128 rows, 256 threads up to 256 rows, 512 above (timed on B300
// for 96 to 384 rows; more threads shorten the segment and running-sum phases that
// every row waits for).
__host__ __device__ __forceinline__ int proj_threads_of(const GeoDev &g) {
    const int need = min(PROJ_MAX_THREADS, 32 * ((g.nv + 31) / 32));
    if (g.proj_threads >= need && g.proj_threads <= PROJ_MAX_THREADS && g.proj_threads % 32 == 0) return g.proj_threads;
    return need <= 128 ? need : need <= 256 ? 256 : PROJ_MAX_THREADS;
}

// Bytes of shared memory the projector tile may use: G.proj_smem if valid, else as much
// as lets as many blocks share an SM as the registers allow (64 per thread, 64 K per
// SM; 228 KB of shared memory per SM, 1 KB of it reserved per block), at most
// PROJ_SMEM.  Larger tables hold whole 32-level bands for longer cell sequences (4 x 56
// KB at 256 threads: 2.3 % faster than 4 x 55 KB on 256x256x64).
// Floats before the chunk offsets: the segment list (exit t and z-column offset per
// slot), rounded up to 16 bytes so that the running sums can be stored as float4.
__host__ __device__ __forceinline__ int proj_list_floats(int slots) { return (2 * slots + 3) & ~3; }

__host__ __device__ __forceinline__ int proj_smem_of(const GeoDev &g) {
    const int slots = g.nx + g.ny + 1;
    const int least = (4 * (proj_list_floats(slots) + slots + (slots + CHUNK - 1) / CHUNK) + 15) & ~15;  // one level per band
    if (g.proj_smem >= least && g.proj_smem <= PROJ_SMEM && g.proj_smem % 16 == 0) return g.proj_smem;
    const int blocks = max(1, 65536 / (64 * proj_threads_of(g)));
    const int fit = ((228 * 1024) / blocks - 1024) & ~1023;
    return max(least, min(PROJ_SMEM, fit));
}

// first s in [0, S) with seg_t[s] >= t (tin <= t <= seg_t[S-1]), from a linear
// estimate corrected by a local walk (segment ends are nearly evenly spaced)
__device__ __forceinline__ int seg_find(const float *seg_t, int S, float tin, float scale, float t) {
    int s = min(max((int)((t - tin) * scale), 0), S - 1);
    while (s < S - 1 && seg_t[s] < t) ++s;
    while (s > 0 && seg_t[s - 1] >= t) --s;
    return s;
}

// Position of t in the segment list: its segment s (seg_t[s-1] < t <= seg_t[s]) and the
// fraction of that segment before t.  The same for every level, so a z-plane crossing
// shared by two consecutive levels is located once.
struct SegPos {
    int s;
    float frac;
};
__device__ __forceinline__ SegPos seg_pos(const float *seg_t, int S, float tin, float scale, float t) {
    SegPos p;
    p.s = seg_find(seg_t, S, tin, scale, t);
    const float tp = p.s > 0 ? seg_t[p.s - 1] : tin;
    const float dt = seg_t[p.s] - tp;
    p.frac = dt > 0.f ? __fdividef(t - tp, dt) : 0.f;
    return p;
}

// Level-kk running integral at position p.  C holds chunk-local running sums;
// coff[chunk][kk] adds the totals of the preceding chunks.  C is piecewise linear in t
// between segment ends.
__device__ __forceinline__ float eval_c(const float *C, const float *coff, int nk, int kk, const SegPos p) {
    const int ch = p.s / CHUNK;
    const float base = coff[ch * nk + kk];
    const bool first = p.s == ch * CHUNK;   // previous value is the chunk's base
    const float cp = first ? base : base + C[(p.s - 1) * nk + kk];
    const float cs = base + C[p.s * nk + kk];
    return __fmaf_rn(p.frac, cs - cp, cp);
}

// One tile: detector column a of view ia, rows [zc T, zc T + T) with T = blockDim.x.
// mode selects the epilogue (uniform per tile).  smem: PROJ_SMEM bytes of dynamic
// shared memory.  Called by the single-request and the batched kernels alike, so a
// request's result does not depend on what else is in the launch.
//
// Only the z-levels [kr0, kr1) are added.  A projection split over several launches of
// consecutive level ranges (so that each launch's slab of the volume stays in L2)
// carries every ray's running sum in out: carry_in starts from out instead of 0,
// carry_out stores the sum there and skips the epilogue.  The levels are added in the
// same ascending order either way, so the split does not change a bit of the result.
// One ray's z-geometry: height at O, cot(phi), and the levels between its xy entry and
// exit (with a level of margin on each side; an empty range when klo > khi).
struct RayZ {
    float zO, cotp;
    int klo, khi;
};
__device__ __forceinline__ RayZ ray_levels(const GeoDev &G, const ColumnRay &c, const float4 rz) {
    RayZ r{rz.x, rz.y, 0, -1};
    const float tanp = rz.w;
    if (r.cotp != 0.f) {
        const float za = __fmaf_rn(c.tin, tanp, r.zO), zb = __fmaf_rn(c.tout, tanp, r.zO);
        r.klo = max((int)floorf((fminf(za, zb) - G.z0) * G.inv_hz) - 1, 0);
        r.khi = min((int)floorf((fmaxf(za, zb) - G.z0) * G.inv_hz) + 1, G.nz - 1);
    } else {
        const int k0 = (int)floorf((r.zO - G.z0) * G.inv_hz);
        if (k0 >= 0 && k0 < G.nz) r.klo = r.khi = k0;
    }
    return r;
}

// VEC: the running sums take 4 levels per lane (float4) where the z-columns come in
// 16-byte pieces; the sums are the same additions in the same order either way.
template <bool VEC = false>
__device__ __forceinline__ void project_tile(const GeoDev &G, const int mode, const float *__restrict__ vol,
                                             const float *__restrict__ y32, const __half *__restrict__ y16,
                                             float *__restrict__ out, double *__restrict__ partial, const int a,
                                             const int ia, const int zc, float *smem, const int kr0 = 0,
                                             int kr1 = -1, const bool carry_in = false,
                                             const bool carry_out = false) {
    if (kr1 < 0) kr1 = G.nz;
    const int slots = G.nx + G.ny + 1;
    const int max_chunks = (slots + CHUNK - 1) / CHUNK;
    float *seg_t = smem;                          // exit t of each segment
    int *seg_off = (int *)(smem + slots);         // z-column offset of each segment's cell
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = T >> 5;
    const ColumnRay c = column_setup(G, ia, a);

    // ---- 1. the column's cell sequence -----------------------------------------------
    int Mx = 0, My = 0;
    if (c.hit) {
        if (c.si != 0) Mx = count_before<true, false>(G, c, c.si > 0 ? G.nx - 1 - c.i0 : c.i0, c.tout);
        if (c.sj != 0) My = count_before<false, false>(G, c, c.sj > 0 ? G.ny - 1 - c.j0 : c.j0, c.tout);
    }
    const int S = c.hit ? Mx + My + 1 : 0;
    for (int m = 1 + tid; m <= Mx; m += T) {
        const float t = x_crossing(G, c, m);
        const int nb = count_before<false, false>(G, c, My, t);   // y crossings strictly before
        seg_t[m - 1 + nb] = t;
        seg_off[m - 1 + nb] = ((c.i0 + c.si * (m - 1)) * G.ny + c.j0 + c.sj * nb) * G.nz;
    }
    for (int n = 1 + tid; n <= My; n += T) {
        const float t = y_crossing(G, c, n);
        const int mb = count_before<true, true>(G, c, Mx, t);     // x crossings at or before
        seg_t[n - 1 + mb] = t;
        seg_off[n - 1 + mb] = ((c.i0 + c.si * mb) * G.ny + c.j0 + c.sj * (n - 1)) * G.nz;
    }
    if (tid == 0 && S > 0) {
        seg_t[S - 1] = c.tout;
        seg_off[S - 1] = ((c.i0 + c.si * Mx) * G.ny + c.j0 + c.sj * My) * G.nz;
    }

    // ---- ray set-up: z-levels between the xy entry and exit ----------------------------
    const int b = zc * T + tid;
    const bool valid = b < G.nv;
    const float4 rz = G.ray_z[(size_t)a * G.nv + (valid ? b : G.nv - 1)];
    const float zO = rz.x, cotp = rz.y, secp = rz.z;
    int klo = 0, khi = -1;
    if (valid && S > 0) {
        const RayZ r0 = ray_levels(G, c, rz);
        klo = r0.klo;
        khi = r0.khi;
    }
    const float scale = S > 0 && c.tout > c.tin ? (float)S / (c.tout - c.tin) : 0.f;
    const size_t o = ((size_t)ia * G.nu + a) * G.nv + (valid ? b : 0);
    float acc = (carry_in && valid) ? out[o] : 0.f;
    __syncthreads();

    // ---- 2./3. bands of z-levels: running slice integrals, then the rays ---------------
    float *coff = smem + proj_list_floats(slots);           // [chunk][level - band start]
    const int c_cap = proj_smem_of(G) / 4 - proj_list_floats(slots);
    const int nr = kr1 - kr0;
    // (VEC: the launcher checked that the z-columns come in 16-byte pieces, that the
    // level range starts at a multiple of 4 and that 4 levels fit; bands then start at
    // multiples of 4)
    int kband = S > 0 ? max(1, min(nr, c_cap / (S + max_chunks))) : nr;
    if (kband >= 32 && kband < nr) kband &= ~31;  // whole 32-level groups: full warps, aligned loads
    else if (VEC && kband < nr) kband = max(4, kband & ~3);
    for (int kb = kr0; kb < kr1 && S > 0; kb += kband) {
        const int nk = min(kband, kr1 - kb);
        float *C = coff + max_chunks * nk;        // [s][kk], chunk-local running sums
        // 2. warps over (32-level group, 16-segment chunk) pairs; lanes over levels, so
        //    each load is a contiguous piece of a z-column
        const int nkg = (nk + 31) >> 5;
        const int nch = (S + CHUNK - 1) / CHUNK;
        if (VEC) {
            // 4 levels per lane (16-byte loads and stores), min(nk, 32)/4 lanes per
            // segment, so one warp instruction serves several chunks; per level the same
            // additions in the same order as the scalar form below
            const int L4 = min(nk, 32) >> 2, Gc = 32 / L4;
            const int gi = lane / L4, q4 = lane - gi * L4;
            const int ncg = (nch + Gc - 1) / Gc;
            for (int w = warp; w < nkg * ncg; w += nwarp) {
                const int kk = (w % nkg) * 32 + 4 * q4, ch = (w / nkg) * Gc + gi;
                const bool on = gi < Gc && ch < nch && kk < nk;
                const int s0 = ch * CHUNK, s1 = on ? min(S, s0 + CHUNK) : s0;
                float4 run = make_float4(0.f, 0.f, 0.f, 0.f);
                float tp = (s1 > s0 && s0 > 0) ? seg_t[s0 - 1] : c.tin;
                for (int q = s0; q < s1; q += PROJ_VBATCH) {
                    float4 v[PROJ_VBATCH];
                    float tq[PROJ_VBATCH];
#pragma unroll
                    for (int u = 0; u < PROJ_VBATCH; ++u) {
                        if (q + u < s1) {
                            tq[u] = seg_t[q + u];
                            v[u] = __ldg(reinterpret_cast<const float4 *>(vol + seg_off[q + u] + kb + kk));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < PROJ_VBATCH; ++u) {
                        if (q + u < s1) {
                            const float dt = tq[u] - tp;
                            run.x = __fmaf_rn(dt, v[u].x, run.x);
                            run.y = __fmaf_rn(dt, v[u].y, run.y);
                            run.z = __fmaf_rn(dt, v[u].z, run.z);
                            run.w = __fmaf_rn(dt, v[u].w, run.w);
                            tp = tq[u];
                            *reinterpret_cast<float4 *>(C + (q + u) * nk + kk) = run;
                        }
                    }
                }
            }
        } else {
            for (int w = warp; w < nkg * nch; w += nwarp) {
                const int kk = (w % nkg) * 32 + lane, ch = w / nkg;
                if (kk >= nk) continue;
                const int s0 = ch * CHUNK, s1 = min(S, s0 + CHUNK);
                float run = 0.f, tp = s0 > 0 ? seg_t[s0 - 1] : c.tin;
                for (int q = s0; q < s1; q += PROJ_BATCH) {
                    float v[PROJ_BATCH], tq[PROJ_BATCH];
#pragma unroll
                    for (int u = 0; u < PROJ_BATCH; ++u) {
                        if (q + u < s1) {
                            tq[u] = seg_t[q + u];
                            v[u] = __ldg(vol + seg_off[q + u] + kb + kk);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < PROJ_BATCH; ++u) {
                        if (q + u < s1) {
                            run = __fmaf_rn(tq[u] - tp, v[u], run);
                            tp = tq[u];
                            C[(q + u) * nk + kk] = run;
                        }
                    }
                }
            }
        }
        __syncthreads();
        // chunk offsets: coff[ch][kk] = sum of the totals of chunks before ch, added in
        // chunk order (the totals loaded four at a time, so that the chain of additions
        // does not wait on each load)
        for (int kk = tid; kk < nk; kk += T) {
            float o = 0.f;
            int ch = 0;
            for (; ch + 4 <= nch; ch += 4) {
                float tt[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) tt[u] = C[(min(S, (ch + u + 1) * CHUNK) - 1) * nk + kk];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    coff[(ch + u) * nk + kk] = o;
                    o += tt[u];
                }
            }
            for (; ch < nch; ++ch) {
                coff[ch * nk + kk] = o;
                o += C[(min(S, (ch + 1) * CHUNK) - 1) * nk + kk];
            }
        }
        __syncthreads();
        // 3. each ray adds C_k(t_exit) - C_k(t_entry) over its levels in this band, in
        //    ascending k (so the sum does not depend on the band size); the plane shared
        //    with the next level is located once
        const int k0 = max(klo, kb), k1 = min(khi, kb + nk - 1);
        if (k0 <= k1) {
            const bool up = cotp >= 0.f;  // rising ray: level k + 1 starts where k ends
            float last_t = -INFINITY;
            SegPos last_p{0, 0.f};
            for (int k = k0; k <= k1; ++k) {
                float ta = c.tin, tb = c.tout;
                if (cotp != 0.f) {
                    const float z1 = t_cross(plane_at(k, G.hz, G.z0), zO, cotp);
                    const float z2 = t_cross(plane_at(k + 1, G.hz, G.z0), zO, cotp);
                    ta = fmaxf(ta, fminf(z1, z2));
                    tb = fminf(tb, fmaxf(z1, z2));
                }
                if (tb > ta) {
                    const SegPos pa = ta == last_t ? last_p : seg_pos(seg_t, S, c.tin, scale, ta);
                    const SegPos pb = tb == last_t ? last_p : seg_pos(seg_t, S, c.tin, scale, tb);
                    const int kq = k - kb;
                    acc += eval_c(C, coff, nk, kq, pb) - eval_c(C, coff, nk, kq, pa);
                    last_t = up ? tb : ta;
                    last_p = up ? pb : pa;
                }
            }
        }
        __syncthreads();
    }

    if (carry_out) {  // uniform per launch: the next level range continues from here
        if (valid) out[o] = acc;
        return;
    }

    // ---- epilogue ----------------------------------------------------------------------
    float r2 = 0.f;
    if (valid) {
        // every rounding spelled out, so no caller's inlining can fuse them differently
        const float p = __fmul_rn(acc, secp);  // horizontal length -> 3D length
        if (mode == PROJ_PLAIN) {
            out[o] = p;
        } else if (mode == PROJ_SCALED) {
            out[o] = __fmul_rn(p, secp);
        } else {
            const float yv = (mode == PROJ_RESID32 || mode == PROJ_RAW32) ? __ldg(y32 + o) : __half2float(y16[o]);
            const float rr = __fsub_rn(p, yv);
            r2 = __fmul_rn(rr, rr);
            out[o] = mode >= PROJ_RAW32 ? rr : __fmul_rn(rr, secp);
        }
    }
    if (proj_is_resid(mode)) {
        // float32 within a warp (pairwise tree), float64 across warps and blocks
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, off);
        double *red = (double *)smem;  // the tables are no longer needed (barrier above)
        if (lane == 0) red[warp] = (double)r2;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < nwarp; ++w) sum += red[w];
            partial[((size_t)zc * G.na + ia) * G.nu + a] = sum;
        }
    }
}


}  // namespace cbct
