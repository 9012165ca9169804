// Device-side body of the fused TV prox sweeps: T consecutive projected-gradient
// steps of step 2 (and 3) of Algorithm A1 in one launch, marching along x.
#pragma once

// The arithmetic per voxel and sweep is that of tv_tile.cuh (same expressions, same
// order): with the own term o(i,j,k) = (p_x, p_y, p_z, -(sum_d g_d / h_d) n) of a voxel
// (tv_own), the divergence of the smoothed gradient is
//   div = o.div + p_x(i-1) / hx + p_y(j-1) / hy + p_z(k-1) / hz   (terms at index 0 absent)
// and the step is f <- max(0, f - s (beta (f - g) + div)).  The other forms recompute
// one of the three neighbour terms (p_x(i-1)); here every voxel's own term is computed
// once per sweep and handed to the three neighbours that need it:
//   * p_x(i-1): the same warp, one step earlier in the x-march (a register);
//   * p_z(k-1): a lane holds VZ consecutive voxels of its z-column (k = VZ l + v), so
//     it is the lane's own previous slot, or one shuffle from the lane below;
//   * p_y(j-1): the warp of the row below, through shared memory.
// The reciprocal square root is the ftz form of the same approximate instruction
// (rsqrt.approx): its argument |grad f|^2 + eps^2 >= eps^2 is never subnormal (the
// launcher requires eps^2 >= FLT_MIN), where both forms agree, so the results are
// bitwise those of the other forms.
//
// Tiles.  A block owns output rows [j0, j0 + by) and planes [x0, x0 + lx) with whole
// z-columns (nz = VZ x active lanes); warp w owns row j0 - T + w (W = by + 2T - 1
// warps).  Sweep t (t = 0..T-1, the input being f^t) updates rows and planes within
// T-1-t of the output tile, and computes own terms one row and one plane further
// down, so that after T sweeps the output tile holds f^T exactly as T separate sweeps
// would give it.  At x-step s, sweep t works on plane s - 1 - t: its +x neighbour
// plane is the one the previous sweep produced at this step (a register), its +y
// neighbour row the one the warp above produced at the previous step (shared memory,
// double-buffered by step parity; the steps run in pairs so that the parity is a
// constant).  A sweep whose plane lies outside its range for the whole block is skipped
// (with its barrier).  Only f^0, g and the output touch global memory: each warp stages
// its rows of f^0 and g one plane ahead into shared memory with asynchronous 16-byte
// copies (three planes in a ring; the last warp also stages the row above the block),
// so the sweeps read only registers and shared memory.  For T = 2, about 4 + 4 + 4
// bytes per voxel (plus the halo share) carry two sweeps instead of 24.
//
// Accumulators (one float64 partial per block): X.e1, the E1 terms |grad f^0|_eps of
// the input over the output tile (sweep 0's own terms); X.step, (f^T - f_k)^2 over the
// output tile, fout holding f_k on entry (overwritten in place: no other block reads
// fout, which must not alias fin).
#include <type_traits>

#include "tv_tile.cuh"

namespace cbct {

struct TvXArgs {
    int W;            // warps per block (by + 2T - 1)
    int by, lx;       // output rows and planes per block
    int nyt;          // blocks along y (the block index runs fastest along y)
    unsigned clamp;   // bit t: clamp at 0 in sweep t of this launch
    int e1, step;     // accumulators (at most one set per launch)
};

constexpr int TVX_MAX_THREADS = 1024;

// Shared floats of one block: the p_y rows of every sweep for two step parities, for
// T > 1 the f rows of sweeps 0..T-2 for two step parities, and the three staged planes
// of f^0 (W + 1 rows) and g (W rows).
__host__ __device__ __forceinline__ size_t tvx_smem_floats(int T, int W, int VZ) {
    return ((size_t)(2 * T + 2 * (T - 1)) * W + 3 * (W + 1) + 3 * W) * 32 * VZ;
}

// Voxels per lane of a column of nz voxels (0: the form does not apply): whole lanes,
// and whole 16-byte pieces for the staging copies.
__host__ __device__ __forceinline__ int tvx_vz(int nz) {
    const int vz = (nz + 31) / 32;
    return (vz >= 1 && vz <= 3 && nz % vz == 0 && nz % 4 == 0) ? vz : 0;
}

__device__ __forceinline__ float tvx_rsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// tv_own with tvx_rsqrt (same expressions and roundings)
template <bool E1, bool ANISO>
__device__ __forceinline__ TvOwn tvx_own(const TvArgs &A, float c, float fxp, float fyp, float fzp) {
    TvOwn o;
    const float gx = __fmul_rn(__fsub_rn(fxp, c), A.ihx);
    const float gy = __fmul_rn(__fsub_rn(fyp, c), A.ihy);
    const float gz = __fmul_rn(__fsub_rn(fzp, c), A.ihz);
    o.e1 = 0.f;
    if (ANISO) {
        const float qx = __fmaf_rn(gx, gx, A.eps2), qy = __fmaf_rn(gy, gy, A.eps2), qz = __fmaf_rn(gz, gz, A.eps2);
        const float rx = tvx_rsqrt(qx), ry = tvx_rsqrt(qy), rz = tvx_rsqrt(qz);
        o.px = __fmul_rn(gx, rx);
        o.py = __fmul_rn(gy, ry);
        o.pz = __fmul_rn(gz, rz);
        o.div = -__fmaf_rn(o.px, A.ihx, __fmaf_rn(o.py, A.ihy, __fmul_rn(o.pz, A.ihz)));
        if (E1) o.e1 = __fadd_rn(__fadd_rn(__fmul_rn(qx, rx), __fmul_rn(qy, ry)), __fmul_rn(qz, rz));
    } else {
        const float q0 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmaf_rn(gz, gz, A.eps2)));
        const float n0 = tvx_rsqrt(q0);
        o.px = __fmul_rn(gx, n0);
        o.py = __fmul_rn(gy, n0);
        o.pz = __fmul_rn(gz, n0);
        o.div = -__fmul_rn(__fmaf_rn(gx, A.ihx, __fmaf_rn(gy, A.ihy, __fmul_rn(gz, A.ihz))), n0);
        if (E1) o.e1 = __fmul_rn(q0, n0);
    }
    return o;
}

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only)
__device__ __forceinline__ void tvx_cp16(float *dst, const float *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void tvx_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void tvx_cp_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int T, int VZ, int W, bool ANISO>
__device__ __forceinline__ void tv_x_tile(const TvArgs &A, const TvXArgs &X, const float *__restrict__ fin,
                                          const float *__restrict__ g, float *__restrict__ fout,
                                          double *__restrict__ partial, float *sm, const int blk) {
    static_assert(T == 1 || T == 2, "at most two sweeps per launch");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int KZ = 32 * VZ;
    constexpr int RING = 3;                         // planes of f^0 and g staged: p - 1, p, p + 1
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int yt = blk % X.nyt, xc = blk / X.nyt;
    const int j0 = yt * X.by, j1 = min(j0 + X.by, A.ny);
    const int x0 = xc * X.lx, x1 = min(x0 + X.lx, A.nx);
    const int j = j0 - T + w;                      // this warp's row
    const bool row = j >= 0 && j < A.ny;
    const bool yp = j + 1 < A.ny;
    const bool jout = j >= j0 && j < j1;
    const int nl = A.nz / VZ;                       // lanes holding voxels
    const bool lon = lane < nl;
    const bool ztop = lane == nl - 1;               // its last slot is the column's top voxel
    const int kb = VZ * (lon ? lane : nl - 1);      // first voxel of the lane (idle lanes mirror the top one)
    const size_t sx = (size_t)A.ny * A.nz;
    const size_t jr = (size_t)(row ? j : 0) * A.nz;
    const int wy = yp ? w + 1 : w;                  // the +y row's slot (row W: the extra row)
    // shared memory: p_y rows [step parity][sweep][warp], f rows of sweeps 0..T-2
    // [sweep][step parity][warp], the staged f^0 rows [ring][warp + the row above the
    // block] and g rows [ring][warp], all rows KZ floats with voxel k at index k
    float *const PYw = sm + w * KZ + kb;
    const float *const PYr = sm + (w > 0 ? w - 1 : 0) * KZ + kb;
    float *const FXw = sm + 2 * T * W * KZ + w * KZ + kb;
    const float *const FXr = sm + 2 * T * W * KZ + (w + 1 < W ? w + 1 : w) * KZ + kb;
    float *const F0 = sm + (2 * T + 2 * (T - 1)) * W * KZ;
    float *const G0 = F0 + RING * (W + 1) * KZ;
    // staging: lanes q < nz / 4 copy 16 bytes each of a row (z-columns are 16-byte aligned)
    const bool cpl = lane < (A.nz >> 2);
    const bool up_row = w == W - 1 && row && yp; // the last warp also stages the row above
    auto stage = [&](const int pf, const int pg) {  // f^0 at plane pf, g at plane pg
        if (row && cpl) {
            if (pf < A.nx) {
                const float *src = fin + (size_t)pf * sx + jr + 4 * lane;
                float *dst = F0 + ((pf % RING) * (W + 1) + w) * KZ + 4 * lane;
                tvx_cp16(dst, src);
                if (up_row) tvx_cp16(dst + KZ, src + A.nz);
            }
            if (pg >= 0 && pg < A.nx)
                tvx_cp16(G0 + ((pg % RING) * W + w) * KZ + 4 * lane, g + (size_t)pg * sx + jr + 4 * lane);
        }
        tvx_cp_commit();
    };
    float cv[T][VZ], pxp[T][VZ];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int v = 0; v < VZ; ++v) cv[t][v] = pxp[t][v] = 0.f;
    // per-sweep ranges: steps whose plane lies in the sweep's planes, own terms and
    // updates (one plane and one row further down for own terms)
    int slo[T], shi[T], sup[T];
    bool ract[T], rupd[T];
    float lo[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int d = T - 1 - t;
        slo[t] = max(x0 - d - 1, 0) + 1 + t;        // plane p = s - 1 - t
        shi[t] = min(x1 + d, A.nx) + 1 + t;
        sup[t] = x0 - d + 1 + t;
        ract[t] = row && j >= j0 - d - 1 && j < j1 + d;
        rupd[t] = row && j >= j0 - d && j < j1 + d;
        lo[t] = ((X.clamp >> t) & 1u) ? 0.f : -INFINITY;   // fmaxf(x, -inf) is x
    }
    float acc = 0.f;
    const int s0 = max(x0 - T, 0) + 1, s1 = x1 - 1 + T;
    float *pout = fout + ((ptrdiff_t)s0 - T) * (ptrdiff_t)sx + (ptrdiff_t)(jr + kb);
    // f^0 at planes s0 - 1 and s0, g at s0 - 1, before the first step
    stage(s0 - 1, s0 - 1);
    stage(s0, -1);
    tvx_cp_wait();
    __syncthreads();

    // one x-step with its step parity PAR fixed at compile time
    auto step = [&](const int s, auto par_tag) {
        constexpr int PAR = decltype(par_tag)::value;
        // this step's staged rows have landed (the lanes' own copies; the barrier of the
        // previous step published the other warps'); then stage the next step's
        tvx_cp_wait();
        __syncwarp();
        stage(s + 1, s);
        const int pT = s - T;                       // the output plane of this step
        const bool out = jout && lon && pT >= x0 && pT < x1;
        float fo[VZ];
#pragma unroll
        for (int v = 0; v < VZ; ++v) fo[v] = (X.step && out) ? pout[v] : 0.f;   // f_k at the output
        const int r0 = (s - 1) % RING, r1 = s % RING;
        const float *c0 = F0 + (r0 * (W + 1) + w) * KZ + kb;      // f^0(s - 1, j)
        float inc[VZ];
        {
            const float *n0 = F0 + (r1 * (W + 1) + w) * KZ + kb;  // f^0(s, j), itself past the last plane
            const bool lin = s < A.nx;
#pragma unroll
            for (int v = 0; v < VZ; ++v) inc[v] = lin ? n0[v] : c0[v];
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int p = s - 1 - t;
            float y[VZ];
            if (t == 0) {
#pragma unroll
                for (int v = 0; v < VZ; ++v) cv[0][v] = c0[v];
            }
            if (s < slo[t] || s >= shi[t]) {
                // the whole block is outside this sweep's planes: nothing to do; past the
                // last plane, the next sweep's +x plane is its own (zero difference)
#pragma unroll
                for (int v = 0; v < VZ; ++v) {
                    y[v] = t + 1 < T ? cv[t + 1 < T ? t + 1 : t][v] : 0.f;
                    cv[t][v] = inc[v];
                    inc[v] = y[v];
                }
                continue;
            }
            const bool act = ract[t];
            const bool upd = rupd[t] && s >= sup[t];
            float fy[VZ], fz[VZ];
            {
                // f^t(p, j+1): the staged row (t = 0), else written by the warp above at
                // the previous step; its own row at the last row
                const float *src = t == 0 ? F0 + (r0 * (W + 1) + wy) * KZ + kb
                                          : (yp ? FXr : FXw) + ((t > 0 ? t - 1 : 0) * 2 + (1 - PAR)) * W * KZ;
#pragma unroll
                for (int v = 0; v < VZ; ++v) fy[v] = src[v];
            }
            // +z neighbours: the next slot, the lane above's first slot, itself at the top
#pragma unroll
            for (int v = 0; v + 1 < VZ; ++v) fz[v] = cv[t][v + 1];
            {
                const float up = __shfl_down_sync(FULL, cv[t][0], 1);
                fz[VZ - 1] = ztop ? cv[t][VZ - 1] : up;
            }
            TvOwn own[VZ];
#pragma unroll
            for (int v = 0; v < VZ; ++v) {
                if (t == 0) own[v] = tvx_own<true, ANISO>(A, cv[t][v], inc[v], fy[v], fz[v]);
                else own[v] = tvx_own<false, ANISO>(A, cv[t][v], inc[v], fy[v], fz[v]);
            }
            const int PYO = (PAR * T + t) * W * KZ;
            if (act) {
#pragma unroll
                for (int v = 0; v < VZ; ++v) PYw[PYO + v] = own[v].py;
            }
            if (t == 0 && X.e1 && jout && lon && p >= x0 && p < x1) {
#pragma unroll
                for (int v = 0; v < VZ; ++v) acc = __fadd_rn(acc, own[v].e1);
            }
            __syncthreads();
            // p_z piece of (k - 1): the previous slot, the lane below's last slot for slot 0
            const float pz_dn = __shfl_up_sync(FULL, own[VZ - 1].pz, 1);
            const bool ypos = upd && j > 0;
            const float *gp = G0 + ((p % RING) * W + w) * KZ + kb;   // g(p, j)
#pragma unroll
            for (int v = 0; v < VZ; ++v) {
                float dv = own[v].div;
                if (p > 0) dv = __fmaf_rn(pxp[t][v], A.ihx, dv);
                if (ypos) dv = __fmaf_rn(PYr[PYO + v], A.ihy, dv);
                if (v > 0) dv = __fmaf_rn(own[v > 0 ? v - 1 : 0].pz, A.ihz, dv);
                else if (lane > 0) dv = __fmaf_rn(pz_dn, A.ihz, dv);
                const float c = cv[t][v];
                const float x = __fmaf_rn(-A.s, __fmaf_rn(A.beta, __fsub_rn(c, gp[v]), dv), c);
                y[v] = fmaxf(x, lo[t]);
            }
            if (upd) {
                if (t < T - 1) {
                    float *dst = FXw + (t * 2 + PAR) * W * KZ;
#pragma unroll
                    for (int v = 0; v < VZ; ++v) dst[v] = y[v];
                } else if (out) {
#pragma unroll
                    for (int v = 0; v < VZ; ++v) {
                        if (X.step) {   // fo: f_k, read before it is overwritten
                            const float dd = __fsub_rn(y[v], fo[v]);
                            acc = __fmaf_rn(dd, dd, acc);
                        }
                        pout[v] = y[v];
                    }
                }
            }
            // the next step of this sweep works on plane p + 1; the next sweep of this
            // step takes f^{t+1}(p) as its +x plane
#pragma unroll
            for (int v = 0; v < VZ; ++v) {
                pxp[t][v] = own[v].px;
                cv[t][v] = inc[v];
                inc[v] = y[v];
            }
        }
        pout += sx;
    };
    // steps in pairs so that the step parity (which shared rows to use) is a constant
    int s = s0;
    if (s & 1) {
        if (s <= s1) step(s, std::integral_constant<int, 1>{});
        ++s;
    }
#pragma unroll 1
    for (; s + 1 <= s1; s += 2) {
        step(s, std::integral_constant<int, 0>{});
        step(s + 1, std::integral_constant<int, 1>{});
    }
    if (s <= s1) step(s, std::integral_constant<int, 0>{});
    tvx_cp_wait();   // (copies past the block's last step, never read)

    if (X.e1 || X.step) {
        // float32 over the block's planes per lane, a pairwise tree over the lanes, then
        // float64 over the warps in order: one partial per block
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(FULL, acc, off);
        __syncthreads();   // the shared rows are no longer read
        double *red = (double *)sm;
        if (lane == 0) red[w] = (double)acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int q = 0; q < W; ++q) sum += red[q];
            partial[blk] = sum;
        }
    }
}

}  // namespace cbct
