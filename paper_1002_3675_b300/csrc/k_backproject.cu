// Adjoint gather launchers (single request).  The arithmetic is in bp_tile.cuh.
#include "bp_tile.cuh"

namespace cbct {

// at most 51 registers per thread (48 used): 10 blocks of 128 threads per SM (64
// registers for 4 voxels per lane); dynamic shared memory: the warps' setup records
template <int MODE, int VPL, bool IL>
__global__ void __launch_bounds__(256, VPL == 4 ? 4 : 5)
k_backproject(GeoDev G, const float *__restrict__ rs, const float *__restrict__ fin,
              float *__restrict__ out, float c) {
    extern __shared__ float4 rec[];
    const long gwarp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gwarp >= bp_warp_tiles<VPL>(G)) return;
    bp_warp<VPL, IL>(G, MODE, rs, fin, out, c, gwarp, rec + (threadIdx.x >> 5) * BP_REC_PER_WARP);
}

template <int VPL>
static void launch_vpl(const GeoDev &g, const float *rs, const float *fin, float *out, float c, int mode,
                       cudaStream_t s) {
    const int T = (g.bp_threads == 64 || g.bp_threads == 256) ? g.bp_threads : BP_THREADS;
    const long nb = (bp_warp_tiles<VPL>(g) * 32 + T - 1) / T;
    const size_t smem = (size_t)(T / 32) * BP_REC_PER_WARP * sizeof(float4);
    const bool il = bp_interleaved(g, VPL);
    if (mode == BP_PLAIN) {
        if (il) k_backproject<BP_PLAIN, VPL, true><<<(unsigned)nb, T, smem, s>>>(g, rs, fin, out, c);
        else k_backproject<BP_PLAIN, VPL, false><<<(unsigned)nb, T, smem, s>>>(g, rs, fin, out, c);
    } else {
        if (il) k_backproject<BP_STEP, VPL, true><<<(unsigned)nb, T, smem, s>>>(g, rs, fin, out, c);
        else k_backproject<BP_STEP, VPL, false><<<(unsigned)nb, T, smem, s>>>(g, rs, fin, out, c);
    }
    count_launch();
}

// Running sums of rs along every detector column, kept as unevaluated sums of two
// float32 (hi + lo, |lo| <= ulp(hi)/2: about 48 bits, as the float64 sum rounded to a
// pair) by error-free transformations in float32 arithmetic (Knuth's TwoSum, then a
// renormalisation), which B300 runs far faster than float64: rowsum[b] = sum_{b' < b}
// rs[b'].  One warp per column: lane l owns the rows [l L, (l + 1) L), L = ceil(nv/32);
// the lane totals are scanned across the warp (fixed order), then every lane re-adds its
// rows from its exclusive prefix and writes them.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_norm(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ DF df_add(DF a, float b) {  // (a.hi + a.lo) + b
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_norm(s, __fadd_rn(e, a.lo));
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__global__ void __launch_bounds__(256)
k_row_prefix(const float *__restrict__ rs, float2 *__restrict__ out, long ncol, int nv) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
    const int L = (nv + 31) >> 5;
    const int b0 = min(lane * L, nv), b1 = min(b0 + L, nv);
    for (long c = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncol; c += nwarps) {
        const float *r = rs + c * nv;
        float2 *o = out + c * (nv + 1);
        DF t = {0.f, 0.f};
        for (int b = b0; b < b1; ++b) t = df_add(t, __ldg(r + b));
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {  // inclusive scan of the lane totals
            DF u;
            u.hi = __shfl_up_sync(FULL, t.hi, d);
            u.lo = __shfl_up_sync(FULL, t.lo, d);
            if (lane >= d) t = df_add(u, t);
        }
        DF run;
        run.hi = __shfl_up_sync(FULL, t.hi, 1);
        run.lo = __shfl_up_sync(FULL, t.lo, 1);
        if (lane == 0) {
            run = {0.f, 0.f};
            o[0] = make_float2(0.f, 0.f);
        }
        for (int b = b0; b < b1; ++b) {
            run = df_add(run, __ldg(r + b));
            o[b + 1] = make_float2(run.hi, run.lo);
        }
    }
}

cudaError_t launch_row_prefix(const GeoDev &g, const float *rs, cudaStream_t s) {
    const long ncol = (long)g.na * g.nu;
    long nb = (ncol + 7) / 8;  // 8 warps (columns) per block
    if (nb > 148 * 32) nb = 148 * 32;
    k_row_prefix<<<(unsigned)nb, 256, 0, s>>>(rs, g.rowsum, ncol, g.nv);
    count_launch();
    return cudaGetLastError();
}

// voxels per lane: cover a z-column with as few warps as possible, up to 4 per lane
int bp_default_vpl(const GeoDev &g) { return min(4, max(1, (g.nz + 31) / 32)); }

// Lane layout: interleaved when one gather of the consecutive layout would span 400
// detector rows or more (32 vpl planes at about hz dsd / (dso dv) rows each, at the
// axis).  Measured on B300: the adjoint 12.5 % faster at 450 rows (3 voxels per lane,
// 0.8 mm rows), slower at 300 (2 per lane, 1.6 mm rows) and 14 % slower at 150, where
// the extra shuffles cost more than the cache lines saved.
bool bp_interleaved(const GeoDev &g, int vpl) {
    if (g.bp_layout == 1) return false;
    if (g.bp_layout == 2) return true;
    const double rows = 32.0 * vpl * (double)g.hz * g.dsd / ((double)g.dso * g.dv);
    return rows >= 400.0;
}

cudaError_t launch_backproject(const GeoDev &g, const float *rs, const float *fin, float *out, float c,
                               int mode, cudaStream_t s) {
    const cudaError_t e = launch_row_prefix(g, rs, s);
    if (e != cudaSuccess) return e;
    const int vpl = (g.bp_vpl >= 1 && g.bp_vpl <= 4) ? g.bp_vpl : bp_default_vpl(g);
    if (vpl == 4) launch_vpl<4>(g, rs, fin, out, c, mode, s);
    else if (vpl == 3) launch_vpl<3>(g, rs, fin, out, c, mode, s);
    else if (vpl == 2) launch_vpl<2>(g, rs, fin, out, c, mode, s);
    else launch_vpl<1>(g, rs, fin, out, c, mode, s);
    return cudaGetLastError();
}

}  // namespace cbct
