// Internal declarations of the sm_103a CBCT library (not part of the C ABI).
//
// Internal layouts (chosen for the kernels, converted at the ABI boundary):
//   volume    float [nx][ny][nz]      (z fastest: a z-column is contiguous)
//   sinogram  float [na][nu][nv]      (v fastest: a detector column is contiguous)
// With these, the 32 lanes of a projector warp (32 consecutive detector rows of one
// column) read neighbouring voxels of one z-column, and the 32 lanes of an adjoint
// warp (32 consecutive voxels of one z-column) write contiguous outputs and read
// contiguous residual rows.
#pragma once
#include <atomic>

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cbct.h"

namespace cbct {

// Kernels this process has launched through the library (every launch site counts
// itself); read with cbct_kernel_launch_count.
extern std::atomic<unsigned long long> g_kernel_launches;
inline void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }


// Ray parameterisation shared by the projector and the adjoint.
//
// All rays of detector column a at view ia share one line in the xy-plane.  It is
// parameterised by t, the horizontal distance (mm) from O, the foot of the
// perpendicular from the rotation axis: p_xy(t) = O + t e.  The ray through row b
// has height z(t) = zO + t tan(phi), and 3D length = dt * sec(phi).  Plane
// crossings are t = (plane - O) / e for x and y planes and t = (plane - zO) cot(phi)
// for z planes; both kernels evaluate them with the same float32 expression, so the
// intersection lengths they use are the same numbers.
struct GeoDev {
    int nx, ny, nz, nu, nv, na;
    float hx, hy, hz;
    float x0, y0, z0;            // lower corner of the volume box
    float inv_hx, inv_hy, inv_hz;
    float du, dv, inv_du, inv_dv;
    float cu, cv;                // (nu-1)/2, (nv-1)/2
    float dso, dsd;
    const float4 *ray_xy;        // [na][nu]  O_x, O_y, 1/e_x, 1/e_y   (1/e = 0: parallel)
    const float2 *ray_e;         // [na][nu]  e_x, e_y
    const float4 *ray_z;         // [nu][nv]  zO, cot(phi), sec(phi), tan(phi)  (cot = 0: v = 0)
    const float2 *ray_zc;        // [nu][nv]  zO, cot(phi) (same values; the adjoint's table)
    const float2 *col;           // [nu]      D = |d_xy|, t_S (source-to-O distance)
    const float2 *view;          // [na]      cos, sin
    float2 *rowsum;              // [na][nu][nv+1] running sums of the scaled residual along each
                                 // detector column, as double-float (hi, lo) float32 pairs (workspace)
    // launch shapes (0 = default); none of them changes any result bit
    int proj_threads;            // projector block size (>= 32 ceil(nv/32) up to 512, multiple of 32)
    int proj_smem;               // projector dynamic shared memory, bytes (0 = default; see proj_smem_of)
    int proj_levels;             // z-levels per projector launch (0 = default; see project_levels_per_launch)
    int bp_vpl;                  // adjoint voxels per lane (1..4)
    int bp_threads;              // adjoint block size (64, 128 or 256)
    int bp_layout;               // adjoint lane layout: 0 by gather span (bp_interleaved), 1 consecutive
                                 // voxels per lane, 2 interleaved
};

__host__ __device__ __forceinline__ size_t vol_elems(const GeoDev &g) { return (size_t)g.nx * g.ny * g.nz; }
__host__ __device__ __forceinline__ size_t sino_elems(const GeoDev &g) { return (size_t)g.na * g.nu * g.nv; }

#ifdef __CUDACC__
// Coordinate of grid plane p (exact expression shared by every kernel).
__device__ __forceinline__ float plane_at(int p, float h, float lo) { return __fmaf_rn((float)p, h, lo); }
// Crossing parameter of a plane: (plane - origin) * inverse direction, no contraction.
__device__ __forceinline__ float t_cross(float plane, float origin, float inv) {
    return __fmul_rn(__fsub_rn(plane, origin), inv);
}
#endif

// One multigrid level: host geometry, device tables, workspaces.
struct Level {
    // host values (float64 for table construction)
    int nx, ny, nz, nu, nv, na;
    double hx, hy, hz, du, dv, dso, dsd;
    GeoDev gd{};
    // device allocations owned by the level
    void *tables = nullptr;
    float *f = nullptr, *g = nullptr, *A = nullptr, *B = nullptr;  // internal volumes
    float *rs = nullptr;          // sec(phi) * residual, internal sinogram
    float *Y = nullptr;           // data, internal sinogram (float32)
    __half *Yh = nullptr;         // data, internal sinogram (half storage variant)
    double *partial = nullptr;    // float64 block partials
    size_t partial_len = 0;
    double lambda = 0.0;          // cached lambda_max(P^T P) (0 = unknown)
    int lambda_iters = 0;
    int tv_sweeps = 0, tv_warps = 0, tv_planes = 0;  // x-marching TV launch shape (0 = default)
    float *eq2p = nullptr;        // zero-bordered residual for the Eq. 2 adjoint, [na][nu+2][nv+2]
    float *mg = nullptr;          // V-cycle volumes: linear term, restricted iterate, 2 scratch
    double *mg_partial = nullptr; // V-cycle dot-product partials
};

struct EventPool {
    std::vector<cudaEvent_t> free_list, used;
    std::vector<int> cls;
    cudaEvent_t get();
    void release_all();
    ~EventPool();
};

}  // namespace cbct

struct cbct_geometry {
    cbct_geometry_desc desc;
    std::vector<double> angles;
    int device = 0;
    std::vector<cbct::Level *> levels;   // index = level, created on demand
    double *dscalars = nullptr;          // small device scratch: trace, counters
    int *dcounter = nullptr;
    double *dtrace = nullptr;            // device energy trace
    size_t dtrace_len = 0;
    cbct::EventPool events;
    // power iterations of the finer levels of a cascade, run on a side stream while the
    // coarser levels iterate (they depend on the geometry alone)
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr;
    cudaEvent_t side_done[13] = {};
    double *host_lam = nullptr;          // pinned host [13]: lambda of each level
};

namespace cbct {

void set_error(const char *fmt, ...);
int device_sm_count();  // SMs of the current device (cached per device)
cbct_status cuda_fail(cudaError_t e, const char *what);

// level management (geometry.cu)
cbct_status ensure_level(cbct_geometry *G, int level, Level **out);
cbct_status ensure_workspace(Level *L, bool need_half);
cbct_status ensure_mg_workspace(Level *L);
// L->eq2p for the Eq. 2 adjoint, its border zeroed on stream s at allocation
cbct_status ensure_eq2_pad(Level *L, cudaStream_t s);
void free_level(Level *L);

// kernel launchers (return cudaError_t of the launch)
// RESID32/RESID16 store sec(phi) * (P f - Y) for the matched gather; the RAW variants
// store P f - Y itself (the Eq. 2 adjoint interpolates the residual).
enum ProjMode { PROJ_PLAIN = 0, PROJ_RESID32 = 1, PROJ_RESID16 = 2, PROJ_SCALED = 3, PROJ_RAW32 = 4, PROJ_RAW16 = 5 };
__host__ __device__ __forceinline__ bool proj_is_resid(int mode) {
    return mode == PROJ_RESID32 || mode == PROJ_RESID16 || mode == PROJ_RAW32 || mode == PROJ_RAW16;
}
cudaError_t launch_project(const GeoDev &g, const float *vol, const float *y32, const __half *y16,
                           float *out, double *partial, int mode, cudaStream_t s, int *nblocks_out);
size_t project_partials(const GeoDev &g);

enum BpMode { BP_PLAIN = 0, BP_STEP = 1 };
// (launches the column running sums of rs into g.rowsum first)
cudaError_t launch_backproject(const GeoDev &g, const float *rs, const float *fin, float *out, float c,
                               int mode, cudaStream_t s);
cudaError_t launch_row_prefix(const GeoDev &g, const float *rs, cudaStream_t s);
int project_threads(const GeoDev &g);

// Eq. 2 adjoint: out = cscale * B' r (BP_PLAIN) or fin - cscale * B' r (BP_STEP), where
// B' is B without its dV/(du dv) factor and r = P f - Y unscaled.  padded (or null): a
// zero-bordered [na][nu + 2][nv + 2] workspace (ensure_eq2_pad); r is copied into its
// interior first and the gather reads its taps without bounds checks (the same result).
cudaError_t launch_backproject_eq2(const GeoDev &g, const float *r, float *padded, const float *fin, float *out,
                                   float cscale, int mode, cudaStream_t s);
double eq2_scale(const Level *L);  // dV / (du dv)
int bp_default_vpl(const GeoDev &g);
// Whether the adjoint's lanes hold interleaved voxels (bp_tile.cuh) with vpl voxels per lane.
bool bp_interleaved(const GeoDev &g, int vpl);

struct TvArgs {
    int nx, ny, nz;          // internal layout [nx][ny][nz]
    float ihx, ihy, ihz;     // 1/h
    float s, beta, eps2;
    int aniso;               // 0: isotropic E1, 1: anisotropic E1
    int jc;                  // rows per warp tile of the sweep (tv_rows_per_tile; 0: per voxel)
    int vz;                  // full-column tiles: voxels per lane in z (tv_col_vz; 0: 32-voxel z-blocks)
    // x-marching fused sweeps (tv_xmarch.cuh; xT = 0: not used): sweeps per launch (1 or 2),
    // warps per block, planes per block
    int xT, xW, xLX;
};
// Forms of the TV sweep, chosen from the sizes alone (so every launch of a level, alone
// or batched, uses the same tiles):
//  * full column (tv_col_vz > 0): a warp owns whole z-columns of at most 96 voxels (up
//    to 3 per lane) and walks jc rows in y; z-neighbours come by shuffle, with no halo.
//    Used when walks of 4 rows still give 8192 warp tiles (3 voxels per lane run with
//    a 64-register cap: 15 % faster than the row walk on 96-voxel columns).
//  * row walk (jc > 0, vz = 0): a warp owns 32 consecutive z-voxels and walks 16 rows;
//    for taller volumes (measured on B300: 1.3-1.5x faster than one thread per voxel
//    from 256x256x48 up).
//  * one thread per voxel (jc = 0): smaller volumes.
__host__ __device__ __forceinline__ int tv_col_vz(int nx, int ny, int nz) {
    return (nz <= 96 && (long)nx * ((ny + 3) / 4) >= 8192) ? (nz + 31) / 32 : 0;
}
__host__ __device__ __forceinline__ int tv_rows_per_tile(int nx, int ny, int nz) {
    if (tv_col_vz(nx, ny, nz)) {
        if ((long)nx * ((ny + 15) / 16) >= 8192) return 16;
        if ((long)nx * ((ny + 7) / 8) >= 8192) return 8;
        return 4;
    }
    return (long)nx * ((ny + 15) / 16) * ((nz + 31) / 32) >= 8192 ? 16 : 0;
}
// x-marching form of a level (tv_xmarch.cuh), from the sizes and the level's launch-shape
// overrides (0 = default): whole z-columns of at most 96 voxels and enough tiles to fill
// the GPU.  Writes the shape into a (xT = 0 when the form does not apply).
void tv_x_shape(TvArgs &a, int sweeps, int warps, int planes);
// One launch of the x-marching form: T (1 or 2) consecutive sweeps fin -> fout, sweep t
// clamping when bit t of clamp is set; partial_e1: E1 partials of fin; partial_step: the
// partials of (fout_new - f_k)^2 with f_k in fout on entry.  *nblocks_out: partials written.
cudaError_t launch_tv_x(const TvArgs &a, int T, unsigned clamp, const float *fin, const float *g, float *fout,
                        double *partial_e1, double *partial_step, cudaStream_t s, int *nblocks_out);
// Partials one x-marching launch of T sweeps writes (the block count).
size_t tv_x_partials(const TvArgs &a, int T);
// Upper bound of tv_x_partials over every shape the level may take (workspace sizing).
size_t tv_x_partials_max(int nx, int ny, int nz);
// The launches of a whole prox (M sweeps) in the x-marching form, from src0: launches of
// up to a.xT sweeps ping-ponging through A and B, the last one writing f (f_k+1 over f_k)
// unless its input is f itself.  Shared by the single-request path and the batch engine,
// so both issue the same launches.
struct XLaunch {
    int T;
    unsigned clamp;          // bit t: sweep t clamps at 0
    const float *fin;
    float *fout;
    bool e1, step;           // accumulators of this launch
};
struct XProxPlan {
    std::vector<XLaunch> launches;
    const float *result;     // where the last launch leaves f_k+1
    bool step_fused;         // the last launch forms the step partials (it overwrites f_k)
    int n_e1, n_step;        // partials of the E1 launch and of the step norm (a step copy's
                             // step_partials when not fused)
};
XProxPlan xprox_plan(const TvArgs &a, int M, int clamp_mode, const float *src0, float *f, float *A, float *B,
                     bool want_e1, bool want_step, size_t nvox);
// One prox sweep fin -> fout.  partial_e1: the E1 partials of fin; partial_step (fout
// then holds f_k and is overwritten in place): the partials of (fout_new - f_k)^2.  At
// most one of the two; tv_partials values either way.
cudaError_t launch_tv_sweep(const TvArgs &a, const float *fin, const float *g, float *fout, bool clamp,
                            double *partial_e1, cudaStream_t s, int *nblocks_out, double *partial_step = nullptr);
size_t tv_partials(int nx, int ny, int nz);         // E1 (or step) partials written by a sweep
size_t tv_blocks(int nx, int ny, int nz);           // blocks of one sweep launch
size_t tv_energy_partials(int nx, int ny, int nz);  // partials written by launch_tv_energy

// layout changes
cudaError_t launch_vol_to_internal(const float *api, float *in, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_vol_to_api(const float *in, float *api, int nx, int ny, int nz, cudaStream_t s);
// sinogram [na][nv][nu] -> [na][nu][nv]; optional sec(phi) scaling from ray_z, optional half output
cudaError_t launch_sino_to_internal(const float *api, float *out32, __half *out16, const float4 *ray_z,
                                    int na, int nu, int nv, cudaStream_t s);
cudaError_t launch_sino_to_api(const float *in, float *api, int na, int nu, int nv, cudaStream_t s);

// multigrid transfers (layout-agnostic: [n0][n1][n2] volumes, [na][n1][n2] stacks)
cudaError_t launch_restrict(const float *y, float *yc, int na, int n1, int n2, cudaStream_t s);
cudaError_t launch_to_half(const float *x, __half *y, size_t n, cudaStream_t s);
cudaError_t launch_prolong(const float *fc, int c0, int c1, int c2, float *f, int n0, int n1, int n2,
                           cudaStream_t s);

// reductions and small kernels
// device energy trace: TRACE_W doubles per iteration: E, E1, mu E2 of the entering
// iterate and |f_k+1 - f_k|_2 of the iteration
constexpr int TRACE_W = 4;
cudaError_t launch_energy_finalize(const double *pe2, int n2, const double *pe1, int n1, double inv_nv,
                                   double mu_over_nr, double *trace, int *counter, cudaStream_t s,
                                   const double *pstep = nullptr, int nstep = 0);
size_t step_partials(size_t n);
// the step-norm partials inside a level's partials buffer (after the projector's and
// the TV sweep's)
double *step_region(Level *L);
size_t tv_region_len(const Level *L);
// The last of M prox sweeps from src0 writes f_k+1 over f_k in place and forms the
// step-norm partials itself unless its input is f_k (M == 1 from f_k); then it goes
// through a buffer and launch_step_copy.  Number of step partials either way:
inline bool prox_step_fused(int M, const float *src0, const float *f) { return M >= 2 || src0 != f; }
cudaError_t launch_step_copy(const float *v, float *f, size_t n, double *partial, cudaStream_t s);
cudaError_t launch_dot2(const float *x, const float *y, size_t n, double *partial, cudaStream_t s,
                        int *nblocks_out);
cudaError_t launch_power_finalize(const double *partial, int nblk, double *lam, float *scale,
                                  cudaStream_t s);
cudaError_t launch_scale(const float *y, const float *scale, float *x, size_t n, cudaStream_t s);
cudaError_t launch_fill(float *x, float v, size_t n, cudaStream_t s);
// seeded uniform(0,1) volume (internal layout) of the power iteration's start
constexpr unsigned long long POWER_SEED = 10023675ull;
cudaError_t launch_fill_uniform(float *x, int nx, int ny, int nz, unsigned long long seed, cudaStream_t s);

// V-cycle kernels (k_mg.cu); volumes [n0][n1][n2], coarse sizes ceil(n / 2)
cudaError_t launch_restrict_vol(const float *f, int n0, int n1, int n2, float *fc, cudaStream_t s);
cudaError_t launch_prolong_adjoint(const float *x, int n0, int n1, int n2, float *out, int c0, int c1, int c2,
                                   cudaStream_t s);
cudaError_t launch_axpy(float *y, const float *x, float a, size_t n, cudaStream_t s);
cudaError_t launch_sub(const float *a, const float *b, float *out, size_t n, cudaStream_t s);
cudaError_t launch_add_clamp(const float *f, const float *c, float *out, size_t n, cudaStream_t s);
size_t dot_partials(size_t n);
cudaError_t launch_dot(const float *x, const float *y, size_t n, double *partial, double *out, cudaStream_t s);
cudaError_t launch_tv_energy(const TvArgs &a, const float *f, double *partial, cudaStream_t s,
                             int *nblocks_out);
// out = (grad TV_eps(f) + gamma bp) / Nv - lin (lin optional; out may alias bp)
cudaError_t launch_energy_grad(const TvArgs &a, const float *f, const float *bp, float gamma, float inv_nv,
                               const float *lin, float *out, cudaStream_t s);


// Solver constants of one level (Algorithm A1, discrete scaling of Eq. 1).
struct SolveParams {
    float c;        // gamma / beta
    float s;        // inner step 1 / (beta + L_TV)
    float beta;
    float eps2;
    int M;
    int clamp_mode;
    int tv_mode;
    int adjoint_mode;  // 0 exact transpose, 1 Eq. 2
    float c_eq2;       // (gamma / beta) dV / (du dv)
    const float *lin;  // V-cycle coarse model: linear term -<lin, f> (null: none)
    float lin_scale;   // Nv / beta: its share of step 1
    bool fp16;
    double inv_nv, mu_over_nr;
};
double default_eps(const Level *L);
double tv_lipschitz(const Level *L, double eps);
double gamma_of(const Level *L, double mu);
cbct_status ensure_trace(cbct_geometry *G, size_t n);
TvArgs tv_args(const Level *L, const SolveParams &P);
cbct_status solve_params(const Level *L, double mu, double beta, double eps, int M, int clamp_mode, bool fp16,
                         SolveParams *P, int tv_mode = 0, int adjoint_mode = 0);
cbct_status get_trace(cbct_geometry *G, size_t n, double **out);
cbct_status copy_trace(const double *dtrace, int iters, double *energy, double *step, cudaStream_t s);

}  // namespace cbct
