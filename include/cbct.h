/*
 * cbct.h -- C ABI of the B300 (sm_103a) TV-regularised cone-beam CT reconstruction
 * library.  The method is that of Jia, Lou, Li, Song and Jiang (2010): minimise
 * E[f] = E1[f] + mu E2[f] subject to f >= 0 (Eq. 1) by forward-backward splitting
 * (Algorithm A1) inside a coarse-to-fine multigrid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Units       millimetres; angles in radians; attenuation in mm^-1, so line
 *              integrals are dimensionless.
 *  Geometry    circular orbit about z.  Source at (dso cos t, dso sin t, 0); flat
 *              imager at distance dsd from the source, centred on the central ray,
 *              axes u = (-sin t, cos t, 0) and v = (0, 0, 1); one ray per pixel
 *              centre.  The volume grid is centred on the origin; voxels are
 *              half-open boxes.
 *  Layouts     volumes   float32 [nz][ny][nx]   (x fastest)
 *              sinograms float32 [n_angles][nv][nu] (u fastest)
 *  Memory      every pointer named *_dev is a CUDA device pointer, 16-byte aligned,
 *              owned by the caller and not retained after the call returns.
 *              *_host pointers are host memory, read (or written) during the call.
 *              Handles (cbct_geometry, cbct_server) and the device workspaces
 *              behind them are owned by the library and freed by the matching
 *              destroy call.
 *  Streams     work is enqueued on `stream` (0 = legacy default stream) and is
 *              asynchronous unless stated; a handle must not be used by two
 *              host threads at the same time.
 *  Errors      every call returns a cbct_status; no exception or abort crosses the
 *              ABI.  cbct_last_error() gives a message for the calling thread.
 *              Invalid arguments are rejected before any work is enqueued.  CUDA
 *              errors raised by the enqueued work are reported by the call that
 *              observes them (CBCT_ERR_CUDA).
 *  Precision   bulk arithmetic float32; global reductions (energies, norms,
 *              step-size estimate) float64.
 */
#ifndef CBCT_H
#define CBCT_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CBCT_OK = 0,
    CBCT_ERR_INVALID_ARG = 1,  /* bad pointer, size, alignment or parameter      */
    CBCT_ERR_OOM = 2,          /* a library workspace could not be allocated     */
    CBCT_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed    */
    CBCT_ERR_TIMEOUT = 4,      /* a bounded wait expired                         */
    CBCT_ERR_UNSUPPORTED = 5,  /* option combination not implemented            */
    CBCT_ERR_BUSY = 6,         /* admission refused (budget or slots exhausted)  */
    CBCT_ERR_CANCELLED = 7     /* request cancelled before it ran                */
} cbct_status;

/* Scan and grid description (problem statement before Eq. 1: P^theta maps f onto
 * an imager at angle theta).  All sizes >= 1; spacings, dso, dsd > 0; the source
 * circle must clear the volume (dso > half diagonal of the xy extent) and the
 * imager must lie beyond it (dsd - dso > half diagonal).  nx*ny*nz and
 * n_angles*nu*nv must each be below 2^31. */
typedef struct {
    int nx, ny, nz;      /* voxels                                    */
    double hx, hy, hz;   /* voxel size, mm                            */
    int nu, nv;          /* imager pixels                             */
    double du, dv;       /* pixel pitch, mm                           */
    double dso, dsd;     /* source-to-axis, source-to-imager (L0), mm */
} cbct_geometry_desc;

typedef struct cbct_geometry cbct_geometry;

/* Solver options for cbct_reconstruct.  A zero-initialised struct selects the
 * defaults given in brackets. */
typedef struct {
    double beta;          /* Algorithm A1's beta for every level; 0 -> per level
                             max(10 mu, 1.05 gamma lambda_max(P^T P)) [auto]      */
    const double *betas;  /* optional host [levels], index 0 = finest; overrides beta */
    double eps;           /* TV smoothing, mm^-2; 0 -> 2e-5 / min(h) per level    */
    int inner_iters;      /* M gradient steps of step 2; 0 -> 10                  */
    int clamp_mode;       /* 0: f >= 0 enforced in every inner step from f_k [default];
                             1: step 2 descends from g without the bound and step 3
                             clamps afterwards (Algorithm A1 read literally)      */
    int sino_fp16;        /* 1: keep the projection data in half precision on the
                             device (the input stays float32)                    */
    int power_iters;      /* power iterations for the automatic beta; 0 -> 30     */
    int start_level;      /* resume: first (coarsest) level to run; 0 -> levels-1
                             with f_init ignored; otherwise f_init seeds it        */
    const float *f_init_dev; /* optional initial volume of level start_level, in
                             that level's [nz][ny][nx] layout (see cbct_level_dims) */
    int use_graphs;       /* 1: replay each FBS iteration as a captured CUDA graph */
    double *energy_trace; /* optional host out [levels][iters][3]: E, E1, mu*E2 of
                             the iterate entering each iteration, coarsest level
                             first; levels not run are left untouched.  Filling it
                             synchronises the stream once per level.              */
    double *beta_out;     /* optional host out [levels]: beta used per level      */
    float *kernel_ms;     /* optional host out [CBCT_NUM_KERNEL_CLASSES]: summed
                             device time per kernel class, measured with CUDA events
                             on `stream` (synchronises at the end of the call)    */
    int *kernel_launches; /* optional host out [CBCT_NUM_KERNEL_CLASSES]: kernels
                             launched per class                                    */
    unsigned kernel_mask; /* kernel classes (bit c: class c) that kernel_ms times with
                             events around each launch; 0 -> all.  Launches of every
                             class are counted.  Timing fewer classes keeps the event
                             overhead out of the others.                         */
    int reuse_lambda;     /* 1: reuse lambda_max(P^T P) of a level computed by an
                             earlier call on this geometry with the same power_iters
                             (the estimate is deterministic, so results are unchanged) */
    int tv_mode;          /* E1 of Eq. 1: 0 isotropic sum_j sqrt(|grad f|_j^2 + eps^2)
                             [default]; 1 anisotropic sum_j sum_d sqrt((D_d f)_j^2 + eps^2)
                             (the l1 norm of the gradient taken per axis)        */
    int adjoint_mode;     /* the adjoint in step 1 of Algorithm A1: 0 the exact transpose
                             P^T [default]; 1 the voxel-driven interpolation of Eq. 2
                             (see cbct_backproject_eq2).  The automatic beta always
                             comes from lambda_max(P^T P).                        */
    int mg_cycle;         /* multigrid: 0 the coarse-to-fine cascade [default]: `iters`
                             iterations of Algorithm A1 per level, coarsest first;
                             1 `iters` V-cycles from f = 0 (or f_init with start_level
                             0) on the finest level: on level l, mg_pre iterations of
                             A1, then the coarse model E_{l+1}(x) - <lin, x> with
                             lin = grad E_{l+1}(R f) - Q^T(grad E_l(f) - lin_l) (R the
                             2x2x2 mean, Q the trilinear prolongation) reduced by a cycle
                             on level l+1 (mg_coarse iterations of A1 on the coarsest),
                             the correction f + Q(x - R f) clamped at 0 and kept when it
                             lowers the level's model, then mg_post iterations.  Needs
                             clamp_mode 0 and adjoint_mode 0; cbct_reconstruct only.
                             energy_trace then receives [iters][3]: E, E1, mu*E2 of the
                             finest iterate after each cycle.                     */
    int mg_pre, mg_post;  /* smoothing iterations per level; 0 -> 2 each             */
    int mg_coarse;        /* iterations on the coarsest level; 0 -> 10               */
    int *mg_accepted;     /* optional host out [levels]: coarse corrections kept     */
    double *step_trace;   /* optional host out [levels][iters]: |f_k+1 - f_k|_2 of each
                             iteration (float64 sum of float32 squares), coarsest
                             level first, like energy_trace; with mg_cycle 1,
                             [iters]: the change of the finest iterate over each cycle */
    int serial_power;     /* 1: the power iterations of the finer levels of a cascade run
                             in level order on `stream`; 0 [default]: they run on a
                             side stream of the geometry while the coarser levels iterate
                             (they depend on the geometry alone; the same results)     */
    float *kernel_ms_finest; /* optional host out [CBCT_NUM_KERNEL_CLASSES]: like
                             kernel_ms, over the finest level's Algorithm A1 iterations
                             alone (no other stream's work runs beside them)           */
    int *kernel_launches_finest; /* optional host out [CBCT_NUM_KERNEL_CLASSES]         */
    float *level_ms;      /* optional host out [levels], index 0 = finest: device time of
                             each level's Algorithm A1 iterations, from one pair of CUDA
                             events on `stream` around them (no event per launch, so the
                             run is otherwise unchanged; synchronises at the end of the
                             call).  The finest level runs after every power iteration
                             has finished, so nothing else shares its window; a coarser
                             level's window may also hold finer levels' power iterations
                             running on the geometry's side stream.  Cascade only.      */
} cbct_options;

/* Kernel classes reported through cbct_options.kernel_ms. */
enum {
    CBCT_K_PROJECT = 0,     /* forward projection + residual          */
    CBCT_K_BACKPROJECT = 1, /* adjoint gather + gradient step         */
    CBCT_K_TV = 2,          /* TV prox sweeps with f >= 0             */
    CBCT_K_REDUCE = 3,      /* float64 reductions and small kernels   */
    CBCT_K_TRANSFER = 4,    /* multigrid transfers and layout changes */
    CBCT_NUM_KERNEL_CLASSES = 5
};

/* Create a geometry for the given angles (host, radians, n_angles >= 1) on the
 * current CUDA device.  Device tables derived from it (ray parameters per view and
 * detector column, per detector pixel) are computed in float64 on the host and
 * stored in float32.  On success *out owns them. */
cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, const double *angles_host,
                                 int n_angles, cbct_geometry **out);
void cbct_geometry_destroy(cbct_geometry *geom);

/* Sizes of multigrid level `level` (0 = the geometry itself): n_l = ceil(n / 2^l),
 * spacing 2^l h, imager ceil(nu / 2^l) x ceil(nv / 2^l) at pitch 2^l du.  dims_out
 * receives {nx, ny, nz, nu, nv}. */
cbct_status cbct_level_dims(const cbct_geometry *geom, int level, int dims_out[5]);

/* Forward projection P^theta for every angle (problem statement before Eq. 1):
 * y = P f with P the exact intersection-length (Siddon) operator, y[ray] =
 * sum_j |ray ∩ voxel_j| f_j.  f_dev: volume; y_dev: sinogram (written). */
cbct_status cbct_project(cbct_geometry *geom, const float *f_dev, float *y_dev, cudaStream_t stream);

/* Adjoint f = P^T y: the exact matrix transpose of cbct_project, i.e. the
 * sum over theta of P^theta^T named before Eq. 2, computed voxel by voxel as a
 * gather over the rays that meet each voxel (the voxel-driven form of Eq. 2) with
 * the same intersection lengths, in a fixed order and without atomics.
 * y_dev: sinogram; f_dev: volume (written). */
cbct_status cbct_backproject(cbct_geometry *geom, const float *y_dev, float *f_dev, cudaStream_t stream);

/* The variation of E2 as Eq. 2 evaluates it, as an operator on projection stacks:
 *   f_j = dV / (du dv) * sum_theta L^3 / (L0 l^2) * y_theta(u*, v*)
 * for every voxel centre x_j, where (u*, v*) is the imager point on the line from the
 * source through x_j, l = |x_j - source|, L = |(u*, v*) - source|, L0 = dsd, and
 * y_theta(u*, v*) interpolates y bilinearly between pixel centres (zero outside the
 * pixel grid).  The factor dV / (du dv) makes it an approximation of P^T y (Eq. 2
 * times Nv with A = nu nv du dv); it is not its exact transpose.
 * y_dev: sinogram; f_dev: volume (written). */
cbct_status cbct_backproject_eq2(cbct_geometry *geom, const float *y_dev, float *f_dev, cudaStream_t stream);

/* Steps 2 and 3 of Algorithm A1 on the geometry's grid: inner_iters projected
 * gradient steps on TV_eps(f) + beta/2 |f - g|^2 over f >= 0, starting from the
 * volume in f_inout_dev, step 1/(beta + (4/eps) sum_d h_d^-2).  TV_eps is the
 * forward-difference TV with Neumann boundary (E1 of Eq. 1): tv_mode 0 isotropic,
 * sqrt(|grad f|^2 + eps^2) per voxel; tv_mode 1 anisotropic, sum over the axes of
 * sqrt((D_d f)^2 + eps^2).  Every output voxel is >= +0.0.  g_dev: volume. */
cbct_status cbct_tv_prox(cbct_geometry *geom, const float *g_dev, float *f_inout_dev, double beta,
                         double eps, int inner_iters, int tv_mode, cudaStream_t stream);

/* Algorithm A1 on a single grid (the geometry's own), `iters` iterations from the
 * volume in f_inout_dev:
 *   g = f - (gamma/beta) P^T (P f - Y),  gamma = 2 mu Nv / (n_angles nu nv)
 *   f = step 2 and 3 as in cbct_tv_prox (clamp_mode, tv_mode as in cbct_options)
 * beta must be > 0 (no automatic choice here).  Y_dev: measured sinogram.
 * energy_trace: optional host [iters][3] (E, E1, mu*E2 of each entering iterate);
 * step_trace: optional host [iters], |f_k+1 - f_k|_2 of each iteration.  Either one
 * synchronises the stream once at the end. */
cbct_status cbct_fbs(cbct_geometry *geom, const float *Y_dev, double mu, double beta, double eps,
                     int inner_iters, int clamp_mode, int tv_mode, int iters, float *f_inout_dev,
                     double *energy_trace, double *step_trace, cudaStream_t stream);

/* Largest eigenvalue of P^T P by `iters` power iterations from a seeded uniform(0,1)
 * volume (value of voxel a, in [nz][ny][nx] order: the top 24 bits of SplitMix64 with
 * seed 10023675 at counter a, over 2^24);
 * the estimate is the Rayleigh quotient of the last normalised iterate.  Writes
 * *lambda_out (host) and synchronises the stream. */
cbct_status cbct_power_iteration(cbct_geometry *geom, int iters, double *lambda_out, cudaStream_t stream);

/* Energy of Eq. 1 on the grid, float64: out_host = {E, E1, mu*E2} with
 * E1 = TV_eps(f) / Nv (tv_mode as in cbct_options) and
 * E2 = |P f - Y|^2 / (n_angles nu nv).  eps >= 0: eps = 0 gives the unsmoothed TV
 * (sum of |grad f|).  Synchronises. */
cbct_status cbct_energy(cbct_geometry *geom, const float *Y_dev, const float *f_dev, double mu,
                        double eps, int tv_mode, double out_host[3], cudaStream_t stream);

/* Full reconstruction (Eq. 1 by Algorithm A1 with multigrid): for level
 * l = levels-1 .. 0 (coarsest first) the data are the 2x2-binned sinogram of the
 * finer level, the start is 0 on the coarsest level and the cell-centred trilinear
 * prolongation of the coarser result elsewhere, and `iters` iterations of A1 run
 * per level.  angles_host must equal the geometry's angles (n_angles of them).
 * Y_dev: measured sinogram of the finest level; f_out_dev: volume (written).
 * levels >= 1 with n >= 2^(levels-1) on every axis of volume and imager. */
cbct_status cbct_reconstruct(cbct_geometry *geom, const float *Y_dev, const double *angles_host,
                             int n_angles, double mu, int iters, int levels, const cbct_options *opts,
                             float *f_out_dev, cudaStream_t stream);

/* Multigrid transfers on caller buffers (layouts as above).
 * cbct_restrict_sino: y_coarse[t][b][a] = mean of y over the existing pixels of
 *   the 2x2 block {2b, 2b+1} x {2a, 2a+1}; output [n_angles][ceil nv/2][ceil nu/2].
 * cbct_prolong_vol: cell-centred trilinear interpolation of the coarse volume
 *   (spacing 2h) at the fine voxel centres, indices clamped at the edges. */
cbct_status cbct_restrict_sino(int n_angles, int nv, int nu, const float *y_dev, float *y_coarse_dev,
                               cudaStream_t stream);
cbct_status cbct_prolong_vol(int nxc, int nyc, int nzc, const float *fc_dev, int nx, int ny, int nz,
                             float *f_dev, cudaStream_t stream);

/* Batched reconstruction (many independent reconstructions, as in a serving batch).
 * Each request is a cbct_reconstruct call; all of them advance together, one
 * Algorithm A1 iteration (or power-iteration step) per tick, every stage of every
 * request in one persistent launch per stage.  Each request's volume, energy trace
 * and betas are bitwise the same as those of its own cbct_reconstruct call.  Every
 * request needs its own geometry handle.  Synchronous: returns when all volumes are
 * written.  use_graphs: replay ticks whose stages repeat as captured CUDA graphs
 * (needs a stream other than 0).  Options honoured per request: as cbct_reconstruct,
 * except kernel_ms / kernel_launches / use_graphs (ignored). */
typedef struct {
    cbct_geometry *geom;
    const float *Y_dev;       /* finest-level sinogram [n_angles][nv][nu]            */
    double mu;
    int iters, levels;
    const cbct_options *opts; /* nullable                                           */
    float *f_out_dev;         /* volume [nz][ny][nx], written                        */
} cbct_request;
cbct_status cbct_reconstruct_batch(const cbct_request *reqs, int n_reqs, int use_graphs, cudaStream_t stream);

/* Launch shapes of one level (0 = the library's default); they change no bit of any
 * volume (the float64 energy and step-norm sums may differ in their last bits, as the
 * partial sums are grouped by tile). */
typedef struct {
    int proj_threads;  /* projector block size: multiple of 32, >= 32 ceil(nv/32), <= 512 */
    int bp_vpl;        /* adjoint voxels per lane, 1..4                                */
    int bp_threads;    /* adjoint block size: 64, 128 or 256                           */
    float proj_ms;     /* autotune: measured time of one projection with the choice    */
    float bp_ms;       /* autotune: measured time of one adjoint with the choice       */
    int proj_smem;     /* projector shared memory per block in bytes (multiple of 16, at
                          most 110 KB); sets how many z-levels one pass holds          */
    int proj_levels;   /* z-levels per projector launch, 1..nz: a projection of a volume
                          larger than the L2 cache runs as consecutive launches over
                          slabs of levels, each ray's sum carried between them        */
    int bp_layout;     /* adjoint lane layout: 1 consecutive voxels per lane, 2 interleaved
                          (0: interleaved when a warp's gathers would span 400 or more
                          detector rows)                                              */
    int tv_sweeps;     /* TV prox of levels with z-columns of at most 96 voxels: prox sweeps
                          fused per x-marching launch, 1 or 2 (0: 2); -1 selects the
                          one-sweep-per-launch warp tiles instead (same volume bits)   */
    int tv_warps;      /* x-marching TV: warps per block, 16 or 32 (0: 32 for two sweeps,
                          16 for one); the block's output rows are warps - 2 sweeps + 1 */
    int tv_planes;     /* x-marching TV: x-planes per block, >= 8 (0: from the size)   */
} cbct_tuning;
/* Time the candidate launch shapes of level `level` with CUDA events on `stream`
 * (synchronises), keep the fastest in the geometry and report it in *out. */
cbct_status cbct_autotune(cbct_geometry *geom, int level, cbct_tuning *out, cudaStream_t stream);
/* Apply launch shapes (e.g. from a cache of earlier autotune results). */
cbct_status cbct_set_tuning(cbct_geometry *geom, int level, const cbct_tuning *tuning);

/* Continuous-batching server.  A worker thread owns a stream and max_slots slots;
 * a slot keeps one geometry (tables and workspaces) resident and serves one request
 * at a time, and later requests with the same scan geometry reuse it.  Requests are
 * admitted in arrival order whenever a slot is free, the device memory of the
 * geometries in use stays within hbm_budget_bytes (idle geometries are released,
 * least recently used first) and the running requests do not already fill the GPU
 * (each is rated by the share of the SMs its finest-level adjoint keeps busy; a new
 * request joins while the shares sum to less than one).  Admitted requests join the
 * running batch between iterations, so small requests that arrive while others run
 * overlap on the device and large ones are served first come, first served; each
 * result is bitwise the one cbct_reconstruct gives for the same request.  The
 * server uses the device that is current when it is created. */
typedef struct cbct_server cbct_server;
typedef struct {
    cbct_geometry_desc desc;  /* scan and grid                                        */
    const double *angles_host;/* n_angles radians, copied at submit                    */
    int n_angles;
    const float *Y_dev;       /* sinogram [n_angles][nv][nu]; valid until completion    */
    double mu;
    int iters, levels;
    cbct_options opts;        /* as for cbct_reconstruct; betas copied at submit;
                                 energy_trace, beta_out, kernel_ms, level_ms ignored   */
    float *f_out_dev;         /* volume [nz][ny][nx]; written before completion        */
} cbct_server_request;
typedef struct {
    cbct_status status;       /* CBCT_OK, or the error that ended the request          */
    double latency_s;         /* submit to completion                                  */
    double queue_s;           /* submit to admission                                   */
    double betas[8];          /* beta used per level (index 0 = finest)                */
} cbct_result;
typedef struct {
    int queued, running, slots_in_use;
    uint64_t completed;
    size_t hbm_in_use;        /* bytes held by resident geometries                     */
    double busy_s;            /* worker time spent issuing and waiting for device work */
} cbct_server_stats;
cbct_status cbct_server_create(size_t hbm_budget_bytes, int max_slots, int use_graphs, cbct_server **out);
/* Queue a request (returns at once).  Malformed requests: CBCT_ERR_INVALID_ARG;
 * requests that could never fit the budget: CBCT_ERR_BUSY. */
cbct_status cbct_server_submit(cbct_server *srv, const cbct_server_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (< 0: no limit) for a ticket; CBCT_ERR_TIMEOUT if it has not
 * finished (the ticket stays valid).  Returns the request's status and fills
 * *result (nullable); a ticket can be collected once. */
cbct_status cbct_server_wait(cbct_server *srv, uint64_t ticket, int timeout_ms, cbct_result *result);
/* Cancel a request that is still queued (CBCT_ERR_BUSY if it already runs). */
cbct_status cbct_server_cancel(cbct_server *srv, uint64_t ticket);
cbct_status cbct_server_get_stats(cbct_server *srv, cbct_server_stats *out);
/* Finish running requests, cancel queued ones, release everything. */
void cbct_server_destroy(cbct_server *srv);
/* Test hook: the next n geometry set-ups inside the server fail as if out of memory
 * (no device memory is touched), so failure handling can be exercised safely. */
void cbct_debug_fail_next_allocations(int n);

/* Largest volume (nx*ny*nz) that cbct_tv_energy_noalloc accepts. */
#define CBCT_NOALLOC_MAX_VOXELS 33554432

/* E1 energy of a volume without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc --
 * real-time or embedded hosts that forbid allocation after start-up, plug-ins that
 * must leave the device heap alone -- and therefore cannot create a cbct_geometry.
 * Writes *e1_dev = TV_eps(f) / (nx ny nz) (device float64, isotropic; same
 * definition and value as element 1 of cbct_energy with tv_mode 0; eps >= 0, eps = 0
 * the unsmoothed TV) for f_dev, a [nz][ny][nx] float32 device volume (4-byte
 * aligned) with spacings hx, hy, hz.  Asynchronous on `stream`.
 * Scratch: a 1 MiB array inside the library, reserved on every GPU that loads the
 * library until the process exits; hence volumes above CBCT_NOALLOC_MAX_VOXELS are
 * rejected with CBCT_ERR_INVALID_ARG.  The first call on a device looks up that
 * array's device address (with that device current); make that first call before
 * any stream capture.  The address is kept for the life of the process: after a
 * device reset (cudaDeviceReset) it is stale, and this entry point must not be called
 * on that device again.  Calls share the array: calls that may overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
cbct_status cbct_tv_energy_noalloc(int nx, int ny, int nz, double hx, double hy, double hz, double eps,
                                   const float *f_dev, double *e1_dev, cudaStream_t stream);

/* Thread-local description of the last error on the calling thread. */
const char *cbct_last_error(void);

/* Library version string. */
const char *cbct_version(void);

/* Kernels launched through the library by this process so far (every launch site
 * counts itself; a captured graph replay adds nothing).  Never fails. */
unsigned long long cbct_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* CBCT_H */
