// Batched reconstruction: many requests advance together, one Algorithm A1
// iteration (or one power-iteration step) per tick.  A stage of a request that fills
// the GPU by itself (enough tiles for several waves) runs as its own single-request
// launch; the stages of the smaller requests share one persistent launch per stage,
// sized to the blocks that stay resident on every SM.
//
// Each persistent launch reads a device table of per-request items (geometry block,
// buffers, mode) and a prefix table of per-request tile counts; a block (or warp)
// maps its global tile index to (request, local tile) and runs the same tile body as
// the single-request kernels.  Every request is computed with exactly the arithmetic of
// a single-request call, in the same order, so its result is bitwise the same alone
// and in any mix.  The item tables are rebuilt only when the set of active stages
// changes; while it does not, a tick's launches can be replayed as a CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "batch.h"
#include "bp_eq2_tile.cuh"
#include "bp_tile.cuh"
#include "project_tile.cuh"
#include "step_tile.cuh"
#include "tv_tile.cuh"

namespace cbct {

// ---------------------------------------------------------------------------------
// batched kernels
// ---------------------------------------------------------------------------------

// largest r with start[r] <= t
__device__ __forceinline__ int find_item(const long *__restrict__ start, int n, long t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void copy_words(void *dst, const void *src, int bytes, int lane, int nthreads) {
    const int *s = (const int *)src;
    int *d = (int *)dst;
    for (int q = lane; q < bytes / 4; q += nthreads) d[q] = s[q];
}

__global__ void __launch_bounds__(PROJ_MAX_THREADS, 2)
k_project_batch(const ProjItem *__restrict__ items, const long *__restrict__ start, int n, long total) {
    extern __shared__ float smem[];
    __shared__ ProjItem it;
    int cur = -1;
    long first = 0, next = 0;
    for (long t = blockIdx.x; t < total; t += gridDim.x) {
        if (cur < 0 || t >= next) {  // the item changes rarely along a block's tiles
            const int r = find_item(start, n, t);
            copy_words(&it, items + r, sizeof(ProjItem), threadIdx.x, blockDim.x);
            __syncthreads();
            cur = r;
            first = __ldg(start + r);
            next = r + 1 < n ? __ldg(start + r + 1) : total;
        }
        const long local = t - first;
        const int a = (int)(local % it.G.nu);
        const long rest = local / it.G.nu;
        const int ia = (int)(rest % it.G.na), zc = (int)(rest / it.G.na);
        project_tile(it.G, it.mode, it.vol, it.y32, it.y16, it.out, it.partial, a, ia, zc, smem);
        __syncthreads();
    }
}

template <int VPL>
__global__ void __launch_bounds__(BP_THREADS, 8)
k_bp_batch(const BpItem *__restrict__ items, const long *__restrict__ start, int n, long total) {
    __shared__ BpItem it[BP_THREADS / 32];
    __shared__ float4 rec[(BP_THREADS / 32) * BP_REC_PER_WARP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long stride = (long)gridDim.x * (BP_THREADS / 32);
    int cur = -1;
    long first = 0, next = 0;
    for (long t = (long)blockIdx.x * (BP_THREADS / 32) + w; t < total; t += stride) {
        if (cur < 0 || t >= next) {  // the item changes rarely along a warp's tiles
            const int r = find_item(start, n, t);
            __syncwarp();
            copy_words(&it[w], items + r, sizeof(BpItem), lane, 32);
            __syncwarp();
            cur = r;
            first = __ldg(start + r);
            next = r + 1 < n ? __ldg(start + r + 1) : total;
        }
        // consecutive layout for every item (the interleaved one gives the same bits)
        bp_warp<VPL, false>(it[w].G, it[w].mode, it[w].rs, it[w].fin, it[w].out, it[w].c, t - first,
                            rec + w * BP_REC_PER_WARP);
    }
}

__global__ void __launch_bounds__(EQ2_THREADS)
k_eq2_batch(const Eq2Item *__restrict__ items, const long *__restrict__ start, int n, long total) {
    __shared__ Eq2Item it;
    for (long t = blockIdx.x; t < total; t += gridDim.x) {
        const int r = find_item(start, n, t);
        copy_words(&it, items + r, sizeof(Eq2Item), threadIdx.x, blockDim.x);
        __syncthreads();
        eq2_block(it.G, it.r, false, it.fin, it.out, it.cscale, it.mode, t - start[r]);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TV_THREADS)
k_tv_batch(const TvItem *__restrict__ items, const long *__restrict__ start, int n, long total) {
    __shared__ TvItem it;
    __shared__ long first;
    int cur = -1;
    for (long t = blockIdx.x; t < total; t += gridDim.x) {
        // the item changes rarely along a block's tiles: look it up only when it does
        const int r = (cur >= 0 && t >= first && (cur + 1 >= n || t < __ldg(start + cur + 1))) ? cur
                                                                                            : find_item(start, n, t);
        if (r != cur) {
            __syncthreads();
            copy_words(&it, items + r, sizeof(TvItem), threadIdx.x, blockDim.x);
            if (threadIdx.x == 0) first = start[r];
            cur = r;
            __syncthreads();
        }
        const long blk = t - first;
        // (a step-norm sweep is the last of its prox, which always clamps)
        if (it.clamp) {
            if (it.acc == TV_ACC_E1) tv_block<true, TV_ACC_E1>(it.A, it.fin, it.g, it.fout, it.partial, blk);
            else if (it.acc == TV_ACC_STEP) tv_block<true, TV_ACC_STEP>(it.A, it.fin, it.g, it.fout, it.partial, blk);
            else tv_block<true, TV_ACC_NONE>(it.A, it.fin, it.g, it.fout, it.partial, blk);
        } else {
            if (it.acc == TV_ACC_E1) tv_block<false, TV_ACC_E1>(it.A, it.fin, it.g, it.fout, it.partial, blk);
            else tv_block<false, TV_ACC_NONE>(it.A, it.fin, it.g, it.fout, it.partial, blk);
        }
        __syncthreads();
    }
}

// per-block partials of <x, y> and <y, y> (same partition and arithmetic as k_dot2)
__global__ void __launch_bounds__(VEC_THREADS)
k_dot_batch(const VecItem *__restrict__ items, const long *__restrict__ start, int n, long total) {
    for (long t = blockIdx.x; t < total; t += gridDim.x) {
        const int r = find_item(start, n, t);
        const VecItem it = items[r];
        dot2_tile(it.x, it.y, it.n, t - start[r], it.partial);
    }
}

__global__ void k_pfin_batch(const VecItem *__restrict__ items) {
    const VecItem it = items[blockIdx.x];
    __shared__ double sh1[256], sh2[256];
    double s1 = 0.0, s2 = 0.0;
    for (int q = threadIdx.x; q < it.nblk; q += 256) {
        s1 += it.partial[2 * q];
        s2 += it.partial[2 * q + 1];
    }
    sh1[threadIdx.x] = s1;
    sh2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
            sh2[threadIdx.x] += sh2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *it.lam = sh1[0];
        *it.scale = sh2[0] > 0.0 ? (float)(1.0 / sqrt(sh2[0])) : 0.f;
    }
}

__global__ void __launch_bounds__(VEC_THREADS)
k_scale_batch(const VecItem *__restrict__ items, const long *__restrict__ start, int n, long total) {
    for (long t = blockIdx.x; t < total; t += gridDim.x) {
        const int r = find_item(start, n, t);
        const VecItem it = items[r];
        scale_tile(it.y, it.scale, it.out, it.n, t - start[r]);
    }
}

// The same sums and trace entries as the single-request energy finalisation.
__global__ void __launch_bounds__(ENERGY_THREADS) k_energy_batch(const EnItem *__restrict__ items) {
    const EnItem it = items[blockIdx.x];
    __shared__ double sums[3];
    sum3_fixed(it.pe2, it.n2, it.pe1, it.n1, it.pstep, it.nstep, sums);
    const double q = sums[0], t = sums[1], d = sums[2];
    if (threadIdx.x == 0) {
        const int k = *it.counter;
        const double e1 = t * it.inv_nv, e2 = q * it.mu_over_nr;
        it.trace[TRACE_W * k + 0] = e1 + e2;
        it.trace[TRACE_W * k + 1] = e1;
        it.trace[TRACE_W * k + 2] = e2;
        it.trace[TRACE_W * k + 3] = sqrt(d);
        *it.counter = k + 1;
    }
}

// Step-norm copies of many requests: one 256-voxel block per tile.
__global__ void __launch_bounds__(STEP_THREADS)
k_step_batch(const StepItem *__restrict__ items, const long *__restrict__ start, int n, long total) {
    for (long t = blockIdx.x; t < total; t += gridDim.x) {
        const int r = find_item(start, n, t);
        const StepItem it = items[r];
        step_block(it.v, it.f, (size_t)it.n, it.partial, (size_t)(t - start[r]));
    }
}

// ---------------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------------

// Step-norm partials of one Algorithm A1 iteration of job j on level L (the rule of
// the single-request path: fused into the last sweep unless M == 1 from f_k).
static bool job_step_fused(const Job *j, const Level *L) {
    return prox_step_fused(j->P.M, j->P.clamp_mode == 0 ? L->f : L->g, L->f);
}
// The x-marching prox plan of job j's current iteration (levels in that form).
static XProxPlan job_xplan(const Job *j, Level *L) {
    return xprox_plan(tv_args(L, j->P), j->P.M, j->P.clamp_mode, j->P.clamp_mode == 0 ? L->f : L->g, L->f, L->A,
                      L->B, j->P.clamp_mode == 0, true, vol_elems(L->gd));
}
static int job_nstep(const Job *j, Level *L) {
    if (tv_args(L, j->P).xT > 0) return job_xplan(j, L).n_step;
    return (int)(job_step_fused(j, L) ? tv_partials(L->nx, L->ny, L->nz) : step_partials(vol_elems(L->gd)));
}
// E1 partials of job j's iteration (literal clamp mode: the separate energy pass)
static int job_ne1(const Job *j, Level *L) {
    if (j->P.clamp_mode == 1) return (int)tv_energy_partials(L->nx, L->ny, L->nz);
    if (tv_args(L, j->P).xT > 0) return job_xplan(j, L).n_e1;
    return (int)tv_partials(L->nx, L->ny, L->nz);
}

// A TV sweep that fills the GPU by itself, or uses full-column tiles (which the batched
// kernel does not carry), runs as a single-request launch.
static bool tv_sweep_solo(int nx, int ny, int nz, long sms) {
    return (long)tv_blocks(nx, ny, nz) >= 16 * sms || tv_col_vz(nx, ny, nz) > 0;
}

static int sm_count() { return device_sm_count(); }

#define ECK(call, what)                                      \
    do {                                                     \
        cudaError_t e__ = (call);                            \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)
#define EST(call)                        \
    do {                                 \
        cbct_status s__ = (call);        \
        if (s__ != CBCT_OK) return s__;  \
    } while (0)

Engine::Engine(cudaStream_t s, bool graphs) : stream(s), use_graphs(graphs && s != 0) {}

Engine::~Engine() {
    reset_graph();
    cudaFree(dblob);
    for (cudaStream_t st : side) cudaStreamDestroy(st);
    for (cudaEvent_t e : side_events) cudaEventDestroy(e);
}

void Engine::reset_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    same_ticks = 0;
}

cbct_status Engine::add(Job *j) {
    if (!j || !j->G) {
        set_error("engine: null job or geometry");
        return CBCT_ERR_INVALID_ARG;
    }
    for (Job *o : jobs)
        if (o->G == j->G) {
            set_error("engine: two jobs in flight on the same geometry");
            return CBCT_ERR_INVALID_ARG;
        }
    j->phase = PH_PREPARE;
    jobs.push_back(j);
    signature.clear();
    return CBCT_OK;
}

void Engine::remove_finished() {
    const size_t before = jobs.size();
    jobs.erase(std::remove_if(jobs.begin(), jobs.end(), [](Job *j) { return j->phase == PH_DONE; }), jobs.end());
    if (jobs.size() != before) signature.clear();
}

// Per-job work outside the batched stages: data pyramid, level start.
cbct_status Engine::prepare(Job *j) {
    cbct_geometry *G = j->G;
    const cbct_options &o = j->o;
    j->M = o.inner_iters > 0 ? o.inner_iters : 10;
    j->K = o.power_iters > 0 ? o.power_iters : 30;
    j->fp16 = o.sino_fp16 != 0;
    j->Ls.assign(j->levels, nullptr);
    for (int l = 0; l < j->levels; ++l) {
        EST(ensure_level(G, l, &j->Ls[l]));
        EST(ensure_workspace(j->Ls[l], j->fp16));
    }
    EST(ensure_trace(G, 0));
    double *dtrace;
    EST(get_trace(G, TRACE_W * (size_t)std::max(j->iters, 1), &dtrace));
    const GeoDev &g0 = j->Ls[0]->gd;
    ECK(launch_sino_to_internal(j->Y, j->Ls[0]->Y, j->fp16 ? j->Ls[0]->Yh : nullptr, nullptr, g0.na, g0.nu, g0.nv,
                                stream),
        "sinogram layout");
    for (int l = 1; l < j->levels; ++l) {
        const GeoDev &gp = j->Ls[l - 1]->gd;
        ECK(launch_restrict(j->Ls[l - 1]->Y, j->Ls[l]->Y, gp.na, gp.nu, gp.nv, stream), "restriction");
        if (j->fp16) ECK(launch_to_half(j->Ls[l]->Y, j->Ls[l]->Yh, sino_elems(j->Ls[l]->gd), stream), "half copy");
    }
    j->level = o.f_init_dev ? o.start_level : j->levels - 1;
    j->phase = PH_START_LEVEL;
    return CBCT_OK;
}

cbct_status Engine::start_level(Job *j) {
    Level *L = j->Ls[j->level];
    const GeoDev &g = L->gd;
    const bool first = (j->level == (j->o.f_init_dev ? j->o.start_level : j->levels - 1));
    if (first) {
        if (j->o.f_init_dev)
            ECK(launch_vol_to_internal(j->o.f_init_dev, L->f, g.nx, g.ny, g.nz, stream), "volume layout");
        else
            ECK(cudaMemsetAsync(L->f, 0, vol_elems(g) * 4, stream), "zero start");
    } else {
        const GeoDev &gc = j->Ls[j->level + 1]->gd;
        ECK(launch_prolong(j->Ls[j->level + 1]->f, gc.nx, gc.ny, gc.nz, L->f, g.nx, g.ny, g.nz, stream),
            "prolongation");
    }
    double beta = 0.0;
    if (j->o.betas) beta = j->o.betas[j->level];
    else if (j->o.beta > 0) beta = j->o.beta;
    if (beta > 0) return begin_fbs(j, beta);
    if (j->o.reuse_lambda && L->lambda_iters == j->K)
        return begin_fbs(j, std::max(10.0 * j->mu, 1.05 * gamma_of(L, j->mu) * L->lambda));
    // the start x = u / |u| in L->A, with the kernels of the single-request path
    ECK(launch_fill_uniform(L->B, g.nx, g.ny, g.nz, POWER_SEED, stream), "start volume");
    int nb = 0;
    ECK(launch_dot2(L->B, L->B, vol_elems(g), L->partial, stream, &nb), "dot");
    ECK(launch_power_finalize(L->partial, nb, j->G->dscalars, (float *)(j->G->dscalars + 1), stream),
        "power finalize");
    ECK(launch_scale(L->B, (float *)(j->G->dscalars + 1), L->A, vol_elems(g), stream), "scale");
    j->pi_it = 0;
    j->phase = PH_POWER;
    return CBCT_OK;
}

cbct_status Engine::begin_fbs(Job *j, double beta) {
    Level *L = j->Ls[j->level];
    j->beta = beta;
    if (j->o.beta_out) j->o.beta_out[j->level] = beta;
    const double eps = j->o.eps > 0 ? j->o.eps : default_eps(L);
    EST(solve_params(L, j->mu, beta, eps, j->M, j->o.clamp_mode, j->fp16, &j->P, j->o.tv_mode, j->o.adjoint_mode));
    ECK(cudaMemsetAsync(j->G->dcounter, 0, sizeof(int), stream), "counter reset");
    j->it = 0;
    j->phase = j->iters > 0 ? PH_FBS : PH_LEVEL_DONE;
    return CBCT_OK;
}

cbct_status Engine::finish_level(Job *j) {
    Level *L = j->Ls[j->level];
    if ((j->o.energy_trace || j->o.step_trace) && j->iters > 0) {
        const size_t lv = (size_t)j->iters * (j->levels - 1 - j->level);
        EST(copy_trace(j->G->dtrace, j->iters, j->o.energy_trace ? j->o.energy_trace + 3 * lv : nullptr,
                       j->o.step_trace ? j->o.step_trace + lv : nullptr, stream));
        ECK(cudaStreamSynchronize(stream), "trace");
    }
    if (j->level == 0) {
        const GeoDev &g = L->gd;
        ECK(launch_vol_to_api(L->f, j->f_out, g.nx, g.ny, g.nz, stream), "volume layout");
        j->phase = PH_DONE;
        j->done_event_pending = true;
        return CBCT_OK;
    }
    j->level -= 1;
    j->phase = PH_START_LEVEL;
    return CBCT_OK;
}

// One TV item as a single-request launch (a sweep, or x-marching fused sweeps).
static cbct_status launch_tv_item(const TvItem &it, cudaStream_t s) {
    if (it.xT > 0) {
        ECK(launch_tv_x(it.A, it.xT, it.xclamp, it.fin, it.g, it.fout, it.acc == TV_ACC_E1 ? it.partial : nullptr,
                        it.acc == TV_ACC_STEP ? it.partial : nullptr, s, nullptr),
            "tv sweeps");
        return CBCT_OK;
    }
    ECK(launch_tv_sweep(it.A, it.fin, it.g, it.fout, it.clamp != 0, it.acc == TV_ACC_E1 ? it.partial : nullptr, s,
                        nullptr, it.acc == TV_ACC_STEP ? it.partial : nullptr),
        "tv sweep");
    return CBCT_OK;
}

// Rebuild the item tables for the current set of (job, phase) pairs.
cbct_status Engine::build_tables() {
    const size_t ALIGN = 256;
    auto align = [&](size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); };
    hproj.clear();
    for (auto &v : hbp) v.clear();
    hdot.clear();
    htv.clear();
    hen.clear();
    std::vector<long> pstart, dstart;
    std::vector<long> bpstart[4], eqstart;
    heq.clear();
    long eqtot = 0;
    std::vector<std::vector<long>> tvstart;
    long ptot = 0, dtot = 0, bptot[4] = {0, 0, 0, 0};
    std::vector<std::pair<ProjItem, long>> pitems;  // item, tiles
    solo_proj.clear();
    solo_bp.clear();
    solo_eq.clear();
    solo_tv.clear();
    chains.clear();
    const long sms = sm_count();
    max_m = 0;
    hstep.clear();
    std::vector<long> sstart;
    long stot = 0;
    tv_energy_jobs.clear();
    for (Job *j : jobs) {
        if (j->phase != PH_POWER && j->phase != PH_FBS) continue;
        Level *L = j->Ls[j->level];
        const GeoDev &g = L->gd;
        const bool power = j->phase == PH_POWER;
        ProjItem pi;
        pi.G = g;
        pi.vol = power ? L->A : L->f;
        pi.y32 = (!power && !j->fp16) ? L->Y : nullptr;
        pi.y16 = (!power && j->fp16) ? L->Yh : nullptr;
        pi.out = L->rs;
        pi.partial = power ? nullptr : L->partial;
        const bool eq2 = !power && j->P.adjoint_mode == 1;
        pi.mode = power ? PROJ_SCALED
                        : (j->fp16 ? (eq2 ? PROJ_RAW16 : PROJ_RESID16) : (eq2 ? PROJ_RAW32 : PROJ_RESID32));
        // a stage that fills the GPU by itself runs as its own single-request launch (the
        // same tile bodies, so the same bits); the others share a persistent launch
        const long ptiles = (long)g.nu * g.na * ((g.nv + project_threads(g) - 1) / project_threads(g));
        const int vpl0 = (g.bp_vpl >= 1 && g.bp_vpl <= 4) ? g.bp_vpl : bp_default_vpl(g);
        const long wt0 = vpl0 == 1 ? bp_warp_tiles<1>(g) : vpl0 == 2 ? bp_warp_tiles<2>(g)
                                                         : vpl0 == 3 ? bp_warp_tiles<3>(g) : bp_warp_tiles<4>(g);
        const long eblocks0 = eq2_tiles(g);
        const bool indep = ptiles >= 8 * sms && (eq2 ? eblocks0 >= 16 * sms : wt0 >= 64 * sms) &&
                           (power || tv_sweep_solo(g.nx, g.ny, g.nz, sms));
        if (indep) {  // the whole tick of this job on a side stream
            Chain ch;
            ch.job = j;
            ch.power = power;
            ch.eq2 = eq2;
            ch.proj = pi;
            if (eq2) {
                ch.eq.G = g;
                ch.eq.r = L->rs;
                ch.eq.fin = L->f;
                ch.eq.out = L->g;
                ch.eq.cscale = j->P.c_eq2;
                ch.eq.mode = BP_STEP;
            } else {
                ch.bp.G = g;
                ch.bp.rs = L->rs;
                ch.bp.fin = power ? nullptr : L->f;
                ch.bp.out = power ? L->B : L->g;
                ch.bp.c = power ? 0.f : j->P.c;
                ch.bp.mode = power ? BP_PLAIN : BP_STEP;
            }
            if (power) {
                ch.vec.x = L->A;
                ch.vec.y = L->B;
                ch.vec.out = L->A;
                ch.vec.partial = L->partial;
                ch.vec.lam = j->G->dscalars;
                ch.vec.scale = (float *)(j->G->dscalars + 1);
                ch.vec.n = (long)vol_elems(g);
                ch.vec.nblk = (int)vec_tiles(ch.vec.n);
            } else {
                max_m = std::max(max_m, j->P.M);
                const size_t np = project_partials(g);
                EnItem ei;
                ei.pe2 = L->partial;
                ei.n2 = (int)np;
                ei.pe1 = L->partial + np;
                ei.n1 = job_ne1(j, L);
                ei.pstep = step_region(L);
                ei.nstep = job_nstep(j, L);
                ei.inv_nv = j->P.inv_nv;
                ei.mu_over_nr = j->P.mu_over_nr;
                ei.trace = j->G->dtrace;
                ei.counter = j->G->dcounter;
                hen.push_back(ei);
            }
            chains.push_back(ch);
            continue;
        }
        if (ptiles >= 8 * sms) solo_proj.push_back(pi);
        else pitems.push_back({pi, ptiles});
        if (eq2) {
            Eq2Item ei;
            ei.G = g;
            ei.r = L->rs;
            ei.fin = L->f;
            ei.out = L->g;
            ei.cscale = j->P.c_eq2;
            ei.mode = BP_STEP;
            const long eblocks = eq2_tiles(g);
            if (eblocks >= 16 * sms) {
                solo_eq.push_back(ei);
            } else {
                heq.push_back(ei);
                eqstart.push_back(eqtot);
                eqtot += eblocks;
            }
        }
        const int vpl = (g.bp_vpl >= 1 && g.bp_vpl <= 4) ? g.bp_vpl : bp_default_vpl(g);
        if (!eq2) {
            BpItem bi;
            bi.G = g;
            bi.rs = L->rs;
            bi.fin = power ? nullptr : L->f;
            bi.out = power ? L->B : L->g;
            bi.c = power ? 0.f : j->P.c;
            bi.mode = power ? BP_PLAIN : BP_STEP;
            long wt = vpl == 1 ? bp_warp_tiles<1>(g) : vpl == 2 ? bp_warp_tiles<2>(g) : vpl == 3 ? bp_warp_tiles<3>(g)
                                                                                          : bp_warp_tiles<4>(g);
            if (wt >= 64 * sms) {
                solo_bp.push_back(bi);
            } else {
                hbp[vpl - 1].push_back(bi);
                bpstart[vpl - 1].push_back(bptot[vpl - 1]);
                bptot[vpl - 1] += wt;
            }
        }
        if (power) {
            VecItem vi;
            vi.x = L->A;
            vi.y = L->B;
            vi.out = L->A;
            vi.partial = L->partial;
            vi.lam = j->G->dscalars;
            vi.scale = (float *)(j->G->dscalars + 1);
            vi.n = (long)vol_elems(g);
            vi.nblk = (int)vec_tiles(vi.n);
            hdot.push_back(vi);
            dstart.push_back(dtot);
            dtot += vi.nblk;
        } else {
            max_m = std::max(max_m, j->P.M);
            if (j->P.clamp_mode == 1) tv_energy_jobs.push_back(j);
            const size_t np = project_partials(g);  // (jobs on side streams took the branch above)
            EnItem ei;
            ei.pe2 = L->partial;
            ei.n2 = (int)np;
            ei.pe1 = L->partial + np;
            ei.n1 = job_ne1(j, L);
            ei.pstep = step_region(L);
            ei.nstep = job_nstep(j, L);
            ei.inv_nv = j->P.inv_nv;
            ei.mu_over_nr = j->P.mu_over_nr;
            ei.trace = j->G->dtrace;
            ei.counter = j->G->dcounter;
            hen.push_back(ei);
        }
    }
    // projector items grouped by block size (the tile height of a request must be its
    // single-request value), one launch per group; resident blocks per SM from the
    // registers (64 per thread) and the group's largest shared-memory size
    std::stable_sort(pitems.begin(), pitems.end(), [](const std::pair<ProjItem, long> &x,
                                                      const std::pair<ProjItem, long> &y) {
        return project_threads(x.first.G) < project_threads(y.first.G);
    });
    pgroups.clear();
    for (const auto &it : pitems) {
        const int T = project_threads(it.first.G);
        if (pgroups.empty() || pgroups.back().threads != T) {
            ProjGroup pg;
            pg.threads = T;
            pg.first = (int)hproj.size();
            pgroups.push_back(pg);
            ptot = 0;
        }
        ProjGroup &pg = pgroups.back();
        pg.smem = std::max(pg.smem, proj_smem_of(it.first.G));
        pstart.push_back(ptot);
        hproj.push_back(it.first);
        ptot += it.second;
        pg.count += 1;
        pg.tiles = ptot;
    }
    for (ProjGroup &pg : pgroups)
        pg.blocks = std::max(1, std::min(65536 / (64 * pg.threads), (227 * 1024) / (pg.smem + 1024)));
    // TV sweeps: for each m, the jobs with m < M (ping-pong as in the single path)
    htv.assign(max_m, {});
    solo_tv.assign(max_m, {});
    tvstart.assign(max_m, {});
    tvtot.assign(max_m, 0);
    for (Job *j : jobs) {
        if (j->phase != PH_FBS) continue;
        Level *L = j->Ls[j->level];
        const TvArgs ta = tv_args(L, j->P);
        Chain *chain = nullptr;
        for (Chain &ch : chains)
            if (ch.job == j) chain = &ch;
        const float *src = j->P.clamp_mode == 0 ? L->f : L->g;
        const long nb = (long)tv_blocks(L->nx, L->ny, L->nz);
        const size_t np = project_partials(L->gd);
        if (ta.xT > 0) {  // x-marching form: the single-request path's launches, solo
            const XProxPlan pl = job_xplan(j, L);
            for (const XLaunch &x : pl.launches) {
                TvItem ti{};
                ti.A = ta;
                ti.fin = x.fin;
                ti.g = L->g;
                ti.fout = x.fout;
                ti.clamp = 1;
                ti.acc = x.e1 ? TV_ACC_E1 : x.step ? TV_ACC_STEP : TV_ACC_NONE;
                ti.partial = x.step ? step_region(L) : L->partial + np;
                ti.xT = x.T;
                ti.xclamp = x.clamp;
                if (chain) chain->tv.push_back(ti);
                else solo_tv[0].push_back(ti);
            }
            if (chain) chain->step = StepItem{};
            if (pl.step_fused || pl.result == L->f) continue;
            StepItem si;
            si.v = pl.result;
            si.f = L->f;
            si.partial = step_region(L);
            si.n = (long)vol_elems(L->gd);
            if (chain) {
                chain->step = si;
            } else {
                hstep.push_back(si);
                sstart.push_back(stot);
                stot += (long)step_partials((size_t)si.n);
            }
            continue;
        }
        const bool fused = job_step_fused(j, L);
        for (int m = 0; m < j->P.M; ++m) {
            const bool last = m == j->P.M - 1;
            float *dst = (last && fused) ? L->f : (m % 2 == 0) ? L->A : L->B;
            if (dst == src) dst = (dst == L->A) ? L->B : L->A;
            TvItem ti{};
            ti.A = ta;
            ti.fin = src;
            ti.g = L->g;
            ti.fout = dst;
            ti.clamp = (j->P.clamp_mode == 0 || last) ? 1 : 0;
            ti.acc = (m == 0 && j->P.clamp_mode == 0) ? TV_ACC_E1 : (last && fused) ? TV_ACC_STEP : TV_ACC_NONE;
            ti.partial = ti.acc == TV_ACC_STEP ? step_region(L) : L->partial + np;
            if (chain) {
                chain->tv.push_back(ti);
            } else if (tv_sweep_solo(L->nx, L->ny, L->nz, sms)) {
                solo_tv[m].push_back(ti);
            } else {
                htv[m].push_back(ti);
                tvstart[m].push_back(tvtot[m]);
                tvtot[m] += nb;
            }
            src = dst;
        }
        if (chain) chain->step = StepItem{};
        if (fused) continue;
        StepItem si;
        si.v = src;
        si.f = L->f;
        si.partial = step_region(L);
        si.n = (long)vol_elems(L->gd);
        if (chain) {
            chain->step = si;
        } else {
            hstep.push_back(si);
            sstart.push_back(stot);
            stot += (long)step_partials((size_t)si.n);
        }
    }
    steptotal = stot;
    dtotal = dtot;
    for (int v = 0; v < 4; ++v) bptotal[v] = bptot[v];
    eqtotal = eqtot;

    // one device blob: items and start tables
    size_t off = 0;
    auto place = [&](size_t bytes) {
        size_t o = off;
        off = align(off + bytes);
        return o;
    };
    const size_t o_proj = place(hproj.size() * sizeof(ProjItem)), o_pst = place(pstart.size() * sizeof(long));
    size_t o_bp[4], o_bst[4];
    for (int v = 0; v < 4; ++v) {
        o_bp[v] = place(hbp[v].size() * sizeof(BpItem));
        o_bst[v] = place(bpstart[v].size() * sizeof(long));
    }
    const size_t o_eq = place(heq.size() * sizeof(Eq2Item)), o_est = place(eqstart.size() * sizeof(long));
    const size_t o_dot = place(hdot.size() * sizeof(VecItem)), o_dst = place(dstart.size() * sizeof(long));
    std::vector<size_t> o_tv(max_m), o_tst(max_m);
    for (int m = 0; m < max_m; ++m) {
        o_tv[m] = place(htv[m].size() * sizeof(TvItem));
        o_tst[m] = place(tvstart[m].size() * sizeof(long));
    }
    const size_t o_en = place(hen.size() * sizeof(EnItem));
    const size_t o_step = place(hstep.size() * sizeof(StepItem)), o_sst = place(sstart.size() * sizeof(long));
    std::vector<char> blob(std::max<size_t>(off, 16));
    auto put = [&](size_t o, const void *src, size_t bytes) {
        if (bytes) memcpy(blob.data() + o, src, bytes);
    };
    put(o_proj, hproj.data(), hproj.size() * sizeof(ProjItem));
    put(o_pst, pstart.data(), pstart.size() * sizeof(long));
    for (int v = 0; v < 4; ++v) {
        put(o_bp[v], hbp[v].data(), hbp[v].size() * sizeof(BpItem));
        put(o_bst[v], bpstart[v].data(), bpstart[v].size() * sizeof(long));
    }
    put(o_eq, heq.data(), heq.size() * sizeof(Eq2Item));
    put(o_est, eqstart.data(), eqstart.size() * sizeof(long));
    put(o_dot, hdot.data(), hdot.size() * sizeof(VecItem));
    put(o_dst, dstart.data(), dstart.size() * sizeof(long));
    for (int m = 0; m < max_m; ++m) {
        put(o_tv[m], htv[m].data(), htv[m].size() * sizeof(TvItem));
        put(o_tst[m], tvstart[m].data(), tvstart[m].size() * sizeof(long));
    }
    put(o_en, hen.data(), hen.size() * sizeof(EnItem));
    put(o_step, hstep.data(), hstep.size() * sizeof(StepItem));
    put(o_sst, sstart.data(), sstart.size() * sizeof(long));
    if (blob.size() > dblob_len) {
        ECK(cudaStreamSynchronize(stream), "engine sync");
        cudaFree(dblob);
        dblob = nullptr;
        dblob_len = 0;
        ECK(cudaMalloc(&dblob, blob.size() * 2), "engine tables");
        dblob_len = blob.size() * 2;
    }
    // the previous tick's launches may still read the old tables
    ECK(cudaStreamSynchronize(stream), "engine sync");
    ECK(cudaMemcpy(dblob, blob.data(), blob.size(), cudaMemcpyHostToDevice), "engine tables");
    char *b = (char *)dblob;
    d_proj = (ProjItem *)(b + o_proj);
    d_pstart = (long *)(b + o_pst);
    for (int v = 0; v < 4; ++v) {
        d_bp[v] = (BpItem *)(b + o_bp[v]);
        d_bstart[v] = (long *)(b + o_bst[v]);
    }
    d_eq = (Eq2Item *)(b + o_eq);
    d_eqstart = (long *)(b + o_est);
    d_dot = (VecItem *)(b + o_dot);
    d_dstart = (long *)(b + o_dst);
    d_tv.assign(max_m, nullptr);
    d_tstart.assign(max_m, nullptr);
    for (int m = 0; m < max_m; ++m) {
        d_tv[m] = (TvItem *)(b + o_tv[m]);
        d_tstart[m] = (long *)(b + o_tst[m]);
    }
    d_en = (EnItem *)(b + o_en);
    d_step = (StepItem *)(b + o_step);
    d_sstart = (long *)(b + o_sst);
    if (!chains.empty()) EST(ensure_side(chains.size()));
    return CBCT_OK;
}

// per device: the attributes belong to the device's context (setting them twice is harmless)
static std::atomic<bool> attr_done[64];

// Blocks of `kernel` that stay resident on one SM with this block size and dynamic
// shared memory (persistent grids are sized to exactly fill the GPU once).
template <class K>
static int resident_blocks(K kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

static long persistent_grid(long tiles, int per_sm) { return std::max(1L, std::min(tiles, (long)sm_count() * per_sm)); }

cbct_status Engine::ensure_side(size_t n) {
    while (side.size() < std::min<size_t>(n, 8)) {
        cudaStream_t st = nullptr;
        ECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "side stream");
        side.push_back(st);
    }
    while (side_events.size() < n + 1) {
        cudaEvent_t e = nullptr;
        ECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "side event");
        side_events.push_back(e);
    }
    return CBCT_OK;
}

// One job's whole tick (every stage its own single-request launch) on stream s.
static cbct_status launch_chain(const Engine::Chain &c, cudaStream_t s) {
    const Job *j = c.job;
    if (!c.power && j->P.clamp_mode == 1) {  // literal clamp mode: E1 of f_k needs its own pass
        Level *L = j->Ls[j->level];
        int nb = 0;
        ECK(launch_tv_energy(tv_args(L, j->P), L->f, L->partial + project_partials(L->gd), s, &nb), "tv energy");
    }
    ECK(launch_project(c.proj.G, c.proj.vol, c.proj.y32, c.proj.y16, c.proj.out, c.proj.partial, c.proj.mode, s,
                       nullptr),
        "projection");
    if (c.eq2)
        ECK(launch_backproject_eq2(c.eq.G, c.eq.r, nullptr, c.eq.fin, c.eq.out, c.eq.cscale, c.eq.mode, s), "eq2 backprojection");
    else
        ECK(launch_backproject(c.bp.G, c.bp.rs, c.bp.fin, c.bp.out, c.bp.c, c.bp.mode, s), "backprojection");
    if (c.power) {  // the same partition and trees as the batched helpers
        int nb = 0;
        ECK(launch_dot2(c.vec.x, c.vec.y, (size_t)c.vec.n, c.vec.partial, s, &nb), "power dot");
        ECK(launch_power_finalize(c.vec.partial, nb, c.vec.lam, c.vec.scale, s), "power finalize");
        ECK(launch_scale(c.vec.y, c.vec.scale, (float *)c.vec.out, (size_t)c.vec.n, s), "power scale");
    }
    for (const TvItem &it : c.tv) EST(launch_tv_item(it, s));
    if (c.step.f) ECK(launch_step_copy(c.step.v, c.step.f, (size_t)c.step.n, c.step.partial, s), "step");
    return CBCT_OK;
}

// The batched stages of one tick (no host synchronisation; capturable).
cbct_status Engine::launch_stages() {
    cudaStream_t s = stream;
    // jobs that fill the GPU by themselves: forked onto side streams
    if (!chains.empty()) {
        ECK(cudaEventRecord(side_events[0], s), "fork");
        for (size_t q = 0; q < chains.size(); ++q) {
            cudaStream_t ss = side[q % side.size()];
            ECK(cudaStreamWaitEvent(ss, side_events[0], 0), "fork wait");
            EST(launch_chain(chains[q], ss));
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        cudaFuncSetAttribute(k_project_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
        attr_done[dev] = true;
    }
    for (Job *j : tv_energy_jobs) {  // literal clamp mode: E1 of f_k needs its own pass
        Level *L = j->Ls[j->level];
        int nb = 0;
        ECK(launch_tv_energy(tv_args(L, j->P), L->f, L->partial + project_partials(L->gd), s, &nb), "tv energy");
    }
    // projection
    for (const ProjItem &it : solo_proj)
        ECK(launch_project(it.G, it.vol, it.y32, it.y16, it.out, it.partial, it.mode, s, nullptr), "projection");
    for (const ProjGroup &pg : pgroups) {
        const int per_sm = resident_blocks(k_project_batch, pg.threads, pg.smem);
        k_project_batch<<<(unsigned)persistent_grid(pg.tiles, per_sm), pg.threads, pg.smem, s>>>(
            d_proj + pg.first, d_pstart + pg.first, pg.count, pg.tiles);
        count_launch();
        ECK(cudaGetLastError(), "batched projection");
    }
    // adjoint (+ gradient step)
    for (const BpItem &it : solo_bp)
        ECK(launch_backproject(it.G, it.rs, it.fin, it.out, it.c, it.mode, s), "backprojection");
    for (const Eq2Item &it : solo_eq)
        ECK(launch_backproject_eq2(it.G, it.r, nullptr, it.fin, it.out, it.cscale, it.mode, s), "eq2 backprojection");
    for (int v = 0; v < 4; ++v)  // column running sums the batched gathers read
        for (const BpItem &it : hbp[v]) ECK(launch_row_prefix(it.G, it.rs, s), "row sums");
    for (int v = 0; v < 4; ++v) {
        if (hbp[v].empty()) continue;
        const int n = (int)hbp[v].size();
        const long warps = bptotal[v];
        const int wpb = BP_THREADS / 32;
        if (v == 0) {
            const long nb = persistent_grid((warps + wpb - 1) / wpb, resident_blocks(k_bp_batch<1>, BP_THREADS, 0));
            k_bp_batch<1><<<(unsigned)nb, BP_THREADS, 0, s>>>(d_bp[0], d_bstart[0], n, warps);
            count_launch();
        } else if (v == 1) {
            const long nb = persistent_grid((warps + wpb - 1) / wpb, resident_blocks(k_bp_batch<2>, BP_THREADS, 0));
            k_bp_batch<2><<<(unsigned)nb, BP_THREADS, 0, s>>>(d_bp[1], d_bstart[1], n, warps);
            count_launch();
        } else if (v == 2) {
            const long nb = persistent_grid((warps + wpb - 1) / wpb, resident_blocks(k_bp_batch<3>, BP_THREADS, 0));
            k_bp_batch<3><<<(unsigned)nb, BP_THREADS, 0, s>>>(d_bp[2], d_bstart[2], n, warps);
            count_launch();
        } else {
            const long nb = persistent_grid((warps + wpb - 1) / wpb, resident_blocks(k_bp_batch<4>, BP_THREADS, 0));
            k_bp_batch<4><<<(unsigned)nb, BP_THREADS, 0, s>>>(d_bp[3], d_bstart[3], n, warps);
            count_launch();
        }
        ECK(cudaGetLastError(), "batched backprojection");
    }
    if (!heq.empty()) {
        const long nb = persistent_grid(eqtotal, resident_blocks(k_eq2_batch, EQ2_THREADS, 0));
        k_eq2_batch<<<(unsigned)nb, EQ2_THREADS, 0, s>>>(d_eq, d_eqstart, (int)heq.size(), eqtotal);
        count_launch();
        ECK(cudaGetLastError(), "batched eq2 backprojection");
    }
    if (!hdot.empty()) {
        const int n = (int)hdot.size();
        k_dot_batch<<<(unsigned)persistent_grid(dtotal, 8), 256, 0, s>>>(d_dot, d_dstart, n, dtotal);
        count_launch();
        k_pfin_batch<<<(unsigned)n, 256, 0, s>>>(d_dot);
        count_launch();
        k_scale_batch<<<(unsigned)persistent_grid(dtotal, 8), 256, 0, s>>>(d_dot, d_dstart, n, dtotal);
        count_launch();
        ECK(cudaGetLastError(), "batched power iteration");
    }
    // TV prox sweeps
    const int tv_per_sm = resident_blocks(k_tv_batch, TV_THREADS, 0);
    for (int m = 0; m < max_m; ++m) {
        for (const TvItem &it : solo_tv[m]) EST(launch_tv_item(it, s));
        if (htv[m].empty()) continue;
        k_tv_batch<<<(unsigned)persistent_grid(tvtot[m], tv_per_sm), TV_THREADS, 0, s>>>(d_tv[m], d_tstart[m],
                                                                                         (int)htv[m].size(), tvtot[m]);
        count_launch();
        ECK(cudaGetLastError(), "batched tv sweep");
    }
    if (!hstep.empty()) {
        const long nb = persistent_grid(steptotal, resident_blocks(k_step_batch, STEP_THREADS, 0));
        k_step_batch<<<(unsigned)nb, STEP_THREADS, 0, s>>>(d_step, d_sstart, (int)hstep.size(), steptotal);
        count_launch();
        ECK(cudaGetLastError(), "batched step");
    }
    // join the side streams before the energies (which read every job's partials)
    for (size_t q = 0; q < side.size() && q < chains.size(); ++q) {
        ECK(cudaEventRecord(side_events[q + 1], side[q]), "join");
        ECK(cudaStreamWaitEvent(s, side_events[q + 1], 0), "join wait");
    }
    if (!hen.empty()) {
        k_energy_batch<<<(unsigned)hen.size(), ENERGY_THREADS, 0, s>>>(d_en);
        count_launch();
        ECK(cudaGetLastError(), "batched energy");
    }
    return CBCT_OK;
}

cbct_status Engine::tick() {
    // per-job transitions that are not batched
    for (Job *j : jobs) {
        if (j->phase == PH_PREPARE) EST(prepare(j));
        if (j->phase == PH_START_LEVEL) EST(start_level(j));
    }
    std::vector<long> sig;
    for (Job *j : jobs) {
        if (j->phase != PH_POWER && j->phase != PH_FBS) continue;
        sig.push_back((long)(uintptr_t)j);
        sig.push_back(j->phase * 16 + j->level);
    }
    if (sig != signature) {
        reset_graph();
        EST(build_tables());
        signature = sig;
    } else {
        ++same_ticks;
    }
    if (!sig.empty()) {
        if (use_graphs && same_ticks >= 1 && !gexec) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                cbct_status st = launch_stages();
                cudaError_t e = cudaStreamEndCapture(stream, &graph);
                if (st != CBCT_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                if (e != cudaSuccess) return cuda_fail(e, "graph capture");
                e = cudaGraphInstantiate(&gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) {
                    gexec = nullptr;
                    return cuda_fail(e, "graph instantiate");
                }
            } else {
                cudaGetLastError();
                use_graphs = false;
            }
        }
        if (gexec) ECK(cudaGraphLaunch(gexec, stream), "graph launch");
        else EST(launch_stages());
    }
    // advance, then one synchronisation for every job that needs host values
    bool need_sync = false;
    for (Job *j : jobs) {
        if (j->phase == PH_POWER && ++j->pi_it == j->K) {
            j->phase = PH_POWER_DONE;
            need_sync = true;
        } else if (j->phase == PH_FBS && ++j->it == j->iters) {
            j->phase = PH_LEVEL_DONE;
            need_sync = true;
        } else if (j->phase == PH_LEVEL_DONE) {
            need_sync = true;
        }
    }
    if (need_sync) {
        ECK(cudaStreamSynchronize(stream), "engine sync");
        for (Job *j : jobs) {
            if (j->phase == PH_POWER_DONE) {
                double lam = 0.0;
                ECK(cudaMemcpy(&lam, j->G->dscalars, sizeof(double), cudaMemcpyDeviceToHost), "lambda");
                Level *L = j->Ls[j->level];
                L->lambda = lam;
                L->lambda_iters = j->K;
                EST(begin_fbs(j, std::max(10.0 * j->mu, 1.05 * gamma_of(L, j->mu) * lam)));
            }
            if (j->phase == PH_LEVEL_DONE) EST(finish_level(j));
        }
    }
    return CBCT_OK;
}

bool Engine::busy() const {
    for (Job *j : jobs)
        if (j->phase != PH_DONE) return true;
    return false;
}

cbct_status Engine::run_all() {
    while (busy()) EST(tick());
    return CBCT_OK;
}

}  // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_reconstruct_batch(const cbct_request *reqs, int n, int use_graphs, cudaStream_t stream) {
    if (!reqs || n < 1) {
        set_error("need at least one request");
        return CBCT_ERR_INVALID_ARG;
    }
    std::vector<Job> jobs(n);
    Engine E(stream, use_graphs != 0);
    for (int q = 0; q < n; ++q) {
        const cbct_request &r = reqs[q];
        cbct_status st = validate_request(r.geom, r.Y_dev, r.mu, r.iters, r.levels, r.opts, r.f_out_dev);
        if (st != CBCT_OK) {
            set_error("request %d: %s", q, cbct_last_error());
            return st;
        }
        Job &j = jobs[q];
        j.G = r.geom;
        j.Y = r.Y_dev;
        j.mu = r.mu;
        j.iters = r.iters;
        j.levels = r.levels;
        if (r.opts) j.o = *r.opts;
        j.f_out = r.f_out_dev;
        st = E.add(&j);
        if (st != CBCT_OK) {
            set_error("request %d: %s", q, cbct_last_error());
            return st;
        }
    }
    return E.run_all();
}

// ---------------------------------------------------------------------------------
// autotuner: launch shapes per level (results are bitwise independent of them)
// ---------------------------------------------------------------------------------

static float time_ms(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    float ms = 0.f;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

extern "C" cbct_status cbct_autotune(cbct_geometry *G, int level, cbct_tuning *out, cudaStream_t s) {
    if (!G || !out) {
        set_error("null argument");
        return CBCT_ERR_INVALID_ARG;
    }
    Level *L;
    EST(ensure_level(G, level, &L));
    EST(ensure_workspace(L, false));
    GeoDev g = L->gd;
    const size_t nv = vol_elems(g);
    ECK(launch_fill(L->A, 1e-3f, nv, s), "fill");
    cudaEvent_t e0, e1;
    ECK(cudaEventCreate(&e0), "event");
    ECK(cudaEventCreate(&e1), "event");
    const int reps = 3;
    // projector block size and shared memory (band size)
    const int need = std::min(PROJ_MAX_THREADS, 32 * ((g.nv + 31) / 32));
    int best_t = 0, best_m = 0;
    float best_p = 1e30f;
    for (int T : {need, 256, 320, 384, 448, 512}) {
        if (T < need || T > PROJ_MAX_THREADS) continue;
        for (int kb : {0, 110, 74, 56, 40}) {
            g.proj_threads = T;
            g.proj_smem = kb * 1024;
            if (kb && proj_smem_of(g) != kb * 1024) continue;   // too small for this geometry
            launch_project(g, L->A, nullptr, nullptr, L->rs, nullptr, PROJ_SCALED, s, nullptr);
            cudaEventRecord(e0, s);
            for (int q = 0; q < reps; ++q) launch_project(g, L->A, nullptr, nullptr, L->rs, nullptr, PROJ_SCALED, s, nullptr);
            cudaEventRecord(e1, s);
            const float ms = time_ms(s, e0, e1) / reps;
            if (ms < best_p) {
                best_p = ms;
                best_t = T;
                best_m = kb * 1024;
            }
        }
    }
    g.proj_threads = best_t;
    g.proj_smem = best_m;
    // adjoint voxels per lane, block size and lane layout
    int best_v = 0, best_b = 0, best_l = 0;
    float best_q = 1e30f;
    const int vmax = std::min(4, (g.nz + 31) / 32);
    for (int v = 1; v <= vmax; ++v)
        for (int T : {64, 128, 256})
            for (int lay : {1, 2}) {
                g.bp_vpl = v;
                g.bp_threads = T;
                g.bp_layout = lay;
                launch_backproject(g, L->rs, nullptr, L->B, 0.f, BP_PLAIN, s);
                cudaEventRecord(e0, s);
                for (int q = 0; q < reps; ++q) launch_backproject(g, L->rs, nullptr, L->B, 0.f, BP_PLAIN, s);
                cudaEventRecord(e1, s);
                const float ms = time_ms(s, e0, e1) / reps;
                if (ms < best_q) {
                    best_q = ms;
                    best_v = v;
                    best_b = T;
                    best_l = lay;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ECK(cudaGetLastError(), "autotune");
    L->gd.proj_threads = best_t;
    L->gd.proj_smem = best_m;
    L->gd.bp_vpl = best_v;
    L->gd.bp_threads = best_b;
    L->gd.bp_layout = best_l;
    out->proj_threads = best_t;
    out->proj_smem = best_m;
    out->proj_levels = L->gd.proj_levels;
    out->bp_vpl = best_v;
    out->bp_threads = best_b;
    out->bp_layout = best_l;
    out->tv_sweeps = L->tv_sweeps;
    out->tv_warps = L->tv_warps;
    out->tv_planes = L->tv_planes;
    out->proj_ms = best_p;
    out->bp_ms = best_q;
    return CBCT_OK;
}

extern "C" cbct_status cbct_set_tuning(cbct_geometry *G, int level, const cbct_tuning *t) {
    if (!G || !t) {
        set_error("null argument");
        return CBCT_ERR_INVALID_ARG;
    }
    Level *L;
    EST(ensure_level(G, level, &L));
    const int need = std::min(PROJ_MAX_THREADS, 32 * ((L->gd.nv + 31) / 32));
    if ((t->proj_threads && (t->proj_threads < need || t->proj_threads > PROJ_MAX_THREADS || t->proj_threads % 32)) ||
        t->bp_vpl < 0 || t->bp_vpl > 4 ||
        (t->bp_threads && t->bp_threads != 64 && t->bp_threads != 128 && t->bp_threads != 256) ||
        t->proj_levels < 0 || t->proj_levels > L->gd.nz || t->bp_layout < 0 || t->bp_layout > 2 ||
        t->tv_sweeps < -1 || t->tv_sweeps > 2 ||
        (t->tv_warps && t->tv_warps != 16 && t->tv_warps != 32) ||
        (t->tv_planes && t->tv_planes < 8)) {
        set_error("tuning values out of range");
        return CBCT_ERR_INVALID_ARG;
    }
    if (t->proj_smem) {
        GeoDev g = L->gd;
        g.proj_smem = t->proj_smem;
        if (proj_smem_of(g) != t->proj_smem) {
            set_error("proj_smem must be a multiple of 16 between the geometry's minimum and %d", PROJ_SMEM);
            return CBCT_ERR_INVALID_ARG;
        }
    }
    L->gd.proj_threads = t->proj_threads;
    L->gd.proj_smem = t->proj_smem;
    L->gd.proj_levels = t->proj_levels;
    L->gd.bp_vpl = t->bp_vpl;
    L->gd.bp_threads = t->bp_threads;
    L->gd.bp_layout = t->bp_layout;
    L->tv_sweeps = t->tv_sweeps;
    L->tv_warps = t->tv_warps;
    L->tv_planes = t->tv_planes;
    return CBCT_OK;
}
