// C ABI of the library and the solver driver: Algorithm A1 (forward-backward
// splitting) of Jia et al. (2010) for E1 + mu E2 with f >= 0 (Eq. 1), on each level
// of a coarse-to-fine multigrid.
//
// Discrete scaling (the paper's functional derivatives on the voxel grid): with
// V = Nv dV and A = Np du dv, multiplying Eq. 1 by Nv gives
//   Nv E = TV_eps(f) + (gamma / 2) |P f - Y|^2,  gamma = 2 mu Nv / (n_angles Np),
// and step 1 becomes g = f - (gamma / beta) P^T (P f - Y); the 1/V of E1 and of E3
// cancel, so beta is the paper's beta.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "batch.h"
#include "cbct_internal.h"

using namespace cbct;

namespace cbct {
const char *last_error();
}

namespace cbct {

double eq2_scale(const Level *L) { return L->hx * L->hy * L->hz / (L->du * L->dv); }

double default_eps(const Level *L) { return 2e-5 / std::min(L->hx, std::min(L->hy, L->hz)); }

double tv_lipschitz(const Level *L, double eps) {
    return 4.0 / eps * (1.0 / (L->hx * L->hx) + 1.0 / (L->hy * L->hy) + 1.0 / (L->hz * L->hz));
}

double gamma_of(const Level *L, double mu) {
    return 2.0 * mu * (double)vol_elems(L->gd) / (double)sino_elems(L->gd);
}

cbct_status ensure_trace(cbct_geometry *G, size_t n) {
    if (!G->dscalars) {
        // layout: [0..63] scalars (lambda etc.), counter separately
        if (cudaMalloc(&G->dscalars, sizeof(double) * 64) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of scalar scratch failed");
            return CBCT_ERR_OOM;
        }
        if (cudaMalloc(&G->dcounter, sizeof(int) * 4) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of counter failed");
            return CBCT_ERR_OOM;
        }
    }
    (void)n;
    return CBCT_OK;
}

TvArgs tv_args(const Level *L, const SolveParams &P) {
    TvArgs a;
    a.nx = L->nx;
    a.ny = L->ny;
    a.nz = L->nz;
    a.ihx = (float)(1.0 / L->hx);
    a.ihy = (float)(1.0 / L->hy);
    a.ihz = (float)(1.0 / L->hz);
    a.s = P.s;
    a.beta = P.beta;
    a.eps2 = P.eps2;
    a.aniso = P.tv_mode;
    a.jc = tv_rows_per_tile(a.nx, a.ny, a.nz);
    a.vz = tv_col_vz(a.nx, a.ny, a.nz);
    tv_x_shape(a, L->tv_sweeps, L->tv_warps, L->tv_planes);
    return a;
}

}  // namespace cbct

namespace {

#define CK(call, what)                                       \
    do {                                                     \
        cudaError_t e__ = (call);                            \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

#define ST(call)                          \
    do {                                  \
        cbct_status s__ = (call);         \
        if (s__ != CBCT_OK) return s__;   \
    } while (0)

bool aligned16(const void *p) { return p && (((uintptr_t)p) & 15u) == 0; }

cbct_status need_ptr(const void *p, const char *name) {
    if (!aligned16(p)) {
        set_error("%s must be a non-null 16-byte aligned device pointer", name);
        return CBCT_ERR_INVALID_ARG;
    }
    return CBCT_OK;
}

// Per-call timing of kernel classes with CUDA events on the caller's stream.
struct Prof {
    cbct_geometry *G = nullptr;
    cudaStream_t s = 0;
    bool on = false;
    unsigned mask = ~0u;     // kernel classes timed with events (all launches are counted)
    bool timing = false;     // the current launch is timed
    int cur = 0;             // class of the current operation
    cudaStream_t cur_s = 0;  // stream of the current operation
    int tag = 0;             // 1 while the finest level's Algorithm A1 iterations are enqueued
    unsigned long long k0 = 0;
    std::vector<int> cls, tags;
    std::vector<cudaEvent_t> a, b;
    int count[CBCT_NUM_KERNEL_CLASSES] = {}, count_tag[CBCT_NUM_KERNEL_CLASSES] = {};
    void begin(int c, cudaStream_t st) {
        if (!on) return;
        cur = c;
        cur_s = st;
        k0 = g_kernel_launches.load(std::memory_order_relaxed);
        timing = (mask >> c) & 1u;
        if (!timing) return;
        cudaEvent_t e0 = G->events.get();
        cudaEventRecord(e0, st);
        a.push_back(e0);
        cls.push_back(c);
        tags.push_back(tag);
    }
    void end() {
        if (!on) return;
        const int n = (int)(g_kernel_launches.load(std::memory_order_relaxed) - k0);  // kernels it launched
        count[cur] += n;
        if (tag) count_tag[cur] += n;
        if (!timing) return;
        cudaEvent_t e1 = G->events.get();
        cudaEventRecord(e1, cur_s);
        b.push_back(e1);
        timing = false;
    }
    // ms/cnt: every timed operation; ms_t/cnt_t: those enqueued with the tag set
    cbct_status collect(float *ms, int *cnt, float *ms_t = nullptr, int *cnt_t = nullptr) {
        if (!on) return CBCT_OK;
        CK(cudaStreamSynchronize(s), "synchronising for kernel timing");
        for (int c = 0; c < CBCT_NUM_KERNEL_CLASSES; ++c) {
            if (ms) ms[c] = 0.f;
            if (ms_t) ms_t[c] = 0.f;
        }
        for (size_t q = 0; q < cls.size() && q < b.size(); ++q) {
            float t = 0.f;
            cudaEventElapsedTime(&t, a[q], b[q]);
            if (ms) ms[cls[q]] += t;
            if (ms_t && tags[q]) ms_t[cls[q]] += t;
        }
        for (int c = 0; c < CBCT_NUM_KERNEL_CLASSES; ++c) {
            if (cnt) cnt[c] = count[c];
            if (cnt_t) cnt_t[c] = count_tag[c];
        }
        G->events.release_all();
        return CBCT_OK;
    }
};

struct Launch {  // wraps one kernel launch with optional timing (on prof's stream, or st)
    Prof &p;
    int c;
    Launch(Prof &pp, int cc, cudaStream_t st = nullptr) : p(pp), c(cc) { p.begin(c, st ? st : p.s); }
    ~Launch() { p.end(); }
};

// Steps 2 and 3: M sweeps from src0 (ping-pong through A and B) into L->f, with the
// partials of |f_k+1 - f_k|^2 (f_k in L->f on entry) in partial_step (*nstep values).
// partial_e1 (optional) receives the E1 partials of the first sweep's input.
cbct_status enqueue_prox(Level *L, const SolveParams &P, const float *src0, double *partial_e1, int *ne1,
                         double *partial_step, int *nstep, Prof &prof, cudaStream_t s) {
    const TvArgs ta = tv_args(L, P);
    if (ta.xT > 0) {  // x-marching form: launches of up to xT fused sweeps
        const XProxPlan pl = xprox_plan(ta, P.M, P.clamp_mode, src0, L->f, L->A, L->B, partial_e1 != nullptr,
                                        partial_step != nullptr, vol_elems(L->gd));
        for (const XLaunch &x : pl.launches) {
            Launch l(prof, CBCT_K_TV);
            CK(launch_tv_x(ta, x.T, x.clamp, x.fin, L->g, x.fout, x.e1 ? partial_e1 : nullptr,
                           x.step ? partial_step : nullptr, s, nullptr),
               "tv sweeps");
        }
        if (ne1) *ne1 = pl.n_e1;
        if (nstep) *nstep = pl.n_step;
        if (pl.step_fused || pl.result == L->f) return CBCT_OK;
        Launch l(prof, CBCT_K_REDUCE);
        CK(launch_step_copy(pl.result, L->f, vol_elems(L->gd), partial_step, s), "step");
        return CBCT_OK;
    }
    const bool fused = prox_step_fused(P.M, src0, L->f);
    const float *src = src0;
    for (int m = 0; m < P.M; ++m) {
        const bool last = m == P.M - 1;
        float *dst = (last && fused) ? L->f : (m % 2 == 0) ? L->A : L->B;
        if (dst == src) dst = (dst == L->A) ? L->B : L->A;
        const bool clamp = P.clamp_mode == 0 || last;
        {
            Launch l(prof, CBCT_K_TV);
            CK(launch_tv_sweep(ta, src, L->g, dst, clamp, m == 0 ? partial_e1 : nullptr, s, m == 0 ? ne1 : nullptr,
                               (last && fused) ? partial_step : nullptr),
               "tv sweep");
        }
        src = dst;
    }
    if (nstep) *nstep = (int)(fused ? tv_partials(L->nx, L->ny, L->nz) : step_partials(vol_elems(L->gd)));
    if (!fused || !partial_step) {
        if (src == L->f) return CBCT_OK;
        Launch l(prof, CBCT_K_REDUCE);
        CK(launch_step_copy(src, L->f, vol_elems(L->gd), partial_step, s), "step");
    }
    return CBCT_OK;
}

// One iteration of Algorithm A1 on level L (state in L->f).
cbct_status enqueue_iteration(cbct_geometry *G, Level *L, const SolveParams &P, double *dtrace, Prof &prof,
                              cudaStream_t s) {
    const GeoDev &gd = L->gd;
    double *pp = L->partial;
    const size_t np = project_partials(gd);
    double *pt = L->partial + np;
    int nb_p = 0, nb_t = 0;
    if (P.clamp_mode == 1) {
        // the prox starts from g, so E1 of f_k needs its own pass
        Launch l(prof, CBCT_K_REDUCE);
        CK(launch_tv_energy(tv_args(L, P), L->f, pt, s, &nb_t), "tv energy");
    }
    const bool eq2 = P.adjoint_mode == 1;
    {
        Launch l(prof, CBCT_K_PROJECT);
        const int mode = P.fp16 ? (eq2 ? PROJ_RAW16 : PROJ_RESID16) : (eq2 ? PROJ_RAW32 : PROJ_RESID32);
        CK(launch_project(gd, L->f, P.fp16 ? nullptr : L->Y, P.fp16 ? L->Yh : nullptr, L->rs, pp, mode, s, &nb_p),
           "projection");
    }
    {
        Launch l(prof, CBCT_K_BACKPROJECT);
        if (eq2)
            CK(launch_backproject_eq2(gd, L->rs, L->eq2p, L->f, L->g, P.c_eq2, BP_STEP, s), "eq2 backprojection");
        else
            CK(launch_backproject(gd, L->rs, L->f, L->g, P.c, BP_STEP, s), "backprojection");
    }
    if (P.lin) {  // coarse model of a V-cycle: step 1 of A1 on E - <lin, f>
        Launch l(prof, CBCT_K_REDUCE);
        CK(launch_axpy(L->g, P.lin, P.lin_scale, vol_elems(gd), s), "linear term");
    }
    double *pstep = step_region(L);
    int nb_s = 0;
    ST(enqueue_prox(L, P, P.clamp_mode == 0 ? L->f : L->g, P.clamp_mode == 0 ? pt : nullptr,
                    P.clamp_mode == 0 ? &nb_t : nullptr, pstep, &nb_s, prof, s));
    {
        Launch l(prof, CBCT_K_REDUCE);
        CK(launch_energy_finalize(pp, nb_p, pt, nb_t, P.inv_nv, P.mu_over_nr, dtrace, G->dcounter, s, pstep, nb_s),
           "energy reduction");
    }
    return CBCT_OK;
}

// `iters` iterations of A1 on level L; trace values land in dtrace[0 .. TRACE_W*iters).
cbct_status run_level(cbct_geometry *G, Level *L, const SolveParams &P, int iters, double *dtrace, bool graphs,
                      Prof &prof, cudaStream_t s) {
    CK(cudaMemsetAsync(G->dcounter, 0, sizeof(int), s), "counter reset");
    if (graphs && !prof.on && s != 0 && iters > 1) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cbct_status st = enqueue_iteration(G, L, P, dtrace, prof, s);
            cudaError_t e2 = cudaStreamEndCapture(s, &graph);
            if (st != CBCT_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e2 != cudaSuccess) return cuda_fail(e2, "graph capture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                return cuda_fail(e, "graph instantiate");
            }
            for (int it = 0; it < iters && e == cudaSuccess; ++it) e = cudaGraphLaunch(exec, s);
            cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            return CBCT_OK;
        }
        cudaGetLastError();  // capture not possible on this stream: run eagerly
    }
    for (int it = 0; it < iters; ++it) ST(enqueue_iteration(G, L, P, dtrace, prof, s));
    return CBCT_OK;
}

// Enqueues K power iterations on level L (no synchronisation): lambda into *dlam, the
// scale scratch at *dscale.
cbct_status enqueue_power(Level *L, int K, double *dlam, float *dscale, Prof &prof, cudaStream_t s) {
    const GeoDev &gd = L->gd;
    const size_t nv = vol_elems(gd);
    float *x = L->A, *y = L->B;
    {
        Launch l(prof, CBCT_K_REDUCE, s);
        // x = u / |u| for the seeded uniform volume u (built in y), by the same reductions
        // as every iteration, so that every estimate is a Rayleigh quotient
        CK(launch_fill_uniform(y, gd.nx, gd.ny, gd.nz, POWER_SEED, s), "start volume");
        int nb = 0;
        CK(launch_dot2(y, y, nv, L->partial, s, &nb), "dot");
        CK(launch_power_finalize(L->partial, nb, dlam, dscale, s), "power finalize");
        CK(launch_scale(y, dscale, x, nv, s), "scale");
    }
    for (int it = 0; it < K; ++it) {
        {
            Launch l(prof, CBCT_K_PROJECT, s);
            CK(launch_project(gd, x, nullptr, nullptr, L->rs, nullptr, PROJ_SCALED, s, nullptr), "projection");
        }
        {
            Launch l(prof, CBCT_K_BACKPROJECT, s);
            CK(launch_backproject(gd, L->rs, nullptr, y, 0.f, BP_PLAIN, s), "backprojection");
        }
        int nb = 0;
        Launch l(prof, CBCT_K_REDUCE, s);
        CK(launch_dot2(x, y, nv, L->partial, s, &nb), "dot");
        CK(launch_power_finalize(L->partial, nb, dlam, dscale, s), "power finalize");
        CK(launch_scale(y, dscale, x, nv, s), "scale");
    }
    return CBCT_OK;
}

// lambda_max(P^T P) by K power iterations from the seeded uniform(0,1) volume.
cbct_status power_iteration(cbct_geometry *G, Level *L, int K, double *lam, Prof &prof, cudaStream_t s) {
    double *dlam = G->dscalars;
    ST(enqueue_power(L, K, dlam, (float *)(G->dscalars + 1), prof, s));
    CK(cudaMemcpyAsync(lam, dlam, sizeof(double), cudaMemcpyDeviceToHost, s), "lambda copy");
    CK(cudaStreamSynchronize(s), "power iteration");
    return CBCT_OK;
}

// The geometry's side stream, its events and the pinned lambda slots (created once).
cbct_status ensure_side(cbct_geometry *G) {
    if (G->side) return CBCT_OK;
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "side stream");
    G->side = st;
    CK(cudaEventCreateWithFlags(&G->side_fork, cudaEventDisableTiming), "side event");
    for (auto &e : G->side_done) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "side event");
    CK(cudaMallocHost(&G->host_lam, 13 * sizeof(double)), "pinned lambda slots");
    return CBCT_OK;
}

cbct_status check_geometry_desc(const cbct_geometry_desc *d) {
    if (!d) {
        set_error("desc is null");
        return CBCT_ERR_INVALID_ARG;
    }
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nu < 1 || d->nv < 1) {
        set_error("sizes must be >= 1");
        return CBCT_ERR_INVALID_ARG;
    }
    if (!(d->hx > 0) || !(d->hy > 0) || !(d->hz > 0) || !(d->du > 0) || !(d->dv > 0) || !(d->dso > 0) ||
        !(d->dsd > 0)) {
        set_error("spacings and distances must be > 0");
        return CBCT_ERR_INVALID_ARG;
    }
    if ((double)d->nx * d->ny * d->nz >= 2147483647.0) {
        set_error("volume must have fewer than 2^31 voxels");
        return CBCT_ERR_INVALID_ARG;
    }
    if (d->ny > 65535) {
        set_error("ny must be <= 65535");
        return CBCT_ERR_INVALID_ARG;
    }
    return CBCT_OK;
}


// ---------------------------------------------------------------------------------
// V-cycle: a full-approximation reading of the multigrid method the paper cites.
// Level l minimises the model E_l(f) - <lin_l, f> (lin_0 = 0); a cycle smooths with
// `pre` iterations of Algorithm A1, builds the coarse model
//   E_{l+1}(x) - <lin_{l+1}, x>,  lin_{l+1} = grad E_{l+1}(R f) - Q^T (grad E_l(f) - lin_l)
// (R: 2x2x2 mean, Q: trilinear prolongation), whose gradient at R f is Q^T of the
// fine model's gradient at f, reduces it by a cycle on level l+1 (`coarse` iterations
// of A1 on the coarsest level), keeps the correction f + Q(x - R f), clamped at 0,
// when it lowers the fine model, and smooths with `post` iterations.
// ---------------------------------------------------------------------------------

struct VCycle {
    cbct_geometry *G;
    std::vector<Level *> Ls;
    std::vector<SolveParams> P;   // per level
    int levels, pre, post, coarse;
    bool graphs;
    double mu;
    double *dtrace;
    Prof *prof;
    cudaStream_t s;
    int accepted[8] = {0, 0, 0, 0, 0, 0, 0, 0};

    float *lin(int l) { return Ls[l]->mg; }
    float *x0(int l) { return Ls[l]->mg + vol_elems(Ls[l]->gd); }
    float *t1(int l) { return Ls[l]->mg + 2 * vol_elems(Ls[l]->gd); }
    float *t2(int l) { return Ls[l]->mg + 3 * vol_elems(Ls[l]->gd); }

    // out = grad E_l(f) - lin (lin may be null); uses the level's residual buffer
    cbct_status grad(int l, const float *f, const float *lv, float *out) {
        Level *L = Ls[l];
        const GeoDev &g = L->gd;
        const SolveParams &Q = P[l];
        {
            Launch lz(*prof, CBCT_K_PROJECT);
            CK(launch_project(g, f, Q.fp16 ? nullptr : L->Y, Q.fp16 ? L->Yh : nullptr, L->rs, L->partial,
                              Q.fp16 ? PROJ_RESID16 : PROJ_RESID32, s, nullptr),
               "projection");
        }
        {
            Launch lz(*prof, CBCT_K_BACKPROJECT);
            CK(launch_backproject(g, L->rs, nullptr, out, 0.f, BP_PLAIN, s), "backprojection");
        }
        Launch lz(*prof, CBCT_K_REDUCE);
        CK(launch_energy_grad(tv_args(L, Q), f, out, (float)gamma_of(L, mu), (float)Q.inv_nv, lv, out, s),
           "energy gradient");
        return CBCT_OK;
    }

    // host values {E, E1, mu E2} of f on level l, and <lin, f> (0 without lin)
    cbct_status energy(int l, const float *f, const float *lv, double out[4]) {
        Level *L = Ls[l];
        const GeoDev &g = L->gd;
        const SolveParams &Q = P[l];
        const size_t np = project_partials(g);
        int nb_p = 0, nb_t = 0;
        double *scratch = G->dscalars + 8;
        CK(cudaMemsetAsync(G->dcounter + 1, 0, sizeof(int), s), "counter");
        {
            Launch lz(*prof, CBCT_K_PROJECT);
            CK(launch_project(g, f, Q.fp16 ? nullptr : L->Y, Q.fp16 ? L->Yh : nullptr, L->rs, L->partial,
                              Q.fp16 ? PROJ_RESID16 : PROJ_RESID32, s, &nb_p),
               "projection");
        }
        Launch lz(*prof, CBCT_K_REDUCE);
        CK(launch_tv_energy(tv_args(L, Q), f, L->partial + np, s, &nb_t), "tv energy");
        CK(launch_energy_finalize(L->partial, nb_p, L->partial + np, nb_t, Q.inv_nv, Q.mu_over_nr, scratch,
                                  G->dcounter + 1, s),
           "energy");
        if (lv) CK(launch_dot(lv, f, vol_elems(g), L->mg_partial, scratch + TRACE_W, s), "linear term");
        else CK(cudaMemsetAsync(scratch + TRACE_W, 0, sizeof(double), s), "linear term");
        CK(cudaMemcpyAsync(out, scratch, 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "energy copy");
        CK(cudaMemcpyAsync(out + 3, scratch + TRACE_W, sizeof(double), cudaMemcpyDeviceToHost, s), "energy copy");
        CK(cudaStreamSynchronize(s), "energy sync");
        return CBCT_OK;
    }

    // *out (host) = |f_l - prev|_2, the change of level l's iterate since prev
    cbct_status change(int l, const float *prev, double *out) {
        Level *L = Ls[l];
        const size_t n = vol_elems(L->gd);
        double *scratch = G->dscalars + 8;
        Launch lz(*prof, CBCT_K_REDUCE);
        CK(launch_sub(L->f, prev, t1(l), n, s), "change");
        CK(launch_dot(t1(l), t1(l), n, L->mg_partial, scratch, s), "change norm");
        double d = 0.0;
        CK(cudaMemcpyAsync(&d, scratch, sizeof(double), cudaMemcpyDeviceToHost, s), "change copy");
        CK(cudaStreamSynchronize(s), "change sync");
        *out = std::sqrt(d);
        return CBCT_OK;
    }

    cbct_status smooth(int l, int iters, const float *lv) {
        if (iters <= 0) return CBCT_OK;
        SolveParams Q = P[l];
        Q.lin = lv;
        Q.lin_scale = lv ? (float)((double)vol_elems(Ls[l]->gd) / (double)Q.beta) : 0.f;
        return run_level(G, Ls[l], Q, iters, dtrace, graphs, *prof, s);
    }

    cbct_status cycle(int l, const float *lv) {
        if (l == levels - 1) return smooth(l, coarse, lv);
        ST(smooth(l, pre, lv));
        Level *Lf = Ls[l], *Lc = Ls[l + 1];
        const GeoDev &gf = Lf->gd, &gc = Lc->gd;
        const size_t nf = vol_elems(gf), nc = vol_elems(gc);
        ST(grad(l, Lf->f, lv, t1(l)));
        {
            Launch lz(*prof, CBCT_K_TRANSFER);
            CK(launch_restrict_vol(Lf->f, gf.nx, gf.ny, gf.nz, x0(l + 1), s), "volume restriction");
            CK(cudaMemcpyAsync(Lc->f, x0(l + 1), nc * 4, cudaMemcpyDeviceToDevice, s), "copy");
            CK(launch_prolong_adjoint(t1(l), gf.nx, gf.ny, gf.nz, t1(l + 1), gc.nx, gc.ny, gc.nz, s),
               "prolongation transpose");
        }
        ST(grad(l + 1, x0(l + 1), nullptr, t2(l + 1)));
        {
            Launch lz(*prof, CBCT_K_REDUCE);
            CK(launch_sub(t2(l + 1), t1(l + 1), lin(l + 1), nc, s), "coarse linear term");
        }
        ST(cycle(l + 1, lin(l + 1)));
        {
            Launch lz(*prof, CBCT_K_TRANSFER);
            CK(launch_sub(Lc->f, x0(l + 1), t1(l + 1), nc, s), "coarse change");
            CK(launch_prolong(t1(l + 1), gc.nx, gc.ny, gc.nz, t1(l), gf.nx, gf.ny, gf.nz, s), "prolongation");
            CK(launch_add_clamp(Lf->f, t1(l), t2(l), nf, s), "correction");
        }
        double e_try[4], e_cur[4];
        ST(energy(l, t2(l), lv, e_try));
        ST(energy(l, Lf->f, lv, e_cur));
        if (e_try[0] - e_try[3] < e_cur[0] - e_cur[3]) {
            CK(cudaMemcpyAsync(Lf->f, t2(l), nf * 4, cudaMemcpyDeviceToDevice, s), "accept correction");
            accepted[l] += 1;
        }
        return smooth(l, post, lv);
    }
};

}  // namespace

// Device energy-trace buffer owned by the geometry (grown on demand).
cbct_status cbct::get_trace(cbct_geometry *G, size_t n, double **out) {
    if (G->dtrace_len < n) {
        cudaFree(G->dtrace);
        G->dtrace = nullptr;
        G->dtrace_len = 0;
        if (cudaMalloc(&G->dtrace, n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of energy trace failed");
            return CBCT_ERR_OOM;
        }
        G->dtrace_len = n;
    }
    *out = G->dtrace;
    return CBCT_OK;
}

// Host copies of `iters` device trace entries: {E, E1, mu E2} into energy (3 per
// iteration) and |f_k+1 - f_k| into step (1 per iteration); either may be null.
cbct_status cbct::copy_trace(const double *dtrace, int iters, double *energy, double *step, cudaStream_t s) {
    if (iters <= 0) return CBCT_OK;
    const size_t w = TRACE_W * sizeof(double);
    if (energy)
        CK(cudaMemcpy2DAsync(energy, 3 * sizeof(double), dtrace, w, 3 * sizeof(double), iters,
                             cudaMemcpyDeviceToHost, s),
           "trace");
    if (step)
        CK(cudaMemcpy2DAsync(step, sizeof(double), dtrace + 3, w, sizeof(double), iters, cudaMemcpyDeviceToHost, s),
           "step trace");
    return CBCT_OK;
}

cbct_status cbct::solve_params(const Level *L, double mu, double beta, double eps, int M, int clamp_mode, bool fp16,
                                SolveParams *P, int tv_mode, int adjoint_mode) {
    if (!(beta > 0) || !isfinite(beta)) {
        set_error("beta must be > 0");
        return CBCT_ERR_INVALID_ARG;
    }
    if (!(eps > 0) || !isfinite(eps)) {
        set_error("eps must be > 0");
        return CBCT_ERR_INVALID_ARG;
    }
    if (M < 1 || M > 10000) {
        set_error("inner_iters must be in 1..10000");
        return CBCT_ERR_INVALID_ARG;
    }
    if (clamp_mode != 0 && clamp_mode != 1) {
        set_error("clamp_mode must be 0 or 1");
        return CBCT_ERR_INVALID_ARG;
    }
    if (tv_mode != 0 && tv_mode != 1) {
        set_error("tv_mode must be 0 or 1");
        return CBCT_ERR_INVALID_ARG;
    }
    if (adjoint_mode != 0 && adjoint_mode != 1) {
        set_error("adjoint_mode must be 0 or 1");
        return CBCT_ERR_INVALID_ARG;
    }
    const double gam = gamma_of(L, mu);
    P->c = (float)(gam / beta);
    P->s = (float)(1.0 / (beta + tv_lipschitz(L, eps)));
    P->beta = (float)beta;
    P->eps2 = (float)(eps * eps);
    P->M = M;
    P->clamp_mode = clamp_mode;
    P->tv_mode = tv_mode;
    P->adjoint_mode = adjoint_mode;
    P->c_eq2 = (float)(gam / beta * eq2_scale(L));
    P->lin = nullptr;
    P->lin_scale = 0.f;
    P->fp16 = fp16;
    P->inv_nv = 1.0 / (double)vol_elems(L->gd);
    P->mu_over_nr = mu / (double)sino_elems(L->gd);
    return CBCT_OK;
}

cbct_status cbct::validate_request(cbct_geometry *G, const float *Y_dev, double mu, int iters, int levels,
                                  const cbct_options *o, float *f_out_dev) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    if (!aligned16(Y_dev) || !aligned16(f_out_dev)) {
        set_error("Y_dev and f_out_dev must be non-null 16-byte aligned device pointers");
        return CBCT_ERR_INVALID_ARG;
    }
    if (!(mu > 0) || !isfinite(mu) || iters < 0) {
        set_error("need mu > 0 and iters >= 0");
        return CBCT_ERR_INVALID_ARG;
    }
    const cbct_geometry_desc &d = G->desc;
    if (levels < 1 || levels > 8) {
        set_error("levels must be in 1..8");
        return CBCT_ERR_INVALID_ARG;
    }
    const int need = 1 << (levels - 1);
    if (d.nx < need || d.ny < need || d.nz < need || d.nu < need || d.nv < need) {
        set_error("every volume and imager axis needs at least 2^(levels-1) = %d samples", need);
        return CBCT_ERR_INVALID_ARG;
    }
    if (o) {
        if (o->clamp_mode != 0 && o->clamp_mode != 1) {
            set_error("clamp_mode must be 0 or 1");
            return CBCT_ERR_INVALID_ARG;
        }
        if (o->tv_mode != 0 && o->tv_mode != 1) {
            set_error("tv_mode must be 0 or 1");
            return CBCT_ERR_INVALID_ARG;
        }
        if (o->adjoint_mode != 0 && o->adjoint_mode != 1) {
            set_error("adjoint_mode must be 0 or 1");
            return CBCT_ERR_INVALID_ARG;
        }
        if (o->mg_cycle != 0) {
            set_error("V-cycles (mg_cycle 1) run through cbct_reconstruct only");
            return CBCT_ERR_UNSUPPORTED;
        }
        if (o->inner_iters < 0 || o->inner_iters > 10000 || o->power_iters < 0) {
            set_error("inner_iters must be in 0..10000 and power_iters >= 0");
            return CBCT_ERR_INVALID_ARG;
        }
        if (o->betas)
            for (int l = 0; l < levels; ++l)
                if (!(o->betas[l] > 0) || !isfinite(o->betas[l])) {
                    set_error("betas[%d] must be > 0", l);
                    return CBCT_ERR_INVALID_ARG;
                }
        if (o->f_init_dev) {
            if (o->start_level < 0 || o->start_level >= levels) {
                set_error("start_level must be in 0..levels-1");
                return CBCT_ERR_INVALID_ARG;
            }
            if (!aligned16(o->f_init_dev)) {
                set_error("f_init_dev must be a 16-byte aligned device pointer");
                return CBCT_ERR_INVALID_ARG;
            }
        }
    }
    return CBCT_OK;
}

extern "C" {

const char *cbct_last_error(void) { return cbct::last_error(); }

const char *cbct_version(void) { return "cbct-fbs-b300 0.1 (sm_103a)"; }

cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, const double *angles_host, int n_angles,
                                 cbct_geometry **out) {
    if (!out) {
        set_error("out is null");
        return CBCT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    ST(check_geometry_desc(desc));
    if (!angles_host || n_angles < 1 || n_angles > 65535) {
        set_error("need 1..65535 angles");
        return CBCT_ERR_INVALID_ARG;
    }
    if ((double)n_angles * desc->nu * desc->nv >= 2147483647.0) {
        set_error("sinogram must have fewer than 2^31 pixels");
        return CBCT_ERR_INVALID_ARG;
    }
    for (int q = 0; q < n_angles; ++q)
        if (!isfinite(angles_host[q])) {
            set_error("angle %d is not finite", q);
            return CBCT_ERR_INVALID_ARG;
        }
    cbct_geometry *G = new cbct_geometry();
    G->desc = *desc;
    G->angles.assign(angles_host, angles_host + n_angles);
    if (cudaGetDevice(&G->device) != cudaSuccess) {
        cudaGetLastError();
        delete G;
        set_error("no CUDA device available");
        return CBCT_ERR_CUDA;
    }
    Level *L = nullptr;
    cbct_status st = ensure_level(G, 0, &L);
    if (st == CBCT_OK) st = ensure_trace(G, 0);
    if (st != CBCT_OK) {
        cbct_geometry_destroy(G);
        return st;
    }
    *out = G;
    return CBCT_OK;
}

void cbct_geometry_destroy(cbct_geometry *G) {
    if (!G) return;
    if (G->side) {
        cudaStreamSynchronize(G->side);
        cudaStreamDestroy(G->side);
        cudaEventDestroy(G->side_fork);
        for (auto e : G->side_done) cudaEventDestroy(e);
        cudaFreeHost(G->host_lam);
    }
    for (auto *L : G->levels) free_level(L);
    cudaFree(G->dscalars);
    cudaFree(G->dcounter);
    cudaFree(G->dtrace);
    delete G;
}

cbct_status cbct_level_dims(const cbct_geometry *G, int level, int dims_out[5]) {
    if (!G || !dims_out || level < 0 || level > 12) {
        set_error("bad arguments to cbct_level_dims");
        return CBCT_ERR_INVALID_ARG;
    }
    const int s = 1 << level;
    const cbct_geometry_desc &d = G->desc;
    dims_out[0] = (d.nx + s - 1) / s;
    dims_out[1] = (d.ny + s - 1) / s;
    dims_out[2] = (d.nz + s - 1) / s;
    dims_out[3] = (d.nu + s - 1) / s;
    dims_out[4] = (d.nv + s - 1) / s;
    return CBCT_OK;
}

cbct_status cbct_project(cbct_geometry *G, const float *f_dev, float *y_dev, cudaStream_t s) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(f_dev, "f_dev"));
    ST(need_ptr(y_dev, "y_dev"));
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    const GeoDev &g = L->gd;
    CK(launch_vol_to_internal(f_dev, L->A, g.nx, g.ny, g.nz, s), "volume layout");
    CK(launch_project(g, L->A, nullptr, nullptr, L->rs, nullptr, PROJ_PLAIN, s, nullptr), "projection");
    CK(launch_sino_to_api(L->rs, y_dev, g.na, g.nu, g.nv, s), "sinogram layout");
    return CBCT_OK;
}

cbct_status cbct_backproject(cbct_geometry *G, const float *y_dev, float *f_dev, cudaStream_t s) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(y_dev, "y_dev"));
    ST(need_ptr(f_dev, "f_dev"));
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    const GeoDev &g = L->gd;
    CK(launch_sino_to_internal(y_dev, L->rs, nullptr, g.ray_z, g.na, g.nu, g.nv, s), "sinogram layout");
    CK(launch_backproject(g, L->rs, nullptr, L->A, 0.f, BP_PLAIN, s), "backprojection");
    CK(launch_vol_to_api(L->A, f_dev, g.nx, g.ny, g.nz, s), "volume layout");
    return CBCT_OK;
}

cbct_status cbct_backproject_eq2(cbct_geometry *G, const float *y_dev, float *f_dev, cudaStream_t s) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(y_dev, "y_dev"));
    ST(need_ptr(f_dev, "f_dev"));
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    ST(ensure_eq2_pad(L, s));
    const GeoDev &g = L->gd;
    CK(launch_sino_to_internal(y_dev, L->rs, nullptr, nullptr, g.na, g.nu, g.nv, s), "sinogram layout");
    CK(launch_backproject_eq2(g, L->rs, L->eq2p, nullptr, L->A, (float)eq2_scale(L), BP_PLAIN, s),
       "eq2 backprojection");
    CK(launch_vol_to_api(L->A, f_dev, g.nx, g.ny, g.nz, s), "volume layout");
    return CBCT_OK;
}


unsigned long long cbct_kernel_launch_count(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

cbct_status cbct_tv_prox(cbct_geometry *G, const float *g_dev, float *f_inout_dev, double beta, double eps,
                         int inner_iters, int tv_mode, cudaStream_t s) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(g_dev, "g_dev"));
    ST(need_ptr(f_inout_dev, "f_inout_dev"));
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    SolveParams P;
    ST(solve_params(L, 1.0, beta, eps, inner_iters, 0, false, &P, tv_mode));
    const GeoDev &g = L->gd;
    CK(launch_vol_to_internal(g_dev, L->g, g.nx, g.ny, g.nz, s), "volume layout");
    CK(launch_vol_to_internal(f_inout_dev, L->f, g.nx, g.ny, g.nz, s), "volume layout");
    Prof prof;
    ST(enqueue_prox(L, P, L->f, nullptr, nullptr, nullptr, nullptr, prof, s));
    CK(launch_vol_to_api(L->f, f_inout_dev, g.nx, g.ny, g.nz, s), "volume layout");
    return CBCT_OK;
}

cbct_status cbct_fbs(cbct_geometry *G, const float *Y_dev, double mu, double beta, double eps, int inner_iters,
                     int clamp_mode, int tv_mode, int iters, float *f_inout_dev, double *energy_trace,
                     double *step_trace, cudaStream_t s) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(Y_dev, "Y_dev"));
    ST(need_ptr(f_inout_dev, "f_inout_dev"));
    if (iters < 0 || !(mu > 0) || !isfinite(mu)) {
        set_error("need iters >= 0 and mu > 0");
        return CBCT_ERR_INVALID_ARG;
    }
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    SolveParams P;
    ST(solve_params(L, mu, beta, eps, inner_iters, clamp_mode, false, &P, tv_mode));
    double *dtrace;
    ST(get_trace(G, TRACE_W * (size_t)std::max(iters, 1), &dtrace));
    const GeoDev &g = L->gd;
    CK(launch_sino_to_internal(Y_dev, L->Y, nullptr, nullptr, g.na, g.nu, g.nv, s), "sinogram layout");
    CK(launch_vol_to_internal(f_inout_dev, L->f, g.nx, g.ny, g.nz, s), "volume layout");
    Prof prof;
    ST(run_level(G, L, P, iters, dtrace, false, prof, s));
    CK(launch_vol_to_api(L->f, f_inout_dev, g.nx, g.ny, g.nz, s), "volume layout");
    if ((energy_trace || step_trace) && iters > 0) {
        ST(copy_trace(dtrace, iters, energy_trace, step_trace, s));
        CK(cudaStreamSynchronize(s), "fbs");
    }
    return CBCT_OK;
}

cbct_status cbct_power_iteration(cbct_geometry *G, int iters, double *lambda_out, cudaStream_t s) {
    if (!G || !lambda_out || iters < 1) {
        set_error("need a geometry, an output pointer and iters >= 1");
        return CBCT_ERR_INVALID_ARG;
    }
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    Prof prof;
    return power_iteration(G, L, iters, lambda_out, prof, s);
}

cbct_status cbct_energy(cbct_geometry *G, const float *Y_dev, const float *f_dev, double mu, double eps,
                        int tv_mode, double out_host[3], cudaStream_t s) {
    if (!G || !out_host) {
        set_error("null argument");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(Y_dev, "Y_dev"));
    ST(need_ptr(f_dev, "f_dev"));
    Level *L;
    ST(ensure_level(G, 0, &L));
    ST(ensure_workspace(L, false));
    if (!(eps >= 0) || !isfinite(eps)) {
        set_error("eps must be >= 0");
        return CBCT_ERR_INVALID_ARG;
    }
    SolveParams P;
    ST(solve_params(L, mu, 1.0, eps > 0 ? eps : 1.0, 1, 0, false, &P, tv_mode));
    P.eps2 = (float)(eps * eps);  // eps = 0: the unsmoothed TV (the energy pass takes square roots in float64)
    double *dtrace;
    ST(get_trace(G, TRACE_W, &dtrace));
    const GeoDev &g = L->gd;
    CK(launch_sino_to_internal(Y_dev, L->Y, nullptr, nullptr, g.na, g.nu, g.nv, s), "sinogram layout");
    CK(launch_vol_to_internal(f_dev, L->A, g.nx, g.ny, g.nz, s), "volume layout");
    int nb_p = 0, nb_t = 0;
    double *pp = L->partial, *pt = L->partial + project_partials(g);
    CK(launch_project(g, L->A, L->Y, nullptr, L->rs, pp, PROJ_RESID32, s, &nb_p), "projection");
    CK(launch_tv_energy(tv_args(L, P), L->A, pt, s, &nb_t), "tv energy");
    CK(cudaMemsetAsync(G->dcounter, 0, sizeof(int), s), "counter");
    CK(launch_energy_finalize(pp, nb_p, pt, nb_t, P.inv_nv, P.mu_over_nr, dtrace, G->dcounter, s), "energy");
    CK(cudaMemcpyAsync(out_host, dtrace, 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "energy copy");
    CK(cudaStreamSynchronize(s), "energy");
    return CBCT_OK;
}

cbct_status cbct_reconstruct(cbct_geometry *G, const float *Y_dev, const double *angles_host, int n_angles,
                             double mu, int iters, int levels, const cbct_options *opts, float *f_out_dev,
                             cudaStream_t s) {
    if (!G) {
        set_error("geometry is null");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(Y_dev, "Y_dev"));
    ST(need_ptr(f_out_dev, "f_out_dev"));
    if (!angles_host || n_angles != (int)G->angles.size()) {
        set_error("angles must be the geometry's %d angles", (int)G->angles.size());
        return CBCT_ERR_INVALID_ARG;
    }
    for (int q = 0; q < n_angles; ++q)
        if (angles_host[q] != G->angles[q]) {
            set_error("angle %d differs from the geometry's", q);
            return CBCT_ERR_INVALID_ARG;
        }
    if (!(mu > 0) || !isfinite(mu) || iters < 0) {
        set_error("need mu > 0 and iters >= 0");
        return CBCT_ERR_INVALID_ARG;
    }
    const cbct_geometry_desc &d = G->desc;
    if (levels < 1 || levels > 8) {
        set_error("levels must be in 1..8");
        return CBCT_ERR_INVALID_ARG;
    }
    const int need = 1 << (levels - 1);
    if (d.nx < need || d.ny < need || d.nz < need || d.nu < need || d.nv < need) {
        set_error("every volume and imager axis needs at least 2^(levels-1) = %d samples", need);
        return CBCT_ERR_INVALID_ARG;
    }
    cbct_options o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    const int M = o.inner_iters > 0 ? o.inner_iters : 10;
    const int K = o.power_iters > 0 ? o.power_iters : 30;
    const bool fp16 = o.sino_fp16 != 0;
    int start = levels - 1;
    if (o.f_init_dev) {
        if (o.start_level < 0 || o.start_level >= levels) {
            set_error("start_level must be in 0..levels-1");
            return CBCT_ERR_INVALID_ARG;
        }
        ST(need_ptr(o.f_init_dev, "f_init_dev"));
        start = o.start_level;
    }

    if (o.mg_cycle != 0 && o.mg_cycle != 1) {
        set_error("mg_cycle must be 0 or 1");
        return CBCT_ERR_INVALID_ARG;
    }
    if (o.mg_cycle == 1) {
        if (o.mg_pre < 0 || o.mg_post < 0 || o.mg_coarse < 0 || (o.f_init_dev && o.start_level != 0)) {
            set_error("V-cycles need mg_pre, mg_post, mg_coarse >= 0 and start from level 0");
            return CBCT_ERR_INVALID_ARG;
        }
        if (o.clamp_mode != 0 || o.adjoint_mode != 0) {
            set_error("V-cycles use clamp_mode 0 and the exact adjoint");
            return CBCT_ERR_UNSUPPORTED;
        }
    }
    std::vector<Level *> Ls(levels);
    for (int l = 0; l < levels; ++l) {
        ST(ensure_level(G, l, &Ls[l]));
        ST(ensure_workspace(Ls[l], fp16));
        if (o.adjoint_mode == 1) ST(ensure_eq2_pad(Ls[l], s));
    }
    double *dtrace;
    ST(get_trace(G, TRACE_W * (size_t)std::max(iters, 1), &dtrace));
    Prof prof;
    prof.G = G;
    prof.s = s;
    prof.on = o.kernel_ms != nullptr || o.kernel_launches != nullptr || o.kernel_ms_finest != nullptr ||
              o.kernel_launches_finest != nullptr;
    if (o.kernel_mask) prof.mask = o.kernel_mask;
    if (prof.on) G->events.release_all();

    // data pyramid: finest level from the caller's stack, coarser by 2x2 binning
    {
        Launch l(prof, CBCT_K_TRANSFER);
        const GeoDev &g0 = Ls[0]->gd;
        CK(launch_sino_to_internal(Y_dev, Ls[0]->Y, fp16 ? Ls[0]->Yh : nullptr, nullptr, g0.na, g0.nu, g0.nv, s),
           "sinogram layout");
    }
    for (int l = 1; l < levels; ++l) {
        Launch lz(prof, CBCT_K_TRANSFER);
        const GeoDev &gp = Ls[l - 1]->gd;
        CK(launch_restrict(Ls[l - 1]->Y, Ls[l]->Y, gp.na, gp.nu, gp.nv, s), "restriction");
        if (fp16) CK(launch_to_half(Ls[l]->Y, Ls[l]->Yh, sino_elems(Ls[l]->gd), s), "half copy");
    }

    // Cascade with the automatic beta: the power iterations of the finer levels depend
    // on the geometry alone, so they run on the geometry's side stream while the
    // coarser levels iterate; a level waits for its own before its buffers are reused.
    // The kernels and their inputs are those of the plain order, so is every bit.
    bool side_lam[13] = {};
    if (o.mg_cycle != 1 && !o.serial_power && !o.betas && !(o.beta > 0) && start > 0) {
        bool any = false;
        for (int l = start - 1; l >= 0; --l) any = any || !(o.reuse_lambda && Ls[l]->lambda_iters == K);
        if (any) {
            ST(ensure_side(G));
            CK(cudaEventRecord(G->side_fork, s), "fork");
            CK(cudaStreamWaitEvent(G->side, G->side_fork, 0), "fork");
            for (int l = start - 1; l >= 0; --l) {
                if (o.reuse_lambda && Ls[l]->lambda_iters == K) continue;
                double *dl = G->dscalars + 16 + 2 * l;
                ST(enqueue_power(Ls[l], K, dl, (float *)(dl + 1), prof, G->side));
                CK(cudaMemcpyAsync(G->host_lam + l, dl, sizeof(double), cudaMemcpyDeviceToHost, G->side),
                   "lambda copy");
                CK(cudaEventRecord(G->side_done[l], G->side), "join");
                side_lam[l] = true;
            }
        }
    }

    auto level_beta = [&](int l, double *beta) -> cbct_status {
        Level *L = Ls[l];
        if (o.betas) {
            *beta = o.betas[l];
        } else if (o.beta > 0) {
            *beta = o.beta;
        } else {
            double lam = 0.0;
            if (side_lam[l]) {  // computed on the side stream
                CK(cudaEventSynchronize(G->side_done[l]), "power iteration");
                CK(cudaStreamWaitEvent(s, G->side_done[l], 0), "join");
                lam = G->host_lam[l];
                L->lambda = lam;
                L->lambda_iters = K;
            } else if (o.reuse_lambda && L->lambda_iters == K) {
                lam = L->lambda;
            } else {
                ST(power_iteration(G, L, K, &lam, prof, s));
                L->lambda = lam;
                L->lambda_iters = K;
            }
            *beta = std::max(10.0 * mu, 1.05 * gamma_of(L, mu) * lam);
        }
        if (o.beta_out) o.beta_out[l] = *beta;
        return CBCT_OK;
    };

    if (o.mg_cycle == 1) {  // V-cycles from f = 0 on the finest level
        VCycle V;
        V.G = G;
        V.Ls = Ls;
        V.levels = levels;
        V.pre = o.mg_pre > 0 ? o.mg_pre : 2;
        V.post = o.mg_post > 0 ? o.mg_post : 2;
        V.coarse = o.mg_coarse > 0 ? o.mg_coarse : 10;
        V.graphs = o.use_graphs != 0;
        V.mu = mu;
        V.prof = &prof;
        V.s = s;
        ST(get_trace(G, TRACE_W * (size_t)std::max({V.pre, V.post, V.coarse, 1}), &V.dtrace));
        V.P.resize(levels);
        for (int l = 0; l < levels; ++l) {
            ST(ensure_mg_workspace(Ls[l]));
            double beta;
            ST(level_beta(l, &beta));
            const double eps = o.eps > 0 ? o.eps : default_eps(Ls[l]);
            ST(solve_params(Ls[l], mu, beta, eps, M, 0, fp16, &V.P[l], o.tv_mode, 0));
        }
        if (o.f_init_dev) {
            const GeoDev &g0 = Ls[0]->gd;
            CK(launch_vol_to_internal(o.f_init_dev, Ls[0]->f, g0.nx, g0.ny, g0.nz, s), "volume layout");
        } else {
            CK(cudaMemsetAsync(Ls[0]->f, 0, vol_elems(Ls[0]->gd) * 4, s), "zero start");
        }
        for (int c = 0; c < iters; ++c) {
            if (o.step_trace) {
                Launch lz(prof, CBCT_K_REDUCE);
                CK(cudaMemcpyAsync(V.x0(0), Ls[0]->f, vol_elems(Ls[0]->gd) * 4, cudaMemcpyDeviceToDevice, s),
                   "copy");
            }
            ST(V.cycle(0, nullptr));
            if (o.step_trace) ST(V.change(0, V.x0(0), &o.step_trace[c]));
            if (o.energy_trace) {
                double e[4];
                ST(V.energy(0, Ls[0]->f, nullptr, e));
                for (int q = 0; q < 3; ++q) o.energy_trace[3 * (size_t)c + q] = e[q];
            }
        }
        if (o.mg_accepted)
            for (int l = 0; l < levels; ++l) o.mg_accepted[l] = V.accepted[l];
        {
            Launch lz(prof, CBCT_K_TRANSFER);
            const GeoDev &g0 = Ls[0]->gd;
            CK(launch_vol_to_api(Ls[0]->f, f_out_dev, g0.nx, g0.ny, g0.nz, s), "volume layout");
        }
        return prof.collect(o.kernel_ms, o.kernel_launches, o.kernel_ms_finest, o.kernel_launches_finest);
    }

    std::vector<cudaEvent_t> lev_a(levels, nullptr), lev_b(levels, nullptr);
    if (o.level_ms && !prof.on) G->events.release_all();
    for (int l = start; l >= 0; --l) {
        Level *L = Ls[l];
        const GeoDev &g = L->gd;
        if (l == start) {
            Launch lz(prof, CBCT_K_TRANSFER);
            if (o.f_init_dev)
                CK(launch_vol_to_internal(o.f_init_dev, L->f, g.nx, g.ny, g.nz, s), "volume layout");
            else
                CK(cudaMemsetAsync(L->f, 0, vol_elems(g) * 4, s), "zero start");
        } else {
            Launch lz(prof, CBCT_K_TRANSFER);
            const GeoDev &gc = Ls[l + 1]->gd;
            CK(launch_prolong(Ls[l + 1]->f, gc.nx, gc.ny, gc.nz, L->f, g.nx, g.ny, g.nz, s), "prolongation");
        }
        double beta;
        ST(level_beta(l, &beta));
        const double eps = o.eps > 0 ? o.eps : default_eps(L);
        SolveParams P;
        ST(solve_params(L, mu, beta, eps, M, o.clamp_mode, fp16, &P, o.tv_mode, o.adjoint_mode));
        prof.tag = l == 0 ? 1 : 0;
        if (o.level_ms) {
            lev_a[l] = G->events.get();
            if (!lev_a[l]) return cuda_fail(cudaErrorMemoryAllocation, "level timing event");
            CK(cudaEventRecord(lev_a[l], s), "level timing");
        }
        ST(run_level(G, L, P, iters, dtrace, o.use_graphs != 0, prof, s));
        if (o.level_ms) {
            lev_b[l] = G->events.get();
            if (!lev_b[l]) return cuda_fail(cudaErrorMemoryAllocation, "level timing event");
            CK(cudaEventRecord(lev_b[l], s), "level timing");
        }
        prof.tag = 0;
        if ((o.energy_trace || o.step_trace) && iters > 0) {
            const size_t lv = (size_t)iters * (levels - 1 - l);
            ST(copy_trace(dtrace, iters, o.energy_trace ? o.energy_trace + 3 * lv : nullptr,
                          o.step_trace ? o.step_trace + lv : nullptr, s));
            CK(cudaStreamSynchronize(s), "trace sync");
        }
    }
    {
        Launch lz(prof, CBCT_K_TRANSFER);
        const GeoDev &g0 = Ls[0]->gd;
        CK(launch_vol_to_api(Ls[0]->f, f_out_dev, g0.nx, g0.ny, g0.nz, s), "volume layout");
    }
    if (o.level_ms) {
        CK(cudaStreamSynchronize(s), "synchronising for level timing");
        for (int l = 0; l < levels; ++l) {
            float t = 0.f;
            if (lev_a[l] && lev_b[l]) CK(cudaEventElapsedTime(&t, lev_a[l], lev_b[l]), "level timing");
            o.level_ms[l] = t;
        }
        if (!prof.on) G->events.release_all();
    }
    return prof.collect(o.kernel_ms, o.kernel_launches, o.kernel_ms_finest, o.kernel_launches_finest);
}

cbct_status cbct_restrict_sino(int n_angles, int nv, int nu, const float *y_dev, float *y_coarse_dev,
                               cudaStream_t s) {
    if (n_angles < 1 || nv < 1 || nu < 1) {
        set_error("sizes must be >= 1");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(y_dev, "y_dev"));
    ST(need_ptr(y_coarse_dev, "y_coarse_dev"));
    CK(launch_restrict(y_dev, y_coarse_dev, n_angles, nv, nu, s), "restriction");
    return CBCT_OK;
}

cbct_status cbct_prolong_vol(int nxc, int nyc, int nzc, const float *fc_dev, int nx, int ny, int nz, float *f_dev,
                             cudaStream_t s) {
    if (nxc < 1 || nyc < 1 || nzc < 1 || nx < 1 || ny < 1 || nz < 1) {
        set_error("sizes must be >= 1");
        return CBCT_ERR_INVALID_ARG;
    }
    ST(need_ptr(fc_dev, "fc_dev"));
    ST(need_ptr(f_dev, "f_dev"));
    CK(launch_prolong(fc_dev, nzc, nyc, nxc, f_dev, nz, ny, nx, s), "prolongation");
    return CBCT_OK;
}

}  // extern "C"
