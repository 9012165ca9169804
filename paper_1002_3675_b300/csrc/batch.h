// Batched execution engine (shared by cbct_reconstruct_batch and the server).
#pragma once

#include <vector>

#include "cbct_internal.h"

namespace cbct {

// Per-request items of the batched launches (device tables hold copies of these).
struct ProjItem {
    GeoDev G;
    const float *vol;
    const float *y32;
    const __half *y16;
    float *out;
    double *partial;
    int mode;
};

struct BpItem {
    GeoDev G;
    const float *rs;
    const float *fin;
    float *out;
    float c;
    int mode;
};

struct Eq2Item {  // Eq. 2 adjoint + gradient step of one request
    GeoDev G;
    const float *r;
    const float *fin;
    float *out;
    float cscale;
    int mode;
};

struct TvItem {
    TvArgs A;
    const float *fin;
    const float *g;
    float *fout;
    double *partial;
    int clamp;
    int acc;  // TV_ACC_NONE, TV_ACC_E1 or TV_ACC_STEP
    int xT;            // > 0: one x-marching launch of xT sweeps (solo only), clamping per xclamp
    unsigned xclamp;
};

struct VecItem {  // power-iteration helpers on one volume
    const float *x;
    const float *y;
    float *out;
    double *partial;
    double *lam;
    float *scale;
    long n;
    int nblk;
};

struct StepItem {  // prox result v moved into the iterate f, with the step-norm partials
    const float *v;
    float *f;
    double *partial;
    long n;
};

struct EnItem {
    const double *pe2;
    const double *pe1;
    const double *pstep;
    int nstep;
    double *trace;
    int *counter;
    double inv_nv, mu_over_nr;
    int n2, n1;
};


enum JobPhase { PH_PREPARE = 0, PH_START_LEVEL, PH_POWER, PH_POWER_DONE, PH_FBS, PH_LEVEL_DONE, PH_DONE };

// One reconstruction in flight: the arguments of cbct_reconstruct and its progress.
struct Job {
    cbct_geometry *G = nullptr;
    const float *Y = nullptr;
    double mu = 0.0;
    int iters = 0, levels = 1;
    cbct_options o{};
    float *f_out = nullptr;
    // progress
    int level = 0, it = 0, pi_it = 0, M = 10, K = 30;
    int phase = PH_PREPARE;
    bool fp16 = false;
    double beta = 0.0;
    SolveParams P{};
    std::vector<Level *> Ls;
    bool done_event_pending = false;
};

// Advances every job by one power-iteration step or one Algorithm A1 iteration per
// tick, all stages of all jobs in one batched launch per stage.
class Engine {
  public:
    Engine(cudaStream_t s, bool graphs);
    ~Engine();
    cbct_status add(Job *j);
    cbct_status tick();
    cbct_status run_all();
    bool busy() const;
    void remove_finished();
    std::vector<Job *> jobs;
    cudaStream_t stream;
    // jobs whose every stage fills the GPU by itself: each runs its whole tick on a
    // side stream (forked from and joined back to the engine's stream), so that the
    // tails of one job's kernels overlap the next job's
    struct Chain {
        Job *job = nullptr;
        bool power = false, eq2 = false;
        ProjItem proj;
        BpItem bp;
        Eq2Item eq;
        VecItem vec;
        std::vector<TvItem> tv;
        StepItem step{};
    };

  private:
    cbct_status prepare(Job *j);
    cbct_status start_level(Job *j);
    cbct_status begin_fbs(Job *j, double beta);
    cbct_status finish_level(Job *j);
    cbct_status build_tables();
    cbct_status launch_stages();
    void reset_graph();

    bool use_graphs;
    std::vector<long> signature;
    int same_ticks = 0;
    cudaGraphExec_t gexec = nullptr;
    // host copies of the item tables and their device blob
    struct ProjGroup {  // projector items with one block size: one launch
        int threads = 0, smem = 0, blocks = 1, first = 0, count = 0;
        long tiles = 0;
    };
    std::vector<ProjGroup> pgroups;
    std::vector<ProjItem> hproj;
    // stages that fill the GPU by themselves: their own single-request launches
    std::vector<ProjItem> solo_proj;
    std::vector<BpItem> solo_bp;
    std::vector<Eq2Item> solo_eq;
    std::vector<std::vector<TvItem>> solo_tv;
    std::vector<Chain> chains;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_events;
    cbct_status ensure_side(size_t n);
    std::vector<BpItem> hbp[4];
    std::vector<Eq2Item> heq;
    std::vector<VecItem> hdot;
    std::vector<std::vector<TvItem>> htv;
    std::vector<EnItem> hen;
    std::vector<long> tvtot;
    std::vector<StepItem> hstep;
    std::vector<Job *> tv_energy_jobs;
    long steptotal = 0;
    StepItem *d_step = nullptr;
    long *d_sstart = nullptr;
    long dtotal = 0, bptotal[4] = {0, 0, 0, 0}, eqtotal = 0;
    int max_m = 0;
    void *dblob = nullptr;
    size_t dblob_len = 0;
    ProjItem *d_proj = nullptr;
    long *d_pstart = nullptr;
    BpItem *d_bp[4] = {nullptr, nullptr, nullptr, nullptr};
    long *d_bstart[4] = {nullptr, nullptr, nullptr, nullptr};
    Eq2Item *d_eq = nullptr;
    long *d_eqstart = nullptr;
    VecItem *d_dot = nullptr;
    long *d_dstart = nullptr;
    std::vector<TvItem *> d_tv;
    std::vector<long *> d_tstart;
    EnItem *d_en = nullptr;
};

// Argument checks shared by cbct_reconstruct, the batch and the server.
cbct_status validate_request(cbct_geometry *G, const float *Y, double mu, int iters, int levels,
                             const cbct_options *o, float *f_out);

}  // namespace cbct
