// Continuous-batching reconstruction server.
//
// A worker thread owns a CUDA stream, a pool of slots and a batched Engine.  A slot
// holds one geometry (ray tables and device workspaces) and serves one request at a
// time; a later request with the same scan geometry reuses it, keeping its tables,
// workspaces and cached step size resident.  Requests are admitted in arrival order
// whenever a slot is free, the device memory of the geometries in use stays within
// the budget (idle geometries are released, least recently used first, to make
// room), and the requests already running do not fill the GPU: each request's
// per-tick work is rated against what keeps every SM busy, and a new request joins
// only while the running ones sum to less than one GPU.  Small requests therefore
// run side by side, large ones one after another (first come, first served).
// Admitted requests join the engine between ticks, so work of requests that arrived
// at different times overlaps on the device; each request's arithmetic is exactly
// that of its own cbct_reconstruct call.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "batch.h"

using namespace cbct;

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct Slot {
    cbct_geometry *G = nullptr;
    cbct_geometry_desc desc{};
    std::vector<double> angles;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct Pending {
    uint64_t ticket = 0;
    cbct_server_request req{};
    std::vector<double> angles;
    std::vector<double> betas;
    Clock::time_point t_submit;
    Clock::time_point t_admit;
    int slot = -1;
    double fill = 0.0;  // share of the GPU one tick of this request keeps busy
    Job job;
    cbct_result result{};
    bool done = false;
};

bool same_geometry(const Slot &s, const cbct_geometry_desc &d, const std::vector<double> &angles) {
    return s.G && memcmp(&s.desc, &d, sizeof(d)) == 0 && s.angles == angles;
}

// Device bytes a geometry needs for `levels` levels (tables and workspaces).
size_t geometry_bytes(const cbct_geometry_desc &d, int n_angles, int levels, bool fp16, bool eq2) {
    size_t total = 0;
    for (int l = 0; l < levels; ++l) {
        const int s = 1 << l;
        const size_t nx = (d.nx + s - 1) / s, ny = (d.ny + s - 1) / s, nz = (d.nz + s - 1) / s;
        const size_t nu = (d.nu + s - 1) / s, nv = (d.nv + s - 1) / s;
        const size_t vol = nx * ny * nz, sino = (size_t)n_angles * nu * nv;
        total += 4 * vol * 4 + sino * (4 + 4 + (fp16 ? 2 : 0));  // f, g, A, B; rs, Y, Yh
        total += (size_t)n_angles * nu * 24 + nu * nv * 24 + (size_t)n_angles * 8;  // ray tables
        total += (size_t)n_angles * nu * (nv + 1) * 8;                            // adjoint row sums
        if (eq2) total += (size_t)n_angles * (nu + 2) * (nv + 2) * 4;              // Eq. 2 padded residual
        total += (sino / 32 + vol / 128 + 4096) * 8;                                             // partials
    }
    return total + (1 << 20);
}

// Share of the GPU the finest level's adjoint of a request keeps busy: its warp tiles
// (z-columns in chunks of 64 voxels) against two waves of 32 resident warps per SM.
double gpu_fill(const cbct_geometry_desc &d, int sm_count) {
    const double tiles = (double)d.nx * d.ny * ((d.nz + 63) / 64);
    return std::min(1.0, tiles / (2.0 * 32.0 * std::max(sm_count, 1)));
}

}  // namespace

struct cbct_server {
    size_t budget = 0;
    int max_slots = 0;
    int device = 0;
    int sm_count = 148;
    cudaStream_t stream = nullptr;
    bool use_graphs = false;
    std::vector<Slot> slots;
    size_t used = 0;
    uint64_t next_ticket = 1, use_clock = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Pending>> queue;
    std::map<uint64_t, std::shared_ptr<Pending>> all;
    std::vector<std::shared_ptr<Pending>> running;
    bool stop = false;
    cbct_status fatal = CBCT_OK;
    std::thread worker;
    uint64_t completed = 0;
    double busy_s = 0.0;

    void run();
    bool try_admit(const std::shared_ptr<Pending> &p, std::unique_lock<std::mutex> &lk);
    void finish(const std::shared_ptr<Pending> &p, cbct_status st);
};

static std::atomic<int> g_fail_allocs{0};  // test hook: make the next n slot set-ups fail as if out of memory

extern "C" void cbct_debug_fail_next_allocations(int n) { g_fail_allocs = n; }

// Takes one injected failure if any is pending (workers may race for the last one).
static bool take_injected_failure() {
    int n = g_fail_allocs.load();
    while (n > 0 && !g_fail_allocs.compare_exchange_weak(n, n - 1)) {
    }
    return n > 0;
}

void cbct_server::finish(const std::shared_ptr<Pending> &p, cbct_status st) {
    p->result.status = st;
    p->result.latency_s = seconds_since(p->t_submit);
    p->result.queue_s = std::chrono::duration<double>(p->t_admit - p->t_submit).count();
    if (p->result.queue_s < 0) p->result.queue_s = 0;
    for (int l = 0; l < 8 && l < p->req.levels; ++l) p->result.betas[l] = p->job.o.beta_out ? p->job.o.beta_out[l] : 0;
    p->done = true;
    if (p->slot >= 0) {
        slots[p->slot].busy = false;
        slots[p->slot].last_use = ++use_clock;
    }
    ++completed;
}

// Admission: a free slot with this geometry, else a free slot and memory within the
// budget (releasing idle geometries, least recently used first).  Called with the
// lock held; slot set-up (allocation) runs with the lock released.
bool cbct_server::try_admit(const std::shared_ptr<Pending> &p, std::unique_lock<std::mutex> &lk) {
    const cbct_server_request &r = p->req;
    for (size_t q = 0; q < slots.size(); ++q)
        if (!slots[q].busy && same_geometry(slots[q], r.desc, p->angles)) {
            p->slot = (int)q;
            slots[q].busy = true;
            return true;
        }
    const size_t need = geometry_bytes(r.desc, r.n_angles, r.levels, r.opts.sino_fp16 != 0, r.opts.adjoint_mode == 1);
    if (need > budget) return false;  // rejected at submit; never admitted
    int free_slot = -1;
    for (size_t q = 0; q < slots.size(); ++q)
        if (!slots[q].busy && !slots[q].G) {
            free_slot = (int)q;
            break;
        }
    // release idle geometries (LRU) until the request fits and a slot is free
    while (used + need > budget || free_slot < 0) {
        int victim = -1;
        for (size_t q = 0; q < slots.size(); ++q)
            if (!slots[q].busy && slots[q].G && (victim < 0 || slots[q].last_use < slots[victim].last_use))
                victim = (int)q;
        if (victim < 0) return false;
        cbct_geometry_destroy(slots[victim].G);
        slots[victim].G = nullptr;
        used -= slots[victim].bytes;
        slots[victim].bytes = 0;
        if (free_slot < 0) free_slot = victim;
    }
    Slot &s = slots[free_slot];
    s.busy = true;
    p->slot = free_slot;
    lk.unlock();
    cbct_geometry *G = nullptr;
    cbct_status st;
    if (take_injected_failure()) {
        set_error("injected allocation failure");
        st = CBCT_ERR_OOM;
    } else {
        cudaSetDevice(device);
        st = cbct_geometry_create(&r.desc, p->angles.data(), r.n_angles, &G);
    }
    lk.lock();
    if (st != CBCT_OK) {
        s.busy = false;
        p->slot = -1;
        finish(p, st);
        return true;  // handled (failed); removed from the queue
    }
    s.G = G;
    s.desc = r.desc;
    s.angles = p->angles;
    s.bytes = need;
    used += need;
    return true;
}

void cbct_server::run() {
    cudaSetDevice(device);
    Engine E(stream, use_graphs);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // admit in arrival order while slots and memory allow and the GPU is not full
        while (!queue.empty() && !stop) {
            std::shared_ptr<Pending> p = queue.front();
            double load = 0.0;
            for (auto &q : running) load += q->fill;
            if (!running.empty() && load >= 1.0) break;
            if (!try_admit(p, lk)) break;
            queue.pop_front();
            if (p->done) {  // set-up failed
                cv_done.notify_all();
                continue;
            }
            p->t_admit = Clock::now();
            p->fill = gpu_fill(p->req.desc, sm_count);
            Job &j = p->job;
            j.G = slots[p->slot].G;
            j.Y = p->req.Y_dev;
            j.mu = p->req.mu;
            j.iters = p->req.iters;
            j.levels = p->req.levels;
            j.o = p->req.opts;
            j.o.betas = p->betas.empty() ? nullptr : p->betas.data();
            j.o.beta_out = p->result.betas;
            j.o.energy_trace = nullptr;
            j.o.step_trace = nullptr;
            j.o.kernel_ms = nullptr;
            j.o.kernel_launches = nullptr;
            j.o.kernel_ms_finest = nullptr;
            j.o.kernel_launches_finest = nullptr;
            j.o.level_ms = nullptr;
            j.f_out = p->req.f_out_dev;
            cbct_status st = E.add(&j);
            if (st != CBCT_OK) {
                finish(p, st);
                cv_done.notify_all();
                continue;
            }
            running.push_back(p);
        }
        if (stop && running.empty()) break;
        if (running.empty()) {
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            continue;
        }
        lk.unlock();
        const Clock::time_point t0 = Clock::now();
        cbct_status st = E.tick();
        bool any_done = false;
        for (auto &p : running)
            if (p->job.phase == PH_DONE) any_done = true;
        if (st == CBCT_OK && any_done) {
            cudaError_t e = cudaStreamSynchronize(stream);  // volumes written before hand-off
            if (e != cudaSuccess) st = cuda_fail(e, "server sync");
        }
        lk.lock();
        busy_s += seconds_since(t0);
        if (st != CBCT_OK) {  // a device error ends every request in flight
            fatal = st;
            for (auto &p : running) finish(p, st);
            running.clear();
            E.jobs.clear();
            cv_done.notify_all();
            continue;
        }
        for (auto &p : running)
            if (p->job.phase == PH_DONE) finish(p, CBCT_OK);
        running.erase(std::remove_if(running.begin(), running.end(), [](const std::shared_ptr<Pending> &p) {
                          return p->done;
                      }),
                      running.end());
        E.remove_finished();
        if (any_done) cv_done.notify_all();
    }
}

extern "C" cbct_status cbct_server_create(size_t hbm_budget_bytes, int max_slots, int use_graphs,
                                          cbct_server **out) {
    if (!out || max_slots < 1 || max_slots > 1024 || hbm_budget_bytes < (1u << 20)) {
        set_error("need an output pointer, 1..1024 slots and a budget of at least 1 MiB");
        return CBCT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cbct_server *S = new cbct_server();
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->slots.resize(max_slots);
    S->use_graphs = use_graphs != 0;
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        set_error("no CUDA device available for the server");
        return CBCT_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device) == cudaSuccess && sms > 0)
        S->sm_count = sms;
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_submit(cbct_server *S, const cbct_server_request *req, uint64_t *ticket) {
    if (!S || !req || !ticket) {
        set_error("null argument");
        return CBCT_ERR_INVALID_ARG;
    }
    if (!req->angles_host || req->n_angles < 1 || req->levels < 1 || req->levels > 8) {
        set_error("request needs angles and 1..8 levels");
        return CBCT_ERR_INVALID_ARG;
    }
    // validate the scan description and the solver arguments before queueing
    if (req->desc.nx < 1 || req->desc.ny < 1 || req->desc.nz < 1 || req->desc.nu < 1 || req->desc.nv < 1 ||
        !(req->desc.hx > 0) || !(req->desc.hy > 0) || !(req->desc.hz > 0) || !(req->desc.du > 0) ||
        !(req->desc.dv > 0) || !(req->desc.dso > 0) || !(req->desc.dsd > 0)) {
        set_error("malformed geometry description");
        return CBCT_ERR_INVALID_ARG;
    }
    cbct_geometry probe;
    probe.desc = req->desc;
    cbct_status st = validate_request(&probe, req->Y_dev, req->mu, req->iters, req->levels, &req->opts,
                                      req->f_out_dev);
    if (st != CBCT_OK) return st;
    const size_t need =
        geometry_bytes(req->desc, req->n_angles, req->levels, req->opts.sino_fp16 != 0, req->opts.adjoint_mode == 1);
    if (need > S->budget) {
        set_error("request needs about %zu bytes of device memory, above the server budget of %zu", need, S->budget);
        return CBCT_ERR_BUSY;
    }
    auto p = std::make_shared<Pending>();
    p->req = *req;
    p->angles.assign(req->angles_host, req->angles_host + req->n_angles);
    if (req->opts.betas) p->betas.assign(req->opts.betas, req->opts.betas + req->levels);
    p->t_submit = Clock::now();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
        set_error("server is shutting down");
        return CBCT_ERR_BUSY;
    }
    p->ticket = S->next_ticket++;
    *ticket = p->ticket;
    S->all[p->ticket] = p;
    S->queue.push_back(p);
    S->cv_work.notify_one();
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_wait(cbct_server *S, uint64_t ticket, int timeout_ms, cbct_result *result) {
    if (!S) {
        set_error("null server");
        return CBCT_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return CBCT_ERR_INVALID_ARG;
    }
    std::shared_ptr<Pending> p = it->second;
    const auto pred = [&] { return p->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        set_error("ticket %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
        return CBCT_ERR_TIMEOUT;
    }
    if (result) *result = p->result;
    S->all.erase(ticket);
    if (p->result.status != CBCT_OK) set_error("request failed with status %d", (int)p->result.status);
    return p->result.status;
}

extern "C" cbct_status cbct_server_cancel(cbct_server *S, uint64_t ticket) {
    if (!S) {
        set_error("null server");
        return CBCT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(S->mu);
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
        if ((*q)->ticket == ticket) {
            std::shared_ptr<Pending> p = *q;
            S->queue.erase(q);
            p->t_admit = p->t_submit;
            S->finish(p, CBCT_ERR_CANCELLED);
            S->cv_done.notify_all();
            return CBCT_OK;
        }
    set_error("ticket %llu is not queued (running, finished or unknown)", (unsigned long long)ticket);
    return CBCT_ERR_BUSY;
}

extern "C" cbct_status cbct_server_get_stats(cbct_server *S, cbct_server_stats *out) {
    if (!S || !out) {
        set_error("null argument");
        return CBCT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(S->mu);
    out->queued = (int)S->queue.size();
    out->running = (int)S->running.size();
    out->completed = S->completed;
    out->hbm_in_use = S->used;
    out->slots_in_use = 0;
    for (const Slot &s : S->slots) out->slots_in_use += s.busy ? 1 : 0;
    out->busy_s = S->busy_s;
    return S->fatal;
}

extern "C" void cbct_server_destroy(cbct_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        for (auto &p : S->queue) S->finish(p, CBCT_ERR_CANCELLED);
        S->queue.clear();
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (Slot &s : S->slots) cbct_geometry_destroy(s.G);
    cudaStreamDestroy(S->stream);
    delete S;
}
