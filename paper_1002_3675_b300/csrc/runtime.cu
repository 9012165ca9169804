// Geometry levels, device tables, workspaces, error state and event pool.
//
// The ray tables are computed in float64 on the host from the scan description
// (problem statement before Eq. 1: source, imager and angle define P^theta) and
// rounded once to float32; the projector and the adjoint read the same tables.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "cbct_internal.h"

namespace cbct {

std::atomic<unsigned long long> g_kernel_launches{0};


static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char *last_error() { return g_err; }

cbct_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CBCT_ERR_OOM : CBCT_ERR_CUDA;
}

cudaEvent_t EventPool::get() {
    cudaEvent_t e;
    if (!free_list.empty()) {
        e = free_list.back();
        free_list.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    used.push_back(e);
    return e;
}

void EventPool::release_all() {
    for (auto e : used) free_list.push_back(e);
    used.clear();
    cls.clear();
}

EventPool::~EventPool() {
    release_all();
    for (auto e : free_list) cudaEventDestroy(e);
}

static cbct_status dmalloc(void **p, size_t bytes, const char *what) {
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return CBCT_ERR_OOM;
    }
    return CBCT_OK;
}

void free_level(Level *L) {
    if (!L) return;
    cudaFree(L->tables);
    cudaFree(L->f);
    cudaFree(L->g);
    cudaFree(L->A);
    cudaFree(L->B);
    cudaFree(L->rs);
    cudaFree(L->gd.rowsum);
    cudaFree(L->Y);
    cudaFree(L->Yh);
    cudaFree(L->partial);
    cudaFree(L->mg);
    cudaFree(L->mg_partial);
    cudaFree(L->eq2p);
    delete L;
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Build the float64 geometry of a level and upload its float32 ray tables.
static cbct_status build_level(const cbct_geometry *G, int level, Level *L) {
    const cbct_geometry_desc &d = G->desc;
    const int s = 1 << level;
    L->nx = (d.nx + s - 1) / s;
    L->ny = (d.ny + s - 1) / s;
    L->nz = (d.nz + s - 1) / s;
    L->nu = (d.nu + s - 1) / s;
    L->nv = (d.nv + s - 1) / s;
    L->na = (int)G->angles.size();
    L->hx = d.hx * s;
    L->hy = d.hy * s;
    L->hz = d.hz * s;
    L->du = d.du * s;
    L->dv = d.dv * s;
    L->dso = d.dso;
    L->dsd = d.dsd;
    const double half_diag = 0.5 * sqrt((L->nx * L->hx) * (L->nx * L->hx) + (L->ny * L->hy) * (L->ny * L->hy));
    if (L->nu > 32767) {
        set_error("level %d: nu = %d above 32767", level, L->nu);
        return CBCT_ERR_INVALID_ARG;
    }
    if (!(L->dso > half_diag) || !(L->dsd - L->dso > half_diag)) {
        set_error("level %d: source circle (dso=%g) and imager (dsd-dso=%g) must clear the volume "
                  "half-diagonal %g", level, L->dso, L->dsd - L->dso, half_diag);
        return CBCT_ERR_INVALID_ARG;
    }

    const int na = L->na, nu = L->nu, nv = L->nv;
    const double cu = 0.5 * (nu - 1), cv = 0.5 * (nv - 1);
    std::vector<float4> ray_xy((size_t)na * nu);
    std::vector<float2> ray_e((size_t)na * nu);
    std::vector<float4> ray_z((size_t)nu * nv);
    std::vector<float2> ray_zc((size_t)nu * nv);
    std::vector<float2> col(nu);
    std::vector<float2> view(na);
    for (int a = 0; a < nu; ++a) {
        double ua = (a - cu) * L->du;
        double D = sqrt(L->dsd * L->dsd + ua * ua);
        double tS = L->dso * L->dsd / D;
        col[a] = make_float2((float)D, (float)tS);
        for (int b = 0; b < nv; ++b) {
            double vb = (b - cv) * L->dv;
            double tanp = vb / D;
            double zO = tS * tanp;
            double cotp = vb != 0.0 ? D / vb : 0.0;
            double secp = sqrt(D * D + vb * vb) / D;
            ray_z[(size_t)a * nv + b] = make_float4((float)zO, (float)cotp, (float)secp, (float)tanp);
            ray_zc[(size_t)a * nv + b] = make_float2((float)zO, (float)cotp);
        }
    }
    for (int ia = 0; ia < na; ++ia) {
        double c = cos(G->angles[ia]), sn = sin(G->angles[ia]);
        view[ia] = make_float2((float)c, (float)sn);
        double Sx = L->dso * c, Sy = L->dso * sn;
        for (int a = 0; a < nu; ++a) {
            double ua = (a - cu) * L->du;
            double dx = -L->dsd * c - ua * sn;
            double dy = -L->dsd * sn + ua * c;
            double D = sqrt(dx * dx + dy * dy);
            double ex = dx / D, ey = dy / D;
            double tS = -(Sx * ex + Sy * ey);
            double Ox = Sx + tS * ex, Oy = Sy + tS * ey;
            double ix = fabs(ex) > 1e-30 ? 1.0 / ex : 0.0;
            double iy = fabs(ey) > 1e-30 ? 1.0 / ey : 0.0;
            ray_xy[(size_t)ia * nu + a] = make_float4((float)Ox, (float)Oy, (float)ix, (float)iy);
            ray_e[(size_t)ia * nu + a] = make_float2((float)ex, (float)ey);
        }
    }
    size_t o_xy = 0;
    size_t o_e = align_up(o_xy + ray_xy.size() * sizeof(float4));
    size_t o_z = align_up(o_e + ray_e.size() * sizeof(float2));
    size_t o_zc = align_up(o_z + ray_z.size() * sizeof(float4));
    size_t o_col = align_up(o_zc + ray_zc.size() * sizeof(float2));
    size_t o_view = align_up(o_col + col.size() * sizeof(float2));
    size_t total = align_up(o_view + view.size() * sizeof(float2));
    cbct_status st = dmalloc(&L->tables, total, "ray tables");
    if (st != CBCT_OK) return st;
    char *base = (char *)L->tables;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(base + o_xy, ray_xy.data(), ray_xy.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_e, ray_e.data(), ray_e.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_z, ray_z.data(), ray_z.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_zc, ray_zc.data(), ray_zc.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_col, col.data(), col.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_view, view.data(), view.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "uploading ray tables");

    GeoDev &g = L->gd;
    g.nx = L->nx; g.ny = L->ny; g.nz = L->nz; g.nu = nu; g.nv = nv; g.na = na;
    g.hx = (float)L->hx; g.hy = (float)L->hy; g.hz = (float)L->hz;
    g.x0 = (float)(-0.5 * L->nx * L->hx);
    g.y0 = (float)(-0.5 * L->ny * L->hy);
    g.z0 = (float)(-0.5 * L->nz * L->hz);
    g.inv_hx = (float)(1.0 / L->hx); g.inv_hy = (float)(1.0 / L->hy); g.inv_hz = (float)(1.0 / L->hz);
    g.du = (float)L->du; g.dv = (float)L->dv;
    g.inv_du = (float)(1.0 / L->du); g.inv_dv = (float)(1.0 / L->dv);
    g.cu = (float)cu; g.cv = (float)cv;
    g.dso = (float)L->dso; g.dsd = (float)L->dsd;
    g.ray_xy = (const float4 *)(base + o_xy);
    g.ray_e = (const float2 *)(base + o_e);
    g.ray_z = (const float4 *)(base + o_z);
    g.ray_zc = (const float2 *)(base + o_zc);
    g.col = (const float2 *)(base + o_col);
    g.view = (const float2 *)(base + o_view);
    return CBCT_OK;
}

cbct_status ensure_level(cbct_geometry *G, int level, Level **out) {
    if (level < 0 || level > 12) {
        set_error("level %d out of range", level);
        return CBCT_ERR_INVALID_ARG;
    }
    if ((int)G->levels.size() <= level) G->levels.resize(level + 1, nullptr);
    if (!G->levels[level]) {
        Level *L = new Level();
        cbct_status st = build_level(G, level, L);
        if (st != CBCT_OK) {
            free_level(L);
            return st;
        }
        G->levels[level] = L;
    }
    *out = G->levels[level];
    return CBCT_OK;
}

cbct_status ensure_eq2_pad(Level *L, cudaStream_t s) {
    if (L->eq2p) return CBCT_OK;
    const size_t bytes = (size_t)L->na * (L->nu + 2) * (L->nv + 2) * sizeof(float);
    const cbct_status st = dmalloc((void **)&L->eq2p, bytes, "Eq. 2 padded residual");
    if (st != CBCT_OK) return st;
    const cudaError_t e = cudaMemsetAsync(L->eq2p, 0, bytes, s);
    if (e != cudaSuccess) {
        cudaFree(L->eq2p);
        L->eq2p = nullptr;
        return cuda_fail(e, "zeroing the Eq. 2 padded residual");
    }
    return CBCT_OK;
}

cbct_status ensure_workspace(Level *L, bool need_half) {
    const size_t nvox = vol_elems(L->gd), nr = sino_elems(L->gd);
    cbct_status st = CBCT_OK;
    if (!L->f && (st = dmalloc((void **)&L->f, nvox * 4, "volume f")) != CBCT_OK) return st;
    if (!L->g && (st = dmalloc((void **)&L->g, nvox * 4, "volume g")) != CBCT_OK) return st;
    if (!L->A && (st = dmalloc((void **)&L->A, nvox * 4, "volume A")) != CBCT_OK) return st;
    if (!L->B && (st = dmalloc((void **)&L->B, nvox * 4, "volume B")) != CBCT_OK) return st;
    if (!L->rs && (st = dmalloc((void **)&L->rs, nr * 4, "residual")) != CBCT_OK) return st;
    if (!L->gd.rowsum &&
        (st = dmalloc((void **)&L->gd.rowsum, (size_t)L->na * L->nu * (L->nv + 1) * sizeof(float2), "row sums")) !=
            CBCT_OK)
        return st;
    if (!L->Y && (st = dmalloc((void **)&L->Y, nr * 4, "data")) != CBCT_OK) return st;
    if (need_half && !L->Yh && (st = dmalloc((void **)&L->Yh, nr * 2, "half data")) != CBCT_OK) return st;
    // [projector partials][TV partials][step-norm partials]; the power iteration
    // reuses the front of the same buffer
    size_t need = project_partials(L->gd) + tv_region_len(L) +
                  std::max({step_partials(nvox), tv_partials(L->nx, L->ny, L->nz),
                            tv_x_partials_max(L->nx, L->ny, L->nz)});
    size_t dp = 2 * ((nvox + 255) / 256) + 16;
    if (dp > need) need = dp;
    need += 64;
    if (L->partial_len < need) {
        cudaFree(L->partial);
        L->partial = nullptr;
        if ((st = dmalloc((void **)&L->partial, need * sizeof(double), "partials")) != CBCT_OK) return st;
        L->partial_len = need;
    }
    return CBCT_OK;
}

// Length of the TV (E1) partials region of a level's partials buffer: enough for every
// sweep form and x-marching launch shape the level may take.
size_t tv_region_len(const Level *L) {
    return std::max({tv_partials(L->nx, L->ny, L->nz), tv_energy_partials(L->nx, L->ny, L->nz),
                     tv_x_partials_max(L->nx, L->ny, L->nz)});
}

// SM count of the current device, looked up once per device (atomics: the server's
// worker threads call this concurrently).
int device_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

double *step_region(Level *L) { return L->partial + project_partials(L->gd) + tv_region_len(L); }

cbct_status ensure_mg_workspace(Level *L) {
    const size_t nvox = vol_elems(L->gd);
    cbct_status st = CBCT_OK;
    if (!L->mg && (st = dmalloc((void **)&L->mg, 4 * nvox * 4, "multigrid volumes")) != CBCT_OK) return st;
    if (!L->mg_partial &&
        (st = dmalloc((void **)&L->mg_partial, (dot_partials(nvox) + 8) * sizeof(double), "multigrid partials")) !=
            CBCT_OK)
        return st;
    return CBCT_OK;
}

}  // namespace cbct
