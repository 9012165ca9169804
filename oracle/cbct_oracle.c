/*
 * FP64 CPU oracle for TV-regularised cone-beam CT reconstruction by forward-backward
 * splitting (Jia, Lou, Li, Song, Jiang, "GPU-based fast cone beam CT reconstruction
 * from undersampled and noisy projection data via total variation", 2010).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plainly written reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never does, and it
 * shares no code, header or table with the CUDA sources.
 *
 * Everything is double precision.  Readings of points the paper leaves open:
 *   - geometry: circular orbit about z, source (dso cos t, dso sin t, 0), flat imager
 *     at distance dsd from the source, one ray per pixel centre; the volume is centred
 *     on the origin, voxels are half-open boxes.  Volumes are [nz][ny][nx], projection
 *     stacks [na][nv][nu].
 *   - P^theta (problem statement before Eq. 1) is the exact intersection-length
 *     projector: (Pf)_ray = sum_j |ray ∩ box_j| f_j, computed by merging the ray's
 *     plane crossings (Siddon's parametric method).
 *   - the adjoint used in step 1 of Algorithm A1 is the exact matrix transpose named
 *     in the paragraph before Eq. 2; here it is a scatter over the same crossings
 *     (adjoint_mode 0).  adjoint_mode 1 takes Eq. 2 itself instead: per voxel centre
 *     and view, the residual bilinearly interpolated at the imager point (u*, v*)
 *     weighted by L^3/(L0 l^2), times dV/(du dv) so that it approximates P^T.
 *   - E1 (Eq. 1) is the isotropic TV with forward differences, Neumann boundary,
 *     smoothed as sqrt(|grad f|^2 + eps^2) (tv_mode 0).  tv_mode 1 is the anisotropic
 *     reading of the l1 norm of the gradient, sum_d sqrt((D_d f)^2 + eps^2).
 *   - step 2 of Algorithm A1 (a plain gradient descent in the paper) is projected gradient on
 *     TV_eps(f) + beta/2 |f - g|^2 over f >= 0 from f0 = f_k, step 1/(beta + L_TV),
 *     L_TV = (4/eps) sum_d h_d^-2; clamp_mode 1 instead descends from g without the
 *     bound and clamps afterwards (step 3 taken literally).
 *   - discrete scaling: Nv E = TV_eps + (gamma/2)|Pf - Y|^2, gamma = 2 mu Nv/(na Np);
 *     step 1 becomes g = f - (gamma/beta) P^T (Pf - Y).
 *   - multigrid (cited method [20]): coarse-to-fine cascade; 2x2 detector binning,
 *     cell-centred trilinear prolongation with edge replication.
 */
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int nu, nv;
    double du, dv;
    double dso, dsd;
    int na;
    const double *angles;
    int tv_mode;      /* 0: isotropic E1, 1: anisotropic E1 */
    int adjoint_mode; /* step 1 adjoint: 0 exact transpose, 1 Eq. 2 interpolation */
} or_geom;

/* ------------------------------------------------------------------------------ */
/* Rays                                                                            */
/* ------------------------------------------------------------------------------ */

/* Source and pixel-centre position of ray (ia, b, a). */
static void ray_endpoints(const or_geom *g, int ia, int b, int a, double S[3], double P[3])
{
    double c = cos(g->angles[ia]), s = sin(g->angles[ia]);
    double ua = (a - 0.5 * (g->nu - 1)) * g->du;
    double vb = (b - 0.5 * (g->nv - 1)) * g->dv;
    S[0] = g->dso * c;
    S[1] = g->dso * s;
    S[2] = 0.0;
    P[0] = S[0] - g->dsd * c - ua * s;
    P[1] = S[1] - g->dsd * s + ua * c;
    P[2] = vb;
}

/*
 * Siddon enumeration: every voxel the segment S->P crosses, with its intersection
 * length in mm.  Writes at most cap entries; returns the count.
 */
static int ray_segments(const or_geom *g, const double S[3], const double P[3],
                        long *idx, double *len, int cap, double *scratch)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const double h[3] = {g->hx, g->hy, g->hz};
    double lo[3], d[3];
    double amin = 0.0, amax = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        lo[ax] = -0.5 * n[ax] * h[ax];
        d[ax] = P[ax] - S[ax];
        double hi = lo[ax] + n[ax] * h[ax];
        if (d[ax] != 0.0) {
            double a1 = (lo[ax] - S[ax]) / d[ax], a2 = (hi - S[ax]) / d[ax];
            double e = a1 < a2 ? a1 : a2, x = a1 < a2 ? a2 : a1;
            if (e > amin) amin = e;
            if (x < amax) amax = x;
        } else if (S[ax] < lo[ax] || S[ax] >= hi) {
            return 0;  /* parallel to this axis' planes and outside the half-open slab */
        }
    }
    if (!(amax > amin)) return 0;
    double dlen = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);

    /*
     * Plane crossings strictly inside (amin, amax), one increasing list per axis, and
     * the number of each axis' planes already crossed at amin.  A segment's voxel index
     * along an axis is fixed by how many of that axis' planes the ray has crossed, so
     * it follows from the same crossing values that delimit the segments.
     */
    int cnt[3] = {0, 0, 0}, before[3] = {0, 0, 0};
    double *lists[3] = {scratch, scratch + n[0] + 1, scratch + n[0] + n[1] + 2};
    long fixed[3] = {0, 0, 0};
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0) {
            fixed[ax] = (long)floor((S[ax] - lo[ax]) / h[ax]);
            continue;
        }
        for (int q = 0; q <= n[ax]; ++q) {
            int p = d[ax] > 0 ? q : n[ax] - q;  /* visit planes in increasing alpha */
            double al = (lo[ax] + p * h[ax] - S[ax]) / d[ax];
            if (al <= amin) before[ax]++;
            else if (al < amax) lists[ax][cnt[ax]++] = al;
        }
    }
    /* Merge the three sorted lists between amin and amax. */
    int pos[3] = {0, 0, 0};
    double prev = amin;
    int out = 0;
    for (;;) {
        double next = amax;
        int which = -1;
        for (int ax = 0; ax < 3; ++ax)
            if (pos[ax] < cnt[ax] && lists[ax][pos[ax]] < next) {
                next = lists[ax][pos[ax]];
                which = ax;
            }
        if (next > prev) {
            long ijk[3];
            for (int ax = 0; ax < 3; ++ax) {
                long crossed = before[ax] + pos[ax];
                long v = d[ax] == 0.0 ? fixed[ax] : (d[ax] > 0 ? crossed - 1 : n[ax] - crossed);
                if (v < 0) v = 0;
                if (v > n[ax] - 1) v = n[ax] - 1;
                ijk[ax] = v;
            }
            if (out < cap) {
                idx[out] = (ijk[2] * g->ny + ijk[1]) * (long)g->nx + ijk[0];
                len[out] = (next - prev) * dlen;
                ++out;
            }
        }
        if (which < 0) break;
        pos[which]++;
        prev = next;
    }
    return out;
}

static int seg_cap(const or_geom *g) { return g->nx + g->ny + g->nz + 8; }

int or_ray_segments(const or_geom *g, int ia, int b, int a, long *idx, double *len, int cap)
{
    double S[3], P[3];
    double *scr = (double *)malloc(sizeof(double) * seg_cap(g));
    ray_endpoints(g, ia, b, a, S, P);
    int m = ray_segments(g, S, P, idx, len, cap, scr);
    free(scr);
    return m;
}

/* Forward projection: y[ia][b][a] = sum over crossed voxels of length * f. */
void or_project(const or_geom *g, const double *f, double *y)
{
    const long nrays = (long)g->na * g->nv * g->nu;
#pragma omp parallel
    {
        int cap = seg_cap(g);
        long *idx = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * 2 * cap);
        double *scr = len + cap;
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; ++r) {
            int a = (int)(r % g->nu), b = (int)((r / g->nu) % g->nv), ia = (int)(r / ((long)g->nu * g->nv));
            double S[3], P[3];
            ray_endpoints(g, ia, b, a, S, P);
            int m = ray_segments(g, S, P, idx, len, cap, scr);
            double acc = 0.0;
            for (int t = 0; t < m; ++t) acc += len[t] * f[idx[t]];
            y[r] = acc;
        }
        free(idx);
        free(len);
    }
}

double or_project_ray(const or_geom *g, const double *f, int ia, int b, int a)
{
    int cap = seg_cap(g);
    long *idx = (long *)malloc(sizeof(long) * cap);
    double *len = (double *)malloc(sizeof(double) * 2 * cap);
    double *scr = len + cap;
    double S[3], P[3];
    ray_endpoints(g, ia, b, a, S, P);
    int m = ray_segments(g, S, P, idx, len, cap, scr);
    double acc = 0.0;
    for (int t = 0; t < m; ++t) acc += len[t] * f[idx[t]];
    free(idx);
    free(len);
    return acc;
}

/* Number of (ray, voxel) pairs with positive intersection length. */
long long or_count_nnz(const or_geom *g)
{
    const long nrays = (long)g->na * g->nv * g->nu;
    long long total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int cap = seg_cap(g);
        long *idx = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * 2 * cap);
        double *scr = len + cap;
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; ++r) {
            int a = (int)(r % g->nu), b = (int)((r / g->nu) % g->nv), ia = (int)(r / ((long)g->nu * g->nv));
            double S[3], P[3];
            ray_endpoints(g, ia, b, a, S, P);
            total += ray_segments(g, S, P, idx, len, cap, scr);
        }
        free(idx);
        free(len);
    }
    return total;
}

/*
 * Adjoint (exact transpose of or_project): f[j] = sum over rays of length * y[ray].
 * Scatter over the same crossings; angles are split over private accumulators that
 * are summed in a fixed order.
 */
void or_backproject(const or_geom *g, const double *y, double *f)
{
    const long nv = (long)g->nx * g->ny * g->nz;
    int nbuf = 1;
#ifdef _OPENMP
    nbuf = omp_get_max_threads();
#endif
    if (nbuf > g->na) nbuf = g->na;
    long maxbuf = (long)(4.0e9 / (8.0 * (double)nv));
    if (maxbuf < 1) maxbuf = 1;
    if (nbuf > maxbuf) nbuf = (int)maxbuf;
    double *acc = (double *)calloc((size_t)nbuf * nv, sizeof(double));
#pragma omp parallel for schedule(static, 1) num_threads(nbuf)
    for (int bi = 0; bi < nbuf; ++bi) {
        int cap = seg_cap(g);
        long *idx = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * 2 * cap);
        double *scr = len + cap;
        double *mine = acc + (size_t)bi * nv;
        for (int ia = bi; ia < g->na; ia += nbuf)
            for (int b = 0; b < g->nv; ++b)
                for (int a = 0; a < g->nu; ++a) {
                    double S[3], P[3];
                    ray_endpoints(g, ia, b, a, S, P);
                    int m = ray_segments(g, S, P, idx, len, cap, scr);
                    double val = y[((long)ia * g->nv + b) * g->nu + a];
                    for (int t = 0; t < m; ++t) mine[idx[t]] += len[t] * val;
                }
        free(idx);
        free(len);
    }
#pragma omp parallel for schedule(static)
    for (long j = 0; j < nv; ++j) {
        double s = 0.0;
        for (int bi = 0; bi < nbuf; ++bi) s += acc[(size_t)bi * nv + j];
        f[j] = s;
    }
    free(acc);
}

/*
 * Eq. 2 read as an operator B on projection stacks (the paper's voxel-driven
 * evaluation of the variation of E2).  With r(u*, v*) the bilinear interpolation of
 * y between pixel centres (samples outside the pixel grid count as 0),
 *   (B y)_j = dV / (du dv) * sum_theta L^3(u*, v*) / (L0 l^2(x_j)) * r_theta(u*, v*),
 * where x_j is the voxel centre, (u*, v*) the imager point on the line from the
 * source through x_j, l = |x_j - S|, L = |(u*, v*) - S| and L0 = dsd.  Multiplying
 * Eq. 2 by Nv and writing A = Np du dv shows that B takes the place of P^T in
 * step 1 (the matched transpose of the problem statement).
 */
void or_backproject_eq2(const or_geom *g, const double *y, double *f)
{
    const double dV = g->hx * g->hy * g->hz;
    const double scale = dV / (g->du * g->dv);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double x = (i - 0.5 * (g->nx - 1)) * g->hx;
                double yy = (j - 0.5 * (g->ny - 1)) * g->hy;
                double z = (k - 0.5 * (g->nz - 1)) * g->hz;
                double acc = 0.0;
                for (int ia = 0; ia < g->na; ++ia) {
                    double c = cos(g->angles[ia]), s = sin(g->angles[ia]);
                    /* source frame: depth along the central ray, offsets along u and v */
                    double depth = g->dso - (x * c + yy * s);
                    double us = g->dsd * (-x * s + yy * c) / depth;
                    double vs = g->dsd * z / depth;
                    double dx = x - g->dso * c, dy = yy - g->dso * s;
                    double l2 = dx * dx + dy * dy + z * z;
                    double L = sqrt(g->dsd * g->dsd + us * us + vs * vs);
                    double w = L * L * L / (g->dsd * l2);
                    /* bilinear interpolation between pixel centres */
                    double fa = us / g->du + 0.5 * (g->nu - 1);
                    double fb = vs / g->dv + 0.5 * (g->nv - 1);
                    int a0 = (int)floor(fa), b0 = (int)floor(fb);
                    double ta = fa - a0, tb = fb - b0;
                    double r = 0.0;
                    for (int db = 0; db <= 1; ++db)
                        for (int da = 0; da <= 1; ++da) {
                            int a = a0 + da, b = b0 + db;
                            if (a < 0 || a >= g->nu || b < 0 || b >= g->nv) continue;
                            double wt = (da ? ta : 1.0 - ta) * (db ? tb : 1.0 - tb);
                            r += wt * y[((long)ia * g->nv + b) * g->nu + a];
                        }
                    acc += w * r;
                }
                f[((long)k * g->ny + j) * g->nx + i] = scale * acc;
            }
}

/*
 * Length of the segment S->P inside the half-open box [lo, hi): the slab method,
 * written independently of the Siddon enumeration above.
 */
static double box_length(const double S[3], const double P[3], const double lo[3], const double hi[3])
{
    double t0 = 0.0, t1 = 1.0, d2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        double d = P[ax] - S[ax];
        d2 += d * d;
        if (d == 0.0) {
            if (S[ax] < lo[ax] || S[ax] >= hi[ax]) return 0.0;
            continue;
        }
        double a = (lo[ax] - S[ax]) / d, b = (hi[ax] - S[ax]) / d;
        if (a > b) { double t = a; a = b; b = t; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
    }
    return t1 > t0 ? (t1 - t0) * sqrt(d2) : 0.0;
}

/* One voxel of the adjoint by brute force over every ray (slab test per ray). */
double or_backproject_voxel(const or_geom *g, const double *y, int i, int j, int k)
{
    double lo[3] = {(-0.5 * g->nx + i) * g->hx, (-0.5 * g->ny + j) * g->hy, (-0.5 * g->nz + k) * g->hz};
    double hi[3] = {lo[0] + g->hx, lo[1] + g->hy, lo[2] + g->hz};
    double *per_view = (double *)calloc(g->na, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int ia = 0; ia < g->na; ++ia) {
        double s = 0.0;
        for (int b = 0; b < g->nv; ++b)
            for (int a = 0; a < g->nu; ++a) {
                double S[3], P[3];
                ray_endpoints(g, ia, b, a, S, P);
                double L = box_length(S, P, lo, hi);
                if (L > 0.0) s += L * y[((long)ia * g->nv + b) * g->nu + a];
            }
        per_view[ia] = s;
    }
    double total = 0.0;
    for (int ia = 0; ia < g->na; ++ia) total += per_view[ia];
    free(per_view);
    return total;
}

/* Length of ray (ia, b, a) inside voxel (i, j, k), by the slab method. */
double or_ray_voxel_length(const or_geom *g, int ia, int b, int a, int i, int j, int k)
{
    double lo[3] = {(-0.5 * g->nx + i) * g->hx, (-0.5 * g->ny + j) * g->hy, (-0.5 * g->nz + k) * g->hz};
    double hi[3] = {lo[0] + g->hx, lo[1] + g->hy, lo[2] + g->hz};
    double S[3], P[3];
    ray_endpoints(g, ia, b, a, S, P);
    return box_length(S, P, lo, hi);
}

/* ------------------------------------------------------------------------------ */
/* Total variation (E1 of Eq. 1)                                                   */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int tv_mode; /* 0: isotropic, 1: anisotropic */
} or_vol;

#define VIDX(v, i, j, k) ((((long)(k)) * (v)->ny + (j)) * (long)(v)->nx + (i))

/* Forward differences / h with zero difference at the last index (Neumann). */
static void grad_at(const or_vol *v, const double *f, int i, int j, int k, double out[3])
{
    double c = f[VIDX(v, i, j, k)];
    out[0] = i < v->nx - 1 ? (f[VIDX(v, i + 1, j, k)] - c) / v->hx : 0.0;
    out[1] = j < v->ny - 1 ? (f[VIDX(v, i, j + 1, k)] - c) / v->hy : 0.0;
    out[2] = k < v->nz - 1 ? (f[VIDX(v, i, j, k + 1)] - c) / v->hz : 0.0;
}

/* Smoothed magnitude of one voxel's gradient: the term of TV_eps at that voxel. */
static double tv_term(const or_vol *v, const double gr[3], double eps)
{
    if (v->tv_mode == 1)
        return sqrt(gr[0] * gr[0] + eps * eps) + sqrt(gr[1] * gr[1] + eps * eps) + sqrt(gr[2] * gr[2] + eps * eps);
    return sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2] + eps * eps);
}

/*
 * TV_eps(f) = sum_j sqrt(|grad f|_j^2 + eps^2) (isotropic) or
 * sum_j sum_d sqrt((D_d f)_j^2 + eps^2) (anisotropic), summed slice by slice in a
 * fixed order.
 */
double or_tv(const or_vol *v, const double *f, double eps)
{
    double *slice = (double *)calloc(v->nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < v->nz; ++k) {
        double s = 0.0;
        for (int j = 0; j < v->ny; ++j)
            for (int i = 0; i < v->nx; ++i) {
                double gr[3];
                grad_at(v, f, i, j, k, gr);
                s += tv_term(v, gr, eps);
            }
        slice[k] = s;
    }
    double total = 0.0;
    for (int k = 0; k < v->nz; ++k) total += slice[k];
    free(slice);
    return total;
}

/*
 * Gradient of TV_eps: sum_d D_d^T p_d with p_d = D_d f / |grad f|_eps (isotropic) or
 * p_d = D_d f / sqrt((D_d f)^2 + eps^2) (anisotropic), and
 * (D_d^T p)_i = (p_{i-1} [i > 0] - p_i [i < n-1]) / h_d.
 */
void or_tv_grad(const or_vol *v, const double *f, double eps, double *out)
{
    const long n = (long)v->nx * v->ny * v->nz;
    double *p = (double *)malloc(sizeof(double) * 3 * n);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < v->nz; ++k)
        for (int j = 0; j < v->ny; ++j)
            for (int i = 0; i < v->nx; ++i) {
                double gr[3];
                grad_at(v, f, i, j, k, gr);
                long q = VIDX(v, i, j, k);
                for (int d = 0; d < 3; ++d) {
                    double nrm = v->tv_mode == 1 ? sqrt(gr[d] * gr[d] + eps * eps)
                                                 : sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2] + eps * eps);
                    p[3 * q + d] = gr[d] / nrm;
                }
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < v->nz; ++k)
        for (int j = 0; j < v->ny; ++j)
            for (int i = 0; i < v->nx; ++i) {
                long q = VIDX(v, i, j, k);
                double s = 0.0;
                s += ((i > 0 ? p[3 * VIDX(v, i - 1, j, k) + 0] : 0.0) - (i < v->nx - 1 ? p[3 * q + 0] : 0.0)) / v->hx;
                s += ((j > 0 ? p[3 * VIDX(v, i, j - 1, k) + 1] : 0.0) - (j < v->ny - 1 ? p[3 * q + 1] : 0.0)) / v->hy;
                s += ((k > 0 ? p[3 * VIDX(v, i, j, k - 1) + 2] : 0.0) - (k < v->nz - 1 ? p[3 * q + 2] : 0.0)) / v->hz;
                out[q] = s;
            }
    free(p);
}

/*
 * Lipschitz bound of grad TV_eps: (4/eps) sum_d h_d^-2 in both modes (each smoothed
 * magnitude has curvature at most 1/eps, and |D_d|^2 <= 4/h_d^2).
 */
double or_tv_lipschitz(const or_vol *v, double eps)
{
    return 4.0 / eps * (1.0 / (v->hx * v->hx) + 1.0 / (v->hy * v->hy) + 1.0 / (v->hz * v->hz));
}

/*
 * Step 2 (and 3) of Algorithm A1: M gradient steps on
 *   Phi(f) = w TV_eps(f) + beta/2 |f - g|^2,  step s = 1/(beta + w L_TV).
 * clamp_mode 0: start from f (the previous iterate, given in f), project onto f >= 0
 *               after every step.
 * clamp_mode 1: start from g, no bound during the descent, clamp once at the end.
 * w is the TV weight (1 for the method; 0 reduces the step to a projection).
 * If phi is non-null it receives Phi at the start and after each step (M + 1 values).
 */
void or_prox(const or_vol *v, const double *g, double *f, double beta, double eps, int M,
             int clamp_mode, double w, double *phi)
{
    const long n = (long)v->nx * v->ny * v->nz;
    double s = 1.0 / (beta + w * or_tv_lipschitz(v, eps));
    double *grad = (double *)malloc(sizeof(double) * n);
    if (clamp_mode == 1) memcpy(f, g, sizeof(double) * n);
    for (int m = 0; m <= M; ++m) {
        if (phi) {
            double q = 0.0;
            for (long j = 0; j < n; ++j) q += (f[j] - g[j]) * (f[j] - g[j]);
            phi[m] = w * or_tv(v, f, eps) + 0.5 * beta * q;
        }
        if (m == M) break;
        or_tv_grad(v, f, eps, grad);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < n; ++j) {
            double x = f[j] - s * (w * grad[j] + beta * (f[j] - g[j]));
            f[j] = (clamp_mode == 0 && x < 0.0) ? 0.0 : x;
        }
    }
    if (clamp_mode == 1)
        for (long j = 0; j < n; ++j)
            if (f[j] < 0.0) f[j] = 0.0;
    free(grad);
}

/* ------------------------------------------------------------------------------ */
/* Energy, step size and Algorithm A1                                              */
/* ------------------------------------------------------------------------------ */

static or_vol vol_of(const or_geom *g)
{
    or_vol v = {g->nx, g->ny, g->nz, g->hx, g->hy, g->hz, g->tv_mode};
    return v;
}

/* gamma = 2 mu Nv / (na Np): the data weight once Eq. 1 is multiplied by Nv. */
double or_gamma(const or_geom *g, double mu)
{
    double nvox = (double)g->nx * g->ny * g->nz;
    double nray = (double)g->na * g->nu * g->nv;
    return 2.0 * mu * nvox / nray;
}

/* Default TV smoothing: 1e-3 * 0.02 mm^-1 / min voxel size. */
double or_default_eps(const or_geom *g)
{
    double h = g->hx;
    if (g->hy < h) h = g->hy;
    if (g->hz < h) h = g->hz;
    return 1e-3 * 0.02 / h;
}

/*
 * Energy of Eq. 1 on the grid: E = TV_eps/Nv + mu/(na Np) |Pf - Y|^2.
 * out = {E, E1, E2-term}; r (optional, size na*nv*nu) receives Pf - Y.
 */
void or_energy(const or_geom *g, const double *Y, const double *f, double mu, double eps,
               double *out, double *r_opt)
{
    const long nr = (long)g->na * g->nv * g->nu;
    double *r = r_opt ? r_opt : (double *)malloc(sizeof(double) * nr);
    or_project(g, f, r);
    double q = 0.0;
    for (long t = 0; t < nr; ++t) {
        r[t] -= Y[t];
        q += r[t] * r[t];
    }
    or_vol v = vol_of(g);
    double e1 = or_tv(&v, f, eps) / ((double)g->nx * g->ny * g->nz);
    double e2 = mu * q / (double)nr;
    out[0] = e1 + e2;
    out[1] = e1;
    out[2] = e2;
    if (!r_opt) free(r);
}

/*
 * The start of the power iteration is a seeded uniform(0,1) volume.  Its values come
 * from SplitMix64 (Steele, Lea and Flood 2014, "Fast splittable pseudorandom number
 * generators"), used as a counter-based generator: value i of seed s is the 64-bit
 * finaliser applied to s + (i + 1) * 0x9E3779B97F4A7C15, and its top 24 bits make a
 * uniform number in [0, 1) that float32 holds exactly.
 */
uint64_t or_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double or_uniform01(uint64_t seed, uint64_t i)
{
    return (double)(or_splitmix64(seed, i) >> 40) * (1.0 / 16777216.0);
}

/* Fixed seed of the power iteration's start volume (voxel index in [nz][ny][nx] order). */
#define OR_POWER_SEED 10023675ull

/*
 * lambda_max(P^T P) by K power iterations (the step-size estimate of beta) from the
 * seeded uniform(0,1) volume, normalised; the estimate is the Rayleigh quotient
 * <x, P^T P x> of the last normalised iterate.
 */
double or_power_iteration(const or_geom *g, int K)
{
    const long nvox = (long)g->nx * g->ny * g->nz;
    const long nr = (long)g->na * g->nv * g->nu;
    double *x = (double *)malloc(sizeof(double) * nvox);
    double *y = (double *)malloc(sizeof(double) * nvox);
    double *p = (double *)malloc(sizeof(double) * nr);
    double uu = 0.0;
    for (long j = 0; j < nvox; ++j) {
        x[j] = or_uniform01(OR_POWER_SEED, (uint64_t)j);
        uu += x[j] * x[j];
    }
    for (long j = 0; j < nvox; ++j) x[j] /= sqrt(uu);  /* |x| = 1 */
    double lam = 0.0;
    for (int it = 0; it < K; ++it) {
        or_project(g, x, p);
        or_backproject(g, p, y);
        double xy = 0.0, yy = 0.0;
        for (long j = 0; j < nvox; ++j) {
            xy += x[j] * y[j];
            yy += y[j] * y[j];
        }
        lam = xy;
        double s = 1.0 / sqrt(yy);
        for (long j = 0; j < nvox; ++j) x[j] = y[j] * s;
    }
    free(x);
    free(y);
    free(p);
    return lam;
}

/* beta = max(10 mu, 1.05 gamma lambda_hat). */
double or_auto_beta(const or_geom *g, double mu, int K)
{
    double b = 1.05 * or_gamma(g, mu) * or_power_iteration(g, K);
    return b > 10.0 * mu ? b : 10.0 * mu;
}

/*
 * Algorithm A1 for `iters` iterations from the volume in f (updated in place).
 * trace (optional, 3 * iters): {E, E1, E2-term} of the iterate entering each iteration.
 * Step 1 uses the exact transpose, or B of Eq. 2 when g->adjoint_mode is 1.
 * lin (optional, one value per voxel) adds the linear term -<lin, f> to the energy
 * (the coarse-level model of a multigrid cycle); the trace reports E without it.
 * step (optional, iters): |f_{k+1} - f_k|_2 of each iteration.
 */
void or_fbs(const or_geom *g, const double *Y, double mu, double beta, double eps, int M,
            int clamp_mode, double tv_weight, int iters, double *f, double *trace, const double *lin,
            double *step)
{
    const long nvox = (long)g->nx * g->ny * g->nz;
    const long nr = (long)g->na * g->nv * g->nu;
    or_vol v = vol_of(g);
    double gamma = or_gamma(g, mu);
    double *r = (double *)malloc(sizeof(double) * nr);
    double *bp = (double *)malloc(sizeof(double) * nvox);
    double *gv = (double *)malloc(sizeof(double) * nvox);
    double *fprev = step ? (double *)malloc(sizeof(double) * nvox) : NULL;
    for (int it = 0; it < iters; ++it) {
        if (step) memcpy(fprev, f, sizeof(double) * nvox);
        /* step 1: g = f - (gamma/beta) P^T (P f - Y) */
        or_project(g, f, r);
        double q = 0.0;
        for (long t = 0; t < nr; ++t) {
            r[t] -= Y[t];
            q += r[t] * r[t];
        }
        if (trace) {
            double e1 = or_tv(&v, f, eps) / (double)nvox;
            double e2 = mu * q / (double)nr;
            trace[3 * it + 0] = e1 + e2;
            trace[3 * it + 1] = e1;
            trace[3 * it + 2] = e2;
        }
        if (g->adjoint_mode == 1)
            or_backproject_eq2(g, r, bp);
        else
            or_backproject(g, r, bp);
        double c = gamma / beta;
        for (long j = 0; j < nvox; ++j) gv[j] = f[j] - c * bp[j];
        if (lin) /* linear term -<lin, f> of a coarse model, times Nv / beta */
            for (long j = 0; j < nvox; ++j) gv[j] += (double)nvox / beta * lin[j];
        /* steps 2 and 3 */
        or_prox(&v, gv, f, beta, eps, M, clamp_mode, tv_weight, NULL);
        if (step) {
            double d = 0.0;
            for (long j = 0; j < nvox; ++j) d += (f[j] - fprev[j]) * (f[j] - fprev[j]);
            step[it] = sqrt(d);
        }
    }
    free(r);
    free(bp);
    free(gv);
    free(fprev);
}

/* ------------------------------------------------------------------------------ */
/* Multigrid transfers and the coarse-to-fine cascade                              */
/* ------------------------------------------------------------------------------ */

/* Mean over the existing pixels of each 2x2 block: [na][nv][nu] -> [na][ceil nv/2][ceil nu/2]. */
void or_restrict_sino(int na, int nv, int nu, const double *y, double *yc)
{
    int nvc = (nv + 1) / 2, nuc = (nu + 1) / 2;
    for (int ia = 0; ia < na; ++ia)
        for (int b = 0; b < nvc; ++b)
            for (int a = 0; a < nuc; ++a) {
                double s = 0.0;
                int c = 0;
                for (int db = 0; db < 2; ++db)
                    for (int da = 0; da < 2; ++da) {
                        int bb = 2 * b + db, aa = 2 * a + da;
                        if (bb < nv && aa < nu) {
                            s += y[((long)ia * nv + bb) * nu + aa];
                            ++c;
                        }
                    }
                yc[((long)ia * nvc + b) * nuc + a] = s / c;
            }
}

/* Coarse coordinate of fine index i (cell-centred grids, spacing ratio 2). */
static void prolong_weights(int i, int n, int nc, int *i0, int *i1, double *w)
{
    double c = (i - 0.5 * (n - 1)) * 0.5 + 0.5 * (nc - 1);
    double fl = floor(c);
    *w = c - fl;
    int a = (int)fl, b = a + 1;
    if (a < 0) a = 0;
    if (a > nc - 1) a = nc - 1;
    if (b < 0) b = 0;
    if (b > nc - 1) b = nc - 1;
    *i0 = a;
    *i1 = b;
}

/* Trilinear, cell-centred, x2 prolongation with edge replication. */
void or_prolong_vol(int nxc, int nyc, int nzc, const double *fc, int nx, int ny, int nz, double *f)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        int k0, k1;
        double wk;
        prolong_weights(k, nz, nzc, &k0, &k1, &wk);
        for (int j = 0; j < ny; ++j) {
            int j0, j1;
            double wj;
            prolong_weights(j, ny, nyc, &j0, &j1, &wj);
            for (int i = 0; i < nx; ++i) {
                int i0, i1;
                double wi;
                prolong_weights(i, nx, nxc, &i0, &i1, &wi);
#define FC(ii, jj, kk) fc[((long)(kk) * nyc + (jj)) * nxc + (ii)]
                double c00 = (1 - wi) * FC(i0, j0, k0) + wi * FC(i1, j0, k0);
                double c10 = (1 - wi) * FC(i0, j1, k0) + wi * FC(i1, j1, k0);
                double c01 = (1 - wi) * FC(i0, j0, k1) + wi * FC(i1, j0, k1);
                double c11 = (1 - wi) * FC(i0, j1, k1) + wi * FC(i1, j1, k1);
#undef FC
                double c0 = (1 - wj) * c00 + wj * c10;
                double c1 = (1 - wj) * c01 + wj * c11;
                f[((long)k * ny + j) * nx + i] = (1 - wk) * c0 + wk * c1;
            }
        }
    }
}

/* Geometry of multigrid level l: sizes ceil(n / 2^l), spacings 2^l h. */
void or_level_geom(const or_geom *g, int l, or_geom *out)
{
    *out = *g;
    int s = 1 << l;
    out->nx = (g->nx + s - 1) / s;
    out->ny = (g->ny + s - 1) / s;
    out->nz = (g->nz + s - 1) / s;
    out->hx = g->hx * s;
    out->hy = g->hy * s;
    out->hz = g->hz * s;
    out->nu = (g->nu + s - 1) / s;
    out->nv = (g->nv + s - 1) / s;
    out->du = g->du * s;
    out->dv = g->dv * s;
}

/*
 * Coarse-to-fine cascade: f = 0 on the coarsest level, `iters` iterations of A1 per
 * level, prolongation to the next finer level.  betas (optional, one per level, index
 * = level, 0 finest) fixes beta; otherwise beta = or_auto_beta(level, mu, K_pi).
 * eps <= 0 takes the per-level default.  trace (optional) gets 3 * iters values per
 * level, coarsest level first.  f_out is the finest volume.
 */
void or_reconstruct(const or_geom *g, const double *Y, double mu, int iters, int levels,
                    const double *betas, double eps, int M, int clamp_mode, int K_pi,
                    double *f_out, double *trace)
{
    or_geom *lg = (or_geom *)malloc(sizeof(or_geom) * levels);
    double **Ys = (double **)malloc(sizeof(double *) * levels);
    for (int l = 0; l < levels; ++l) or_level_geom(g, l, &lg[l]);
    Ys[0] = (double *)Y;
    for (int l = 1; l < levels; ++l) {
        Ys[l] = (double *)malloc(sizeof(double) * (size_t)g->na * lg[l].nv * lg[l].nu);
        or_restrict_sino(g->na, lg[l - 1].nv, lg[l - 1].nu, Ys[l - 1], Ys[l]);
    }
    double *f = NULL;
    for (int l = levels - 1; l >= 0; --l) {
        long nvox = (long)lg[l].nx * lg[l].ny * lg[l].nz;
        double *fl = (double *)calloc(nvox, sizeof(double));
        if (f) {
            or_prolong_vol(lg[l + 1].nx, lg[l + 1].ny, lg[l + 1].nz, f, lg[l].nx, lg[l].ny, lg[l].nz, fl);
            free(f);
        }
        f = fl;
        double beta = betas ? betas[l] : or_auto_beta(&lg[l], mu, K_pi);
        double e = eps > 0 ? eps : or_default_eps(&lg[l]);
        double *tr = trace ? trace + 3 * iters * (levels - 1 - l) : NULL;
        or_fbs(&lg[l], Ys[l], mu, beta, e, M, clamp_mode, 1.0, iters, f, tr, NULL, NULL);
    }
    memcpy(f_out, f, sizeof(double) * (size_t)g->nx * g->ny * g->nz);
    free(f);
    for (int l = 1; l < levels; ++l) free(Ys[l]);
    free(Ys);
    free(lg);
}

/* ------------------------------------------------------------------------------ */
/* V-cycle (a full-approximation reading of the cited multigrid method)            */
/* ------------------------------------------------------------------------------ */

/* Mean over the existing fine voxels of each 2x2x2 block: [nz][ny][nx] -> ceil halves. */
void or_restrict_vol(int nx, int ny, int nz, const double *f, double *fc)
{
    int nxc = (nx + 1) / 2, nyc = (ny + 1) / 2, nzc = (nz + 1) / 2;
    for (int k = 0; k < nzc; ++k)
        for (int j = 0; j < nyc; ++j)
            for (int i = 0; i < nxc; ++i) {
                double s = 0.0;
                int c = 0;
                for (int dk = 0; dk < 2; ++dk)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di) {
                            int ii = 2 * i + di, jj = 2 * j + dj, kk = 2 * k + dk;
                            if (ii < nx && jj < ny && kk < nz) {
                                s += f[((long)kk * ny + jj) * nx + ii];
                                ++c;
                            }
                        }
                fc[((long)k * nyc + j) * nxc + i] = s / c;
            }
}

/* Transpose of or_prolong_vol: fc[c] = sum over fine voxels of (weight of coarse voxel c
 * in that fine voxel) * x[fine]; accumulated serially in fine raster order. */
void or_prolong_vol_adjoint(int nxc, int nyc, int nzc, int nx, int ny, int nz, const double *x, double *fc)
{
    memset(fc, 0, sizeof(double) * (size_t)nxc * nyc * nzc);
    for (int k = 0; k < nz; ++k) {
        int k0, k1;
        double wk;
        prolong_weights(k, nz, nzc, &k0, &k1, &wk);
        for (int j = 0; j < ny; ++j) {
            int j0, j1;
            double wj;
            prolong_weights(j, ny, nyc, &j0, &j1, &wj);
            for (int i = 0; i < nx; ++i) {
                int i0, i1;
                double wi;
                prolong_weights(i, nx, nxc, &i0, &i1, &wi);
                double xv = x[((long)k * ny + j) * nx + i];
                int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
                double w_i[2] = {1 - wi, wi}, w_j[2] = {1 - wj, wj}, w_k[2] = {1 - wk, wk};
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            fc[((long)kk[c] * nyc + jj[b]) * nxc + ii[a]] += w_k[c] * w_j[b] * w_i[a] * xv;
            }
        }
    }
}

/* Gradient of the grid energy of Eq. 1: (grad TV_eps(f) + gamma P^T (P f - Y)) / Nv. */
void or_energy_grad(const or_geom *g, const double *Y, const double *f, double mu, double eps, double *grad)
{
    const long nvox = (long)g->nx * g->ny * g->nz;
    const long nr = (long)g->na * g->nv * g->nu;
    or_vol v = vol_of(g);
    double *r = (double *)malloc(sizeof(double) * nr);
    double *bp = (double *)malloc(sizeof(double) * nvox);
    or_project(g, f, r);
    for (long t = 0; t < nr; ++t) r[t] -= Y[t];
    or_backproject(g, r, bp);
    or_tv_grad(&v, f, eps, grad);
    double gam = or_gamma(g, mu);
    for (long j = 0; j < nvox; ++j) grad[j] = (grad[j] + gam * bp[j]) / (double)nvox;
    free(r);
    free(bp);
}

/* E(f) - <v, f> (v may be null). */
static double model_energy(const or_geom *g, const double *Y, const double *f, double mu, double eps,
                           const double *v)
{
    double e[3];
    or_energy(g, Y, f, mu, eps, e, NULL);
    double lin = 0.0;
    if (v)
        for (long j = 0; j < (long)g->nx * g->ny * g->nz; ++j) lin += v[j] * f[j];
    return e[0] - lin;
}

typedef struct {
    const or_geom *lg;
    double **Ys;
    const double *betas, *epss;
    double mu;
    int levels, M, pre, post, coarse;
    int *accepted; /* per level: coarse corrections taken */
} vc_ctx;

/*
 * One V-cycle on level l for the model E_l(f) - <v, f> (v null on the finest level):
 * `pre` iterations of Algorithm A1; then the coarse model
 *   E_{l+1}(x) - <v_c, x>,  v_c = grad E_{l+1}(R f) - Q^T (grad E_l(f) - v),
 * with R the 2x2x2 mean and Q^T the transpose of the trilinear prolongation Q, whose
 * gradient at R f equals Q^T of the fine model's gradient at f (first-order
 * coherence); it is reduced by a V-cycle on level l+1 (`coarse` iterations of A1 on
 * the coarsest), and the correction f + Q(x - R f), clamped at 0, is kept when it
 * lowers the fine model; then `post` iterations of A1.
 */
static void vcycle(const vc_ctx *C, int l, double *f, const double *v)
{
    const or_geom *g = &C->lg[l];
    if (l == C->levels - 1) {
        or_fbs(g, C->Ys[l], C->mu, C->betas[l], C->epss[l], C->M, 0, 1.0, C->coarse, f, NULL, v, NULL);
        return;
    }
    or_fbs(g, C->Ys[l], C->mu, C->betas[l], C->epss[l], C->M, 0, 1.0, C->pre, f, NULL, v, NULL);
    const or_geom *gc = &C->lg[l + 1];
    const long n = (long)g->nx * g->ny * g->nz, nc = (long)gc->nx * gc->ny * gc->nz;
    double *gr = (double *)malloc(sizeof(double) * n);
    double *x0 = (double *)malloc(sizeof(double) * nc);
    double *x = (double *)malloc(sizeof(double) * nc);
    double *vc = (double *)malloc(sizeof(double) * nc);
    double *gc_grad = (double *)malloc(sizeof(double) * nc);
    double *corr = (double *)malloc(sizeof(double) * n);
    double *ftry = (double *)malloc(sizeof(double) * n);
    or_energy_grad(g, C->Ys[l], f, C->mu, C->epss[l], gr);
    if (v)
        for (long j = 0; j < n; ++j) gr[j] -= v[j];
    or_restrict_vol(g->nx, g->ny, g->nz, f, x0);
    or_prolong_vol_adjoint(gc->nx, gc->ny, gc->nz, g->nx, g->ny, g->nz, gr, vc);
    or_energy_grad(gc, C->Ys[l + 1], x0, C->mu, C->epss[l + 1], gc_grad);
    for (long j = 0; j < nc; ++j) {
        vc[j] = gc_grad[j] - vc[j];
        x[j] = x0[j];
    }
    vcycle(C, l + 1, x, vc);
    for (long j = 0; j < nc; ++j) x[j] -= x0[j];
    or_prolong_vol(gc->nx, gc->ny, gc->nz, x, g->nx, g->ny, g->nz, corr);
    for (long j = 0; j < n; ++j) {
        double t = f[j] + corr[j];
        ftry[j] = t > 0.0 ? t : 0.0;
    }
    if (model_energy(g, C->Ys[l], ftry, C->mu, C->epss[l], v) < model_energy(g, C->Ys[l], f, C->mu, C->epss[l], v)) {
        memcpy(f, ftry, sizeof(double) * n);
        if (C->accepted) C->accepted[l] += 1;
    }
    or_fbs(g, C->Ys[l], C->mu, C->betas[l], C->epss[l], C->M, 0, 1.0, C->post, f, NULL, v, NULL);
    free(gr);
    free(x0);
    free(x);
    free(vc);
    free(gc_grad);
    free(corr);
    free(ftry);
}

/*
 * `cycles` V-cycles over `levels` levels from f = 0 on the finest level.  betas
 * (optional, per level) as in or_reconstruct; eps <= 0 takes the per-level default.
 * trace (optional, 3 * cycles): {E, E1, E2-term} of the finest iterate after each
 * cycle; accepted (optional, levels values) counts the coarse corrections taken.
 */
void or_vcycle(const or_geom *g, const double *Y, double mu, int cycles, int levels, const double *betas,
               double eps, int M, int pre, int post, int coarse, int K_pi, double *f_out, double *trace,
               int *accepted)
{
    or_geom *lg = (or_geom *)malloc(sizeof(or_geom) * levels);
    double **Ys = (double **)malloc(sizeof(double *) * levels);
    double *bt = (double *)malloc(sizeof(double) * levels);
    double *ep = (double *)malloc(sizeof(double) * levels);
    for (int l = 0; l < levels; ++l) {
        or_level_geom(g, l, &lg[l]);
        bt[l] = betas ? betas[l] : or_auto_beta(&lg[l], mu, K_pi);
        ep[l] = eps > 0 ? eps : or_default_eps(&lg[l]);
    }
    Ys[0] = (double *)Y;
    for (int l = 1; l < levels; ++l) {
        Ys[l] = (double *)malloc(sizeof(double) * (size_t)g->na * lg[l].nv * lg[l].nu);
        or_restrict_sino(g->na, lg[l - 1].nv, lg[l - 1].nu, Ys[l - 1], Ys[l]);
    }
    if (accepted) memset(accepted, 0, sizeof(int) * levels);
    vc_ctx C = {lg, Ys, bt, ep, mu, levels, M, pre, post, coarse, accepted};
    memset(f_out, 0, sizeof(double) * (size_t)g->nx * g->ny * g->nz);
    for (int c = 0; c < cycles; ++c) {
        vcycle(&C, 0, f_out, NULL);
        if (trace) or_energy(&lg[0], Y, f_out, mu, ep[0], trace + 3 * c, NULL);
    }
    for (int l = 1; l < levels; ++l) free(Ys[l]);
    free(Ys);
    free(lg);
    free(bt);
    free(ep);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
