/*
 * FP64 reference implementation of the per-ray and tomographic parts of one
 * UDM(m)-PCG(n) ADMM iteration (Li et al., "A splitting-based iterative
 * algorithm for GPU-accelerated statistical dual-energy X-ray CT
 * reconstruction", Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle that the GPU library is
 * checked against. It is plain, slow and written to be read against the paper:
 * one loop per definition, no blocking or fusion. Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load it. It shares no code with
 * the CUDA library.
 *
 *  - og_project / og_backproject: the forward projection matrix R (Eq. 2, Eq. 3)
 *    as Joseph's ray-driven linear-interpolation projector, and its transpose
 *    R^T written as the scatter of the very same weights.
 *  - og_forward_model: f_{h/l}(a) of Eq. 3 and its Jacobian for per-ray line
 *    integrals a = (a_c, a_p), with the integral over E as a sum over bins and
 *    C_{h/l} = ln sum_E S = 0 for unit-sum spectra.
 *  - og_udm: the per-ray decomposition subproblem, Eq. 13, by
 *    Levenberg-Marquardt (damped Gauss-Newton), 4 evaluations of f per
 *    iteration (Table 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int kind;                  /* 0 = parallel beam, 1 = fan beam, flat detector */
    int nx, ny, nv, nb;        /* image columns, rows; views; detector bins */
    double pix;                /* pixel side (cm) */
    double ang0, span;         /* theta_v = ang0 + v * span / nv */
    double du, uoff;           /* u_k = (k - (nb-1)/2) du + uoff */
    double sod, sdd;           /* fan beam: source-isocentre, source-detector (cm) */
} og_geom;

int og_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* A point on ray (v, k) and its unit direction. */
static void og_ray(const og_geom* g, int v, int k, double* px, double* py, double* dx, double* dy) {
    double th = g->ang0 + v * (g->span / g->nv);
    double c = cos(th), s = sin(th);
    double u = (k - 0.5 * (g->nb - 1)) * g->du + g->uoff;
    if (g->kind == 0) {
        *px = u * c;
        *py = u * s;
        *dx = -s;
        *dy = c;
    } else {
        double sx = g->sod * c, sy = g->sod * s;
        double qx = -(g->sdd - g->sod) * c - u * s;
        double qy = -(g->sdd - g->sod) * s + u * c;
        double ex = qx - sx, ey = qy - sy;
        double len = sqrt(ex * ex + ey * ey);
        *px = sx;
        *py = sy;
        *dx = ex / len;
        *dy = ey / len;
    }
}

/*
 * Joseph's method. If |dx| >= |dy| the ray is sampled once per image column i:
 * its height there, in fractional row units fy, is interpolated linearly
 * between rows floor(fy) and floor(fy)+1 (zero outside the image), and the sum
 * is scaled by pix/|dx|, the path length per column. Otherwise the roles of
 * rows and columns swap. Each call visits the ray's non-zero weights
 * w(ray, pixel) once; `mode` 0 gathers sum w*img, mode 1 scatters val*w.
 */
static double og_joseph(const og_geom* g, int v, int k, const double* img, double* out, double val, int mode) {
    double px, py, dx, dy;
    og_ray(g, v, k, &px, &py, &dx, &dy);
    const int nx = g->nx, ny = g->ny;
    double acc = 0.0;
    if (fabs(dx) >= fabs(dy)) {
        double step = g->pix / fabs(dx);
        for (int i = 0; i < nx; i++) {
            double xi = (i - 0.5 * (nx - 1)) * g->pix;
            double y = py + (xi - px) * (dy / dx);
            double fy = y / g->pix + 0.5 * (ny - 1);
            double fl = floor(fy);
            if (fl < -1.0 || fl > ny - 1) continue;
            int j0 = (int)fl;
            double f = fy - fl;
            if (j0 >= 0) {
                if (mode == 0) acc += (1.0 - f) * img[(size_t)j0 * nx + i];
                else out[(size_t)j0 * nx + i] += val * step * (1.0 - f);
            }
            if (j0 + 1 <= ny - 1) {
                if (mode == 0) acc += f * img[(size_t)(j0 + 1) * nx + i];
                else out[(size_t)(j0 + 1) * nx + i] += val * step * f;
            }
        }
        return acc * step;
    } else {
        double step = g->pix / fabs(dy);
        for (int j = 0; j < ny; j++) {
            double yj = (j - 0.5 * (ny - 1)) * g->pix;
            double x = px + (yj - py) * (dx / dy);
            double fx = x / g->pix + 0.5 * (nx - 1);
            double fl = floor(fx);
            if (fl < -1.0 || fl > nx - 1) continue;
            int i0 = (int)fl;
            double f = fx - fl;
            if (i0 >= 0) {
                if (mode == 0) acc += (1.0 - f) * img[(size_t)j * nx + i0];
                else out[(size_t)j * nx + i0] += val * step * (1.0 - f);
            }
            if (i0 + 1 <= nx - 1) {
                if (mode == 0) acc += f * img[(size_t)j * nx + i0 + 1];
                else out[(size_t)j * nx + i0 + 1] += val * step * f;
            }
        }
        return acc * step;
    }
}

/* Loops over fewer rays than this run on one thread: thread start-up would dominate them. */
#define OG_PAR_MIN 8192

/* sino[v][k] = (R img)[v][k] for an image [ny][nx]. */
void og_project(const og_geom* g, const double* img, double* sino) {
    const long nr = (long)g->nv * g->nb;
#pragma omp parallel for schedule(dynamic, 64) if (nr >= OG_PAR_MIN)
    for (long r = 0; r < nr; r++) {
        int v = (int)(r / g->nb), k = (int)(r % g->nb);
        sino[r] = og_joseph(g, v, k, img, NULL, 0.0, 0);
    }
}

/* Single ray, for sampled checks: returns (R img)[v][k]. */
double og_project_ray(const og_geom* g, const double* img, int v, int k) {
    return og_joseph(g, v, k, img, NULL, 0.0, 0);
}

/*
 * img = R^T sino: every ray scatters its value times the same weights the
 * projector uses. Views are split over threads, each with a private image;
 * the private images are summed in thread order.
 */
void og_backproject(const og_geom* g, const double* sino, double* img) {
    const size_t np = (size_t)g->nx * g->ny;
    int nt = og_num_threads();
    double* part = (double*)calloc((size_t)nt * np, sizeof(double));
#pragma omp parallel if ((long)g->nv * g->nb >= OG_PAR_MIN)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* mine = part + (size_t)t * np;
#pragma omp for schedule(static)
        for (int v = 0; v < g->nv; v++)
            for (int k = 0; k < g->nb; k++) {
                double s = sino[(size_t)v * g->nb + k];
                if (s != 0.0) og_joseph(g, v, k, NULL, mine, s, 1);
            }
    }
    memset(img, 0, np * sizeof(double));
    for (int t = 0; t < nt; t++)
        for (size_t p = 0; p < np; p++) img[p] += part[(size_t)t * np + p];
    free(part);
}

/* Explicit sparse row of R for ray (v, k): writes up to cap (pixel, weight) pairs, returns count. */
int og_ray_weights(const og_geom* g, int v, int k, int64_t* pix_idx, double* wts, int cap) {
    double* dense = (double*)calloc((size_t)g->nx * g->ny, sizeof(double));
    og_joseph(g, v, k, NULL, dense, 1.0, 1);
    int n = 0;
    for (long p = 0; p < (long)g->nx * g->ny; p++)
        if (dense[p] != 0.0) {
            if (n < cap) { pix_idx[n] = p; wts[n] = dense[p]; }
            n++;
        }
    free(dense);
    return n;
}

/* ---------------------------------------------------------------------- */
/* Spectral forward model, Eq. 3. S_h, S_l are normalised to unit sum here. */

typedef struct {
    int ne;
    const double *sh, *sl, *fkn, *fp; /* unit-sum spectra and basis functions */
} og_spec;

/* f_h, f_l at a and, if jac != NULL, jac = {df_h/da_c, df_h/da_p, df_l/da_c, df_l/da_p}. */
static void og_fwd(const og_spec* sp, double ac, double ap, double* fh, double* fl, double* jac) {
    double sh = 0, sl = 0, shc = 0, shp = 0, slc = 0, slp = 0;
    for (int e = 0; e < sp->ne; e++) {
        double t = exp(-sp->fkn[e] * ac - sp->fp[e] * ap);
        sh += sp->sh[e] * t;
        sl += sp->sl[e] * t;
        if (jac) {
            shc += sp->sh[e] * sp->fkn[e] * t;
            shp += sp->sh[e] * sp->fp[e] * t;
            slc += sp->sl[e] * sp->fkn[e] * t;
            slp += sp->sl[e] * sp->fp[e] * t;
        }
    }
    *fh = -log(sh);
    *fl = -log(sl);
    if (jac) {
        jac[0] = shc / sh;
        jac[1] = shp / sh;
        jac[2] = slc / sl;
        jac[3] = slp / sl;
    }
}

static double* og_normalised(const double* s, int ne) {
    double tot = 0;
    for (int e = 0; e < ne; e++) tot += s[e];
    double* out = (double*)malloc(sizeof(double) * ne);
    for (int e = 0; e < ne; e++) out[e] = s[e] / tot;
    return out;
}

void og_forward_model(int ne, const double* S_h, const double* S_l, const double* fkn, const double* fp,
                      long n, const double* ac, const double* ap, double* fh, double* fl, double* jac) {
    double* sh = og_normalised(S_h, ne);
    double* sl = og_normalised(S_l, ne);
    og_spec sp = {ne, sh, sl, fkn, fp};
#pragma omp parallel for schedule(static) if (n >= OG_PAR_MIN)
    for (long r = 0; r < n; r++) og_fwd(&sp, ac[r], ap[r], fh + r, fl + r, jac ? jac + 4 * r : NULL);
    free(sh);
    free(sl);
}

/* Per-ray cost of Eq. 13. */
static double og_cost(double fh, double fl, double mh, double ml, double wh, double wl,
                      double ac, double ap, double vc, double vp, double rc, double rp) {
    double rh = fh - mh, rl = fl - ml;
    return 0.5 * (wh * rh * rh + wl * rl * rl) + 0.5 * (rc * (ac - vc) * (ac - vc) + rp * (ap - vp) * (ap - vp));
}

/*
 * Eq. 13 per ray by Levenberg-Marquardt, `iters` iterations from the warm start
 * (a_c, a_p). One iteration:
 *   1. f_h, f_l and the Jacobian J at a (2 evaluations of f);
 *   2. g = sum_k w_k (f_k - m_k) J_k + rho (a - v),  A = sum_k w_k J_k J_k^T + diag(rho);
 *   3. solve (A + mu diag(A)) delta = -g;
 *   4. f_h, f_l at a + delta (2 evaluations); accept if the cost decreased
 *      (mu /= 10), else keep a (mu *= 10); mu is clamped to [1e-10, 1e10].
 * mu[] is per ray and carried between calls. status: 0 = last step accepted,
 * 1 = last step rejected, 2 = non-finite or singular system met (a kept).
 */
void og_udm(int ne, const double* S_h, const double* S_l, const double* fkn, const double* fp,
            long n, const double* mh, const double* ml, const double* wh, const double* wl,
            const double* vc, const double* vp, double rho_c, double rho_p, int iters,
            double* ac, double* ap, double* mu, uint8_t* status) {
    double* sh = og_normalised(S_h, ne);
    double* sl = og_normalised(S_l, ne);
    og_spec sp = {ne, sh, sl, fkn, fp};
#pragma omp parallel for schedule(static) if (n >= OG_PAR_MIN)
    for (long r = 0; r < n; r++) {
        double a0 = ac[r], a1 = ap[r], m = mu[r];
        uint8_t st = 0;
        for (int it = 0; it < iters; it++) {
            double fh, fl, J[4];
            og_fwd(&sp, a0, a1, &fh, &fl, J);
            double rh = fh - mh[r], rl = fl - ml[r];
            double g0 = wh[r] * rh * J[0] + wl[r] * rl * J[2] + rho_c * (a0 - vc[r]);
            double g1 = wh[r] * rh * J[1] + wl[r] * rl * J[3] + rho_p * (a1 - vp[r]);
            double A00 = wh[r] * J[0] * J[0] + wl[r] * J[2] * J[2] + rho_c;
            double A01 = wh[r] * J[0] * J[1] + wl[r] * J[2] * J[3];
            double A11 = wh[r] * J[1] * J[1] + wl[r] * J[3] * J[3] + rho_p;
            double B00 = A00 * (1.0 + m), B11 = A11 * (1.0 + m);
            double det = B00 * B11 - A01 * A01;
            double cost0 = og_cost(fh, fl, mh[r], ml[r], wh[r], wl[r], a0, a1, vc[r], vp[r], rho_c, rho_p);
            if (!(det > 0.0) || !isfinite(det) || !isfinite(cost0)) { st = 2; break; }
            double d0 = (-g0 * B11 + g1 * A01) / det;
            double d1 = (-g1 * B00 + g0 * A01) / det;
            double t0 = a0 + d0, t1 = a1 + d1;
            double fh1, fl1;
            og_fwd(&sp, t0, t1, &fh1, &fl1, NULL);
            double cost1 = og_cost(fh1, fl1, mh[r], ml[r], wh[r], wl[r], t0, t1, vc[r], vp[r], rho_c, rho_p);
            if (!isfinite(cost1)) { m *= 10.0; st = 2; }
            else if (cost1 < cost0) { a0 = t0; a1 = t1; m /= 10.0; st = 0; }
            else { m *= 10.0; st = 1; }
            if (m < 1e-10) m = 1e-10;
            if (m > 1e10) m = 1e10;
        }
        ac[r] = a0;
        ap[r] = a1;
        mu[r] = m;
        if (status) status[r] = st;
    }
    free(sh);
    free(sl);
}

/* Eq. 13's cost for given a (used by the brute-force checks). */
void og_udm_cost(int ne, const double* S_h, const double* S_l, const double* fkn, const double* fp,
                 long n, const double* mh, const double* ml, const double* wh, const double* wl,
                 const double* vc, const double* vp, double rho_c, double rho_p,
                 const double* ac, const double* ap, double* cost) {
    double* sh = og_normalised(S_h, ne);
    double* sl = og_normalised(S_l, ne);
    og_spec sp = {ne, sh, sl, fkn, fp};
#pragma omp parallel for schedule(static) if (n >= OG_PAR_MIN)
    for (long r = 0; r < n; r++) {
        double fh, fl;
        og_fwd(&sp, ac[r], ap[r], &fh, &fl, NULL);
        cost[r] = og_cost(fh, fl, mh[r], ml[r], wh[r], wl[r], ac[r], ap[r], vc[r], vp[r], rho_c, rho_p);
    }
    free(sh);
    free(sl);
}
