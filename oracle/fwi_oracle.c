/*
 * fwi_oracle.c -- plain FP64 CPU oracle of the preconditioned time-domain FWI
 * gradient of Huang, Wang & Ren, "Two New Gradient Precondition Schemes for
 * Full Waveform Inversion" (arXiv:1406.1864).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the bench's CPU
 * baseline load this library. It shares no code, header, table or helper with
 * the CUDA library and is written straight from the definitions below, one
 * grid point at a time, in double precision. It is slow on purpose.
 *
 * What it computes (paper sections / equations in brackets):
 *   - the constant-density acoustic wave equation 1/v^2 u_tt - lap u = delta f
 *     [Sec. 2, below the OLS misfit]; the paper names only a time-domain
 *     finite-difference scheme, so this one is a reading: 8th-order centred
 *     Laplacian, second-order leapfrog in time, and an absorbing sponge
 *     u_tt + 2 eta u_t outside the physical model, the model padded by edge
 *     replication;
 *   - synthetic traces d = R u at the receivers [Sec. 2, OLS misfit];
 *   - the adjoint (back-propagated residual) wavefield and the zero-lag
 *     cross-correlation gradient g = 2/v^3 sum_s int u_tt v_s dt [Sec. 2],
 *     here as the exact derivative of the discrete misfit: the adjoint of the
 *     discrete update and g = sum_s sum_n psi^{n+1} (2/v) (L u^n + s^n);
 *   - the shot illumination / pseudo-diagonal Hessian [Eq. 1] as
 *     sum_s sum_n u_s^n(x)^2 dt (or the omega^4-weighted form via u_tt);
 *   - the diagonal of the localized subsurface-offset Hessian [Sec. 3, the
 *     Hessian obtained by substituting Eq. 5 into Eq. 6, diagonal part] as
 *     sum_s sum_n u_s^n(x + h e_x) u_s^n(x - h e_x) dt for h = 0..hmax;
 *   - the Born (tangent-linear) operator [Eq. 4] for the Jacobian dot test;
 *   - extended Born modelling [Eq. 5]: the velocity perturbation dv(x, h)
 *     carries a horizontal subsurface offset h; the incident field at x + h
 *     scatters from x - h, and extended migration [Eq. 6] is its exact
 *     adjoint, the correlation of the adjoint field at x - h with the
 *     incident field at x + h.
 * The misfits (OLS and the time-integral misfit of Eq. 2), their adjoint
 * sources and the preconditioning division are done in oracle/__init__.py.
 *
 * Conventions: physical grid nz x ny x nx (ny = 1 and no y axis in 2D), padded
 * by P cells on every side of every axis; the padded velocity replicates the
 * nearest physical cell. Coordinates are (z, y, x) triples of physical indices.
 * Time levels u^0..u^{nt-1}, u^{-1} = u^0 = 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 8th-order centred second-derivative weights (Taylor expansion to h^8). */
static const double W8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

typedef struct {
    int ndim, nz, ny, nx, P;
    int nzp, nyp, nxp, nt;
    long npad;
    double dx, dt, etamax;
} grid_t;

static int setup_grid(grid_t *g, int ndim, int nz, int ny, int nx, int P, double dx, double dt,
                      int nt, double vref, double R)
{
    if ((ndim != 2 && ndim != 3) || nz < 1 || nx < 1 || ny < 1 || P < 1 || nt < 1) return -1;
    if (ndim == 2 && ny != 1) return -1;
    if (!(dx > 0.0) || !(dt > 0.0) || !(vref > 0.0) || !(R > 0.0 && R < 1.0)) return -1;
    g->ndim = ndim; g->nz = nz; g->ny = ny; g->nx = nx; g->P = P; g->nt = nt;
    g->nzp = nz + 2 * P;
    g->nyp = (ndim == 3) ? ny + 2 * P : 1;
    g->nxp = nx + 2 * P;
    g->npad = (long)g->nzp * g->nyp * g->nxp;
    g->dx = dx; g->dt = dt;
    /* damping strength that gives a normal-incidence reflection ~R for a
       quadratic profile of width P*dx at speed vref */
    g->etamax = 3.0 * vref * log(1.0 / R) / (2.0 * P * dx);
    return 0;
}

static long ID(const grid_t *g, int i, int k, int j) { return ((long)i * g->nyp + k) * g->nxp + j; }

/* value of a padded field, zero outside the padded grid */
static double at(const grid_t *g, const double *u, int i, int k, int j)
{
    if (i < 0 || i >= g->nzp || k < 0 || k >= g->nyp || j < 0 || j >= g->nxp) return 0.0;
    return u[ID(g, i, k, j)];
}

/* discrete Laplacian (1/dx^2 included) at padded point (i,k,j) */
static double lap(const grid_t *g, const double *u, int i, int k, int j)
{
    double s = g->ndim * W8[0] * u[ID(g, i, k, j)];
    for (int m = 1; m <= 4; ++m) {
        s += W8[m] * (at(g, u, i + m, k, j) + at(g, u, i - m, k, j));
        s += W8[m] * (at(g, u, i, k, j + m) + at(g, u, i, k, j - m));
        if (g->ndim == 3) s += W8[m] * (at(g, u, i, k + m, j) + at(g, u, i, k - m, j));
    }
    return s / (g->dx * g->dx);
}

/* cells into the sponge along one axis (0 inside the physical range) */
static int depth_in_sponge(int i, int P, int n)
{
    if (i < P) return P - i;
    if (i >= P + n) return i - (P + n - 1);
    return 0;
}

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* padded velocity (edge replication) and damping profile */
static void pad_model(const grid_t *g, const double *v, double *vp, double *eta)
{
    for (int i = 0; i < g->nzp; ++i)
        for (int k = 0; k < g->nyp; ++k)
            for (int j = 0; j < g->nxp; ++j) {
                int iz = clampi(i - g->P, 0, g->nz - 1);
                int iy = (g->ndim == 3) ? clampi(k - g->P, 0, g->ny - 1) : 0;
                int ix = clampi(j - g->P, 0, g->nx - 1);
                vp[ID(g, i, k, j)] = v[((long)iz * g->ny + iy) * g->nx + ix];
                double dz = depth_in_sponge(i, g->P, g->nz) / (double)g->P;
                double dxs = depth_in_sponge(j, g->P, g->nx) / (double)g->P;
                double dy = (g->ndim == 3) ? depth_in_sponge(k, g->P, g->ny) / (double)g->P : 0.0;
                eta[ID(g, i, k, j)] = g->etamax * (dz * dz + dy * dy + dxs * dxs);
            }
}

/* physical (z,y,x) triple -> padded linear index */
static long padded_index(const grid_t *g, const int *c)
{
    int k = (g->ndim == 3) ? c[1] + g->P : 0;
    return ID(g, c[0] + g->P, k, c[2] + g->P);
}

static int check_coord(const grid_t *g, const int *c)
{
    if (c[0] < 0 || c[0] >= g->nz || c[2] < 0 || c[2] >= g->nx) return -1;
    if (g->ndim == 3 && (c[1] < 0 || c[1] >= g->ny)) return -1;
    if (g->ndim == 2 && c[1] != 0) return -1;
    return 0;
}

/* one leapfrog step of the damped wave equation
     (1 + eta dt) u^{n+1} = 2 u^n - (1 - eta dt) u^{n-1} + (v dt)^2 (L u^n + s^n)
   with s^n = srcval at the source point (srcval = f(t_n)/dx^ndim). */
static void leapfrog(const grid_t *g, const double *vp, const double *eta, const double *um1,
                     const double *u0, double *up1, long src, double srcval)
{
    const double dt = g->dt;
    for (int i = 0; i < g->nzp; ++i)
        for (int k = 0; k < g->nyp; ++k)
            for (int j = 0; j < g->nxp; ++j) {
                long p = ID(g, i, k, j);
                double q = lap(g, u0, i, k, j) + (p == src ? srcval : 0.0);
                double c2 = vp[p] * vp[p] * dt * dt;
                up1[p] = (2.0 * u0[p] - (1.0 - eta[p] * dt) * um1[p] + c2 * q) / (1.0 + eta[p] * dt);
            }
}

/* Forward modelling of one shot. Records traces (seis [nt][nrec]), adds the
   illumination and offset-Hessian sums of this shot into the physical-grid
   accumulators, and optionally stores every time level (hist [nt][npad]). */
static void forward_shot(const grid_t *g, const double *vp, const double *eta, long src,
                         const double *wav, int nrec, const long *rec, double *seis,
                         double *illum, int illum_utt, int hmax, double *offh, double *hist)
{
    const long N = g->npad;
    const double dt = g->dt;
    const double sscale = 1.0 / pow(g->dx, g->ndim);
    double *um1 = calloc(N, sizeof(double));
    double *u0 = calloc(N, sizeof(double));
    double *up1 = calloc(N, sizeof(double));
    for (int n = 0; n < g->nt; ++n) {
        if (hist) memcpy(hist + (long)n * N, u0, N * sizeof(double));
        if (seis)
            for (int r = 0; r < nrec; ++r) seis[(long)n * nrec + r] = u0[rec[r]];
        if (n < g->nt - 1) leapfrog(g, vp, eta, um1, u0, up1, src, wav[n] * sscale);
        if (illum) {
            for (int iz = 0; iz < g->nz; ++iz)
                for (int iy = 0; iy < g->ny; ++iy)
                    for (int ix = 0; ix < g->nx; ++ix) {
                        long p = ID(g, iz + g->P, g->ndim == 3 ? iy + g->P : 0, ix + g->P);
                        long o = ((long)iz * g->ny + iy) * g->nx + ix;
                        if (!illum_utt) {
                            illum[o] += u0[p] * u0[p] * dt;
                        } else if (n < g->nt - 1) {
                            double utt = (up1[p] - 2.0 * u0[p] + um1[p]) / (dt * dt);
                            illum[o] += utt * utt * dt;
                        }
                    }
        }
        if (offh) {
            const long nphys = (long)g->nz * g->ny * g->nx;
            for (int h = 0; h <= hmax; ++h)
                for (int iz = 0; iz < g->nz; ++iz)
                    for (int iy = 0; iy < g->ny; ++iy)
                        for (int ix = 0; ix < g->nx; ++ix) {
                            int i = iz + g->P, k = (g->ndim == 3) ? iy + g->P : 0, j = ix + g->P;
                            long o = ((long)iz * g->ny + iy) * g->nx + ix;
                            offh[h * nphys + o] += at(g, u0, i, k, j + h) * at(g, u0, i, k, j - h) * dt;
                        }
        }
        double *t = um1; um1 = u0; u0 = up1; up1 = t;
    }
    free(um1); free(u0); free(up1);
}

/* Adjoint of the discrete forward map for one shot, and its imaging.
   adj [nt][nrec] is the adjoint source a^n = dJ/dd^n at the receivers.
     psi^{nt} = psi^{nt+1} = 0,
     (1 + eta dt) psi^m = 2 psi^{m+1} - (1 - eta dt) psi^{m+2} + (v dt)^2 (L psi^{m+1} + R^T a^m),
   m = nt-1..1 (psi = -(v dt)^2 * Lagrange multiplier of the update);
     gpad += psi^{m} (2/v) (L u^{m-1} + s^{m-1}).
   psi_src[n] = psi^{n+1}(x_s)/dx^ndim is the adjoint of the source-to-trace map. */
static void adjoint_shot(const grid_t *g, const double *vp, const double *eta, long src,
                         const double *wav, int nrec, const long *rec, const double *adj,
                         double *gpad, double *psi_src)
{
    const long N = g->npad;
    const double dt = g->dt;
    const double sscale = 1.0 / pow(g->dx, g->ndim);
    double *hist = malloc((size_t)g->nt * N * sizeof(double));
    forward_shot(g, vp, eta, src, wav, 0, NULL, NULL, NULL, 0, 0, NULL, hist);
    double *p2 = calloc(N, sizeof(double)); /* psi^{m+2} */
    double *p1 = calloc(N, sizeof(double)); /* psi^{m+1} */
    double *p0 = calloc(N, sizeof(double)); /* psi^{m}   */
    double *inj = calloc(N, sizeof(double));
    if (psi_src) psi_src[g->nt - 1] = 0.0;
    for (int m = g->nt - 1; m >= 1; --m) {
        memset(inj, 0, N * sizeof(double));
        for (int r = 0; r < nrec; ++r) inj[rec[r]] += adj[(long)m * nrec + r];
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    double c2 = vp[p] * vp[p] * dt * dt;
                    p0[p] = (2.0 * p1[p] - (1.0 - eta[p] * dt) * p2[p] +
                             c2 * (lap(g, p1, i, k, j) + inj[p])) /
                            (1.0 + eta[p] * dt);
                }
        const double *um = hist + (long)(m - 1) * N;
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    double q = lap(g, um, i, k, j) + (p == src ? wav[m - 1] * sscale : 0.0);
                    gpad[p] += p0[p] * (2.0 / vp[p]) * q;
                }
        if (psi_src) psi_src[m - 1] = p0[src] * sscale;
        double *t = p2; p2 = p1; p1 = p0; p0 = t;
    }
    free(p2); free(p1); free(p0); free(inj); free(hist);
}

/* Born (tangent-linear) modelling of one shot: derivative of the traces with
   respect to the velocity along dv (edge-replicated like v). */
static void born_shot(const grid_t *g, const double *vp, const double *dvp, const double *eta,
                      long src, const double *wav, int nrec, const long *rec, double *dseis)
{
    const long N = g->npad;
    const double dt = g->dt;
    const double sscale = 1.0 / pow(g->dx, g->ndim);
    double *u[3], *du[3];
    for (int a = 0; a < 3; ++a) { u[a] = calloc(N, sizeof(double)); du[a] = calloc(N, sizeof(double)); }
    double *um1 = u[0], *u0 = u[1], *up1 = u[2];
    double *dum1 = du[0], *du0 = du[1], *dup1 = du[2];
    for (int n = 0; n < g->nt; ++n) {
        for (int r = 0; r < nrec; ++r) dseis[(long)n * nrec + r] = du0[rec[r]];
        if (n == g->nt - 1) break;
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    double q = lap(g, u0, i, k, j) + (p == src ? wav[n] * sscale : 0.0);
                    double c2 = vp[p] * vp[p] * dt * dt;
                    double dc2 = 2.0 * vp[p] * dvp[p] * dt * dt;
                    double a = 1.0 + eta[p] * dt, b = 1.0 - eta[p] * dt;
                    up1[p] = (2.0 * u0[p] - b * um1[p] + c2 * q) / a;
                    dup1[p] = (2.0 * du0[p] - b * dum1[p] + c2 * lap(g, du0, i, k, j) + dc2 * q) / a;
                }
        double *t = um1; um1 = u0; u0 = up1; up1 = t;
        t = dum1; dum1 = du0; du0 = dup1; dup1 = t;
    }
    for (int a = 0; a < 3; ++a) { free(u[a]); free(du[a]); }
}

/* Extended Born modelling of one shot [Eq. 5]: as born_shot, with the
   scattering source at padded point y
     S^n(y) = sum_{h=-he..he} 2 v(y + h e_x) dv(y + h e_x, h) dt^2 q^n(y + 2h e_x),
   q^n = L u^n + s^n, zero where y + h or y + 2h leaves the padded grid.
   dvp [2he+1][npad] holds dv(., h) for h = -he..he, edge-replicated. */
static void ext_born_shot(const grid_t *g, const double *vp, const double *dvp, int he, const double *eta,
                          long src, const double *wav, int nrec, const long *rec, double *dseis)
{
    const long N = g->npad;
    const double dt = g->dt;
    const double sscale = 1.0 / pow(g->dx, g->ndim);
    double *u[3], *du[3];
    for (int a = 0; a < 3; ++a) { u[a] = calloc(N, sizeof(double)); du[a] = calloc(N, sizeof(double)); }
    double *q = calloc(N, sizeof(double));
    double *um1 = u[0], *u0 = u[1], *up1 = u[2];
    double *dum1 = du[0], *du0 = du[1], *dup1 = du[2];
    for (int n = 0; n < g->nt; ++n) {
        for (int r = 0; r < nrec; ++r) dseis[(long)n * nrec + r] = du0[rec[r]];
        if (n == g->nt - 1) break;
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    q[p] = lap(g, u0, i, k, j) + (p == src ? wav[n] * sscale : 0.0);
                }
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    double S = 0.0;
                    for (int h = -he; h <= he; ++h) {
                        int jx = j + h, jq = j + 2 * h;
                        if (jx < 0 || jx >= g->nxp || jq < 0 || jq >= g->nxp) continue;
                        long x = ID(g, i, k, jx);
                        S += 2.0 * vp[x] * dvp[(long)(h + he) * N + x] * dt * dt * q[ID(g, i, k, jq)];
                    }
                    double c2 = vp[p] * vp[p] * dt * dt;
                    double a = 1.0 + eta[p] * dt, b = 1.0 - eta[p] * dt;
                    up1[p] = (2.0 * u0[p] - b * um1[p] + c2 * q[p]) / a;
                    dup1[p] = (2.0 * du0[p] - b * dum1[p] + c2 * lap(g, du0, i, k, j) + S) / a;
                }
        double *t = um1; um1 = u0; u0 = up1; up1 = t;
        t = dum1; dum1 = du0; du0 = dup1; dup1 = t;
    }
    for (int a = 0; a < 3; ++a) { free(u[a]); free(du[a]); }
    free(q);
}

/* Extended migration of one shot [Eq. 6], the adjoint of ext_born_shot: the
   adjoint field psi of adjoint_shot correlated across offsets,
     gext[h][x] += psi^m(x - h e_x) q^{m-1}(x + h e_x) 2 v(x) / v(x - h e_x)^2,
   for padded x with x - h and x + h inside the padded grid (at h = 0 the
   gradient's imaging term). */
static void ext_migration_shot(const grid_t *g, const double *vp, const double *eta, long src,
                               const double *wav, int nrec, const long *rec, const double *adj, int he,
                               double *gext)
{
    const long N = g->npad;
    const double dt = g->dt;
    const double sscale = 1.0 / pow(g->dx, g->ndim);
    double *hist = malloc((size_t)g->nt * N * sizeof(double));
    forward_shot(g, vp, eta, src, wav, 0, NULL, NULL, NULL, 0, 0, NULL, hist);
    double *p2 = calloc(N, sizeof(double));
    double *p1 = calloc(N, sizeof(double));
    double *p0 = calloc(N, sizeof(double));
    double *inj = calloc(N, sizeof(double));
    double *q = calloc(N, sizeof(double));
    for (int m = g->nt - 1; m >= 1; --m) {
        memset(inj, 0, N * sizeof(double));
        for (int r = 0; r < nrec; ++r) inj[rec[r]] += adj[(long)m * nrec + r];
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    double c2 = vp[p] * vp[p] * dt * dt;
                    p0[p] = (2.0 * p1[p] - (1.0 - eta[p] * dt) * p2[p] +
                             c2 * (lap(g, p1, i, k, j) + inj[p])) /
                            (1.0 + eta[p] * dt);
                }
        const double *um = hist + (long)(m - 1) * N;
        for (int i = 0; i < g->nzp; ++i)
            for (int k = 0; k < g->nyp; ++k)
                for (int j = 0; j < g->nxp; ++j) {
                    long p = ID(g, i, k, j);
                    q[p] = lap(g, um, i, k, j) + (p == src ? wav[m - 1] * sscale : 0.0);
                }
        for (int h = -he; h <= he; ++h)
            for (int i = 0; i < g->nzp; ++i)
                for (int k = 0; k < g->nyp; ++k)
                    for (int j = 0; j < g->nxp; ++j) {
                        int jm = j - h, jp = j + h;
                        if (jm < 0 || jm >= g->nxp || jp < 0 || jp >= g->nxp) continue;
                        long x = ID(g, i, k, j), y = ID(g, i, k, jm);
                        gext[(long)(h + he) * N + x] += p0[y] * q[ID(g, i, k, jp)] * 2.0 * vp[x] / (vp[y] * vp[y]);
                    }
        double *t = p2; p2 = p1; p1 = p0; p0 = t;
    }
    free(p2); free(p1); free(p0); free(inj); free(q); free(hist);
}

/* shared argument checks; fills padded source/receiver indices */
static int prepare(grid_t *g, int ndim, int nz, int ny, int nx, int P, double dx, double dt,
                   int nt, double vref, double R, int ns, const int *src, int nrec, const int *rec,
                   long **src_p, long **rec_p)
{
    if (setup_grid(g, ndim, nz, ny, nx, P, dx, dt, nt, vref, R)) return -1;
    if (ns < 1 || nrec < 0) return -1;
    *src_p = malloc(ns * sizeof(long));
    *rec_p = malloc(((size_t)ns * nrec + 1) * sizeof(long));
    for (int s = 0; s < ns; ++s) {
        if (check_coord(g, src + 3 * s)) return -2;
        (*src_p)[s] = padded_index(g, src + 3 * s);
        for (int r = 0; r < nrec; ++r) {
            const int *c = rec + 3 * ((long)s * nrec + r);
            if (check_coord(g, c)) return -3;
            (*rec_p)[(long)s * nrec + r] = padded_index(g, c);
        }
    }
    return 0;
}

static int nthreads_used(int want)
{
#ifdef _OPENMP
    return want > 0 ? want : omp_get_max_threads();
#else
    (void)want;
    return 1;
#endif
}

/* Forward modelling of all shots. Outputs (each may be NULL):
     seis  [ns][nt][nrec]             traces d_s^n(r) = u_s^n(x_r)
     illum [nz][ny][nx]               sum_s sum_n u^2 dt (illum_utt: u_tt^2 dt)
     offh  [hmax+1][nz][ny][nx]       sum_s sum_n u(x+h e_x) u(x-h e_x) dt
     dump  [nt][nzp][nyp][nxp]        every padded time level of shot dump_shot
   Returns 0, or a negative code for invalid arguments. */
int oracle_forward(int ndim, int nz, int ny, int nx, int P, double dx, double dt, int nt,
                   double vref, double R, const double *v, int ns, const int *src,
                   const double *wav, int nrec, const int *rec, double *seis, double *illum,
                   int illum_utt, int hmax, double *offh, double *dump, int dump_shot,
                   int nthreads)
{
    grid_t g;
    long *src_p = NULL, *rec_p = NULL;
    int rc = prepare(&g, ndim, nz, ny, nx, P, dx, dt, nt, vref, R, ns, src, nrec, rec, &src_p, &rec_p);
    if (rc) { free(src_p); free(rec_p); return rc; }
    if (hmax < 0) { free(src_p); free(rec_p); return -1; }
    const long nphys = (long)nz * ny * nx;
    double *vp = malloc(g.npad * sizeof(double));
    double *eta = malloc(g.npad * sizeof(double));
    pad_model(&g, v, vp, eta);
    int T = nthreads_used(nthreads);
    double *ill_t = illum ? calloc((size_t)T * nphys, sizeof(double)) : NULL;
    double *off_t = offh ? calloc((size_t)T * (hmax + 1) * nphys, sizeof(double)) : NULL;
#pragma omp parallel for schedule(static) num_threads(T)
    for (int s = 0; s < ns; ++s) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        forward_shot(&g, vp, eta, src_p[s], wav + (long)s * nt, nrec, rec_p + (long)s * nrec,
                     seis ? seis + (long)s * nt * nrec : NULL, ill_t ? ill_t + t * nphys : NULL,
                     illum_utt, hmax, off_t ? off_t + (long)t * (hmax + 1) * nphys : NULL,
                     (dump && s == dump_shot) ? dump : NULL);
    }
    if (illum) {
        memset(illum, 0, nphys * sizeof(double));
        for (int t = 0; t < T; ++t)
            for (long o = 0; o < nphys; ++o) illum[o] += ill_t[t * nphys + o];
    }
    if (offh) {
        long m = (long)(hmax + 1) * nphys;
        memset(offh, 0, m * sizeof(double));
        for (int t = 0; t < T; ++t)
            for (long o = 0; o < m; ++o) offh[o] += off_t[t * m + o];
    }
    free(ill_t); free(off_t); free(vp); free(eta); free(src_p); free(rec_p);
    return 0;
}

/* Gradient of sum_s sum_n sum_r a_s^n(r) d_s^n(r) with respect to the physical
   velocity, for a given adjoint source adj [ns][nt][nrec] (the residual for the
   OLS misfit, C^T C r for the time-integral misfit). The padded-grid gradient
   of each sponge cell is added to the physical edge cell it replicates.
     grad     [nz][ny][nx]   folded gradient
     grad_pad [npad]         gradient on the padded grid before folding (or NULL)
     psi_src  [ns][nt]       adjoint of the source-to-trace map (or NULL) */
int oracle_gradient(int ndim, int nz, int ny, int nx, int P, double dx, double dt, int nt,
                    double vref, double R, const double *v, int ns, const int *src,
                    const double *wav, int nrec, const int *rec, const double *adj, double *grad,
                    double *grad_pad, double *psi_src, int nthreads)
{
    grid_t g;
    long *src_p = NULL, *rec_p = NULL;
    int rc = prepare(&g, ndim, nz, ny, nx, P, dx, dt, nt, vref, R, ns, src, nrec, rec, &src_p, &rec_p);
    if (rc) { free(src_p); free(rec_p); return rc; }
    double *vp = malloc(g.npad * sizeof(double));
    double *eta = malloc(g.npad * sizeof(double));
    pad_model(&g, v, vp, eta);
    int T = nthreads_used(nthreads);
    double *g_t = calloc((size_t)T * g.npad, sizeof(double));
#pragma omp parallel for schedule(static) num_threads(T)
    for (int s = 0; s < ns; ++s) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        adjoint_shot(&g, vp, eta, src_p[s], wav + (long)s * nt, nrec, rec_p + (long)s * nrec,
                     adj + (long)s * nt * nrec, g_t + t * g.npad, psi_src ? psi_src + (long)s * nt : NULL);
    }
    double *gp = calloc(g.npad, sizeof(double));
    for (int t = 0; t < T; ++t)
        for (long p = 0; p < g.npad; ++p) gp[p] += g_t[t * g.npad + p];
    if (grad_pad) memcpy(grad_pad, gp, g.npad * sizeof(double));
    memset(grad, 0, (size_t)nz * ny * nx * sizeof(double));
    for (int i = 0; i < g.nzp; ++i)
        for (int k = 0; k < g.nyp; ++k)
            for (int j = 0; j < g.nxp; ++j) {
                int iz = clampi(i - P, 0, nz - 1);
                int iy = (ndim == 3) ? clampi(k - P, 0, ny - 1) : 0;
                int ix = clampi(j - P, 0, nx - 1);
                grad[((long)iz * ny + iy) * nx + ix] += gp[ID(&g, i, k, j)];
            }
    free(gp); free(g_t); free(vp); free(eta); free(src_p); free(rec_p);
    return 0;
}

/* Born modelling [Eq. 4]: dseis [ns][nt][nrec] = (d traces / d v) dv. */
int oracle_born(int ndim, int nz, int ny, int nx, int P, double dx, double dt, int nt,
                double vref, double R, const double *v, const double *dv, int ns, const int *src,
                const double *wav, int nrec, const int *rec, double *dseis, int nthreads)
{
    grid_t g;
    long *src_p = NULL, *rec_p = NULL;
    int rc = prepare(&g, ndim, nz, ny, nx, P, dx, dt, nt, vref, R, ns, src, nrec, rec, &src_p, &rec_p);
    if (rc) { free(src_p); free(rec_p); return rc; }
    double *vp = malloc(g.npad * sizeof(double));
    double *dvp = malloc(g.npad * sizeof(double));
    double *eta = malloc(g.npad * sizeof(double));
    pad_model(&g, v, vp, eta);
    pad_model(&g, dv, dvp, eta); /* same eta (independent of v) */
    int T = nthreads_used(nthreads);
#pragma omp parallel for schedule(static) num_threads(T)
    for (int s = 0; s < ns; ++s)
        born_shot(&g, vp, dvp, eta, src_p[s], wav + (long)s * nt, nrec, rec_p + (long)s * nrec,
                  dseis + (long)s * nt * nrec);
    free(vp); free(dvp); free(eta); free(src_p); free(rec_p);
    return 0;
}

/* Extended Born modelling [Eq. 5]: dseis [ns][nt][nrec] from the extended
   perturbation dv_ext [2he+1][nz][ny][nx] (offsets h = -he..he along x). */
int oracle_ext_born(int ndim, int nz, int ny, int nx, int P, double dx, double dt, int nt,
                    double vref, double R, const double *v, const double *dv_ext, int he, int ns,
                    const int *src, const double *wav, int nrec, const int *rec, double *dseis, int nthreads)
{
    grid_t g;
    long *src_p = NULL, *rec_p = NULL;
    int rc = prepare(&g, ndim, nz, ny, nx, P, dx, dt, nt, vref, R, ns, src, nrec, rec, &src_p, &rec_p);
    if (rc || he < 0) { free(src_p); free(rec_p); return rc ? rc : -1; }
    const long nphys = (long)nz * ny * nx;
    double *vp = malloc(g.npad * sizeof(double));
    double *eta = malloc(g.npad * sizeof(double));
    double *dvp = malloc((size_t)(2 * he + 1) * g.npad * sizeof(double));
    pad_model(&g, v, vp, eta);
    for (int h = 0; h <= 2 * he; ++h) pad_model(&g, dv_ext + h * nphys, dvp + h * g.npad, eta);
    int T = nthreads_used(nthreads);
#pragma omp parallel for schedule(static) num_threads(T)
    for (int s = 0; s < ns; ++s)
        ext_born_shot(&g, vp, dvp, he, eta, src_p[s], wav + (long)s * nt, nrec, rec_p + (long)s * nrec,
                      dseis + (long)s * nt * nrec);
    free(vp); free(dvp); free(eta); free(src_p); free(rec_p);
    return 0;
}

/* Extended migration [Eq. 6] of the adjoint source adj [ns][nt][nrec]: the
   image [2he+1][nz][ny][nx], the padded image of each sponge cell added to the
   physical edge cell it replicates (the adjoint of the edge replication of
   oracle_ext_born's dv_ext). */
int oracle_ext_migration(int ndim, int nz, int ny, int nx, int P, double dx, double dt, int nt,
                         double vref, double R, const double *v, int ns, const int *src, const double *wav,
                         int nrec, const int *rec, const double *adj, int he, double *image, int nthreads)
{
    grid_t g;
    long *src_p = NULL, *rec_p = NULL;
    int rc = prepare(&g, ndim, nz, ny, nx, P, dx, dt, nt, vref, R, ns, src, nrec, rec, &src_p, &rec_p);
    if (rc || he < 0) { free(src_p); free(rec_p); return rc ? rc : -1; }
    const long nphys = (long)nz * ny * nx;
    const long NE = (long)(2 * he + 1) * g.npad;
    double *vp = malloc(g.npad * sizeof(double));
    double *eta = malloc(g.npad * sizeof(double));
    pad_model(&g, v, vp, eta);
    int T = nthreads_used(nthreads);
    double *g_t = calloc((size_t)T * NE, sizeof(double));
#pragma omp parallel for schedule(static) num_threads(T)
    for (int s = 0; s < ns; ++s) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        ext_migration_shot(&g, vp, eta, src_p[s], wav + (long)s * nt, nrec, rec_p + (long)s * nrec,
                           adj + (long)s * nt * nrec, he, g_t + t * NE);
    }
    memset(image, 0, (size_t)(2 * he + 1) * nphys * sizeof(double));
    for (int t = 0; t < T; ++t)
        for (int h = 0; h <= 2 * he; ++h)
            for (int i = 0; i < g.nzp; ++i)
                for (int k = 0; k < g.nyp; ++k)
                    for (int j = 0; j < g.nxp; ++j) {
                        int iz = clampi(i - P, 0, nz - 1);
                        int iy = (ndim == 3) ? clampi(k - P, 0, ny - 1) : 0;
                        int ix = clampi(j - P, 0, nx - 1);
                        image[h * nphys + ((long)iz * ny + iy) * nx + ix] += g_t[t * NE + h * g.npad + ID(&g, i, k, j)];
                    }
    free(g_t); free(vp); free(eta); free(src_p); free(rec_p);
    return 0;
}

/* Damping profile eta on the padded grid (for tests of the sponge reading). */
int oracle_eta(int ndim, int nz, int ny, int nx, int P, double dx, double vref, double R,
               double *eta_out)
{
    grid_t g;
    if (setup_grid(&g, ndim, nz, ny, nx, P, dx, 1.0, 1, vref, R)) return -1;
    double *vp = malloc(g.npad * sizeof(double));
    double *v = malloc((size_t)nz * ny * nx * sizeof(double));
    for (long o = 0; o < (long)nz * ny * nx; ++o) v[o] = vref;
    pad_model(&g, v, vp, eta_out);
    free(vp); free(v);
    return 0;
}
