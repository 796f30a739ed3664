/*
 * hj_oracle3d.c -- plain CPU reference for the 3D seven-point extension of
 * hierarchical Jacobi (Islam & Wang, arXiv 2006.16465, Sections 4 and 4.1
 * carried from five to seven points: the paper's 2D stencil plus a bottom and
 * a top neighbour; the paper itself stops at 2D).
 *
 * TEST INFRASTRUCTURE ONLY (see hj_oracle.c): only tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs may load it; it shares no
 * code with the CUDA path.  Binary64, compiled with -ffp-contract=off.
 *
 * Grid layout: (nz + 2) planes x (ny + 2) rows x W doubles, W = nx + 2,
 * x fastest, then y, then z; interior [1..nz] x [1..ny] x [1..nx]; the ghost
 * shell holds Dirichlet data.  Index q = (z * (ny + 2) + y) * W + x.
 *
 * Operator:
 *   (A u)_p = d_p u_p + cW u_W + cE u_E + cS u_S + cN u_N + cB u_B + cT u_T,
 *   d_p = cD + sigma_const + sigma_p (sigma nullable),
 * with W/E = x -/+ 1, S/N = y -/+ 1, B/T = z -/+ 1.
 *
 * Jacobi update, one fixed association order (the 2D order of hj_oracle.c
 * extended by the two new terms):
 *   acc = cW*uW; acc = acc + cE*uE; acc = acc + cS*uS; acc = acc + cN*uN;
 *   acc = acc + cB*uB; acc = acc + cT*uT;   u' = (f - acc) * (1.0 / d_p)
 *
 * Parity: pinned by tests/test_oracle_pins.py (dense operator, dense Jacobi
 * step, closed-form decay of the lowest sine mode, k = 1 equals a classic
 * sweep, large k equals a per-subdomain direct solve, the discrete solution
 * is a fixed point).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;      /* interior sizes */
    double cW, cE, cS, cN, cB, cT, cD;
    double sigma_const;  /* constant screening added to every diagonal entry */
    const double *sigma; /* nullable, grid-shaped, per-point screening */
} hjo3_problem;

static long w3(const hjo3_problem *p) { return (long)p->nx + 2; }
static long plane3(const hjo3_problem *p) { return w3(p) * ((long)p->ny + 2); }
static long size3(const hjo3_problem *p) { return plane3(p) * ((long)p->nz + 2); }

static double diag3(const hjo3_problem *p, long q)
{
    double d = p->cD + p->sigma_const;
    if (p->sigma) d = d + p->sigma[q];
    return d;
}

static double point3(const hjo3_problem *p, double f, double d, double uW, double uE, double uS,
                     double uN, double uB, double uT)
{
    double acc = p->cW * uW;
    acc = acc + p->cE * uE;
    acc = acc + p->cS * uS;
    acc = acc + p->cN * uN;
    acc = acc + p->cB * uB;
    acc = acc + p->cT * uT;
    return (f - acc) * (1.0 / d);
}

static double apply3(const hjo3_problem *p, const double *u, long q)
{
    const long W = w3(p), P = plane3(p);
    double au = diag3(p, q) * u[q];
    au = au + p->cW * u[q - 1];
    au = au + p->cE * u[q + 1];
    au = au + p->cS * u[q - W];
    au = au + p->cN * u[q + W];
    au = au + p->cB * u[q - P];
    au = au + p->cT * u[q + P];
    return au;
}

/* out = A u on interior points, 0 elsewhere.  Parity: pinned (dense matrix). */
void hjo3_apply(const hjo3_problem *p, const double *u, double *out)
{
    const long W = w3(p), P = plane3(p);
    memset(out, 0, sizeof(double) * (size_t)size3(p));
    for (long z = 1; z <= p->nz; ++z)
        for (long y = 1; y <= p->ny; ++y)
            for (long x = 1; x <= p->nx; ++x)
                out[z * P + y * W + x] = apply3(p, u, z * P + y * W + x);
}

/* ||f - A u||_2^2 over interior points, summed in x-fastest order. */
double hjo3_residual_sq(const hjo3_problem *p, const double *f, const double *u)
{
    const long W = w3(p), P = plane3(p);
    double s = 0.0;
    for (long z = 1; z <= p->nz; ++z)
        for (long y = 1; y <= p->ny; ++y)
            for (long x = 1; x <= p->nx; ++x) {
                const long q = z * P + y * W + x;
                const double r = f[q] - apply3(p, u, q);
                s = s + r * r;
            }
    return s;
}

/* dst := src everywhere (the ghost shell carries over; the interior is then
 * overwritten by the caller). */
static void copy_all3(const hjo3_problem *p, const double *src, double *dst)
{
    memcpy(dst, src, sizeof(double) * (size_t)size3(p));
}

/* One classic Jacobi sweep: every interior point reads u_in only. */
void hjo3_jacobi_sweep(const hjo3_problem *p, const double *f, const double *uin, double *uout)
{
    const long W = w3(p), P = plane3(p);
    copy_all3(p, uin, uout);
    for (long z = 1; z <= p->nz; ++z)
        for (long y = 1; y <= p->ny; ++y)
            for (long x = 1; x <= p->nx; ++x) {
                const long q = z * P + y * W + x;
                uout[q] = point3(p, f[q], diag3(p, q), uin[q - 1], uin[q + 1], uin[q - W], uin[q + W],
                                 uin[q - P], uin[q + P]);
            }
}

/* One hierarchical cycle on tx x ty x tz subdomains (Sections 3.3 and 4.1
 * in three dimensions): each subdomain (the last one along an axis truncated
 * at the grid edge) is copied with a one-point halo into two local
 * containers, k Jacobi subiterations run on its interior with the halo
 * frozen, reading container s mod 2 and writing (s + 1) mod 2, and the
 * interior of the latest container goes to u_out.  Every subdomain reads u_in
 * only.  Parity: pinned (k = 1 is a classic sweep; large k is a
 * per-subdomain direct solve; fixed point). */
void hjo3_hier_cycle(const hjo3_problem *p, const double *f, const double *uin, double *uout,
                     int tx, int ty, int tz, int k)
{
    const long W = w3(p), P = plane3(p);
    copy_all3(p, uin, uout);
    const long lw = tx + 2, lh = ty + 2, ld = tz + 2, lp = lw * lh;
    double *L[2];
    L[0] = (double *)malloc(sizeof(double) * (size_t)(lp * ld));
    L[1] = (double *)malloc(sizeof(double) * (size_t)(lp * ld));
    for (long z0 = 1; z0 <= p->nz; z0 += tz) {
        const long z1 = z0 + tz - 1 < p->nz ? z0 + tz - 1 : p->nz;
        for (long y0 = 1; y0 <= p->ny; y0 += ty) {
            const long y1 = y0 + ty - 1 < p->ny ? y0 + ty - 1 : p->ny;
            for (long x0 = 1; x0 <= p->nx; x0 += tx) {
                const long x1 = x0 + tx - 1 < p->nx ? x0 + tx - 1 : p->nx;
                /* local index of global (x, y, z): halo starts at x0-1, y0-1, z0-1 */
#define LOC(x, y, z) (((z) - (z0 - 1)) * lp + ((y) - (y0 - 1)) * lw + ((x) - (x0 - 1)))
                for (long z = z0 - 1; z <= z1 + 1; ++z)
                    for (long y = y0 - 1; y <= y1 + 1; ++y)
                        for (long x = x0 - 1; x <= x1 + 1; ++x) {
                            L[0][LOC(x, y, z)] = uin[z * P + y * W + x];
                            L[1][LOC(x, y, z)] = uin[z * P + y * W + x];
                        }
                for (int s = 0; s < k; ++s) {
                    const double *src = L[s % 2];
                    double *dst = L[(s + 1) % 2];
                    for (long z = z0; z <= z1; ++z)
                        for (long y = y0; y <= y1; ++y)
                            for (long x = x0; x <= x1; ++x) {
                                const long l = LOC(x, y, z), q = z * P + y * W + x;
                                dst[l] = point3(p, f[q], diag3(p, q), src[l - 1], src[l + 1], src[l - lw],
                                                src[l + lw], src[l - lp], src[l + lp]);
                            }
                }
                const double *fin = L[k % 2];
                for (long z = z0; z <= z1; ++z)
                    for (long y = y0; y <= y1; ++y)
                        for (long x = x0; x <= x1; ++x)
                            uout[z * P + y * W + x] = fin[LOC(x, y, z)];
#undef LOC
            }
        }
    }
    free(L[0]);
    free(L[1]);
}

/* Cycles until ||r_c|| <= tol ||r_0|| (status 0), a non-finite residual
 * (status 2) or max_cycles (status 1); the same stopping rule as hjo_solve.
 * Returns c; u holds u_c; hist[c] = ||r_c|| for c < hist_cap. */
long hjo3_solve(const hjo3_problem *p, const double *f, double *u, int classic, int tx, int ty, int tz,
                int k, double tol, long max_cycles, double *hist, long hist_cap, int *status)
{
    const size_t n = (size_t)size3(p);
    double *v = (double *)malloc(sizeof(double) * n);
    memcpy(v, u, sizeof(double) * n);
    const double r0 = sqrt(hjo3_residual_sq(p, f, u));
    long c = 0;
    int st = 1;
    double *cur = u, *nxt = v;
    for (;;) {
        const double rc = (c == 0) ? r0 : sqrt(hjo3_residual_sq(p, f, cur));
        if (hist && c < hist_cap) hist[c] = rc;
        if (!isfinite(rc)) { st = 2; break; }
        if (rc <= tol * r0) { st = 0; break; }
        if (c >= max_cycles) { st = 1; break; }
        if (classic) hjo3_jacobi_sweep(p, f, cur, nxt);
        else hjo3_hier_cycle(p, f, cur, nxt, tx, ty, tz, k);
        double *t = cur; cur = nxt; nxt = t;
        ++c;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * n);
    free(v);
    if (status) *status = st;
    return c;
}

/* Exactly ncycles cycles (or classic sweeps) from u (in/out). */
void hjo3_run_fixed(const hjo3_problem *p, const double *f, double *u, int classic, int tx, int ty, int tz,
                    int k, long ncycles)
{
    const size_t n = (size_t)size3(p);
    double *v = (double *)malloc(sizeof(double) * n);
    double *cur = u, *nxt = v;
    for (long c = 0; c < ncycles; ++c) {
        if (classic) hjo3_jacobi_sweep(p, f, cur, nxt);
        else hjo3_hier_cycle(p, f, cur, nxt, tx, ty, tz, k);
        double *t = cur; cur = nxt; nxt = t;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * n);
    free(v);
}
