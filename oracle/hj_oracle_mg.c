/*
 * hj_oracle_mg.c -- plain CPU reference for hierarchical Jacobi used as the
 * smoother of a geometric multigrid V-cycle (Islam & Wang, arXiv 2006.16465:
 * the conclusion names this use; the V-cycle itself is the textbook one of
 * the multigrid tutorial the paper cites, Briggs et al. 2000).
 *
 * TEST INFRASTRUCTURE ONLY (see hj_oracle.c): only tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs may load it; it shares no
 * code with the CUDA path.  Binary64, compiled with -ffp-contract=off; every
 * sum below is written in the order it is evaluated.
 *
 * Problem: 2D, constant coefficients, (A u)_p = d u_p + cW u_W + cE u_E +
 * cS u_S + cN u_N, d = cD + sigma_const, on a grid of (ny + 2) rows of
 * W = nx + 2 values (x fastest) with a Dirichlet ghost ring.
 *
 * Levels: level 0 is the given grid; level l + 1 has nx_{l+1} = (nx_l - 1)/2
 * and ny_{l+1} = (ny_l - 1)/2 interior points (nx_l, ny_l odd), coarse point
 * (I, J) sitting on fine point (2I, 2J).  The coarse operator rediscretises
 * the stencil on the doubled spacing: every h^-2 term is divided by 4,
 *   cX_{l+1} = cX_l / 4 (X = W, E, S, N),  cD_{l+1} = cD_l / 4,
 * and sigma_const stays (the screening term does not scale with h).
 *
 * Smoother: weighted hierarchical cycles.  A cycle is the hierarchical cycle
 * of hj_oracle.c (tx x ty subdomains, halo frozen, k subiterations in two
 * local containers, u_in -> u_out) whose subiteration is damped Jacobi:
 *   jac = (f - (((cW uW + cE uE) + cS uS) + cN uN)) * (1/d)
 *   u'  = u + omega * (jac - u)
 * Restriction: full weighting of the fine residual r = f - A u,
 *   f_c(I, J) = (4 r00 + 2 s1 + s2) * (1/16),
 *   s1 = ((r(-1,0) + r(1,0)) + r(0,-1)) + r(0,1),
 *   s2 = ((r(-1,-1) + r(1,-1)) + r(-1,1)) + r(1,1)   (offsets from (2I, 2J)),
 * with r = f - ((((d u + cW uW) + cE uE) + cS uS) + cN uN).
 * Prolongation: bilinear interpolation of the coarse correction e (zero on
 * the coarse ghost ring), added to u:
 *   (even, even): e(I, J);  (odd, even): (e(a, J) + e(a+1, J)) * 0.5;
 *   (even, odd): (e(I, b) + e(I, b+1)) * 0.5;
 *   (odd, odd): (((e(a,b) + e(a+1,b)) + e(a,b+1)) + e(a+1,b+1)) * 0.25,
 * a = (i - 1)/2, b = (j - 1)/2.
 *
 * V-cycle on level l < L - 1: pre smoothing cycles, restrict, zero the coarse
 * correction, V-cycle on level l + 1, prolongate and add, post smoothing
 * cycles.  On the coarsest level (l = L - 1): coarse_cycles undamped cycles
 * (omega = 1) of coarse_k subiterations on one subdomain covering the level.
 *
 * Parity: pinned by tests/test_oracle_pins_mg.py (dense restriction and
 * prolongation matrices, dense damped Jacobi step, a two-level cycle as a
 * dense affine map, the V-cycle's contraction on Poisson, convergence to the
 * dense solution).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny;
    double cW, cE, cS, cN, cD;
    double sigma_const;
} hjo_mg_problem;

static long mw(const hjo_mg_problem *p) { return (long)p->nx + 2; }
static long msize(const hjo_mg_problem *p) { return mw(p) * ((long)p->ny + 2); }
static double mdiag(const hjo_mg_problem *p) { return p->cD + p->sigma_const; }

static double mg_resid(const hjo_mg_problem *p, const double *f, const double *u, long q)
{
    const long W = mw(p);
    double au = mdiag(p) * u[q];
    au = au + p->cW * u[q - 1];
    au = au + p->cE * u[q + 1];
    au = au + p->cS * u[q - W];
    au = au + p->cN * u[q + W];
    return f[q] - au;
}

/* One weighted hierarchical cycle (u_in -> u_out; ghosts copied). */
void hjo_mg_wcycle(const hjo_mg_problem *p, const double *f, const double *uin, double *uout, int tx, int ty,
                   int k, double omega)
{
    const long W = mw(p);
    memcpy(uout, uin, sizeof(double) * (size_t)msize(p));
    const long lw = tx + 2, lh = ty + 2;
    double *L[2];
    L[0] = (double *)malloc(sizeof(double) * (size_t)(lw * lh));
    L[1] = (double *)malloc(sizeof(double) * (size_t)(lw * lh));
    const double invd = 1.0 / mdiag(p);
    for (long j0 = 1; j0 <= p->ny; j0 += ty) {
        const long j1 = j0 + ty - 1 < p->ny ? j0 + ty - 1 : p->ny;
        for (long i0 = 1; i0 <= p->nx; i0 += tx) {
            const long i1 = i0 + tx - 1 < p->nx ? i0 + tx - 1 : p->nx;
            for (long j = j0 - 1; j <= j1 + 1; ++j)
                for (long i = i0 - 1; i <= i1 + 1; ++i) {
                    const long l = (j - (j0 - 1)) * lw + (i - (i0 - 1));
                    L[0][l] = uin[j * W + i];
                    L[1][l] = uin[j * W + i];
                }
            for (int s = 0; s < k; ++s) {
                const double *src = L[s % 2];
                double *dst = L[(s + 1) % 2];
                for (long j = j0; j <= j1; ++j)
                    for (long i = i0; i <= i1; ++i) {
                        const long l = (j - (j0 - 1)) * lw + (i - (i0 - 1));
                        double acc = p->cW * src[l - 1];
                        acc = acc + p->cE * src[l + 1];
                        acc = acc + p->cS * src[l - lw];
                        acc = acc + p->cN * src[l + lw];
                        const double jac = (f[j * W + i] - acc) * invd;
                        dst[l] = src[l] + omega * (jac - src[l]);
                    }
            }
            const double *fin = L[k % 2];
            for (long j = j0; j <= j1; ++j)
                for (long i = i0; i <= i1; ++i) uout[j * W + i] = fin[(j - (j0 - 1)) * lw + (i - (i0 - 1))];
        }
    }
    free(L[0]);
    free(L[1]);
}

/* f_c = full weighting of r = f - A u (coarse interior; coarse ghosts 0). */
void hjo_mg_restrict(const hjo_mg_problem *p, const double *f, const double *u, double *fc)
{
    const long W = mw(p);
    const long ncx = (p->nx - 1) / 2, ncy = (p->ny - 1) / 2, Wc = ncx + 2;
    memset(fc, 0, sizeof(double) * (size_t)(Wc * (ncy + 2)));
    for (long J = 1; J <= ncy; ++J)
        for (long I = 1; I <= ncx; ++I) {
            const long q = 2 * J * W + 2 * I;
            const double r00 = mg_resid(p, f, u, q);
            double s1 = mg_resid(p, f, u, q - 1) + mg_resid(p, f, u, q + 1);
            s1 = s1 + mg_resid(p, f, u, q - W);
            s1 = s1 + mg_resid(p, f, u, q + W);
            double s2 = mg_resid(p, f, u, q - W - 1) + mg_resid(p, f, u, q - W + 1);
            s2 = s2 + mg_resid(p, f, u, q + W - 1);
            s2 = s2 + mg_resid(p, f, u, q + W + 1);
            double t = 4.0 * r00;
            t = t + 2.0 * s1;
            t = t + s2;
            fc[J * Wc + I] = t * 0.0625;
        }
}

/* u += bilinear interpolation of the coarse correction e (coarse ghosts 0). */
void hjo_mg_prolong_add(const hjo_mg_problem *p, const double *e, double *u)
{
    const long W = mw(p);
    const long ncx = (p->nx - 1) / 2, Wc = ncx + 2;
    for (long j = 1; j <= p->ny; ++j)
        for (long i = 1; i <= p->nx; ++i) {
            double v;
            const long a = (i - 1) / 2, b = (j - 1) / 2;
            if (i % 2 == 0 && j % 2 == 0) {
                v = e[(j / 2) * Wc + i / 2];
            } else if (j % 2 == 0) {
                v = (e[(j / 2) * Wc + a] + e[(j / 2) * Wc + a + 1]) * 0.5;
            } else if (i % 2 == 0) {
                v = (e[b * Wc + i / 2] + e[(b + 1) * Wc + i / 2]) * 0.5;
            } else {
                double s = e[b * Wc + a] + e[b * Wc + a + 1];
                s = s + e[(b + 1) * Wc + a];
                s = s + e[(b + 1) * Wc + a + 1];
                v = s * 0.25;
            }
            u[j * W + i] = u[j * W + i] + v;
        }
}

/* Number of levels available: halve while both sizes are odd and > 1. */
int hjo_mg_max_levels(int nx, int ny)
{
    int L = 1;
    while (nx > 1 && ny > 1 && nx % 2 == 1 && ny % 2 == 1) {
        nx = (nx - 1) / 2;
        ny = (ny - 1) / 2;
        ++L;
    }
    return L;
}

static hjo_mg_problem coarse_of(const hjo_mg_problem *p)
{
    hjo_mg_problem c = *p;
    c.nx = (p->nx - 1) / 2;
    c.ny = (p->ny - 1) / 2;
    c.cW = p->cW / 4.0;
    c.cE = p->cE / 4.0;
    c.cS = p->cS / 4.0;
    c.cN = p->cN / 4.0;
    c.cD = p->cD / 4.0;
    return c;
}

static void smooth(const hjo_mg_problem *p, const double *f, double *u, int cycles, int tx, int ty, int k,
                   double omega)
{
    if (cycles <= 0) return;
    double *t = (double *)malloc(sizeof(double) * (size_t)msize(p));
    for (int c = 0; c < cycles; ++c) {
        hjo_mg_wcycle(p, f, u, t, tx, ty, k, omega);
        memcpy(u, t, sizeof(double) * (size_t)msize(p));
    }
    free(t);
}

static void vcycle(const hjo_mg_problem *p, const double *f, double *u, int level, int levels, int pre,
                   int post, int tx, int ty, int k, double omega, int coarse_k, int coarse_cycles)
{
    if (level == levels - 1) {
        smooth(p, f, u, coarse_cycles, p->nx, p->ny, coarse_k, 1.0);
        return;
    }
    smooth(p, f, u, pre, tx, ty, k, omega);
    const hjo_mg_problem c = coarse_of(p);
    const size_t nc = (size_t)(mw(&c) * ((long)c.ny + 2));
    double *fc = (double *)malloc(sizeof(double) * nc);
    double *ec = (double *)calloc(nc, sizeof(double));
    hjo_mg_restrict(p, f, u, fc);
    vcycle(&c, fc, ec, level + 1, levels, pre, post, tx, ty, k, omega, coarse_k, coarse_cycles);
    hjo_mg_prolong_add(p, ec, u);
    free(fc);
    free(ec);
    smooth(p, f, u, post, tx, ty, k, omega);
}

/* One V-cycle over `levels` levels, u in/out. */
void hjo_mg_vcycle(const hjo_mg_problem *p, const double *f, double *u, int levels, int pre, int post, int tx,
                   int ty, int k, double omega, int coarse_k, int coarse_cycles)
{
    vcycle(p, f, u, 0, levels, pre, post, tx, ty, k, omega, coarse_k, coarse_cycles);
}

/* V-cycles until ||r_c|| <= tol ||r_0|| (status 0), non-finite (2) or
 * max_vcycles (1); hist[c] = ||r_c||.  Returns c. */
long hjo_mg_solve(const hjo_mg_problem *p, const double *f, double *u, int levels, int pre, int post, int tx,
                  int ty, int k, double omega, int coarse_k, int coarse_cycles, double tol, long max_vcycles,
                  double *hist, long hist_cap, int *status)
{
    const long W = mw(p);
    long c = 0;
    int st = 1;
    double r0 = 0.0;
    for (;;) {
        double s = 0.0;
        for (long j = 1; j <= p->ny; ++j)
            for (long i = 1; i <= p->nx; ++i) {
                const double r = mg_resid(p, f, u, j * W + i);
                s = s + r * r;
            }
        const double rc = sqrt(s);
        if (c == 0) r0 = rc;
        if (hist && c < hist_cap) hist[c] = rc;
        if (!isfinite(rc)) { st = 2; break; }
        if (rc <= tol * r0) { st = 0; break; }
        if (c >= max_vcycles) { st = 1; break; }
        hjo_mg_vcycle(p, f, u, levels, pre, post, tx, ty, k, omega, coarse_k, coarse_cycles);
        ++c;
    }
    if (status) *status = st;
    return c;
}
