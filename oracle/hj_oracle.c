/*
 * hj_oracle.c -- plain, slow, obviously-correct CPU reference for hierarchical
 * Jacobi iteration (Islam & Wang, "Hierarchical Jacobi Iteration for Structured
 * Matrices on GPUs using Shared Memory", arXiv 2006.16465).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library.  It shares no code, header, helper or
 * constant with the CUDA path in paper_2006_16465_gb300/, and it includes
 * nothing from include/.
 *
 * Arithmetic is IEEE binary64 (binary32 where a function says so), compiled
 * with -ffp-contract=off so that no multiply-add is ever fused; every loop runs
 * in a fixed order, so results are bitwise reproducible.
 *
 * Grid layout: rows x W doubles, W = nx + 2, row-major, x fastest.
 *   2D: rows = ny + 2, interior [1..ny] x [1..nx], ghost ring = Dirichlet data.
 *   1D: rows = ny independent copies, interior columns 1..nx, ghosts 0, nx+1.
 *
 * Operator (Section 3, Eq. jacobi-stencil-equation-1d; Section 4,
 * Eq. 2d-jacobi-stencil, with a,c,e,f,d named cW,cE,cS,cN,cD):
 *   (A u)_p = d_p u_p + cW u_W + cE u_E + cS u_S + cN u_N,
 *   d_p = cD + sigma_const + sigma_p   (sigma: screening, nullable),
 * with ghost values taken as known Dirichlet data.
 *
 * Canonical Jacobi update (Eq. jacobi-elemental restated for the stencil):
 *   acc = cW*uW; acc = acc + cE*uE; [2D: acc = acc + cS*uS; acc = acc + cN*uN;]
 *   u'  = (f - acc) * (1.0 / d_p)
 * This is the paper's x_i = (1/d)(b - a x_W - c x_E - e x_S - f x_N) with one
 * fixed association order; the GPU FP64 path evaluates the same order.
 *
 * Parity status of each function is stated beside it; all are pinned by the
 * not-gpu tests (closed-form Jacobi decay, Thomas vs banded LU, DST and dense
 * direct solves, per-tile dense solves for the large-k limit, the k = 1
 * equivalence of Section 3.3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int dim;            /* 1 or 2 */
    int nx, ny;         /* interior sizes; 1D: ny = number of independent copies */
    double cW, cE, cS, cN, cD;
    double sigma_const; /* constant screening added to every diagonal entry */
    const double *sigma;/* nullable, grid-shaped, per-point screening */
    const double *coef; /* nullable: per-point neighbour coefficients, grid-shaped
                           planes W, E (1D) or W, E, S, N (2D) that replace cW..cN;
                           the general tridiagonal a_i, c_i of Section 3 */
} hjo_problem;

static long rows_of(const hjo_problem *p) { return p->dim == 2 ? (long)p->ny + 2 : (long)p->ny; }
static long width_of(const hjo_problem *p) { return (long)p->nx + 2; }
static long first_row(const hjo_problem *p) { return p->dim == 2 ? 1 : 0; }
static long last_row(const hjo_problem *p) { return p->dim == 2 ? (long)p->ny : (long)p->ny - 1; }

/* diagonal entry d_p of row-major grid index q */
static double diag_at(const hjo_problem *p, long q)
{
    double d = p->cD + p->sigma_const;
    if (p->sigma) d = d + p->sigma[q];
    return d;
}

/* neighbour coefficient m (0 = W, 1 = E, 2 = S, 3 = N) of grid index q */
static double coef_at(const hjo_problem *p, int m, long q)
{
    if (p->coef) return p->coef[(long)m * rows_of(p) * width_of(p) + q];
    return m == 0 ? p->cW : m == 1 ? p->cE : m == 2 ? p->cS : p->cN;
}

/* One Jacobi point update of grid index q from the four (two in 1D)
 * neighbour values. */
static double jacobi_point(const hjo_problem *p, long q, double f, double d,
                           double uW, double uE, double uS, double uN)
{
    double acc = coef_at(p, 0, q) * uW;
    acc = acc + coef_at(p, 1, q) * uE;
    if (p->dim == 2) {
        acc = acc + coef_at(p, 2, q) * uS;
        acc = acc + coef_at(p, 3, q) * uN;
    }
    return (f - acc) * (1.0 / d);
}

/* (A u)_p for an interior grid index q (fixed evaluation order). */
static double apply_point(const hjo_problem *p, const double *u, long q)
{
    const long W = width_of(p);
    double au = diag_at(p, q) * u[q];
    au = au + coef_at(p, 0, q) * u[q - 1];
    au = au + coef_at(p, 1, q) * u[q + 1];
    if (p->dim == 2) {
        au = au + coef_at(p, 2, q) * u[q - W];
        au = au + coef_at(p, 3, q) * u[q + W];
    }
    return au;
}

/* out = A u on interior points, 0 elsewhere.  Parity: pinned (dense matrix). */
void hjo_apply(const hjo_problem *p, const double *u, double *out)
{
    const long W = width_of(p), R = rows_of(p);
    memset(out, 0, sizeof(double) * (size_t)(W * R));
    for (long j = first_row(p); j <= last_row(p); ++j)
        for (long i = 1; i <= p->nx; ++i)
            out[j * W + i] = apply_point(p, u, j * W + i);
}

/* ||f - A u||_2^2 over interior points, summed in row-major order.
 * The stopping quantity of Sections 3.5 and 4.2 is the L2 norm of this
 * residual relative to that of the initial guess. */
double hjo_residual_sq(const hjo_problem *p, const double *f, const double *u)
{
    const long W = width_of(p);
    double s = 0.0;
    for (long j = first_row(p); j <= last_row(p); ++j)
        for (long i = 1; i <= p->nx; ++i) {
            const long q = j * W + i;
            const double r = f[q] - apply_point(p, u, q);
            s = s + r * r;
        }
    return s;
}

/* Copy the ghost ring (Dirichlet data) of src into dst. */
static void copy_ghosts(const hjo_problem *p, const double *src, double *dst)
{
    const long W = width_of(p), R = rows_of(p);
    for (long j = 0; j < R; ++j) {
        const int ghost_row = (p->dim == 2) && (j == 0 || j == R - 1);
        if (ghost_row) {
            memcpy(dst + j * W, src + j * W, sizeof(double) * (size_t)W);
        } else {
            dst[j * W] = src[j * W];
            dst[j * W + W - 1] = src[j * W + W - 1];
        }
    }
}

/* One classic Jacobi sweep (Section 3.1, two containers): every interior
 * point reads u_in only.  Parity: pinned (closed-form decay, Thomas, DST). */
void hjo_jacobi_sweep(const hjo_problem *p, const double *f, const double *uin, double *uout)
{
    const long W = width_of(p);
    copy_ghosts(p, uin, uout);
    /* rows are independent (every point reads u_in only): an OpenMP build
     * may split them over threads with the same result bit for bit */
#pragma omp parallel for schedule(static)
    for (long j = first_row(p); j <= last_row(p); ++j)
        for (long i = 1; i <= p->nx; ++i) {
            const long q = j * W + i;
            const double uS = p->dim == 2 ? uin[q - W] : 0.0;
            const double uN = p->dim == 2 ? uin[q + W] : 0.0;
            uout[q] = jacobi_point(p, q, f[q], diag_at(p, q), uin[q - 1], uin[q + 1], uS, uN);
        }
}

/* One cycle of the hierarchical method (Sections 3.3 and 4.1, Appendix A):
 *   1. partition the interior into tx (x ty) subdomains starting at interior
 *      index 1 (a last partial subdomain is truncated at the grid edge) and
 *      copy each subdomain plus a one-point halo into BOTH local containers;
 *   2. run k Jacobi subiterations on the subdomain interior, reading container
 *      s mod 2 and writing container (s+1) mod 2; halo values stay frozen;
 *   3. copy the subdomain interior of the latest container into u_out.
 * Every subdomain reads u_in, and the result goes to a separate array u_out
 * (double-buffered global state).  Parity: pinned (k = 1 equals a classic
 * sweep; large k equals a per-subdomain direct solve; fixed point). */
void hjo_hier_cycle(const hjo_problem *p, const double *f, const double *uin, double *uout,
                    int tx, int ty, int k)
{
    const long W = width_of(p);
    if (p->dim == 1) ty = 1;
    copy_ghosts(p, uin, uout);
    const long lw = tx + 2, lh = (p->dim == 2) ? ty + 2 : 1;
    const long jlo = first_row(p), jhi = last_row(p);
    const long jstep = (p->dim == 2) ? ty : 1;
    const long nbx = (p->nx + tx - 1) / tx;                 /* subdomains along x */
    const long nby = (jhi - jlo + jstep) / jstep;           /* subdomain rows (1D: copies) */
    /* Subdomains are independent within a cycle (each reads u_in only and
     * writes its own interior of u_out), so an OpenMP build may run them on
     * several threads; the result is the same bit for bit. */
#pragma omp parallel
    {
        double *L[2];
        L[0] = (double *)malloc(sizeof(double) * (size_t)(lw * lh));
        L[1] = (double *)malloc(sizeof(double) * (size_t)(lw * lh));
#pragma omp for schedule(static)
        for (long t = 0; t < nbx * nby; ++t) {
            const long j0 = jlo + (t / nbx) * jstep;
            const long j1 = (p->dim == 2) ? (j0 + ty - 1 < jhi ? j0 + ty - 1 : jhi) : j0;
            const long i0 = 1 + (t % nbx) * tx;
            const long i1 = (i0 + tx - 1 < p->nx) ? i0 + tx - 1 : p->nx;
            const long hj0 = (p->dim == 2) ? j0 - 1 : j0;   /* first staged row */
            const long hj1 = (p->dim == 2) ? j1 + 1 : j1;   /* last staged row  */
            /* step 1: stage subdomain + halo into both containers */
            for (long j = hj0; j <= hj1; ++j)
                for (long i = i0 - 1; i <= i1 + 1; ++i) {
                    const long l = (j - hj0) * lw + (i - (i0 - 1));
                    L[0][l] = uin[j * W + i];
                    L[1][l] = uin[j * W + i];
                }
            /* step 2: k subiterations with a frozen halo */
            for (int s = 0; s < k; ++s) {
                const double *src = L[s % 2];
                double *dst = L[(s + 1) % 2];
                for (long j = j0; j <= j1; ++j)
                    for (long i = i0; i <= i1; ++i) {
                        const long l = (j - hj0) * lw + (i - (i0 - 1));
                        const double uS = p->dim == 2 ? src[l - lw] : 0.0;
                        const double uN = p->dim == 2 ? src[l + lw] : 0.0;
                        dst[l] = jacobi_point(p, j * W + i, f[j * W + i], diag_at(p, j * W + i),
                                              src[l - 1], src[l + 1], uS, uN);
                    }
            }
            /* step 3: write the subdomain interior of the latest container */
            const double *fin = L[k % 2];
            for (long j = j0; j <= j1; ++j)
                for (long i = i0; i <= i1; ++i)
                    uout[j * W + i] = fin[(j - hj0) * lw + (i - (i0 - 1))];
        }
        free(L[0]);
        free(L[1]);
    }
}

/* Subdomains along one dimension with overlap (Sections 3.4 and 4.3).
 * Subdomain j of J spans [start, end] of the interior 1..n: T points at
 * stride S = T - o, the last one clamped so that it ends at n (with o = 0 the
 * last one is truncated instead, as in hjo_hier_cycle).  Neighbouring
 * subdomains share the points of their overlap; the left one keeps the left
 * half of them and the right one the right half (with an odd count the right
 * one keeps the middle point), so every interior point is owned by exactly
 * one subdomain: [own_lo, own_hi]. */
static long ovl_count(long n, long T, long o)
{
    if (n <= T) return 1;
    if (o == 0) return (n + T - 1) / T;
    return (n - T + (T - o) - 1) / (T - o) + 1;
}

static void ovl_span(long j, long J, long n, long T, long o, long *start, long *end, long *own_lo, long *own_hi)
{
    const long S = T - o;
    long st = 1 + j * S;
    if (o > 0 && J > 1 && j == J - 1) st = n - T + 1;
    *start = st;
    *end = st + T - 1 < n ? st + T - 1 : n;
    if (j == 0) {
        *own_lo = 1;
    } else {
        long ps, pe, d1, d2;
        ovl_span(j - 1, J, n, T, o, &ps, &pe, &d1, &d2);   /* previous subdomain's span only */
        *own_lo = st + (pe - st + 1) / 2;
    }
    if (j == J - 1) {
        *own_hi = n;
    } else {
        const long ns = (o > 0 && J > 1 && j + 1 == J - 1) ? n - T + 1 : 1 + (j + 1) * S;
        *own_hi = ns + (*end - ns + 1) / 2 - 1;
    }
}

/* One hierarchical cycle with overlapping subdomains (Sections 3.4 and 4.3):
 * every subdomain stages its points plus the one-point halo from u_in, runs k
 * Jacobi subiterations on all its points with the halo frozen, and writes
 * only the points it owns (ovl_span) to u_out.  ox = oy = 0 is the cycle of
 * hjo_hier_cycle.  Parity: pinned (ox = oy = 0 equals hjo_hier_cycle; k = 1
 * equals a classic sweep for any overlap; large k equals restricted additive
 * Schwarz with dense subdomain solves; k steps of local Jacobi then owner
 * selection at finite k; the cycle count of an independent probe of the
 * Section 3.5 problem). */
void hjo_hier_cycle_ovl(const hjo_problem *p, const double *f, const double *uin, double *uout,
                        int tx, int ty, int k, int ox, int oy)
{
    const long W = width_of(p);
    if (p->dim == 1) { ty = 1; oy = 0; }
    copy_ghosts(p, uin, uout);
    const long lw = tx + 2, lh = (p->dim == 2) ? ty + 2 : 1;
    double *L[2];
    L[0] = (double *)malloc(sizeof(double) * (size_t)(lw * lh));
    L[1] = (double *)malloc(sizeof(double) * (size_t)(lw * lh));
    const long Jx = ovl_count(p->nx, tx, ox);
    /* 2D: subdomains in y as in x; 1D: every copy (row) on its own */
    const long Jy = (p->dim == 2) ? ovl_count(p->ny, ty, oy) : p->ny;
    for (long jy = 0; jy < Jy; ++jy) {
        long j0, j1, oj0, oj1;
        if (p->dim == 2) {
            ovl_span(jy, Jy, p->ny, ty, oy, &j0, &j1, &oj0, &oj1);
        } else {
            j0 = j1 = oj0 = oj1 = jy;
        }
        for (long jx = 0; jx < Jx; ++jx) {
            long i0, i1, oi0, oi1;
            ovl_span(jx, Jx, p->nx, tx, ox, &i0, &i1, &oi0, &oi1);
            const long hj0 = (p->dim == 2) ? j0 - 1 : j0;
            const long hj1 = (p->dim == 2) ? j1 + 1 : j1;
            for (long j = hj0; j <= hj1; ++j)
                for (long i = i0 - 1; i <= i1 + 1; ++i) {
                    const long l = (j - hj0) * lw + (i - (i0 - 1));
                    L[0][l] = uin[j * W + i];
                    L[1][l] = uin[j * W + i];
                }
            for (int s = 0; s < k; ++s) {
                const double *src = L[s % 2];
                double *dst = L[(s + 1) % 2];
                for (long j = j0; j <= j1; ++j)
                    for (long i = i0; i <= i1; ++i) {
                        const long l = (j - hj0) * lw + (i - (i0 - 1));
                        const double uS = p->dim == 2 ? src[l - lw] : 0.0;
                        const double uN = p->dim == 2 ? src[l + lw] : 0.0;
                        dst[l] = jacobi_point(p, j * W + i, f[j * W + i], diag_at(p, j * W + i),
                                              src[l - 1], src[l + 1], uS, uN);
                    }
            }
            const double *fin = L[k % 2];
            for (long j = oj0; j <= oj1; ++j)
                for (long i = oi0; i <= oi1; ++i)
                    uout[j * W + i] = fin[(j - hj0) * lw + (i - (i0 - 1))];
        }
    }
    free(L[0]);
    free(L[1]);
}

/* Iterate classic sweeps (classic != 0) or hierarchical cycles from u (in/out)
 * until ||r_c|| <= tol * ||r_0|| (L2 residual reduced by the factor tol,
 * Sections 3.5 and 4.2), or max_cycles.  On return u holds u_c for the
 * returned c (the first iterate that met the tolerance, else the last one);
 * hist[c] = ||r_c|| for c < hist_cap.  *status: 0 converged, 1 not converged,
 * 2 diverged (non-finite residual).  Parity: pinned through its parts. */
long hjo_solve_ovl(const hjo_problem *p, const double *f, double *u, int classic,
                   int tx, int ty, int k, int ox, int oy, double tol, long max_cycles,
                   double *hist, long hist_cap, int *status);

long hjo_solve(const hjo_problem *p, const double *f, double *u, int classic,
               int tx, int ty, int k, double tol, long max_cycles,
               double *hist, long hist_cap, int *status)
{
    const size_t n = (size_t)(rows_of(p) * width_of(p));
    double *v = (double *)malloc(sizeof(double) * n);
    memcpy(v, u, sizeof(double) * n);
    const double r0 = sqrt(hjo_residual_sq(p, f, u));
    long c = 0;
    int st = 1;
    double *cur = u, *nxt = v;
    for (;;) {
        const double rc = (c == 0) ? r0 : sqrt(hjo_residual_sq(p, f, cur));
        if (hist && c < hist_cap) hist[c] = rc;
        if (!isfinite(rc)) { st = 2; break; }
        if (rc <= tol * r0) { st = 0; break; }
        if (c >= max_cycles) { st = 1; break; }
        if (classic) hjo_jacobi_sweep(p, f, cur, nxt);
        else hjo_hier_cycle(p, f, cur, nxt, tx, ty, k);
        double *t = cur; cur = nxt; nxt = t;
        ++c;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * n);
    free(v);
    if (status) *status = st;
    return c;
}

/* Run exactly ncycles cycles (or classic sweeps) from u (in/out). */
void hjo_run_fixed(const hjo_problem *p, const double *f, double *u, int classic,
                   int tx, int ty, int k, long ncycles)
{
    const size_t n = (size_t)(rows_of(p) * width_of(p));
    double *v = (double *)malloc(sizeof(double) * n);
    double *cur = u, *nxt = v;
    for (long c = 0; c < ncycles; ++c) {
        if (classic) hjo_jacobi_sweep(p, f, cur, nxt);
        else hjo_hier_cycle(p, f, cur, nxt, tx, ty, k);
        double *t = cur; cur = nxt; nxt = t;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * n);
    free(v);
}

/* hjo_solve / hjo_run_fixed with overlapping subdomains (ox, oy points). */
long hjo_solve_ovl(const hjo_problem *p, const double *f, double *u, int classic,
                   int tx, int ty, int k, int ox, int oy, double tol, long max_cycles,
                   double *hist, long hist_cap, int *status)
{
    const size_t n = (size_t)(rows_of(p) * width_of(p));
    double *v = (double *)malloc(sizeof(double) * n);
    memcpy(v, u, sizeof(double) * n);
    const double r0 = sqrt(hjo_residual_sq(p, f, u));
    long c = 0;
    int st = 1;
    double *cur = u, *nxt = v;
    for (;;) {
        const double rc = (c == 0) ? r0 : sqrt(hjo_residual_sq(p, f, cur));
        if (hist && c < hist_cap) hist[c] = rc;
        if (!isfinite(rc)) { st = 2; break; }
        if (rc <= tol * r0) { st = 0; break; }
        if (c >= max_cycles) { st = 1; break; }
        if (classic) hjo_jacobi_sweep(p, f, cur, nxt);
        else hjo_hier_cycle_ovl(p, f, cur, nxt, tx, ty, k, ox, oy);
        double *t = cur; cur = nxt; nxt = t;
        ++c;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * n);
    free(v);
    if (status) *status = st;
    return c;
}

void hjo_run_fixed_ovl(const hjo_problem *p, const double *f, double *u, int tx, int ty, int k, int ox, int oy,
                       long ncycles)
{
    const size_t n = (size_t)(rows_of(p) * width_of(p));
    double *v = (double *)malloc(sizeof(double) * n);
    double *cur = u, *nxt = v;
    for (long c = 0; c < ncycles; ++c) {
        hjo_hier_cycle_ovl(p, f, cur, nxt, tx, ty, k, ox, oy);
        double *t = cur; cur = nxt; nxt = t;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * n);
    free(v);
}

/* Threads the subdomain loop of hjo_hier_cycle and the row loop of
 * hjo_jacobi_sweep may use (an OpenMP build; 1 otherwise).  Results do not
 * depend on it.  Returns the count in effect. */
int hjo_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Thomas algorithm (tridiagonal direct solve, named in Section 3 as the direct
 * alternative for 1D): a = sub-diagonal (a[0] unused), d = diagonal,
 * c = super-diagonal (c[n-1] unused), b = RHS.  Used only to pin the 1D fixed
 * point.  Parity: pinned against a banded LU solve. */
void hjo_thomas(long n, const double *a, const double *d, const double *c,
                const double *b, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * (size_t)n);
    double *bp = (double *)malloc(sizeof(double) * (size_t)n);
    cp[0] = c[0] / d[0];
    bp[0] = b[0] / d[0];
    for (long i = 1; i < n; ++i) {
        const double m = d[i] - a[i] * cp[i - 1];
        cp[i] = (i < n - 1) ? c[i] / m : 0.0;
        bp[i] = (b[i] - a[i] * bp[i - 1]) / m;
    }
    x[n - 1] = bp[n - 1];
    for (long i = n - 2; i >= 0; --i) x[i] = bp[i] - cp[i] * x[i + 1];
    free(cp);
    free(bp);
}

/* ------------------------------------------------------------------------- */
/* Mixed-precision iterative refinement (not in the paper; the refinement
 * wrapper of the GPU path).  Inner arithmetic is binary32; with bf16 != 0 the
 * correction is rounded to bfloat16 (round to nearest even) every time a cycle
 * stores it, i.e. it is *stored* in bfloat16 between cycles.
 * Parity: pinned (converges to the DST / dense solution within the tolerance). */

static float bf16_round(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) == 0x7f800000u) {          /* Inf / NaN: keep, quiet NaN */
        if (b & 0x007fffffu) b |= 0x00400000u;
        b &= 0xffff0000u;
    } else {
        const uint32_t lsb = (b >> 16) & 1u;
        b = b + 0x7fffu + lsb;                        /* round half to even */
        b &= 0xffff0000u;
    }
    float y;
    memcpy(&y, &b, 4);
    return y;
}

float hjo_bf16_round(float x) { return bf16_round(x); }

/* binary32 version of jacobi_point: same association order, float operands */
static float jacobi_point_f32(int dim, float cW, float cE, float cS, float cN,
                              float rhs, float invd, float uW, float uE, float uS, float uN)
{
    float acc = cW * uW;
    acc = acc + cE * uE;
    if (dim == 2) {
        acc = acc + cS * uS;
        acc = acc + cN * uN;
    }
    return (rhs - acc) * invd;
}

/* One hierarchical cycle on the correction equation A d = rhs in binary32
 * (same subdomains, halos and container rule as hjo_hier_cycle). */
void hjo_hier_cycle_f32(const hjo_problem *p, const float *rhs, const float *din, float *dout,
                        int tx, int ty, int k, int bf16)
{
    const long W = width_of(p), R = rows_of(p);
    if (p->dim == 1) ty = 1;
    const float cW = (float)p->cW, cE = (float)p->cE, cS = (float)p->cS, cN = (float)p->cN;
    /* ghost ring of the correction is copied through unchanged */
    for (long q = 0; q < W * R; ++q) dout[q] = din[q];
    const long lw = tx + 2, lh = (p->dim == 2) ? ty + 2 : 1;
    float *L[2];
    L[0] = (float *)malloc(sizeof(float) * (size_t)(lw * lh));
    L[1] = (float *)malloc(sizeof(float) * (size_t)(lw * lh));
    const long jlo = first_row(p), jhi = last_row(p);
    const long jstep = (p->dim == 2) ? ty : 1;
    for (long j0 = jlo; j0 <= jhi; j0 += jstep) {
        const long j1 = (p->dim == 2) ? (j0 + ty - 1 < jhi ? j0 + ty - 1 : jhi) : j0;
        for (long i0 = 1; i0 <= p->nx; i0 += tx) {
            const long i1 = (i0 + tx - 1 < p->nx) ? i0 + tx - 1 : p->nx;
            const long hj0 = (p->dim == 2) ? j0 - 1 : j0;
            const long hj1 = (p->dim == 2) ? j1 + 1 : j1;
            for (long j = hj0; j <= hj1; ++j)
                for (long i = i0 - 1; i <= i1 + 1; ++i) {
                    const long l = (j - hj0) * lw + (i - (i0 - 1));
                    L[0][l] = din[j * W + i];
                    L[1][l] = din[j * W + i];
                }
            for (int s = 0; s < k; ++s) {
                const float *src = L[s % 2];
                float *dst = L[(s + 1) % 2];
                for (long j = j0; j <= j1; ++j)
                    for (long i = i0; i <= i1; ++i) {
                        const long l = (j - hj0) * lw + (i - (i0 - 1));
                        const float invd = (float)(1.0 / diag_at(p, j * W + i));
                        const float uS = p->dim == 2 ? src[l - lw] : 0.0f;
                        const float uN = p->dim == 2 ? src[l + lw] : 0.0f;
                        dst[l] = jacobi_point_f32(p->dim, cW, cE, cS, cN, rhs[j * W + i], invd,
                                                  src[l - 1], src[l + 1], uS, uN);
                    }
            }
            const float *fin = L[k % 2];
            for (long j = j0; j <= j1; ++j)
                for (long i = i0; i <= i1; ++i) {
                    const float v = fin[(j - hj0) * lw + (i - (i0 - 1))];
                    dout[j * W + i] = bf16 ? bf16_round(v) : v;
                }
        }
    }
    free(L[0]);
    free(L[1]);
}

/* ||rhs - A d||^2 for binary32 data, evaluated in binary64. */
double hjo_residual_sq_f32(const hjo_problem *p, const float *rhs, const float *d)
{
    const long W = width_of(p), R = rows_of(p);
    double *dd = (double *)malloc(sizeof(double) * (size_t)(W * R));
    double *rr = (double *)malloc(sizeof(double) * (size_t)(W * R));
    for (long q = 0; q < W * R; ++q) { dd[q] = (double)d[q]; rr[q] = (double)rhs[q]; }
    const double s = hjo_residual_sq(p, rr, dd);
    free(dd);
    free(rr);
    return s;
}

/* Iterative refinement: u (binary64, in/out) solves A u = f.
 *   outer step: r = f - A u (binary64); stop if ||r|| <= tol ||r_0||;
 *               rhs = (float) r; d = 0;
 *               inner: binary32 hierarchical cycles on A d = rhs until
 *                      ||rhs - A d|| <= inner_tol ||rhs||, or (stall_window > 0)
 *                      ||rhs - A d_c|| differs by at most stall_rtol (relative)
 *                      from its value stall_window cycles earlier (checked at
 *                      c = W, 2W, ...: the stored correction has reached its
 *                      fixed point), or inner_max cycles;
 *               u = u + (double) d   (interior points).
 * Returns the number of outer steps taken (== max_outer if not converged,
 * *status = 1).  hist[o] = ||r_o||; *inner_total = total inner cycles. */
long hjo_ir_solve(const hjo_problem *p, const double *f, double *u,
                  int tx, int ty, int k, double tol, double inner_tol, long inner_max,
                  long max_outer, int bf16, long stall_window, double stall_rtol,
                  double *hist, long hist_cap, long *inner_total, int *status)
{
    if (p->coef) {   /* refinement is defined here for constant neighbour coefficients */
        if (status) *status = 3;
        return -1;
    }
    const long W = width_of(p), R = rows_of(p);
    const size_t n = (size_t)(W * R);
    float *rhs = (float *)calloc(n, sizeof(float));
    float *d0 = (float *)calloc(n, sizeof(float));
    float *d1 = (float *)calloc(n, sizeof(float));
    const double r0 = sqrt(hjo_residual_sq(p, f, u));
    long total = 0, o = 0;
    int st = 1;
    for (;; ++o) {
        /* binary64 residual */
        double r2 = 0.0;
        for (long q = 0; q < (long)n; ++q) rhs[q] = 0.0f;
        for (long j = first_row(p); j <= last_row(p); ++j)
            for (long i = 1; i <= p->nx; ++i) {
                const long q = j * W + i;
                const double r = f[q] - apply_point(p, u, q);
                r2 = r2 + r * r;
                rhs[q] = (float)r;
            }
        const double rn = sqrt(r2);
        if (hist && o < hist_cap) hist[o] = rn;
        if (!isfinite(rn)) { st = 2; break; }
        if (rn <= tol * r0) { st = 0; break; }
        if (o >= max_outer) { st = 1; break; }
        /* binary32 inner solve from d = 0 */
        memset(d0, 0, n * sizeof(float));
        memset(d1, 0, n * sizeof(float));
        float *cur = d0, *nxt = d1;
        const double ri0 = sqrt(hjo_residual_sq_f32(p, rhs, cur));
        double mark = ri0;
        long mark_c = 0;
        for (long c = 0; c < inner_max; ++c) {
            const double ri = (c == 0) ? ri0 : sqrt(hjo_residual_sq_f32(p, rhs, cur));
            if (ri <= inner_tol * ri0) break;
            if (stall_window > 0 && c > 0 && c - mark_c >= stall_window) {
                const int stop = fabs(ri - mark) <= stall_rtol * ri;
                mark = ri;
                mark_c = c;
                if (stop) break;
            }
            hjo_hier_cycle_f32(p, rhs, cur, nxt, tx, ty, k, bf16);
            float *t = cur; cur = nxt; nxt = t;
            ++total;
        }
        /* binary64 update */
        for (long j = first_row(p); j <= last_row(p); ++j)
            for (long i = 1; i <= p->nx; ++i) {
                const long q = j * W + i;
                u[q] = u[q] + (double)cur[q];
            }
    }
    free(rhs);
    free(d0);
    free(d1);
    if (inner_total) *inner_total = total;
    if (status) *status = st;
    return o;
}

/* ------------------------------------------------------------------------- */
/* Implicit adjoint of A(sigma) u = f (not in the paper; the differentiation
 * wrapper of the GPU path).  For L(u(f, sigma)):
 *   A^T lambda = dL/du,  dL/df = lambda,  dL/dsigma_p = -lambda_p u_p,
 * because dA/dsigma_p = e_p e_p^T.  A^T of the constant stencil swaps the
 * coefficients cW <-> cE and cS <-> cN; lambda has a zero ghost ring.
 * The adjoint system is solved with binary64 hierarchical cycles to tol.
 * Parity: pinned (dense A^{-T}, central finite differences). */
long hjo_adjoint(const hjo_problem *p, const double *g, const double *u,
                 double *lam, double *dl_dsigma, int tx, int ty, int k,
                 double tol, long max_cycles, int *status)
{
    if (p->coef) {   /* the transposed stencil is built for constant neighbour coefficients */
        if (status) *status = 3;
        return -1;
    }
    const long W = width_of(p), R = rows_of(p);
    hjo_problem pt = *p;
    pt.cW = p->cE; pt.cE = p->cW;
    pt.cS = p->cN; pt.cN = p->cS;
    memset(lam, 0, sizeof(double) * (size_t)(W * R));
    const long c = hjo_solve(&pt, g, lam, 0, tx, ty, k, tol, max_cycles, NULL, 0, status);
    if (dl_dsigma) {
        memset(dl_dsigma, 0, sizeof(double) * (size_t)(W * R));
        for (long j = first_row(p); j <= last_row(p); ++j)
            for (long i = 1; i <= p->nx; ++i) {
                const long q = j * W + i;
                dl_dsigma[q] = -lam[q] * u[q];
            }
    }
    return c;
}

/* Shared memory of the paper's own kernel layout (Sections 3.3 and 4.1): two
 * containers of the halo-augmented subdomain plus the interior RHS values,
 * times the element size.  Pinned by the printed 800 B and 26.688 kB. */
long hjo_paper_smem_bytes(int dim, int tx, int ty, int esize)
{
    if (dim == 1) return (long)(2 * (tx + 2) + tx) * esize;
    return (long)(2 * (tx + 2) * (ty + 2) + tx * ty) * esize;
}
