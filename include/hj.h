/*
 * hj.h -- C ABI of the GB300 hierarchical Jacobi solver.
 *
 * Method: Islam & Wang, "Hierarchical Jacobi Iteration for Structured Matrices
 * on GPUs using Shared Memory" (arXiv 2006.16465).  A cycle partitions the grid
 * into subdomains (tiles), stages each tile plus a one-point halo on chip, runs
 * k Jacobi subiterations there with the halo frozen, and writes the tile
 * interior back (Section 3.3 for 1D, Section 4.1 for 2D).  Cycles repeat until
 * the L2 residual has dropped by the requested factor (Sections 3.5, 4.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Operator.  For interior point p with neighbours W,E (x-1, x+1) and S,N
 * (y-1, y+1):
 *     (A u)_p = d_p u_p + cW u_W + cE u_E + cS u_S + cN u_N,
 *     d_p     = cD + sigma_const + sigma_p          (sigma_p = 0 if sigma NULL)
 * This is the tridiagonal stencil of Section 3 (Eq. jacobi-stencil-equation-1d,
 * a = cW, c = cE, d = cD) and the pentadiagonal stencil of Section 4
 * (Eq. 2d-jacobi-stencil, a,c,e,f,d = cW,cE,cS,cN,cD), plus a screening term.
 * 2D Poisson on the unit square (Eq. 2d-poisson): cW = cE = -1/hx^2,
 * cS = cN = -1/hy^2, cD = 2/hx^2 + 2/hy^2, hx = 1/(nx+1), hy = 1/(ny+1).
 * The stencil must be diagonally dominant, |d_p| >= |cW|+|cE|+|cS|+|cN| with
 * d_p > 0 (the convergence condition of Section 2.1); hj_create checks it.
 *
 * Grid arrays (f, u, g, sigma, dl_df, dl_dsigma).  Row-major, x fastest, with a
 * one-point ghost ring holding Dirichlet data:
 *     2D: (ny + 2) rows, element (row j, column i) at index j*ld + i,
 *         interior j = 1..ny, i = 1..nx.
 *     1D: ny rows; every row is an independent 1D problem (the paper's 1024
 *         simultaneous copies, Section 3.5), interior i = 1..nx, ghosts at
 *         i = 0 and i = nx + 1.
 * ld (elements) >= nx + 2.  Base pointers must be 16-byte aligned and
 * ld * element_size a multiple of 16 bytes.  Element type: double for
 * HJ_F64, float for HJ_F32; sigma is always double.
 * Ghost-ring entries of f and sigma are ignored.
 *
 * Memory.  Pointers passed to the solve calls are device pointers, except
 * that hj_solve also accepts host pointers for f and u (it then copies them
 * through its own device buffers, see hj_solve).  The caller owns every
 * array it passes; the handle owns its workspace (second iterate buffer,
 * residual partials, refinement buffers, CUDA graphs) and frees it in
 * hj_destroy.  sigma must stay valid for the life of the handle.
 *
 * Streams.  Every call is ordered on the given stream (NULL = the legacy
 * default stream).  hj_solve, hj_solve_adjoint and hj_residual synchronise
 * with that stream to read convergence state and return results, so they
 * block the calling host thread.
 *
 * Errors.  Every int-returning call returns an hj_status code; HJ_OK = 0.
 * hj_last_error() gives a one-line description of the most recent failure on
 * the calling thread.  A handle stays usable after HJ_ERR_NOT_CONVERGED,
 * HJ_ERR_DIVERGED and HJ_ERR_INVALID_ARG; after HJ_ERR_CUDA or
 * HJ_ERR_TIMEOUT only hj_destroy is safe.
 */
#ifndef HJ_H
#define HJ_H

#ifdef __cplusplus
extern "C" {
#endif

/* Entry points are the only symbols the shared library exports. */
#if defined(__GNUC__)
#define HJ_API __attribute__((visibility("default")))
#else
#define HJ_API
#endif

typedef struct hj_handle hj_handle;

/* A cudaStream_t passed as an opaque pointer (NULL = legacy default stream). */
typedef void *hj_stream;

enum hj_status {
    HJ_OK = 0,
    HJ_ERR_INVALID_ARG = 1,      /* bad size, pointer, alignment or parameter     */
    HJ_ERR_NOT_DIAG_DOMINANT = 2,/* stencil fails the Section 2.1 condition        */
    HJ_ERR_UNSUPPORTED = 3,      /* tile shape / mode combination not built        */
    HJ_ERR_CUDA = 4,             /* a CUDA runtime call failed                     */
    HJ_ERR_NOT_CONVERGED = 5,    /* max_cycles reached; u holds the last iterate   */
    HJ_ERR_DIVERGED = 6,         /* residual became NaN or Inf                     */
    HJ_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up             */
    HJ_ERR_NO_MEMORY = 8,        /* workspace allocation failed                    */
    HJ_ERR_BOUNDS = 9            /* debug builds: an index check or guard band
                                    failed (hj_debug_check)                       */
};

enum hj_dtype { HJ_F64 = 0, HJ_F32 = 1 };

/* Arithmetic of the solve.
 *   HJ_PREC_F64          : binary64 cycles; the update is evaluated in the fixed
 *                          order  acc = cW*uW; acc += cE*uE; acc += cS*uS;
 *                          acc += cN*uN; u' = (f - acc) * (1/d_p)  with no fused
 *                          multiply-add, so results are reproducible bit for bit.
 *   HJ_PREC_F32          : binary32 cycles on binary32 f and u (fused multiply-
 *                          add allowed).  Attainable relative residual ~1e-6.
 *   HJ_PREC_F32_IR       : binary64 f and u; mixed-precision iterative
 *                          refinement: binary64 residual r = f - A u and binary64
 *                          update u += d are the only binary64 steps; the
 *                          correction equation A d = r is solved by binary32
 *                          hierarchical cycles.
 *   HJ_PREC_BF16CORR_IR  : as F32_IR, but the correction d is stored in
 *                          bfloat16 between cycles (arithmetic stays binary32). */
enum hj_precision { HJ_PREC_F64 = 0, HJ_PREC_F32 = 1, HJ_PREC_F32_IR = 2, HJ_PREC_BF16CORR_IR = 3 };

/* HJ_METHOD_HIER: hierarchical cycles (Sections 3.3, 4.1).
 * HJ_METHOD_CLASSIC: one global-memory Jacobi sweep per step (Section 3.2);
 * every point reads the previous iterate only (a true grid-wide step).
 * HJ_METHOD_MG: geometric multigrid V-cycles whose smoother is the
 * hierarchical cycle with damped Jacobi subiterations (the use the paper's
 * conclusion names).  2D, constant coefficients, sigma_const only, odd nx and
 * ny; level l + 1 has (n_l - 1) / 2 points per axis (coarse point I on fine
 * point 2I), its operator rediscretises the stencil (cW..cN and cD divided by
 * 4, sigma_const kept); full-weighting restriction of the residual, bilinear
 * prolongation, the coarsest level solved by mg_coarse_cycles undamped
 * cycles of mg_coarse_k subiterations on one subdomain.  A "cycle" in
 * hj_stats and max_cycles / fixed_cycles is one V-cycle; a solve also ends
 * (HJ_ERR_NOT_CONVERGED) when ||r|| fell by less than 1 % over 4 V-cycles,
 * the floor that the storage precision sets. */
enum hj_method { HJ_METHOD_HIER = 0, HJ_METHOD_CLASSIC = 1, HJ_METHOD_MG = 2 };

typedef struct {
    int dim;              /* 1, 2 or 3 (3: the seven-point extension, see nz)    */
    int nx, ny;           /* interior points; 1D: ny = number of independent rows */
    long long ld;         /* row pitch of every grid array, in elements          */
    double cW, cE, cS, cN, cD;  /* stencil (cS, cN ignored in 1D)                */
    double sigma_const;   /* constant screening added to the diagonal            */
    const double *sigma;  /* device, grid layout, per-point screening; nullable  */
    int dtype;            /* hj_dtype of f and u                                 */
    const double *coef;   /* device, nullable: per-point neighbour coefficients
                             replacing cW..cN (the general tridiagonal a_i, c_i
                             of Section 3 and its 2D analogue): planes W, E
                             (1D) or W, E, S, N (2D), each rows x ld binary64 in
                             the grid layout, one after another.  The diagonal
                             stays cD + sigma_const + sigma_p.  Runs on the
                             one-thread-per-point kernels under CUDA graphs;
                             HJ_PREC_F64 and HJ_PREC_F32 only, no overlap, no
                             adjoint, no batched solves (HJ_ERR_UNSUPPORTED)  */
    int nz;               /* dim = 3: interior planes (1 <= nz <= 65535).  A 3D
                             grid array is (nz + 2) planes of (ny + 2) rows of
                             ld elements (x fastest, then y, then z) with a
                             one-point ghost shell of Dirichlet data; the
                             operator is Section 4's five-point stencil plus
                             cB u_{z-1} + cT u_{z+1} (an extension: the paper
                             stops at 2D).  3D takes constant coefficients and
                             sigma_const only (sigma, coef NULL), HJ_PREC_F64
                             or HJ_PREC_F32, hierarchical or classic, on CUDA
                             graphs; no refinement, overlap, in-place, adjoint,
                             autotune or batched solves (HJ_ERR_UNSUPPORTED)  */
    double cB, cT;        /* dim = 3: bottom (z - 1) and top (z + 1) coefficients */
} hj_desc;

typedef struct {
    int method;           /* hj_method                                           */
    int tile_x, tile_y;   /* subdomain interior size (the paper's blockDim.x,
                             blockDim.y); 1D ignores tile_y.  Built shapes are
                             listed by hj_tile_shapes().                          */
    int k;                /* subiterations per cycle (>= 1)                      */
    int precision;        /* hj_precision                                        */
    int check_every;      /* cycles per host convergence check (CUDA graph
                             length); rounded up to an even number                */
    long long max_cycles; /* cap on cycles (classic: sweeps)                     */
    double tol;           /* stop at the first iterate with
                             ||f - A u_c||_2 <= tol * ||f - A u_0||_2             */
    long long fixed_cycles; /* > 0: run exactly this many cycles, check nothing  */
    double inner_tol;     /* refinement: inner relative residual target          */
    long long inner_max_cycles; /* refinement: cap on inner cycles per outer step */
    int max_outer;        /* refinement: cap on outer steps                      */
    int persistent;       /* 1: single persistent launch looping over cycles with
                             a device-side grid barrier (needs all tiles resident);
                             0: one launch per cycle inside CUDA graphs;
                             -1: choose automatically                            */
    int autotune;         /* 1: pick tile shape and k by measurement (hj_autotune)
                             at hj_create; 2: keep tile_x, tile_y and tune k only
                             (both also pick the overlap, replacing overlap_x/y);
                             3: keep tile and k, tune only the pipelined kernel's
                             launch (threads per subdomain, copy stages, CTAs
                             per SM; 1 and 2 tune it too after their pick);
                             hj_solve_batched: tile from the largest problem,
                             k per size class                                   */
    int pipeline;         /* 2D cycles: 1 = TMA-pipelined kernel (CTAs walk tile
                             lists, next tile staged while the current one
                             sweeps), 0 = one CTA per tile, -1 = automatic.
                             3D: 1 = persistent warps that prefetch the next
                             subdomain with cp.async; 0 = one warp per
                             subdomain; -1 = automatic: binary32 grids of at
                             least 8 subdomains per SM (subdomains at least 16
                             wide) run the TMA-pipelined kernel (one warp per
                             CTA walking subdomains), others one warp per
                             subdomain                                        */
    int tile_threads;     /* threads per subdomain (one warp per band of rows);
                             0 = the default for the tile shape; the built
                             combinations are listed by hj_tile_variants()      */
    int pipeline_stages;  /* TMA-pipelined kernel: shared-memory stages per CTA
                             (binary32 / bfloat16: 1 or 2, binary64: 2; 0 = the
                             default, the first built).  With one stage the
                             next tile is copied in while the current one
                             sweeps in registers                               */
    int inner_stall;      /* refinement: an inner solve also stops when ||r|| has
                             changed by <= 1e-3 (relative) over this many cycles,
                             i.e. the correction has reached the fixed point its
                             storage precision allows; 0 = off                 */
    int ctas_per_sm;      /* TMA-pipelined kernel: resident CTAs per SM (0 = as
                             many as fit).  Fewer CTAs keep fewer copies in
                             flight, which HBM can serve at a higher rate     */
    int overlap_x;        /* overlapping subdomains (Sections 3.4 and 4.3):
                             points shared by neighbouring subdomains along x
                             (0 <= overlap_x < tile_x).  Starts advance by
                             tile_x - overlap_x, the last subdomain ends at nx,
                             and each shared point is written by the subdomain
                             in which it lies further from an edge (an overlap
                             is split at its midpoint).  Runs on CUDA graphs of
                             the one-CTA-per-subdomain kernels; persistent = 1,
                             pipeline = 1 and classic reject it; batched
                             solves run without overlap                      */
    int overlap_y;        /* the same along y (2D; 0 <= overlap_y < tile_y)   */
    int in_place;         /* 1: one global iterate array, as the listing of
                             Appendix A has it: a subdomain may stage halo
                             values that a neighbour already overwrote in the
                             same cycle, so results depend on scheduling and
                             are not reproducible bit for bit.  The stopping
                             test uses the fused residual of the staged data;
                             res0 and res_final are exact residuals of the
                             initial and the returned array (which may be one
                             cycle past the checked one).  0 (default): u_c
                             and u_{c+1} in separate arrays, deterministic   */
    int tile_z;           /* 3D: subdomain depth; 0 = the default 3D shape of
                             the precision (binary32 16 x 8 x 8, binary64
                             16 x 4 x 8), which replaces tile_x and tile_y.
                             Built shapes are listed by hj_tile_shapes3d()    */
    int mg_levels;        /* HJ_METHOD_MG: levels including the given grid (>= 2;
                             0 = as many as the sizes allow).  The coarsest
                             level must hold at most 1024 points             */
    int mg_pre, mg_post;  /* HJ_METHOD_MG: smoothing cycles before and after the
                             coarse correction (>= 0); each cycle runs k damped
                             subiterations on tile_x x tile_y subdomains
                             (tile_x * tile_y <= 1024)                       */
    double mg_omega;      /* HJ_METHOD_MG: Jacobi damping, 0 < omega <= 1
                             (u' = u + omega (jac - u))                       */
    int mg_coarse_k;      /* HJ_METHOD_MG: subiterations per coarsest-level cycle */
    int mg_coarse_cycles; /* HJ_METHOD_MG: cycles on the coarsest level        */
} hj_params;

typedef struct {
    long long cycles;         /* cycles (classic: sweeps) up to the returned iterate */
    long long cycles_launched;/* cycles issued, including skipped overshoot        */
    long long inner_cycles;   /* refinement: total binary32 cycles               */
    int outer_steps;          /* refinement: outer steps taken                   */
    double res0;              /* ||f - A u_0||_2                                  */
    double res_final;         /* ||f - A u||_2 of the returned iterate            */
    double rel_final;         /* res_final / res0 (0 if res0 == 0)                */
    double *history;          /* caller-owned host array (nullable): ||r_c||_2 per
                                 checked iterate (refinement: per outer step)     */
    long long history_cap;    /* capacity of history                             */
    long long history_len;    /* entries written                                 */
    double wall_ms;           /* host wall time of the call                      */
    int tile_x, tile_y, k;    /* configuration actually used                     */
    int tile_threads;         /* threads per subdomain actually used             */
    int persistent;           /* 1 if the persistent path ran                    */
    int pipeline_stages;      /* copy stages of the pipelined kernel if it runs, else 0 */
    int ctas_per_sm;          /* its CTAs-per-SM cap (0 = as many as fit)         */
    int overlap_x, overlap_y; /* overlapping points used (Sections 3.4, 4.3)      */
    int tile_z;               /* 3D: subdomain depth used (1 otherwise)           */
    /* hj_solve_batched / hj_solve_adjoint_batched: */
    int graphed;              /* 1 if every refinement step ran as a replay of one
                                 captured CUDA graph (zero the corrections, the
                                 persistent inner launch, the binary64 update and
                                 residual, the retirement decisions)              */
    double *cycle_ms;         /* caller-owned host array (nullable): duration of
                                 each batch cycle (every active problem advances
                                 one inner cycle), refinement steps one after
                                 another                                          */
    long long *cycle_points;  /* caller-owned host array (nullable): interior
                                 points of the problems active in that cycle      */
    long long cycle_cap;      /* capacity of cycle_ms and cycle_points            */
    long long cycle_len;      /* batch cycles recorded (at most cycle_cap)        */
} hj_stats;

/* Fill p with defaults: hierarchical, 32 x 32 tiles, k = 16, HJ_PREC_F64,
 * check_every = 64, max_cycles = 10^7, tol = 1e-6, fixed_cycles = 0,
 * inner_tol = 1e-4, inner_max_cycles = 10^6, max_outer = 60, persistent = -1,
 * autotune = 0, pipeline = -1, tile_threads = 0, pipeline_stages = 0,
 * inner_stall = 32, ctas_per_sm = 0, overlap_x = overlap_y = 0, in_place = 0,
 * tile_z = 0, mg_levels = 0, mg_pre = mg_post = 1, mg_omega = 0.8,
 * mg_coarse_k = 64, mg_coarse_cycles = 4. */
HJ_API void hj_default_params(hj_params *p);

/* Create a solver for one problem shape.  Validates the descriptor and
 * parameters (HJ_ERR_INVALID_ARG, HJ_ERR_NOT_DIAG_DOMINANT, HJ_ERR_UNSUPPORTED),
 * allocates the workspace on the current device (HJ_ERR_NO_MEMORY) and
 * precomputes the diagonal of a per-point sigma.  *out is NULL on failure. */
HJ_API int hj_create(hj_handle **out, const hj_desc *desc, const hj_params *params);

/* Solve A u = f.  u: in = initial guess whose ghost ring holds the Dirichlet
 * data; out = the first iterate u_c with ||r_c|| <= tol ||r_0|| (c in
 * stats->cycles), or the last iterate (HJ_ERR_NOT_CONVERGED, HJ_ERR_DIVERGED).
 * With params.fixed_cycles > 0 exactly that many cycles run and no residual is
 * tested.  f and u may both be host pointers (pageable or pinned): they are
 * then copied to and from device buffers inside the call.  stats: nullable. */
HJ_API int hj_solve(hj_handle *h, const void *f, void *u, hj_stream stream, hj_stats *stats);

/* ||f - A u||_2 over interior points (binary64 accumulation, deterministic
 * order) into *abs_l2, and *rel_l2 = abs / ||f||_2 (abs itself if f = 0).
 * Device pointers; either output pointer may be NULL. */
HJ_API int hj_residual(hj_handle *h, const void *f, const void *u, double *abs_l2, double *rel_l2,
                hj_stream stream);

/* Implicit adjoint of the solve for a loss L(u).  Given g = dL/du (grid,
 * device, same dtype as u) and the solution u, solves A^T lambda = g with a
 * zero ghost ring by the same hierarchical cycles and precision as hj_solve
 * (A^T of the stencil swaps cW<->cE and cS<->cN), then writes
 *     dl_df     = lambda                (dL/df)
 *     dl_dsigma = -lambda * u  pointwise (dL/dsigma_p, since dA/dsigma_p = e_p e_p^T)
 * dl_dsigma (binary64 grid) may be NULL.  Ghost entries of the outputs are 0.
 * No iterate of the forward solve is stored or needed besides u. */
HJ_API int hj_solve_adjoint(hj_handle *h, const void *g, const void *u, void *dl_df, void *dl_dsigma,
                     hj_stream stream, hj_stats *stats);

/* Solve nprob independent 2D problems (each with its own hj_desc: sizes, ld,
 * stencil, sigma_const, per-point sigma or NULL; dtype HJ_F64) in one
 * persistent launch per refinement phase, fed by a device work queue of
 * (problem, tile) items; problems retire independently when they meet
 * params.tol.  The handle must come from hj_create with a 2D descriptor and
 * HJ_PREC_F32_IR or HJ_PREC_BF16CORR_IR (it supplies params; autotune = 1
 * tunes one tile variant for the launch and k per size class).  f[i], u[i]
 * are device pointers.  stats (nullable) receives totals (rel_final = the
 * worst relative residual); per-problem inner cycle counts go to cycles_out
 * (host, nprob entries, nullable). */
HJ_API int hj_solve_batched(hj_handle *h, int nprob, const hj_desc *descs, const void *const *f,
                     void *const *u, hj_stream stream, hj_stats *stats, long long *cycles_out);

/* Adjoint of a batch of nrhs solves that share the handle's operator A(sigma)
 * (the handle's descriptor, sigma included): solves A^T lambda_b = g_b for
 * every b in one persistent launch per refinement phase (handle precision
 * HJ_PREC_F32_IR or HJ_PREC_BF16CORR_IR, 2D), writes dl_df[b] = lambda_b and
 * accumulates dl_dsigma = -sum_b lambda_b * u_b (binary64 grid, nullable) by
 * the fused gradient kernel.  g, u, dl_df: device grids in the handle's layout.
 * Same errors as hj_solve_batched. */
HJ_API int hj_solve_adjoint_batched(hj_handle *h, int nrhs, const void *const *g, const void *const *u,
                                    void *const *dl_df, void *dl_dsigma, hj_stream stream, hj_stats *stats);

/* Free the handle and its workspace (NULL is ignored). */
HJ_API void hj_destroy(hj_handle *h);

/* Static description of a status code. */
HJ_API const char *hj_error_string(int status);

/* One-line description of the last error on the calling thread ("" if none). */
HJ_API const char *hj_last_error(void);

/* Pick the subdomain shape (tile_x, tile_y; threads per subdomain follow from
 * it) and the subiteration count k for desc and params->precision/tol by
 * measurement on the device, and write them into *params (other fields are
 * left alone).  k trades in-chip work against halo staleness (Section 3.3);
 * each candidate is scored by its measured time per cycle times the cycles
 * its measured contraction rate needs to reach tol.  Results are cached per
 * process and, when the environment variable HJ_AUTOTUNE_CACHE names a file,
 * in that file.  *predicted_ms (nullable) receives the predicted time to
 * tolerance, or -1 for a cache hit.  hj_create runs this when
 * params->autotune is 1; params->autotune = 2 keeps tile_x, tile_y and tunes
 * k only.  Modes 1 and 2 also pick the overlap of neighbouring subdomains
 * (Sections 3.4, 4.3) from {0, 2, 4, 8} points (below half the subdomain
 * side) and write it into overlap_x (and overlap_y in 2D).  Where the TMA-pipelined kernel runs the cycles (2D grids of at least
 * 8 subdomains per SM, or pipeline = 1), every mode then measures its launch
 * shapes for the chosen subdomain and k (threads per subdomain, copy stages,
 * CTAs per SM) and writes the fastest into tile_threads, pipeline_stages and
 * ctas_per_sm; params->autotune = 3 does only that.  1D and 2D grids with
 * constant coefficients and hierarchical cycles only: a 3D descriptor, per-point
 * coefficients or HJ_METHOD_MG give HJ_ERR_UNSUPPORTED before any GPU work. */
HJ_API int hj_autotune(const hj_desc *desc, hj_params *params, double *predicted_ms);

/* Runs params->fixed_cycles cycles (hierarchical, or classic sweeps with
 * params->method) on u in place, like hj_solve with fixed_cycles, but
 * allocates nothing: no handle, no workspace, no graph.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory
 * when they need cycles (a device-memory budget fixed at start-up, a real-time
 * loop that cannot afford cudaMalloc, memory owned by another allocator).
 * The second iterate buffer comes from a static 16 MiB device array inside
 * the library, so the grid must satisfy rows * ld * element size <= 16 MiB
 * (2D: rows = ny + 2), else HJ_ERR_INVALID_ARG.  desc->sigma must be NULL
 * (sigma_const is fine); params->precision is HJ_PREC_F64 or HJ_PREC_F32 to
 * match desc->dtype; tile_x, tile_y, k, method as for hj_create.  f and u are
 * device pointers (same layout rules).  Stream-ordered; does not wait.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture; after
 * cudaDeviceReset the next call on that device looks it up again (the same
 * rule applies to it).  in_place, persistent = 1, pipeline = 1 and autotune
 * give HJ_ERR_UNSUPPORTED (they need a handle's workspace).  All
 * calls share the array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and corrupt each other's results. */
HJ_API int hj_cycles_noalloc(const hj_desc *desc, const hj_params *params, const void *f, void *u,
                             hj_stream stream);

/* Memory checks of debug builds (the library compiled with -DHJ_DEBUG, see
 * the package's build script), a stand-in for an external memory checker; no
 * counterpart in the paper.  In such builds the cycle kernels (2D and 1D
 * subdomain kernels, the pipelined and persistent engines, the classic sweep)
 * check every staging, exchange and write-back index against the extent of
 * the array or shared box it addresses, skip an access that fails and record
 * the first failure in a device word; every device allocation of the library
 * is surrounded by guard bands of a fixed byte pattern.  hj_debug_check waits
 * for the device, then reports the first recorded failure: *site = the kernel
 * site (> 0) and *index = the failing index, or *site = -2 and *index = the
 * byte offset (from the start of the allocation) of an overwritten guard byte;
 * it returns HJ_ERR_BOUNDS for either and clears it (so each is reported
 * once), HJ_OK with *site = 0 when clean.  Release builds return HJ_OK with
 * *site = -1: no checks are compiled in.  Either pointer may be NULL.  The
 * device word lives on the device current at the first debug-build call. */
HJ_API int hj_debug_check(long long *site, long long *index);

/* Debug builds: shows that both checks catch what they are for, without any
 * access out of bounds: a kernel checks one index outside its range (no
 * memory is addressed), and the host overwrites one byte of a fresh
 * allocation's trailing guard band with cudaMemset.  HJ_OK if both were
 * reported, HJ_ERR_BOUNDS if not; HJ_ERR_UNSUPPORTED in release builds. */
HJ_API int hj_debug_selftest(void);

/* Built (tile_x, tile_y, threads) combinations for (dim, precision): writes
 * up to cap triples into txt[3*i .. 3*i+2] and returns how many exist. */
HJ_API int hj_tile_variants(int dim, int precision, int *txt, int cap);

/* Tile shapes built for (dim, precision): writes up to cap (tile_x, tile_y)
 * pairs into xy[2*i], xy[2*i+1] and returns how many exist. */
HJ_API int hj_tile_shapes(int dim, int precision, int *xy, int cap);

/* 3D subdomain shapes built for a precision (HJ_PREC_F64 or HJ_PREC_F32):
 * writes up to cap (tile_x, tile_y, tile_z) triples into xyz[3*i .. 3*i+2]
 * and returns how many exist (0 for other precisions). */
HJ_API int hj_tile_shapes3d(int precision, int *xyz, int cap);

#ifdef __cplusplus
}
#endif

#endif /* HJ_H */
