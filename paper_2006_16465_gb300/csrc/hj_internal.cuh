// hj_internal.cuh -- shared device/host pieces of the GB300 hierarchical Jacobi
// library: kernel argument blocks, the device-side convergence control block,
// and the deterministic two-level residual reduction fused into every cycle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/hj.h"

namespace hj {

// ---------------------------------------------------------------------------
// Device-side convergence control.  One per handle.  The last CTA to finish a
// cycle folds the residual of the cycle's *input* iterate u_c into it, so the
// host only reads it every check_every cycles, and launches queued after
// convergence return at once (the graph may overshoot without touching u).
// ---------------------------------------------------------------------------
struct Ctl {
    int done;            // -1 while iterating; else index c of the iterate to return
    int status;          // HJ_OK, HJ_ERR_DIVERGED or HJ_ERR_NOT_CONVERGED
    long long cycle;     // index of the iterate whose residual the next cycle computes
    double res2_0;       // ||r_0||^2
    double res2_last;    // ||r_c||^2 of the last reduced cycle
    int err;             // HJ_ERR_TIMEOUT if a bounded device wait expired
    int pad;
    double res2_mark;    // stagnation rule: ||r||^2 at cycle mark_cycle
    long long mark_cycle;
    // deferred fold (TMA-pipelined kernel): launches started, and per launch
    // parity whether the launch only folds its predecessor's partials
    long long launch;
    int fold_only[2];
};

constexpr int kHistCap = 1 << 17;  // device ring of per-cycle ||r_c||^2 (power of two)
constexpr int kGroup = 256;        // CTAs per first-level reduction group

enum RedMode { RED_CYCLE = 0, RED_STORE = 1 };

struct RedArgs {
    double *partials;    // one per CTA (NV per CTA)
    double *gpart;       // one per group (NV per group)
    unsigned *gcnt;      // arrival counters per group (zero between uses)
    unsigned *fcnt;      // final arrival counter (zero between uses)
    double *hist;        // RED_CYCLE: ring of ||r_c||^2, kHistCap entries
    double *out;         // RED_STORE: NV results
    Ctl *ctl;            // RED_CYCLE: control block
    double tol;          // stop at ||r_c|| <= tol ||r_0||
    double scale;        // RED_CYCLE: the reduced sum is multiplied by this (d^2 for the fast path)
    long long stall_window;  // > 0: also stop when ||r|| moved by <= stall_rtol relative over this many cycles
    double stall_rtol;
    long long max_cycles;
    int mode;            // RedMode
};

// Arguments of one cycle (or one classic sweep).
// Debug builds (compiled with -DHJ_DEBUG) stand in for a memory checker:
// every staging, exchange and write-back index of the cycle kernels is
// checked against the extent of the array it addresses; a failure records
// the first (site, index) in a device word and skips the access instead of
// trapping, and hj_debug_check reports it.  Release builds compile the
// checks away (HJ_IN is the constant true).
struct DbgWord {
    unsigned long long site;   // 0 = clean
    long long index;
};
#ifdef HJ_DEBUG
__device__ __forceinline__ bool dbg_in(DbgWord *w, long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    if (w && atomicCAS(&w->site, 0ull, (unsigned long long)site) == 0ull) w->index = i;
    return false;
}
#define HJ_IN(w, i, n, site) ::hj::dbg_in((w), (long long)(i), (long long)(n), (site))
#else
#define HJ_IN(w, i, n, site) true
#endif

// Classic 2D sweep (classic2d_kernel): rows per thread, and the block of
// points one CTA of 32 x 8 threads covers per step of its grid-stride loop
// (columns counted from the ghost column 0, 16 bytes of storage per thread).
constexpr int kClassicRows = 4;
inline int classic2d_block_cols(int storage_bytes) { return 32 * (16 / storage_bytes); }
inline int classic2d_block_rows() { return 8 * kClassicRows; }
inline long long classic2d_blocks(int nx, int ny, int storage_bytes) {
    const int bx = classic2d_block_cols(storage_bytes), by = classic2d_block_rows();
    return (long long)((nx + 2 + bx - 1) / bx) * ((ny + by - 1) / by);
}

struct CycArgs {
    const void *f;       // right-hand side, compute type (grid layout)
    const void *uin;     // iterate u_c, storage type
    void *uout;          // iterate u_{c+1}, storage type
    const void *dinv;    // per-point 1/d_p in compute type (grid layout), or null
    long long ld;        // row pitch (elements)
    int nx, ny, k;       // interior size, subiterations
    double cW, cE, cS, cN;   // stencil
    double invd;         // 1/(cD + sigma_const) when dinv is null
    double dconst;       // cD + sigma_const
    // binary32 copies precomputed on the host (binary64 arithmetic is slow on
    // this part, so no kernel derives its binary32 coefficients in double)
    float fW, fE, fS, fN;        // stencil
    float gW, gE, gS, gN;        // -c * (1/d)
    float finvd, fdconst;
    RedArgs red;
    int *err;            // device error word (bounded waits), nullable
    // overlapping subdomains (Sections 3.4, 4.3): points shared with each
    // neighbour along x / y, and subdomains along x / y (2D; 1D: along x)
    int ox, oy, jx, jy;
    // variable neighbour coefficients (null: constant cW..cN above): planes of
    // rows * ld elements, vcs apart.  binary64: the caller's W, E[, S, N]
    // coefficients, with d_p = dconst + sigma_p (vsig, nullable); binary32:
    // -cW/d, -cE/d[, -cS/d, -cN/d], 1/d, d per point, precomputed
    const void *vc;
    const double *vsig;
    long long vcs;
    // debug builds: the device word of failed index checks (nullable)
    DbgWord *dbg;
    // fused residual with a deferred fold (part_w non-null): this launch
    // writes one partial of ||f - A u_c||^2 per CTA into part_w; the last CTA
    // of the next launch folds them (part_r there) into the control block;
    // parity = launch index mod 2 selects the launch's fold_only flag
    double *part_w;
    const double *part_r;
    int parity;
    // 3D seven-point extension: interior planes, plane pitch (elements) and
    // the bottom (z - 1) / top (z + 1) coefficients with their binary32 copies
    int nz;
    long long ps;
    double cB, cT;
    float fB, fT, gB, gT;
};

// Elements of one grid array of a 2D problem ((ny + 2) rows) and of a 1D one
// (ny independent rows), at the pitch the arguments carry.
__device__ __forceinline__ long long grid_elems2d(const CycArgs &a) { return (long long)(a.ny + 2) * a.ld; }
__device__ __forceinline__ long long grid_elems1d(const CycArgs &a) { return (long long)a.ny * a.ld; }

// Subdomain j of J along one dimension of n interior points, T points each,
// overlapping its neighbours by o points: it spans [start, end] and owns
// [lo, hi].  Starts advance by T - o; with o > 0 the last subdomain is moved
// back to end at n (o = 0: truncated at n).  Each overlap is split at its
// midpoint, the left subdomain keeping the left half (the right one keeps the
// middle point of an odd overlap), so every point has exactly one owner: the
// subdomain in which it lies further from an edge.
struct Span {
    int start, end, lo, hi;
};
__host__ __device__ __forceinline__ int span_start(int j, int J, int n, int T, int o) {
    return (o > 0 && J > 1 && j == J - 1) ? n - T + 1 : 1 + j * (T - o);
}
__host__ __device__ __forceinline__ Span subdomain_span(int j, int J, int n, int T, int o) {
    Span s;
    s.start = span_start(j, J, n, T, o);
    s.end = s.start + T - 1 < n ? s.start + T - 1 : n;
    if (j == 0) {
        s.lo = 1;
    } else {
        const int ps = span_start(j - 1, J, n, T, o);
        const int pe = ps + T - 1 < n ? ps + T - 1 : n;
        s.lo = s.start + (pe - s.start + 1) / 2;
    }
    if (j == J - 1) {
        s.hi = n;
    } else {
        const int ns = span_start(j + 1, J, n, T, o);
        s.hi = ns + (s.end - ns + 1) / 2 - 1;
    }
    return s;
}
// Subdomains along a dimension of n points.
__host__ __device__ __forceinline__ int subdomain_count(int n, int T, int o) {
    if (n <= T) return 1;
    if (o == 0) return (n + T - 1) / T;
    return (n - T + (T - o) - 1) / (T - o) + 1;
}

// ---------------------------------------------------------------------------
// storage <-> compute conversions
// ---------------------------------------------------------------------------
template <typename S, typename T> __device__ __forceinline__ T ld_s(const S *p) { return (T)__ldg(p); }
template <> __device__ __forceinline__ float ld_s<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <typename S, typename T> __device__ __forceinline__ void st_s(S *p, T v) { *p = (S)v; }
template <> __device__ __forceinline__ void st_s<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// Deterministic reductions.  Within a warp: xor butterfly (every lane ends with
// the same value, independent of which CTA performs it).  Across CTAs: the last
// CTA of each group of kGroup CTAs sums the group's partials in a fixed order,
// the last group sums the group results in a fixed order.  The order depends
// only on the grid shape, so results are bitwise reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Stagnation rule of the refinement's inner solves: every stall_window cycles,
// compare ||r_c|| with its value stall_window cycles earlier; a relative change
// of at most stall_rtol means the iterate has reached the fixed point that its
// storage precision allows (bitwise, in practice), so further cycles are wasted.
__device__ __forceinline__ bool stalled(const RedArgs &r, long long c, double res2, volatile double *mark,
                                        volatile long long *mark_c) {
    if (r.stall_window <= 0) return false;
    if (c == 0) {
        *mark = res2;
        *mark_c = 0;
        return false;
    }
    if (c - *mark_c < r.stall_window) return false;
    const double a = sqrt(res2), b = sqrt(*mark);
    *mark = res2;
    *mark_c = c;
    return fabs(a - b) <= r.stall_rtol * a;
}

// Fold ||r_c||^2 of the cycle into the control block (runs on one thread).
__device__ __forceinline__ void finish_cycle(const RedArgs &r, double res2) {
    volatile Ctl *ctl = r.ctl;   // written by earlier launches: bypass L1
    const long long c = ctl->cycle;
    r.hist[c & (kHistCap - 1)] = res2;
    if (c == 0) ctl->res2_0 = res2;
    const double r0 = sqrt(c == 0 ? res2 : ctl->res2_0);
    const double rc = sqrt(res2);
    ctl->res2_last = res2;
    if (!isfinite(rc)) {
        ctl->status = HJ_ERR_DIVERGED;
        ctl->done = (int)c;
    } else if (rc <= r.tol * r0) {
        ctl->done = (int)c;
    } else if (stalled(r, c, res2, &ctl->res2_mark, &ctl->mark_cycle)) {
        ctl->done = (int)c;
    } else if (c + 1 >= r.max_cycles) {
        ctl->status = HJ_ERR_NOT_CONVERGED;
        ctl->done = (int)(c + 1);
    }
    ctl->cycle = c + 1;
}

// Block-level reduction of NV per-thread values followed by the grid-level
// group/final steps.  Must be called by every thread of the CTA.  nwarps =
// blockDim.x*blockDim.y/32 (<= 32).
template <int NV>
__device__ __forceinline__ void reduce_grid(const RedArgs &r, const double (&val)[NV]) {
    __shared__ double s_w[32][NV];
    __shared__ int s_flag;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
    double v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(val[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) s_w[warp][i] = v[i];
    }
    __syncthreads();
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned g = blk / kGroup;
    const unsigned gsize = min((unsigned)kGroup, nblk - g * kGroup);
    const unsigned ngroups = (nblk + kGroup - 1) / kGroup;
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += s_w[w][i];
            r.partials[(size_t)blk * NV + i] = s;
        }
        __threadfence();
        const unsigned t = atomicAdd(&r.gcnt[g], 1u);
        s_flag = (t == gsize - 1);
    }
    __syncthreads();
    if (!s_flag || warp != 0) return;
    // last CTA of group g: sum the group's partials in a fixed order
    __threadfence();
    double gs[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (unsigned b = lane; b < gsize; b += 32) s += __ldcg(&r.partials[(size_t)(g * kGroup + b) * NV + i]);
        gs[i] = warp_sum(s);
    }
    int last = 0;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) r.gpart[(size_t)g * NV + i] = gs[i];
        r.gcnt[g] = 0u;
        __threadfence();
        const unsigned t2 = atomicAdd(r.fcnt, 1u);
        last = (t2 == ngroups - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    double fs[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (unsigned b = lane; b < ngroups; b += 32) s += __ldcg(&r.gpart[(size_t)b * NV + i]);
        fs[i] = warp_sum(s);
    }
    if (lane == 0) {
        *r.fcnt = 0u;
        if (r.mode == RED_CYCLE) {
            finish_cycle(r, fs[0] * r.scale);
        } else {
#pragma unroll
            for (int i = 0; i < NV; ++i) r.out[i] = fs[i];
        }
        __threadfence();
    }
}

// Deferred fold: one warp sums n per-CTA partials written by the previous
// launch (fixed order: lane-strided, four interleaved accumulators, then the
// butterfly) and folds ||r||^2 into the control block.  The kernel boundary
// orders those writes before these loads; __ldcg skips stale L1 lines.
__device__ __forceinline__ void fold_partials(const RedArgs &r, const double *part, int n) {
    const int lane = threadIdx.x & 31;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int b = lane;
    for (; b + 96 < n; b += 128) {
        const double x0 = __ldcg(part + b), x1 = __ldcg(part + b + 32);
        const double x2 = __ldcg(part + b + 64), x3 = __ldcg(part + b + 96);
        s0 += x0;
        s1 += x1;
        s2 += x2;
        s3 += x3;
    }
    for (; b < n; b += 32) s0 += __ldcg(part + b);
    const double s = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) finish_cycle(r, s * r.scale);
}

// Deferred fold, run by one warp of the last CTA of a launch: fold the
// previous launch's partials (nparts of them: the residual of the iterate that
// launch staged), then decide whether the next launch only folds (its iterate
// would lie beyond max_cycles).  The launch counter and the flags are touched
// by this warp only, one launch after another.
__device__ __forceinline__ void deferred_fold_parts(const RedArgs &red, const double *part_r, int nparts,
                                                    int parity) {
    volatile Ctl *ctl = red.ctl;
    const long long l = ctl->launch;
    if (l >= 1) fold_partials(red, part_r, nparts);
    if ((threadIdx.x & 31) == 0) {
        ctl->fold_only[parity ^ 1] = (l + 1 >= red.max_cycles) ? 1 : 0;
        ctl->launch = l + 1;
    }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Per-thread residual contribution -> grid reduction.  binary32 contributions
// are summed within the warp in binary32 first (one conversion per warp).
template <typename A>
__device__ __forceinline__ void reduce_grid_acc(const RedArgs &r, A acc) {
    double v;
    if constexpr (std::is_same<A, float>::value) {
        const float w = warp_sum_f(acc);
        v = ((threadIdx.x + threadIdx.y * blockDim.x) & 31) == 0 ? (double)w : 0.0;
    } else {
        v = acc;
    }
    const double vals[1] = {v};
    reduce_grid<1>(r, vals);
}

// Launch-side description of one compiled cycle kernel.
typedef void (*CycKernel)(CycArgs);

struct PpcArgs;
typedef void (*PpcKernel)(PpcArgs);

// TMA-pipelined 2D cycle kernel (hj_tma.cuh).
struct PpcKernelInfo {
    int tx, ty, threads, stages;
    int smem[2];        // dynamic shared memory bytes [sig]
    int bwu, bwf;       // box widths (elements) of the iterate / RHS boxes
    PpcKernel fn[2][2]; // [sig][res]
};

struct TileKernelInfo {
    int dim;            // 1 or 2
    int tx, ty;         // tile interior shape (1D: ty = 1)
    int threads;        // threads per CTA
    int tiles_per_cta;  // 1D packs several tiles per CTA
    CycKernel fn[2][2]; // [sig][res]
    CycKernel ovl[2][2];// [sig][res] overlapping subdomains (null for classic kernels)
};

// Variable-coefficient kernels: [dim - 1][res], one thread per point, dynamic
// shared memory 2 * (tile_x + 2) * (tile_y + 2) elements of the compute type.
struct VcKernelInfo {
    CycKernel fn[2][2];
};
const VcKernelInfo *vc_kernels_f64();
const VcKernelInfo *vc_kernels_f32();

// 3D seven-point kernels: one warp per TX x TY x TZ subdomain, NW subdomains
// per CTA of 32 * NW threads, grid ceil(subdomains / NW) CTAs; fn[res].
struct Tile3Info {
    int tx, ty, tz, threads, nw;
    CycKernel fn[2];
    CycKernel pf[2];   // prefetching persistent variant: grid <= resident CTAs, dynamic smem pf_smem
    int pf_smem;
    PpcKernel ppc[2];  // TMA-pipelined variant (binary32; null otherwise): one warp per CTA, dynamic smem ppc_smem
    int ppc_smem;
    int ppc_cps;       // its resident CTAs per SM unless the caller sets ctas_per_sm (0: as many as fit)
};
const Tile3Info *tiles3d_f64(int *n);
const Tile3Info *tiles3d_f32(int *n);
// classic seven-point sweep: block (32, 8), grid (ceil(nx/32), ceil(ny/8), nz); fn[res]
CycKernel classic3d_kernel_of(int fam, int res);
cudaError_t launch_residual3d(int user_f64, const void *f, const void *u, long long ld, long long ps, int nx,
                              int ny, int nz, double cW, double cE, double cS, double cN, double cB, double cT,
                              double dconst, int with_fnorm, RedArgs red, cudaStream_t s);
int aux_max_blocks3(int nx, int ny, int nz);

// Kernel registries (one per storage/compute combination).
enum KernelFamily { FAM_F64 = 0, FAM_F32 = 1, FAM_BF16 = 2 };
const TileKernelInfo *tile_kernels_f64(int *n);
const TileKernelInfo *tile_kernels_f32(int *n);
const TileKernelInfo *tile_kernels_bf16(int *n);
const TileKernelInfo *classic_kernels_f64(int *n);
const TileKernelInfo *classic_kernels_f32(int *n);
const TileKernelInfo *classic_kernels_bf16(int *n);
const PpcKernelInfo *ppc_kernels_f64(int *n);
const PpcKernelInfo *ppc_kernels_f32(int *n);
const PpcKernelInfo *ppc_kernels_bf16(int *n);

// Grid-wide helper kernels (hj_aux.cu).
cudaError_t launch_make_dinv_box(const double *sigma, double dconst, long long ld, long long ld2, int row0, int rows,
                                 int col0, int cols, int family, void *dinv, cudaStream_t s);
// coef (nullable): per-point W, E[, S, N] coefficient planes cps elements apart
cudaError_t launch_residual_ex(int dim, int user_f64, const void *f, const void *u, const double *sigma,
                               long long ld, long long ld2, int nx, int ny, double cW, double cE, double cS,
                               double cN, double dconst, int with_fnorm, float *r32, RedArgs red, cudaStream_t s,
                               const double *coef = nullptr, long long cps = 0);
// binary32 factors of the variable-coefficient kernels (vc_kernel)
cudaError_t launch_vc_prep(int dim, const double *coef, const double *sigma, double dconst, long long ld,
                           long long ps, int nx, int ny, float *out, cudaStream_t s);
cudaError_t launch_update_residual_ex(int dim, const double *f, const double *uin, const void *d, int d_bf16,
                                      double *uout, const double *sigma, float *r32, long long ld, long long ld2,
                                      int nx, int ny, double cW, double cE, double cS, double cN, double dconst,
                                      RedArgs red, cudaStream_t s);
cudaError_t launch_grad_sigma_ex(int dim, int user_f64, const void *lam, const void *u, double *dsig, long long ld,
                                 int nx, int ny, int accumulate, cudaStream_t s);
int aux_max_blocks(int dim, int nx, int ny);
int aux_sm_count();

}  // namespace hj
