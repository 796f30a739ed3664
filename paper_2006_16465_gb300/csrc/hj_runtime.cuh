// hj_runtime.cuh -- host runtime internals shared by the C-ABI translation
// units: the handle, error reporting, and the engines the solve calls use.
#pragma once

#include <cuda.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "hj_internal.cuh"
#include "hj_persist.cuh"

namespace hj {

int seterr(int code, const char *fmt, ...);

// Device allocations of the library (handle workspaces): plain cudaMalloc /
// cudaFree in release builds; debug builds add guard bands around each one
// (hj_debug.cu, checked by hj_debug_check).
cudaError_t dmalloc(void **p, size_t bytes);
cudaError_t dfree(void *p);
// Device word of the index checks of debug builds (nullptr in release builds).
DbgWord *debug_word();
const char *last_error_text();

#define CKR(call)                                                                                           \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return ::hj::seterr(HJ_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                                __LINE__);                                                                  \
    } while (0)

#define CKS(expr)                     \
    do {                              \
        int st_ = (expr);             \
        if (st_ != HJ_OK) return st_; \
    } while (0)

// A captured graph of M alternating launches, keyed by the kernel, the launch
// shape and the bytes of both argument blocks.
struct GraphEntry {
    const void *fn;
    dim3 grid, block;
    int smem;
    std::vector<unsigned char> key;
    int M;
    cudaGraphExec_t exec;
    unsigned long long stamp;
};

const TileKernelInfo *family_tiles(int fam, int *n);
const PersistKernelInfo *family_persist(int fam, int *n);
const PersistKernelInfo *find_persist(int fam, int dim, int tx, int ty, int threads = 0);
const PersistKernelInfo *persist_kernels_f64(int *n);
const PersistKernelInfo *persist_kernels_f32(int *n);
const PersistKernelInfo *persist_kernels_bf16(int *n);
const PersistClassicInfo *persist_classic_f64();
const PersistClassicInfo *persist_classic_f32();
const PersistClassicInfo *persist_classic_bf16();

// One multigrid level: sizes, pitch, the two iterate buffers and the
// right-hand side, and the rediscretised stencil (sigma_const is shared).
struct MgLevel {
    int nx = 0, ny = 0;
    long long ld = 0;
    void *a = nullptr, *b = nullptr, *f = nullptr;
    double cW = 0, cE = 0, cS = 0, cN = 0, cD = 0;
};

}  // namespace hj

struct hj_handle {
    hj_desc d;
    hj_params p;
    int dev = 0, nsm = 0;
    int rows = 0;
    size_t esz = 0, grid_elems = 0, grid_bytes = 0;
    int fam_outer = hj::FAM_F64, fam_inner = hj::FAM_F32;
    bool ir = false;
    const hj::TileKernelInfo *k_outer = nullptr, *k_inner = nullptr, *k_classic = nullptr, *k_classic_inner = nullptr;
    const hj::PpcKernelInfo *p_outer = nullptr, *p_inner = nullptr;   // TMA-pipelined variants (2D)
    const hj::Tile3Info *k3 = nullptr;                                 // 3D seven-point kernel (hierarchical)
    long long ld_in = 0;          // row pitch of the refinement's binary32 / bfloat16 arrays
    void *ubuf = nullptr;
    void *ubuf2 = nullptr;        // third iterate buffer (pipelined kernel, deferred residual fold)
    float *vcf = nullptr;         // binary32 factors of the variable-coefficient kernels
    void *dinv_outer = nullptr;   // per-point 1/d in the outer compute type (sigma given)
    float *dinv32 = nullptr;      // per-point 1/d in binary32 (refinement, sigma given)
    float *r32 = nullptr;         // refinement: binary32 residual (inner RHS)
    void *dA = nullptr, *dB = nullptr;  // refinement: correction buffers
    void *dC = nullptr;                 // refinement: third correction buffer (as ubuf2)
    void *hf = nullptr, *hu = nullptr;  // staging for host-pointer solves
    double *partials = nullptr, *gpart = nullptr, *hist = nullptr, *rstore = nullptr;
    unsigned *gcnt = nullptr, *fcnt = nullptr;
    hj::Ctl *ctl = nullptr;
    hj::Ctl *h_ctl = nullptr, *h_ctl_init = nullptr;   // h_ctl: two slots (pipelined checks)
    double *h_hist = nullptr, *h_rstore = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    std::vector<hj::GraphEntry> graphs;
    unsigned long long stamp = 0;
    size_t max_blocks = 0, max_groups = 0;
    // persistent engine scratch (device) and its pinned staging copy
    void *pscratch = nullptr;
    unsigned char *h_pstage = nullptr;
    size_t pscratch_bytes = 0;
    // batched solves: per-problem arrays and norms
    void *barena = nullptr;
    size_t barena_bytes = 0;
    double *rs = nullptr, *h_rs = nullptr;
    size_t nrs = 0;
    // batched solves: device metadata of the batch (per-problem buffers and
    // refinement state, residual shares, the per-cycle log) and its pinned copy
    void *bmeta = nullptr;
    unsigned char *h_bmeta = nullptr;
    size_t bmeta_bytes = 0;
    // multigrid (HJ_METHOD_MG): levels, their buffers and the V-cycle graph
    std::vector<hj::MgLevel> mg;
    void *mg_arena = nullptr;
    cudaGraphExec_t mg_exec = nullptr;         // V-cycle + level-0 residual (converging runs)
    cudaGraphExec_t mg_exec_fixed = nullptr;   // V-cycle alone (fixed-cycle runs)
};

namespace hj {
int mg_levels_of(int nx, int ny);
int mg_setup(hj_handle *h, int levels);
int solve_mg(hj_handle *h, const void *f, void *u, cudaStream_t s, hj_stats *st);
}  // namespace hj

namespace hj {

// 2D tiled tensor map over a grid array: dims (cols, rows), row stride
// ld*esz bytes, box (bw, bh), zero fill out of bounds.  False if the encoder
// is unavailable or rejects the arguments (alignment, pitch).
bool make_tmap(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int esz, long long ld, int cols, int rows,
               int bw, int bh);
// Element type of a family's storage (iterate) or compute (RHS, 1/d) arrays.
CUtensorMapDataType tmap_type(int fam, bool storage);

// Grow the grid-reduction workspace so that a launch of `blocks` CTAs fits.
int ensure_reduction(hj_handle *h, size_t blocks);
// Grow the persistent-engine scratch (items, states, partials, barrier words).
int ensure_scratch(hj_handle *h, size_t bytes);

// Persistent engine: run cycles of several problems in one cooperative launch.
struct PersistProblem {
    CycArgs a;        // f, uin (= u_0 buffer), uout (= other buffer), dinv, geometry, k, coefficients,
                      // red.tol, red.max_cycles, red.scale (red.hist for a single problem)
    int blocks_x;     // CTAs along x (2D tiles, or 1D groups of tiles)
    int blocks;       // CTAs in total
};
// classic: run the grid-sync classic kernel (one problem, blocks of points as items)
// fam >= 0 (the kernels' family) lets 2D problems stage by TMA (pipeline != 0).
int run_persistent(hj_handle *h, const PersistKernelInfo *ki, bool sig, std::vector<PersistProblem> &probs,
                   cudaStream_t s, std::vector<ProbState> *out, PersistKernel classic = nullptr, int fam = -1);
int persist_capacity(hj_handle *h, const PersistKernelInfo *ki, bool sig, int *ctas);

// Batched tuning (hj_autotune.cu): tile variant with a persistent kernel and
// k per size class; cls[p] in [0, ncls).
int autotune_batched(const hj_desc *descs, int nprob, const std::vector<int> &cls, int ncls, hj_params *par,
                     std::vector<int> *kcls);

}  // namespace hj
