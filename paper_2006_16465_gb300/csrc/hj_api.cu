// hj_api.cu -- host runtime and C ABI (include/hj.h).
//
// The cycle loop: a CUDA graph of M launches alternates the two iterate
// buffers (u_c -> u_{c+1} -> u_c ...).  Each launch folds ||f - A u_c||^2 into
// the device control block; once an iterate meets the tolerance, the control
// block records its index and later launches return immediately, so the host
// only synchronises once per graph (M cycles) and the returned iterate is the
// exact first one that met the tolerance (Sections 3.5 and 4.2 stop on the L2
// residual reduced by a factor).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "hj_runtime.cuh"
#include "hj_tma.cuh"

using namespace hj;

namespace hj {

thread_local char g_err[512] = "";

int seterr(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

const char *last_error_text() { return g_err; }

}  // namespace hj

namespace hj {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D tiled map over a grid array: dims (cols, rows), row stride ld*esz bytes,
// box (bw, bh); out-of-bounds elements read as zero.
bool make_tmap(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int esz, long long ld, int cols, int rows,
               int bw, int bh) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[2] = {1, 1};
    memset(m, 0, sizeof(*m));
    return enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D tiled map over a grid array: dims (cols, rows, planes), row stride
// ld*esz and plane stride ps*esz bytes, box (bw, bh, bd); out-of-bounds
// elements read as zero.
bool make_tmap3(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int esz, long long ld, long long ps,
                int cols, int rows, int planes, int bw, int bh, int bd) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * esz), (cuuint64_t)(ps * esz)};
    cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bd};
    cuuint32_t estr[3] = {1, 1, 1};
    memset(m, 0, sizeof(*m));
    return enc(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

CUtensorMapDataType tmap_type(int fam, bool storage) {
    if (fam == FAM_F64) return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (fam == FAM_BF16 && storage) return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
}

}  // namespace hj

namespace {

}  // namespace

const TileKernelInfo *hj::family_tiles(int fam, int *n) {
    switch (fam) {
    case FAM_F64: return tile_kernels_f64(n);
    case FAM_F32: return tile_kernels_f32(n);
    default: return tile_kernels_bf16(n);
    }
}
const PersistKernelInfo *hj::family_persist(int fam, int *n) {
    switch (fam) {
    case FAM_F64: return persist_kernels_f64(n);
    case FAM_F32: return persist_kernels_f32(n);
    default: return persist_kernels_bf16(n);
    }
}
const PersistKernelInfo *hj::find_persist(int fam, int dim, int tx, int ty, int threads) {
    int n = 0;
    const PersistKernelInfo *k = family_persist(fam, &n);
    for (int i = 0; i < n; ++i)
        if (k[i].dim == dim && k[i].tx == tx && (dim == 1 || k[i].ty == ty) &&
            (!threads || k[i].threads / k[i].tiles_per_cta == threads))
            return &k[i];
    return nullptr;
}

namespace {
const TileKernelInfo *family_classic(int fam, int dim) {
    int n = 0;
    const TileKernelInfo *k = fam == FAM_F64 ? classic_kernels_f64(&n)
                              : fam == FAM_F32 ? classic_kernels_f32(&n)
                                               : classic_kernels_bf16(&n);
    for (int i = 0; i < n; ++i)
        if (k[i].dim == dim) return &k[i];
    return nullptr;
}
const PpcKernelInfo *family_ppc(int fam, int *n) {
    switch (fam) {
    case FAM_F64: return ppc_kernels_f64(n);
    case FAM_F32: return ppc_kernels_f32(n);
    default: return ppc_kernels_bf16(n);
    }
}
// threads / stages 0 = the first (default) entry for the shape
const PpcKernelInfo *find_ppc(int fam, int tx, int ty, int threads, int stages) {
    int n = 0;
    const PpcKernelInfo *k = family_ppc(fam, &n);
    for (int i = 0; i < n; ++i)
        if (k[i].tx == tx && k[i].ty == ty && (!threads || k[i].threads == threads) &&
            (!stages || k[i].stages == stages))
            return &k[i];
    return nullptr;
}



// threads: threads per subdomain (a CTA of a 1D kernel may hold several
// subdomains); 0 = the first (default) entry for the shape
const TileKernelInfo *find_tile(int fam, int dim, int tx, int ty, int threads = 0) {
    int n = 0;
    const TileKernelInfo *k = family_tiles(fam, &n);
    for (int i = 0; i < n; ++i)
        if (k[i].dim == dim && k[i].tx == tx && (dim == 1 || k[i].ty == ty) &&
            (!threads || k[i].threads / k[i].tiles_per_cta == threads))
            return &k[i];
    return nullptr;
}



double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace



namespace {

// ---------------------------------------------------------------------------
// kernel arguments and launch geometry
// ---------------------------------------------------------------------------
CycArgs base_args(const hj_handle *h, bool transpose) {
    CycArgs a;
    memset(&a, 0, sizeof(a));
    a.ld = h->d.ld;
    a.nx = h->d.nx;
    a.ny = h->d.ny;
    a.k = h->p.k;
    a.cW = transpose ? h->d.cE : h->d.cW;
    a.cE = transpose ? h->d.cW : h->d.cE;
    a.cS = h->d.dim >= 2 ? (transpose ? h->d.cN : h->d.cS) : 0.0;
    a.cN = h->d.dim >= 2 ? (transpose ? h->d.cS : h->d.cN) : 0.0;
    a.dconst = h->d.cD + h->d.sigma_const;
    a.invd = 1.0 / a.dconst;
    a.fW = (float)a.cW; a.fE = (float)a.cE; a.fS = (float)a.cS; a.fN = (float)a.cN;
    a.gW = (float)(-a.cW * a.invd); a.gE = (float)(-a.cE * a.invd);
    a.gS = (float)(-a.cS * a.invd); a.gN = (float)(-a.cN * a.invd);
    a.finvd = (float)a.invd;
    a.fdconst = (float)a.dconst;
    a.dbg = debug_word();
    a.ox = h->p.overlap_x;
    a.oy = h->d.dim == 2 ? h->p.overlap_y : 0;
    a.jx = subdomain_count(h->d.nx, h->p.tile_x, a.ox);
    a.jy = h->d.dim == 2 ? subdomain_count(h->d.ny, h->p.tile_y, a.oy) : h->d.ny;
    if (h->d.coef) {
        a.vc = h->fam_outer == FAM_F64 ? (const void *)h->d.coef : (const void *)h->vcf;
        a.vsig = h->d.sigma;
        a.vcs = (long long)h->rows * h->d.ld;
    }
    if (h->d.dim == 3) {
        a.nz = h->d.nz;
        a.ps = (long long)(h->d.ny + 2) * h->d.ld;
        a.cB = transpose ? h->d.cT : h->d.cB;
        a.cT = transpose ? h->d.cB : h->d.cT;
        a.fB = (float)a.cB; a.fT = (float)a.cT;
        a.gB = (float)(-a.cB * a.invd); a.gT = (float)(-a.cT * a.invd);
    }
    return a;
}

bool overlapped(const hj_handle *h) { return h->p.overlap_x > 0 || (h->d.dim == 2 && h->p.overlap_y > 0); }

RedArgs red_args(const hj_handle *h, int mode, double tol, long long max_cycles) {
    RedArgs r;
    memset(&r, 0, sizeof(r));
    r.partials = h->partials;
    r.gpart = h->gpart;
    r.gcnt = h->gcnt;
    r.fcnt = h->fcnt;
    r.hist = h->hist;
    r.out = h->rstore;
    r.ctl = h->ctl;
    r.tol = tol;
    r.max_cycles = max_cycles;
    r.mode = mode;
    r.scale = 1.0;
    return r;
}

void geometry(const hj_handle *h, const TileKernelInfo *ki, bool classic, dim3 *grid, dim3 *block) {
    const int nx = h->d.nx, ny = h->d.ny;
    if (classic) {
        // grid-stride kernels over blocks of points (2D: classic2d_blocks; an
        // upper bound for every storage type) or 256 (1D) points, bounded to 8
        // CTAs per SM so the residual is reduced once per CTA
        const long long nb = h->d.dim == 2 ? classic2d_blocks(nx, ny, 8) : (long long)((nx + 255) / 256) * ny;
        *grid = dim3((unsigned)std::min<long long>(nb, 8LL * h->nsm));
        *block = h->d.dim == 2 ? dim3(32, 8) : dim3(256);
        return;
    }
    const bool ovl = overlapped(h);
    if (h->d.dim == 2) {
        *grid = ovl ? dim3(subdomain_count(nx, ki->tx, h->p.overlap_x), subdomain_count(ny, ki->ty, h->p.overlap_y))
                    : dim3((nx + ki->tx - 1) / ki->tx, (ny + ki->ty - 1) / ki->ty);
    } else {
        const int tiles = ovl ? subdomain_count(nx, ki->tx, h->p.overlap_x) : (nx + ki->tx - 1) / ki->tx;
        *grid = dim3((tiles + ki->tiles_per_cta - 1) / ki->tiles_per_cta, ny);
    }
    *block = dim3(ki->threads);
}

// Graph of M launches of fn; launch i takes args[i % period].
template <typename Args>
int get_graph(hj_handle *h, void (*fn)(Args), dim3 grid, dim3 block, int smem, const Args *args, int period,
              int M, cudaGraphExec_t *out) {
    std::vector<unsigned char> key(period * sizeof(Args));
    for (int j = 0; j < period; ++j) memcpy(key.data() + j * sizeof(Args), &args[j], sizeof(Args));
    for (auto &g : h->graphs) {
        if (g.fn == (const void *)fn && g.M == M && g.smem == smem && g.grid.x == grid.x && g.grid.y == grid.y &&
            g.block.x == block.x && g.block.y == block.y && g.key == key) {
            g.stamp = ++h->stamp;
            *out = g.exec;
            return HJ_OK;
        }
    }
    if (h->graphs.size() >= 16) {
        auto it = std::min_element(h->graphs.begin(), h->graphs.end(),
                                   [](const GraphEntry &x, const GraphEntry &y) { return x.stamp < y.stamp; });
        cudaGraphExecDestroy(it->exec);
        h->graphs.erase(it);
    }
    cudaGraph_t graph;
    CKR(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < M; ++i) fn<<<grid, block, smem, h->cap>>>(args[i % period]);
    cudaError_t le = cudaGetLastError();
    cudaError_t ee = cudaStreamEndCapture(h->cap, &graph);
    if (le != cudaSuccess) return seterr(HJ_ERR_CUDA, "kernel launch during capture: %s", cudaGetErrorString(le));
    if (ee != cudaSuccess) return seterr(HJ_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
    cudaGraphExec_t exec;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return seterr(HJ_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
    GraphEntry e;
    e.fn = (const void *)fn;
    e.grid = grid;
    e.block = block;
    e.smem = smem;
    e.key = std::move(key);
    e.M = M;
    e.exec = exec;
    e.stamp = ++h->stamp;
    h->graphs.push_back(std::move(e));
    *out = exec;
    return HJ_OK;
}

// Launch plan for one iteration kernel: either the one-CTA-per-tile kernel
// (CycArgs) or the TMA-pipelined kernel (PpcArgs) with its two argument blocks.
// Converging runs of the pipelined kernel rotate three iterate buffers and
// two partial slots (period 6): launch c reads B[c % 3], writes B[(c+1) % 3]
// and its residual partials to slot c % 2.  Its residual is folded by launch
// c + 1 while that launch writes B[(c+2) % 3], so the iterate u_c whose
// residual met the tolerance is still intact when the fold decides.
constexpr int kPpcPeriod = 6;

struct Plan {
    bool ppc = false;
    bool deferred = false;   // fused residual with the deferred fold (three iterate buffers)
    int period = 2;          // argument blocks launches cycle through
    CycKernel fn = nullptr;
    PpcKernel pfn = nullptr;
    dim3 grid, block;
    int smem = 0;
    CycArgs a[kPpcPeriod];
    PpcArgs p[kPpcPeriod];
};

// Largest grid of the one-CTA-per-subdomain kernels that folds its residual
// in the next launch (one warp sums one partial per CTA; larger grids keep the
// grid reduction at the launch's end).
constexpr long long kDeferMaxBlocks = 4096;

// 3D: whether the prefetching (persistent-warp, cp.async) kernel runs.  Only
// on request (pipeline = 1): measured at 512^3 binary32 it is slower than the
// one-warp-per-subdomain kernel (755 against 625 us a cycle at k = 1).
bool use_pf3(const hj_handle *h) {
    return h->k3 && h->d.dim == 3 && h->p.method == HJ_METHOD_HIER && h->p.pipeline == 1;
}

// Id of the calling thread's current CUDA context (cuCtxGetId through the
// runtime's driver entry points), or 0 if it cannot be had.  A context made
// after cudaDeviceReset gets a new id, so settings recorded for the old one
// are not taken for it.
unsigned long long context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_cuCtxGetCurrent_v4000)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id + 1;
}

// Raise a kernel's dynamic shared-memory limit (an attribute of the function
// in the current context) to at least `bytes`, never lowering it: a kernel
// whose shared memory depends on the subdomain shape may serve several
// handles, and graphs built earlier keep launching with their own sizes.
// Recorded per (context, device, function); without a context id it is set
// every time.
cudaError_t ensure_dyn_smem(int dev, const void *fn, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<unsigned long long, const void *>, std::pair<int, int>>> set;
    const unsigned long long ctx = context_id();
    if (ctx == 0) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    std::lock_guard<std::mutex> lk(mu);
    for (auto &e : set)
        if (e.first.first == ctx && e.first.second == fn && e.second.first == dev) {
            if (bytes <= e.second.second) return cudaSuccess;
            const cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (r == cudaSuccess) e.second.second = bytes;
            return r;
        }
    const cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (r == cudaSuccess) set.push_back({{ctx, fn}, {dev, bytes}});
    return r;
}

// 3D: whether the TMA-pipelined kernel runs the hierarchical cycles (binary32,
// automatic pipeline choice, at least 8 subdomains per SM, as in 2D).
bool want_ppc3(const hj_handle *h, bool classic) {
    if (classic || !h->k3 || h->d.dim != 3 || h->p.method != HJ_METHOD_HIER || !h->k3->ppc[0]) return false;
    if (h->p.pipeline != -1) return false;
    const Tile3Info *t3 = h->k3;
    const long long nsub = (long long)((h->d.nx + t3->tx - 1) / t3->tx) * ((h->d.ny + t3->ty - 1) / t3->ty) *
                           ((h->d.nz + t3->tz - 1) / t3->tz);
    return nsub >= 8LL * h->nsm;
}

// Whether the TMA-pipelined kernel runs this plan's cycles.
bool want_ppc(const hj_handle *h, const PpcKernelInfo *pi, bool classic) {
    if (classic || !pi || h->d.dim != 2 || overlapped(h) || h->d.coef) return false;
    if (h->p.pipeline == 1) return true;
    if (h->p.pipeline != -1) return false;
    const long long ntiles = (long long)((h->d.nx + pi->tx - 1) / pi->tx) * ((h->d.ny + pi->ty - 1) / pi->ty);
    return ntiles >= 8LL * h->nsm;
}

// Whether a converging run of the one-CTA-per-subdomain 2D kernels folds its
// residual in the next launch (as the pipelined kernel always does): 2D
// hierarchical cycles with constant coefficients on grids of at most
// kDeferMaxBlocks subdomains.
bool defer_hier(const hj_handle *h, const TileKernelInfo *ki, bool classic) {
    if (classic || !ki || h->d.dim != 2 || h->d.coef) return false;
    dim3 g, b;
    geometry(h, ki, false, &g, &b);
    return (long long)g.x * g.y <= kDeferMaxBlocks;
}

// Whether a converging run of this plan needs the third iterate buffer.
bool deferred_run(const hj_handle *h, const TileKernelInfo *ki, const PpcKernelInfo *pi, bool classic) {
    return want_ppc(h, pi, classic) || defer_hier(h, ki, classic) || want_ppc3(h, classic);
}


// b2: third iterate buffer (same ghost ring as b0), required when the
// pipelined kernel runs with the fused residual.
int make_plan(hj_handle *h, const TileKernelInfo *ki, const PpcKernelInfo *pi, int fam, bool classic, bool sig,
              bool res, const CycArgs &base, void *b0, void *b1, void *b2, Plan *pl) {
    pl->a[0] = base;
    pl->a[1] = base;
    pl->a[0].uin = b0; pl->a[0].uout = b1;
    pl->a[1].uin = b1; pl->a[1].uout = b0;
    pl->period = 2;
    pl->deferred = false;
    const int nx = h->d.nx, ny = h->d.ny;
    if (h->d.dim == 3) {
        // seven-point extension: warp-per-subdomain register kernel, or the
        // classic thread-per-point sweep
        if (want_ppc3(h, classic)) {
            // TMA-pipelined: one warp per CTA walks subdomains, the next one's
            // boxes copied in while the current one sweeps; residual folded by
            // the next launch over three rotating iterate buffers
            if (res && !b2) return seterr(HJ_ERR_CUDA, "internal: pipelined residual runs need a third iterate buffer");
            const Tile3Info *t3 = h->k3;
            PpcKernel fn = t3->ppc[res];
            const int smem = t3->ppc_smem;
            CKR(ensure_dyn_smem(h->dev, (const void *)fn, smem));
            int occ = 0;
            CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32, smem));
            if (occ < 1) return seterr(HJ_ERR_UNSUPPORTED, "3D pipelined kernel does not fit on an SM");
            if (h->p.ctas_per_sm > 0) occ = std::min(occ, h->p.ctas_per_sm);
            else if (t3->ppc_cps > 0) occ = std::min(occ, t3->ppc_cps);
            const int tiles_x = (nx + t3->tx - 1) / t3->tx, tiles_y = (ny + t3->ty - 1) / t3->ty;
            const int ntiles = tiles_x * tiles_y * ((h->d.nz + t3->tz - 1) / t3->tz);
            const int grid = std::min(ntiles, occ * h->nsm);
            const int bw = (t3->tx + 2 + 3) / 4 * 4;   // box width: the kernel's BX
            void *bufs[3] = {b0, b1, b2};
            pl->deferred = res;
            pl->period = res ? kPpcPeriod : 2;
            if (res) CKS(ensure_reduction(h, (size_t)grid));
            for (int j = 0; j < pl->period; ++j) {
                PpcArgs &P = pl->p[j];
                memset(&P, 0, sizeof(P));
                P.a = base;
                P.a.uin = res ? bufs[j % 3] : bufs[j & 1];
                P.a.uout = res ? bufs[(j + 1) % 3] : bufs[(j + 1) & 1];
                P.tiles_x = tiles_x;
                P.tiles_y = tiles_y;
                P.ntiles = ntiles;
                P.spin_limit = 1LL << 26;
                P.parity = j & 1;
                P.part_w = h->partials + (size_t)(j & 1) * grid;
                P.part_r = h->partials + (size_t)((j + 1) & 1) * grid;
                const long long ld = base.ld, ps = base.ps;
                if (!make_tmap3(&P.mu, P.a.uin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ld, ps, nx + 2, ny + 2, h->d.nz + 2,
                                bw, t3->ty + 2, t3->tz + 2) ||
                    !make_tmap3(&P.mf, P.a.f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ld, ps, nx + 2, ny + 2, h->d.nz + 2,
                                bw, t3->ty, t3->tz))
                    return seterr(HJ_ERR_CUDA, "cuTensorMapEncodeTiled failed (3D map: pointer alignment or pitch)");
            }
            pl->ppc = true;
            pl->pfn = fn;
            pl->smem = smem;
            pl->grid = dim3(grid);
            pl->block = dim3(32);
            return HJ_OK;
        }
        if (classic) {
            pl->fn = classic3d_kernel_of(fam, res);
            pl->grid = dim3((nx + 31) / 32, (ny + 7) / 8, h->d.nz);
            pl->block = dim3(32, 8);
        } else {
            const Tile3Info *t3 = h->k3;
            const long long nsub = (long long)((nx + t3->tx - 1) / t3->tx) * ((ny + t3->ty - 1) / t3->ty) *
                                   ((h->d.nz + t3->tz - 1) / t3->tz);
            const long long nblk = (nsub + t3->nw - 1) / t3->nw;
            pl->block = dim3(t3->threads);
            pl->smem = 0;
            if (use_pf3(h)) {
                // persistent warps: at most the resident CTAs, each walking subdomains
                pl->fn = t3->pf[res];
                pl->smem = t3->pf_smem;
                if (pl->smem > 48 * 1024)
                    CKR(cudaFuncSetAttribute(pl->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem));
                int occ = 0;
                CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pl->fn, t3->threads, pl->smem));
                if (occ < 1) return seterr(HJ_ERR_UNSUPPORTED, "3D prefetching kernel does not fit on an SM");
                pl->grid = dim3((unsigned)std::min<long long>(nblk, (long long)occ * h->nsm));
            } else {
                pl->fn = t3->fn[res];
                pl->grid = dim3((unsigned)nblk);
            }
        }
        if (classic) pl->smem = 0;
        pl->ppc = false;
        return HJ_OK;
    }
    if (h->d.coef) {
        // variable coefficients: one thread per point; classic Jacobi is the
        // same kernel with one subiteration (a k = 1 cycle is a classic sweep)
        const VcKernelInfo *vk = fam == FAM_F64 ? vc_kernels_f64() : vc_kernels_f32();
        const int tx = h->p.tile_x, ty = h->d.dim == 2 ? h->p.tile_y : 1;
        pl->fn = vk->fn[h->d.dim - 1][res];
        pl->grid = h->d.dim == 2 ? dim3((nx + tx - 1) / tx, (ny + ty - 1) / ty) : dim3((nx + tx - 1) / tx, ny);
        pl->block = h->d.dim == 2 ? dim3(tx, ty) : dim3(tx);
        pl->smem = 2 * (tx + 2) * (h->d.dim == 2 ? ty + 2 : 1) * (fam == FAM_F64 ? 8 : 4);
        if (classic) pl->a[0].k = pl->a[1].k = 1;
        pl->ppc = false;
        return HJ_OK;
    }
    if (!want_ppc(h, pi, classic)) {
        geometry(h, ki, classic, &pl->grid, &pl->block);
        pl->fn = (!classic && overlapped(h)) ? ki->ovl[sig][res] : ki->fn[sig][res];
        if (res && defer_hier(h, ki, classic)) {
            // deferred fold: launch c reads B[c % 3], writes B[(c+1) % 3] and
            // its per-CTA partials to slot c % 2, folded by launch c + 1
            if (!b2) return seterr(HJ_ERR_CUDA, "internal: deferred residual runs need a third iterate buffer");
            const long long nb = (long long)pl->grid.x * pl->grid.y;
            CKS(ensure_reduction(h, (size_t)nb));
            void *bufs[3] = {b0, b1, b2};
            pl->deferred = true;
            pl->period = kPpcPeriod;
            for (int j = 0; j < kPpcPeriod; ++j) {
                CycArgs &A = pl->a[j];
                A = base;
                A.uin = bufs[j % 3];
                A.uout = bufs[(j + 1) % 3];
                A.part_w = h->partials + (size_t)(j & 1) * nb;
                A.part_r = h->partials + (size_t)((j + 1) & 1) * nb;
                A.parity = j & 1;
            }
        }
        if (classic && h->d.dim == 2) {
            // one wave of resident CTAs: every CTA of the grid-stride sweep gets
            // the same share of blocks, so a partial last wave would idle SMs
            int occ = 0;
            CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pl->fn, pl->block.x * pl->block.y, 0));
            pl->grid.x = (unsigned)std::max(1, std::min<int>((int)pl->grid.x, std::max(occ, 1) * h->nsm));
        }
        pl->ppc = false;
        return HJ_OK;
    }
    if (res && !b2) return seterr(HJ_ERR_CUDA, "internal: pipelined residual runs need a third iterate buffer");
    PpcKernel fn = pi->fn[sig][res];
    const int smem = pi->smem[sig];
    CKR(ensure_dyn_smem(h->dev, (const void *)fn, smem));
    int occ = 0;
    CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, pi->threads, smem));
    if (occ < 1) return seterr(HJ_ERR_UNSUPPORTED, "pipelined kernel does not fit on an SM");
    if (h->p.ctas_per_sm > 0) occ = std::min(occ, h->p.ctas_per_sm);
    const int tiles_x = (nx + pi->tx - 1) / pi->tx;
    const int ntiles = tiles_x * ((ny + pi->ty - 1) / pi->ty);
    const int ssz = fam == FAM_F64 ? 8 : fam == FAM_BF16 ? 2 : 4;
    const int tsz = fam == FAM_F64 ? 8 : 4;
    const long long ld = base.ld;
    const int grid = std::min(ntiles, occ * h->nsm);
    void *bufs[3] = {b0, b1, b2};
    pl->deferred = res;
    pl->period = res ? kPpcPeriod : 2;
    if (res) CKS(ensure_reduction(h, (size_t)grid));   // two slots of one partial per CTA
    for (int j = 0; j < pl->period; ++j) {
        PpcArgs &P = pl->p[j];
        memset(&P, 0, sizeof(P));
        P.a = base;
        P.a.uin = res ? bufs[j % 3] : bufs[j & 1];
        P.a.uout = res ? bufs[(j + 1) % 3] : bufs[(j + 1) & 1];
        P.tiles_x = tiles_x;
        P.ntiles = ntiles;
        P.spin_limit = 1LL << 26;
        P.parity = j & 1;
        P.part_w = h->partials + (size_t)(j & 1) * grid;
        P.part_r = h->partials + (size_t)((j + 1) & 1) * grid;
        if (!make_tmap(&P.mu, P.a.uin, tmap_type(fam, true), ssz, ld, nx + 2, ny + 2, pi->bwu, pi->ty + 2) ||
            !make_tmap(&P.mf, P.a.f, tmap_type(fam, false), tsz, ld, nx + 2, ny + 2, pi->bwf, pi->ty))
            return seterr(HJ_ERR_CUDA, "cuTensorMapEncodeTiled failed (pointer alignment or pitch)");
        if (sig && !make_tmap(&P.md, P.a.dinv, tmap_type(fam, false), tsz, ld, nx + 2, ny + 2, pi->bwf, pi->ty))
            return seterr(HJ_ERR_CUDA, "cuTensorMapEncodeTiled failed for 1/d");
    }
    pl->ppc = true;
    pl->pfn = fn;
    pl->smem = smem;
    pl->grid = dim3(grid);
    pl->block = dim3(pi->threads);
    return HJ_OK;
}

int plan_graph(hj_handle *h, const Plan &pl, int M, cudaGraphExec_t *ex) {
    if (pl.ppc) return get_graph<PpcArgs>(h, pl.pfn, pl.grid, pl.block, pl.smem, pl.p, pl.period, M, ex);
    return get_graph<CycArgs>(h, pl.fn, pl.grid, pl.block, pl.smem, pl.a, pl.period, M, ex);
}

void plan_launch(const Plan &pl, long long c, cudaStream_t s) {
    if (pl.ppc) pl.pfn<<<pl.grid, pl.block, pl.smem, s>>>(pl.p[c % pl.period]);
    else pl.fn<<<pl.grid, pl.block, pl.smem, s>>>(pl.a[c % pl.period]);
}

struct RunOut {
    long long c;        // index of the returned iterate
    int status;
    long long launched; // cycles issued
    double res2_0;      // ||r_0||^2 (converging mode)
    double res2_c;      // ||r_c||^2 of the returned iterate if known, else -1
    void *buf;          // the buffer that holds iterate c
};

// Where a converging run keeps its third iterate buffer (allocated on first
// use: only the pipelined kernel's deferred residual fold needs it).
struct ThirdBuffer {
    void **slot;
    size_t bytes;
    void *alias;   // in-place runs: every iterate buffer is this array
};

// Iterate cycles (or classic sweeps) from b0 (holds u_0) and b1 (the other
// buffer, same ghost ring).  fixed > 0: exactly `fixed` cycles, no residual.
// Otherwise until ||r_c|| <= tol ||r_0|| or max_cycles.
int run_cycles(hj_handle *h, const TileKernelInfo *ki, const PpcKernelInfo *pi, int fam, bool classic, bool sig,
               const CycArgs &base_in, void *b0, void *b1, ThirdBuffer third, double tol, long long max_cycles,
               long long fixed, cudaStream_t s, RunOut *ro, double *hist_out, long long hist_cap,
               long long *hist_len) {
    int M = h->p.check_every;
    ro->res2_0 = -1.0;
    ro->res2_c = -1.0;
    CycArgs base = base_in;
    base.err = &h->ctl->err;
    *h->h_ctl_init = Ctl{-1, HJ_OK, 0, 0.0, 0.0, 0, 0, 0.0, 0, 0, {0, 0}};
    CKR(cudaMemcpyAsync(h->ctl, h->h_ctl_init, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    if (fixed > 0) {
        Plan pl;
        CKS(make_plan(h, ki, pi, fam, classic, sig, false, base, b0, b1, nullptr, &pl));
        const long long reps = fixed / M;
        if (reps > 0) {
            cudaGraphExec_t ex;
            CKS(plan_graph(h, pl, M, &ex));
            for (long long r = 0; r < reps; ++r) CKR(cudaGraphLaunch(ex, s));
        }
        for (long long c = reps * M; c < fixed; ++c) plan_launch(pl, c, s);
        CKR(cudaGetLastError());
        CKR(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CKR(cudaEventRecord(h->ev, s));
        CKR(cudaEventSynchronize(h->ev));
        if (h->h_ctl->err) return seterr(HJ_ERR_TIMEOUT, "a bounded device wait expired (tile pipeline)");
        ro->c = fixed;
        ro->status = HJ_OK;
        ro->launched = fixed;
        ro->buf = (fixed & 1) ? b1 : b0;
        return HJ_OK;
    }
    {
        const long long sw = base.red.stall_window;
        base.red = red_args(h, RED_CYCLE, tol, max_cycles);
        base.red.stall_window = sw;
        base.red.stall_rtol = 1e-3;
    }
    // binary32 kernels with a constant diagonal accumulate (u' - u)^2; r = d (u' - u)
    // (the variable-coefficient kernels scale by their own d_p)
    if (fam != FAM_F64 && !sig && !h->d.coef) base.red.scale = base.dconst * base.dconst;
    if (max_cycles <= 0) {
        // no cycle may run: the residual of u_0 is all there is
        ro->c = 0;
        ro->status = HJ_ERR_NOT_CONVERGED;
        ro->launched = 0;
        ro->buf = b0;
        return HJ_OK;
    }
    // the pipelined kernel folds each launch's residual in the next launch:
    // a third buffer keeps u_c intact until that fold has decided
    void *b2 = nullptr;
    if (third.alias) {
        b2 = third.alias;
    } else if (deferred_run(h, ki, pi, classic)) {
        if (!third.slot) return seterr(HJ_ERR_CUDA, "internal: no slot for the third iterate buffer");
        if (!*third.slot) {
            if (dmalloc(third.slot, third.bytes) != cudaSuccess) {
                cudaGetLastError();
                *third.slot = nullptr;
                return seterr(HJ_ERR_NO_MEMORY, "third iterate buffer (%zu bytes)", third.bytes);
            }
        }
        b2 = *third.slot;
        CKR(cudaMemcpyAsync(b2, b0, third.bytes, cudaMemcpyDeviceToDevice, s));   // same ghost ring
    }
    Plan pl;
    CKS(make_plan(h, ki, pi, fam, classic, sig, true, base, b0, b1, b2, &pl));
    // residual of launch c's input is known after launch c + 1 (deferred fold)
    const int lag = pl.deferred ? 1 : 0;
    if (pl.deferred) M = (M + kPpcPeriod - 1) / kPpcPeriod * kPpcPeriod;
    cudaGraphExec_t ex;
    CKS(plan_graph(h, pl, M, &ex));
    const long long mask = kHistCap - 1;
    // Replays are pipelined two deep: replay i+1 is queued before the host
    // waits for replay i's control block, so the GPU does not idle while the
    // host checks.  Replay r copies its control block into slot r % 2 and the
    // entries of the residual ring it may have written into the pinned ring.
    // No replay starts beyond the launch that settles max_cycles, and launches
    // after convergence return at once.
    long long issued = 0;   // replays queued
    auto copy_ring = [&](long long lo, long long n) -> int {
        while (n > 0) {
            const long long p0 = lo & mask;
            const long long k = std::min<long long>(n, kHistCap - p0);
            CKR(cudaMemcpyAsync(h->h_hist + p0, h->hist + p0, k * sizeof(double), cudaMemcpyDeviceToHost, s));
            lo += k;
            n -= k;
        }
        return HJ_OK;
    };
    auto issue = [&]() -> int {
        const long long r = issued;
        CKR(cudaGraphLaunch(ex, s));
        const long long lo = std::max(0LL, r * M - lag);
        CKS(copy_ring(lo, (r + 1) * M - lo));
        CKR(cudaMemcpyAsync(h->h_ctl + (r & 1), h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CKR(cudaEventRecord(h->evs[r & 1], s));
        ++issued;
        return HJ_OK;
    };
    CKS(issue());
    long long copied = 0, checked = 0;
    const Ctl *last = nullptr;
    for (;;) {
        if (issued * M < max_cycles + lag) CKS(issue());
        CKR(cudaEventSynchronize(h->evs[checked & 1]));
        last = h->h_ctl + (checked & 1);
        ++checked;
        if (last->err) return seterr(HJ_ERR_TIMEOUT, "a bounded device wait expired (tile pipeline)");
        const long long ncomp = last->cycle;
        if (hist_out) {
            for (; copied < ncomp; ++copied)
                if (copied < hist_cap) hist_out[copied] = sqrt(h->h_hist[copied & mask]);
        }
        if (last->done >= 0) break;
        if (checked >= issued)
            return seterr(HJ_ERR_CUDA, "cycle loop did not terminate (device control block not updated)");
    }
    // the replay queued behind the converged one returns at once; wait for it
    // so that no copy into the pinned slots is still pending when we return
    if (issued > checked) CKR(cudaEventSynchronize(h->evs[(issued - 1) & 1]));
    const long long launched = issued * M;   // kernels launched, including returns-at-once overshoot
    if (hist_len) *hist_len = std::min(copied, hist_cap);
    ro->c = last->done;
    ro->status = last->status;
    ro->launched = launched;
    ro->res2_0 = last->res2_0;
    if (ro->status == HJ_OK || ro->status == HJ_ERR_DIVERGED) ro->res2_c = h->h_hist[ro->c & mask];
    if (pl.deferred) {
        void *bufs[3] = {b0, b1, b2};
        ro->buf = bufs[ro->c % 3];
    } else {
        ro->buf = (ro->c & 1) ? b1 : b0;
    }
    return HJ_OK;
}

// Iterate with the persistent engine when every block of the grid can be
// resident at once (or when forced), else with graph-captured launches.
int iterate(hj_handle *h, const TileKernelInfo *ki, const PpcKernelInfo *pi, int fam, bool classic, bool sig,
            const CycArgs &base, void *b0, void *b1, ThirdBuffer third, double tol, long long max_cycles,
            long long fixed, cudaStream_t s, RunOut *ro, double *hist_out, long long hist_cap, long long *hist_len,
            int *used_persistent) {
    if (h->d.coef || h->d.dim == 3) {   // variable coefficients and 3D: graph-captured launches only
        if (used_persistent) *used_persistent = 0;
        return run_cycles(h, ki, pi, fam, classic, sig, base, b0, b1, third, tol, max_cycles, fixed, s, ro,
                          hist_out, hist_cap, hist_len);
    }
    const PersistKernelInfo *pk =
        classic ? nullptr : find_persist(fam, h->d.dim, ki->tx, ki->ty, ki->threads / ki->tiles_per_cta);
    PersistKernel pclassic = nullptr;
    if (classic) {
        const PersistClassicInfo *pc = fam == FAM_F64 ? persist_classic_f64()
                                       : fam == FAM_F32 ? persist_classic_f32() : persist_classic_bf16();
        pclassic = pc->fn[h->d.dim - 1][sig ? 1 : 0];
    }
    dim3 g, bb;
    geometry(h, ki, classic, &g, &bb);
    // classic: items are blocks of points (the grid-stride launch shape is bounded)
    const long long cblocks = h->d.dim == 2 ? (long long)((h->d.nx + 31) / 32) * ((h->d.ny + 7) / 8)
                                            : (long long)((h->d.nx + 255) / 256) * h->d.ny;
    bool use = false;
    if ((pk || pclassic) && fixed <= 0 && max_cycles > 0 && h->p.persistent != 0 && !overlapped(h) && !h->d.coef) {
        int cap = 0;
        if (pclassic) {
            int occ = 0;
            CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pclassic, 256, 0));
            cap = occ * h->nsm;
        } else {
            CKS(persist_capacity(h, pk, sig, &cap));
        }
        const long long blocks = pclassic ? cblocks : (long long)g.x * g.y;
        if (h->p.persistent == 1) {
            if (blocks > 64LL * cap) return seterr(HJ_ERR_UNSUPPORTED, "grid too large for the persistent engine");
            use = true;
        } else {
            use = blocks <= cap;
        }
    }
    if (used_persistent) *used_persistent = use ? 1 : 0;
    if (!use)
        return run_cycles(h, ki, pi, fam, classic, sig, base, b0, b1, third, tol, max_cycles, fixed, s, ro,
                          hist_out, hist_cap, hist_len);
    std::vector<PersistProblem> v(1);
    PersistProblem &q = v[0];
    q.a = base;
    q.a.uin = b0;
    q.a.uout = b1;
    q.a.red = red_args(h, RED_CYCLE, tol, max_cycles);
    q.a.red.stall_window = base.red.stall_window;
    q.a.red.stall_rtol = 1e-3;
    if (fam != FAM_F64 && !sig) q.a.red.scale = base.dconst * base.dconst;
    q.blocks_x = pclassic ? 1 : g.x;
    q.blocks = pclassic ? (int)cblocks : g.x * g.y;
    std::vector<ProbState> st;
    CKS(run_persistent(h, pk, sig, v, s, &st, pclassic, fam));
    ro->c = st[0].done;
    ro->status = st[0].status;
    ro->launched = st[0].cycle;
    ro->res2_0 = st[0].res2_0;
    ro->res2_c = (ro->status == HJ_OK || ro->status == HJ_ERR_DIVERGED) ? st[0].res2_last : -1.0;
    ro->buf = (ro->c & 1) ? b1 : b0;
    if (hist_out) {
        const long long ncomp = st[0].cycle;
        const long long lo = std::max(0LL, ncomp - (long long)kHistCap);
        const long long mask = kHistCap - 1;
        CKR(cudaMemcpyAsync(h->h_hist, h->hist, kHistCap * sizeof(double), cudaMemcpyDeviceToHost, s));
        CKR(cudaStreamSynchronize(s));
        for (long long c = lo; c < ncomp && c < hist_cap; ++c) hist_out[c] = sqrt(h->h_hist[c & mask]);
        if (hist_len) *hist_len = std::min(ncomp, hist_cap);
    }
    return HJ_OK;
}

int residual_of(hj_handle *h, const void *f, const void *u, bool transpose, double *rr, double *ff, cudaStream_t s) {
    const CycArgs a = base_args(h, transpose);
    const RedArgs red = red_args(h, RED_STORE, 0.0, 0);
    if (h->d.dim == 3)
        CKR(launch_residual3d(h->d.dtype == HJ_F64, f, u, h->d.ld, a.ps, h->d.nx, h->d.ny, h->d.nz, a.cW, a.cE,
                              a.cS, a.cN, a.cB, a.cT, a.dconst, 1, red, s));
    else
        CKR(launch_residual_ex(h->d.dim, h->d.dtype == HJ_F64, f, u, h->d.sigma, h->d.ld, h->d.ld, h->d.nx,
                               h->d.ny, a.cW, a.cE, a.cS, a.cN, a.dconst, 1, nullptr, red, s, h->d.coef,
                               (long long)h->rows * h->d.ld));
    CKR(cudaMemcpyAsync(h->h_rstore, h->rstore, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev, s));
    CKR(cudaEventSynchronize(h->ev));
    if (rr) *rr = h->h_rstore[0];
    if (ff) *ff = h->h_rstore[1];
    return HJ_OK;
}

// Plain (binary64 or binary32) solve of A u = f, u in/out (device).
int solve_plain(hj_handle *h, const void *f, void *u, bool transpose, cudaStream_t s, hj_stats *st) {
    const bool classic = h->p.method == HJ_METHOD_CLASSIC;
    const TileKernelInfo *ki = classic ? h->k_classic : h->k_outer;
    const bool sig = h->d.sigma != nullptr;
    CycArgs base = base_args(h, transpose);
    base.f = f;
    base.dinv = h->dinv_outer;
    const bool inplace = h->p.in_place != 0;
    if (!inplace) CKR(cudaMemcpyAsync(h->ubuf, u, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    // in place, even the first cycle's staged data may mix u_0 and u_1: take
    // ||r_0|| exactly for the final status
    double r0_exact = -1.0;
    if (inplace && h->p.fixed_cycles <= 0) {
        double rr;
        CKS(residual_of(h, f, u, transpose, &rr, nullptr, s));
        r0_exact = sqrt(rr);
    }
    RunOut ro;
    long long hl = 0;
    int persist = 0;
    CKS(iterate(h, ki, classic ? nullptr : h->p_outer, h->fam_outer, classic, sig, base, u, inplace ? u : h->ubuf,
                ThirdBuffer{&h->ubuf2, h->grid_bytes, inplace ? u : nullptr}, h->p.tol, h->p.max_cycles,
                h->p.fixed_cycles, s, &ro, st ? st->history : nullptr, st ? st->history_cap : 0, &hl, &persist));
    if (ro.buf != u) CKR(cudaMemcpyAsync(u, ro.buf, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    double res0 = -1.0, resc = -1.0;
    if (h->p.fixed_cycles <= 0) {
        res0 = inplace ? r0_exact : sqrt(std::max(ro.res2_0, 0.0));
        if (ro.res2_c >= 0.0 && !inplace) {
            resc = sqrt(ro.res2_c);
        } else {
            // in place, the fused residuals belong to staged data, not to one
            // iterate: the exact residual of the returned array decides
            double rr;
            CKS(residual_of(h, f, u, transpose, &rr, nullptr, s));
            resc = sqrt(rr);
            if (ro.launched == 0) res0 = resc;
            if (resc <= h->p.tol * res0 && ro.status != HJ_ERR_DIVERGED) ro.status = HJ_OK;
        }
    }
    CKR(cudaStreamSynchronize(s));
    if (st) {
        st->cycles = ro.c;
        st->cycles_launched = ro.launched;
        st->inner_cycles = 0;
        st->outer_steps = 0;
        st->res0 = res0;
        st->res_final = resc;
        st->rel_final = res0 > 0 ? resc / res0 : 0.0;
        st->history_len = hl;
        st->persistent = persist;
    }
    if (ro.status == HJ_ERR_DIVERGED) return seterr(HJ_ERR_DIVERGED, "residual became non-finite at cycle %lld", ro.c);
    if (ro.status == HJ_ERR_NOT_CONVERGED)
        return seterr(HJ_ERR_NOT_CONVERGED, "tolerance %g not met after %lld cycles (rel %g)", h->p.tol, ro.c,
                      res0 > 0 ? resc / res0 : 0.0);
    return HJ_OK;
}

// Mixed-precision iterative refinement, u (binary64, device) in/out.
int solve_ir(hj_handle *h, const double *f, double *u, bool transpose, cudaStream_t s, hj_stats *st) {
    const bool sig = h->d.sigma != nullptr;
    const CycArgs geo = base_args(h, transpose);
    const bool bf16 = h->fam_inner == FAM_BF16;
    const size_t dsz = bf16 ? 2 : 4;
    CKR(cudaMemcpyAsync(h->ubuf, u, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    // outer residual of u_0 -> r32
    {
        const RedArgs red = red_args(h, RED_STORE, 0.0, 0);
        CKR(launch_residual_ex(h->d.dim, 1, f, u, h->d.sigma, h->d.ld, h->ld_in, h->d.nx, h->d.ny, geo.cW, geo.cE,
                               geo.cS, geo.cN, geo.dconst, 0, h->r32, red, s));
        CKR(cudaMemcpyAsync(h->h_rstore, h->rstore, sizeof(double), cudaMemcpyDeviceToHost, s));
        CKR(cudaEventRecord(h->ev, s));
        CKR(cudaEventSynchronize(h->ev));
    }
    double *cur = u, *other = (double *)h->ubuf;
    double r0 = sqrt(h->h_rstore[0]), rn = r0;
    long long inner_total = 0, inner_launched = 0;
    int o = 0, status = HJ_OK, persist = 0;
    long long hl = 0;
    CycArgs base = geo;
    base.ld = h->ld_in;
    base.f = h->r32;
    base.dinv = h->dinv32;
    base.red.stall_window = h->p.inner_stall;
    for (;; ++o) {
        if (st && st->history && o < st->history_cap) { st->history[o] = rn; hl = o + 1; }
        if (!std::isfinite(rn)) { status = HJ_ERR_DIVERGED; break; }
        if (rn <= h->p.tol * r0) { status = HJ_OK; break; }
        if (o >= h->p.max_outer) { status = HJ_ERR_NOT_CONVERGED; break; }
        CKR(cudaMemsetAsync(h->dA, 0, (size_t)h->rows * h->ld_in * dsz, s));
        RunOut ro;
        const bool inplace = h->p.in_place != 0;
        CKS(iterate(h, h->k_inner, h->p_inner, h->fam_inner, false, sig, base, h->dA, inplace ? h->dA : h->dB,
                    ThirdBuffer{&h->dC, (size_t)h->rows * h->ld_in * dsz, inplace ? h->dA : nullptr},
                    h->p.inner_tol, h->p.inner_max_cycles, 0, s, &ro, nullptr, 0, nullptr, &persist));
        inner_total += ro.c;
        inner_launched += ro.launched;
        const void *dsel = ro.buf;
        const RedArgs red = red_args(h, RED_STORE, 0.0, 0);
        CKR(launch_update_residual_ex(h->d.dim, f, cur, dsel, bf16 ? 1 : 0, other, h->d.sigma, h->r32, h->d.ld,
                                      h->ld_in, h->d.nx, h->d.ny, geo.cW, geo.cE, geo.cS, geo.cN, geo.dconst, red,
                                      s));
        CKR(cudaMemcpyAsync(h->h_rstore, h->rstore, sizeof(double), cudaMemcpyDeviceToHost, s));
        CKR(cudaEventRecord(h->ev, s));
        CKR(cudaEventSynchronize(h->ev));
        rn = sqrt(h->h_rstore[0]);
        std::swap(cur, other);
    }
    if (cur != u) CKR(cudaMemcpyAsync(u, cur, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    CKR(cudaStreamSynchronize(s));
    if (st) {
        st->cycles = inner_total;
        st->cycles_launched = inner_launched;
        st->inner_cycles = inner_total;
        st->outer_steps = o;
        st->res0 = r0;
        st->res_final = rn;
        st->rel_final = r0 > 0 ? rn / r0 : 0.0;
        st->history_len = hl;
        st->persistent = persist;
    }
    if (status == HJ_ERR_DIVERGED) return seterr(HJ_ERR_DIVERGED, "refinement residual became non-finite");
    if (status == HJ_ERR_NOT_CONVERGED)
        return seterr(HJ_ERR_NOT_CONVERGED, "refinement: tolerance %g not met after %d outer steps (rel %g)",
                      h->p.tol, o, r0 > 0 ? rn / r0 : 0.0);
    return HJ_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_ptr(const hj_handle *h, const void *p, const char *name) {
    if (!p) return seterr(HJ_ERR_INVALID_ARG, "%s is NULL", name);
    if (((uintptr_t)p) & 15) return seterr(HJ_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
    (void)h;
    return HJ_OK;
}

void fill_stats_config(const hj_handle *h, hj_stats *st, double t0) {
    if (!st) return;
    st->wall_ms = now_ms() - t0;
    st->tile_x = h->p.tile_x;
    st->tile_y = h->d.dim == 2 ? h->p.tile_y : 1;
    st->k = h->p.k;
    const TileKernelInfo *tk = h->ir ? h->k_inner : h->k_outer;
    st->tile_threads = tk ? tk->threads / tk->tiles_per_cta
                          : (h->d.coef || h->p.method == HJ_METHOD_MG) ? h->p.tile_x * (h->d.dim == 2 ? h->p.tile_y : 1)
                          : h->k3                                      ? 32
                                                                       : 0;
    st->tile_y = h->d.dim >= 2 ? h->p.tile_y : 1;
    st->tile_z = h->d.dim == 3 ? h->p.tile_z : 1;
    const PpcKernelInfo *pk = h->ir ? h->p_inner : h->p_outer;
    const bool ppc = want_ppc(h, pk, h->p.method == HJ_METHOD_CLASSIC);
    st->pipeline_stages = ppc ? pk->stages : (use_pf3(h) || want_ppc3(h, h->p.method == HJ_METHOD_CLASSIC)) ? 1 : 0;
    st->ctas_per_sm = ppc ? h->p.ctas_per_sm : 0;
    st->overlap_x = h->p.overlap_x;
    st->overlap_y = h->d.dim == 2 ? h->p.overlap_y : 0;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void hj_default_params(hj_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->method = HJ_METHOD_HIER;
    p->tile_x = 32;
    p->tile_y = 32;
    p->k = 16;
    p->precision = HJ_PREC_F64;
    p->check_every = 64;
    p->max_cycles = 10000000;
    p->tol = 1e-6;
    p->fixed_cycles = 0;
    p->inner_tol = 1e-4;
    p->inner_max_cycles = 1000000;
    p->max_outer = 60;
    p->persistent = -1;
    p->autotune = 0;
    p->pipeline = -1;
    p->inner_stall = 32;
    p->ctas_per_sm = 0;
    p->mg_levels = 0;
    p->mg_pre = 1;
    p->mg_post = 1;
    p->mg_omega = 0.8;
    p->mg_coarse_k = 64;
    p->mg_coarse_cycles = 4;
}

const char *hj_error_string(int s) {
    switch (s) {
    case HJ_OK: return "success";
    case HJ_ERR_INVALID_ARG: return "invalid argument";
    case HJ_ERR_NOT_DIAG_DOMINANT: return "stencil is not diagonally dominant";
    case HJ_ERR_UNSUPPORTED: return "unsupported tile shape or mode";
    case HJ_ERR_CUDA: return "CUDA error";
    case HJ_ERR_NOT_CONVERGED: return "not converged";
    case HJ_ERR_DIVERGED: return "diverged";
    case HJ_ERR_TIMEOUT: return "device wait timed out";
    case HJ_ERR_NO_MEMORY: return "out of device memory";
    case HJ_ERR_BOUNDS: return "debug check failed (index out of range or guard band overwritten)";
    default: return "unknown status";
    }
}

const char *hj_last_error(void) { return g_err; }

int hj_tile_variants(int dim, int precision, int *txt, int cap) {
    const int fam = precision == HJ_PREC_F64 ? FAM_F64 : precision == HJ_PREC_BF16CORR_IR ? FAM_BF16 : FAM_F32;
    int n = 0, m = 0;
    const TileKernelInfo *k = family_tiles(fam, &n);
    for (int i = 0; i < n; ++i) {
        if (k[i].dim != dim) continue;
        if (txt && m < cap) {
            txt[3 * m] = k[i].tx;
            txt[3 * m + 1] = k[i].ty;
            txt[3 * m + 2] = k[i].threads / k[i].tiles_per_cta;
        }
        ++m;
    }
    return m;
}

int hj_tile_shapes(int dim, int precision, int *xy, int cap) {
    const int fam = precision == HJ_PREC_F64 ? FAM_F64 : precision == HJ_PREC_BF16CORR_IR ? FAM_BF16 : FAM_F32;
    int n = 0, m = 0;
    const TileKernelInfo *k = family_tiles(fam, &n);
    for (int i = 0; i < n; ++i) {
        if (k[i].dim != dim) continue;
        bool dup = false;
        for (int j = 0; j < i; ++j) dup |= k[j].dim == dim && k[j].tx == k[i].tx && k[j].ty == k[i].ty;
        if (dup) continue;
        if (xy && m < cap) {
            xy[2 * m] = k[i].tx;
            xy[2 * m + 1] = k[i].ty;
        }
        ++m;
    }
    return m;
}

int hj_tile_shapes3d(int precision, int *xyz, int cap) {
    if (precision != HJ_PREC_F64 && precision != HJ_PREC_F32) return 0;
    int n = 0;
    const Tile3Info *k = precision == HJ_PREC_F64 ? tiles3d_f64(&n) : tiles3d_f32(&n);
    for (int i = 0; i < n && xyz && i < cap; ++i) {
        xyz[3 * i] = k[i].tx;
        xyz[3 * i + 1] = k[i].ty;
        xyz[3 * i + 2] = k[i].tz;
    }
    return n;
}

void hj_destroy(hj_handle *h) {
    if (!h) return;
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    if (h->mg_exec) cudaGraphExecDestroy(h->mg_exec);
    if (h->mg_exec_fixed) cudaGraphExecDestroy(h->mg_exec_fixed);
    if (h->mg_arena) dfree(h->mg_arena);
    void *dev[] = {h->ubuf, h->ubuf2, h->dC, h->vcf, h->dinv_outer, h->dinv32, h->r32, h->dA, h->dB, h->hf, h->hu, h->partials, h->gpart,
                   h->hist, h->rstore, h->gcnt, h->fcnt, h->ctl, h->pscratch, h->barena, h->rs, h->bmeta};
    for (void *p : dev)
        if (p) dfree(p);
    void *pin[] = {h->h_ctl, h->h_ctl_init, h->h_hist, h->h_rstore, h->h_pstage, h->h_rs, h->h_bmeta};
    for (void *p : pin)
        if (p) cudaFreeHost(p);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev) cudaEventDestroy(h->ev);
    for (cudaEvent_t e : h->evs)
        if (e) cudaEventDestroy(e);
    delete h;
}

int hj_create(hj_handle **out, const hj_desc *desc, const hj_params *params) {
    if (!out) return seterr(HJ_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return seterr(HJ_ERR_INVALID_ARG, "desc is NULL");
    hj_params p;
    if (params) p = *params;
    else hj_default_params(&p);
    const hj_desc &d = *desc;
    if (d.dim < 1 || d.dim > 3) return seterr(HJ_ERR_INVALID_ARG, "dim must be 1, 2 or 3 (got %d)", d.dim);
    if (d.nx < 1 || d.ny < 1) return seterr(HJ_ERR_INVALID_ARG, "nx, ny must be >= 1 (got %d, %d)", d.nx, d.ny);
    if (d.dtype != HJ_F64 && d.dtype != HJ_F32) return seterr(HJ_ERR_INVALID_ARG, "dtype must be HJ_F64 or HJ_F32");
    const size_t esz = d.dtype == HJ_F64 ? 8 : 4;
    if (d.ld < (long long)d.nx + 2) return seterr(HJ_ERR_INVALID_ARG, "ld (%lld) < nx + 2", d.ld);
    if ((d.ld * (long long)esz) % 16) return seterr(HJ_ERR_INVALID_ARG, "ld * element size must be a multiple of 16 bytes");
    if (d.dim == 1 && d.ny > 65535) return seterr(HJ_ERR_INVALID_ARG, "1D: at most 65535 rows");
    if (d.dim >= 2 && (d.ny + 7) / 8 > 65535) return seterr(HJ_ERR_INVALID_ARG, "2D/3D: ny must be <= 524280");
    if (p.precision < HJ_PREC_F64 || p.precision > HJ_PREC_BF16CORR_IR)
        return seterr(HJ_ERR_INVALID_ARG, "unknown precision %d", p.precision);
    const bool ir = p.precision == HJ_PREC_F32_IR || p.precision == HJ_PREC_BF16CORR_IR;
    if ((p.precision == HJ_PREC_F32) != (d.dtype == HJ_F32))
        return seterr(HJ_ERR_INVALID_ARG, "dtype HJ_F32 goes with precision HJ_PREC_F32 only (binary64 arrays otherwise)");
    if (p.method != HJ_METHOD_HIER && p.method != HJ_METHOD_CLASSIC && p.method != HJ_METHOD_MG)
        return seterr(HJ_ERR_INVALID_ARG, "unknown method %d", p.method);
    int mg_levels = 0;
    if (p.method == HJ_METHOD_MG) {
        if (d.dim != 2) return seterr(HJ_ERR_UNSUPPORTED, "multigrid: 2D only");
        if (d.sigma || d.coef)
            return seterr(HJ_ERR_UNSUPPORTED, "multigrid: constant coefficients and sigma_const (sigma, coef NULL)");
        if (p.precision != HJ_PREC_F64 && p.precision != HJ_PREC_F32)
            return seterr(HJ_ERR_UNSUPPORTED, "multigrid: HJ_PREC_F64 or HJ_PREC_F32");
        if (p.overlap_x > 0 || p.overlap_y > 0 || p.in_place || p.persistent == 1 || p.pipeline == 1 ||
            p.autotune != 0)
            return seterr(HJ_ERR_UNSUPPORTED, "multigrid: no overlap, in-place, persistent, pipeline or autotune");
        if (p.tile_x < 1 || p.tile_y < 1 || (long long)p.tile_x * p.tile_y > 1024)
            return seterr(HJ_ERR_INVALID_ARG, "multigrid: smoother subdomain of 1 to 1024 points");
        if (p.mg_pre < 0 || p.mg_post < 0 || p.mg_coarse_k < 1 || p.mg_coarse_cycles < 1)
            return seterr(HJ_ERR_INVALID_ARG, "multigrid: mg_pre, mg_post >= 0, mg_coarse_k, mg_coarse_cycles >= 1");
        if (!(p.mg_omega > 0.0 && p.mg_omega <= 1.0))
            return seterr(HJ_ERR_INVALID_ARG, "multigrid: 0 < mg_omega <= 1");
        const int avail = mg_levels_of(d.nx, d.ny);
        if (avail < 2) return seterr(HJ_ERR_INVALID_ARG, "multigrid needs odd nx, ny > 1 (got %d x %d)", d.nx, d.ny);
        if (p.mg_levels < 0 || p.mg_levels == 1 || p.mg_levels > avail)
            return seterr(HJ_ERR_INVALID_ARG, "multigrid: mg_levels must be 0 or in [2, %d]", avail);
        mg_levels = p.mg_levels ? p.mg_levels : avail;
        int cx = d.nx, cy = d.ny;
        for (int l = 1; l < mg_levels; ++l) {
            cx = (cx - 1) / 2;
            cy = (cy - 1) / 2;
        }
        if ((long long)cx * cy > 1024)
            return seterr(HJ_ERR_UNSUPPORTED, "multigrid: coarsest level %d x %d exceeds 1024 points (add levels)", cx, cy);
        p.mg_levels = mg_levels;
    }
    if (p.k < 1) return seterr(HJ_ERR_INVALID_ARG, "k must be >= 1");
    if (!(p.tol >= 0.0)) return seterr(HJ_ERR_INVALID_ARG, "tol must be >= 0");
    if (p.max_cycles < 0) return seterr(HJ_ERR_INVALID_ARG, "max_cycles must be >= 0");
    if (ir && !(p.inner_tol > 0.0 && p.inner_tol < 1.0)) return seterr(HJ_ERR_INVALID_ARG, "inner_tol must be in (0,1)");
    if (ir && p.inner_max_cycles < 1) return seterr(HJ_ERR_INVALID_ARG, "inner_max_cycles must be >= 1");
    if (p.inner_stall < 0) return seterr(HJ_ERR_INVALID_ARG, "inner_stall must be >= 0");
    if (p.ctas_per_sm < 0) return seterr(HJ_ERR_INVALID_ARG, "ctas_per_sm must be >= 0");
    if (p.in_place != 0 && p.in_place != 1) return seterr(HJ_ERR_INVALID_ARG, "in_place must be 0 or 1");
    // 3D seven-point extension: constant coefficients, graphs, F64 / F32
    const Tile3Info *k3 = nullptr;
    if (d.dim == 3) {
        if (d.nz < 1 || d.nz > 65535) return seterr(HJ_ERR_INVALID_ARG, "3D: nz must be in [1, 65535] (got %d)", d.nz);
        if (d.sigma || d.coef)
            return seterr(HJ_ERR_UNSUPPORTED, "3D takes constant coefficients and sigma_const (sigma, coef NULL)");
        if (ir) return seterr(HJ_ERR_UNSUPPORTED, "3D: HJ_PREC_F64 or HJ_PREC_F32");
        if (p.overlap_x > 0 || p.overlap_y > 0) return seterr(HJ_ERR_UNSUPPORTED, "3D: no overlapping subdomains");
        if (p.in_place) return seterr(HJ_ERR_UNSUPPORTED, "3D: no in-place variant");
        if (p.persistent == 1) return seterr(HJ_ERR_UNSUPPORTED, "3D runs on graphs (persistent must not be 1)");
        if (p.autotune != 0) return seterr(HJ_ERR_UNSUPPORTED, "3D: no autotuner");
        const double off = fabs(d.cW) + fabs(d.cE) + fabs(d.cS) + fabs(d.cN) + fabs(d.cB) + fabs(d.cT);
        const double dc = d.cD + d.sigma_const;
        if (!(dc > 0.0) || dc < off)
            return seterr(HJ_ERR_NOT_DIAG_DOMINANT, "diagonal %g < sum |off-diagonal| %g", dc, off);
        if (p.method == HJ_METHOD_HIER) {
            int n3 = 0;
            const Tile3Info *t3 = p.precision == HJ_PREC_F64 ? tiles3d_f64(&n3) : tiles3d_f32(&n3);
            if (p.tile_z == 0) k3 = &t3[0];
            for (int i = 0; i < n3 && !k3; ++i)
                if (t3[i].tx == p.tile_x && t3[i].ty == p.tile_y && t3[i].tz == p.tile_z) k3 = &t3[i];
            if (!k3)
                return seterr(HJ_ERR_UNSUPPORTED, "3D subdomain %dx%dx%d not built for this precision (hj_tile_shapes3d)",
                              p.tile_x, p.tile_y, p.tile_z);
            p.tile_x = k3->tx;
            p.tile_y = k3->ty;
            p.tile_z = k3->tz;
        }
    } else {
        p.tile_z = 1;
    }
    if (d.dim == 1) p.overlap_y = 0;
    if (p.overlap_x < 0 || p.overlap_y < 0) return seterr(HJ_ERR_INVALID_ARG, "overlaps must be >= 0");
    if (p.overlap_x > 0 || p.overlap_y > 0) {
        if (p.method == HJ_METHOD_CLASSIC) return seterr(HJ_ERR_INVALID_ARG, "overlap applies to hierarchical cycles");
        if (p.persistent == 1 || p.pipeline == 1)
            return seterr(HJ_ERR_UNSUPPORTED, "overlapping subdomains run on graphs (persistent and pipeline must not be 1)");
    }
    if (ir && p.method == HJ_METHOD_CLASSIC) return seterr(HJ_ERR_UNSUPPORTED, "refinement uses hierarchical cycles");
    if (p.check_every < 1) p.check_every = 1;
    if (p.check_every > 4096) p.check_every = 4096;
    p.check_every += p.check_every & 1;
    if (d.dim == 1) p.tile_y = 1;
    if (p.autotune < 0 || p.autotune > 3) return seterr(HJ_ERR_INVALID_ARG, "autotune must be 0, 1, 2 or 3");
    if (p.autotune != 0 && !d.coef) {   // (variable coefficients: kept as given)
        hj_params tp = p;
        const int st = hj_autotune(&d, &tp, nullptr);
        if (st != HJ_OK) return st;
        p.tile_x = tp.tile_x;
        p.tile_y = tp.tile_y;
        p.tile_threads = tp.tile_threads;
        p.k = tp.k;
        p.pipeline_stages = tp.pipeline_stages;
        p.ctas_per_sm = tp.ctas_per_sm;
        p.overlap_x = tp.overlap_x;
        p.overlap_y = tp.overlap_y;
    }
    if (p.overlap_x >= p.tile_x || (d.dim == 2 && p.overlap_y >= p.tile_y))
        return seterr(HJ_ERR_INVALID_ARG, "overlap (%d, %d) must be smaller than the subdomain (%d, %d)", p.overlap_x,
                      p.overlap_y, p.tile_x, p.tile_y);

    const int rows = d.dim >= 2 ? d.ny + 2 : d.ny;
    if (d.coef) {
        if (ir) return seterr(HJ_ERR_UNSUPPORTED, "variable coefficients: HJ_PREC_F64 or HJ_PREC_F32 only");
        if (p.overlap_x > 0 || p.overlap_y > 0)
            return seterr(HJ_ERR_UNSUPPORTED, "variable coefficients do not take overlapping subdomains");
        if (p.persistent == 1 || p.pipeline == 1)
            return seterr(HJ_ERR_UNSUPPORTED, "variable coefficients run on graphs (persistent and pipeline must not be 1)");
        if (p.tile_x < 1 || p.tile_y < 1) return seterr(HJ_ERR_INVALID_ARG, "tile sizes must be >= 1");
        if ((long long)p.tile_x * (d.dim == 2 ? p.tile_y : 1) > 1024)
            return seterr(HJ_ERR_UNSUPPORTED, "variable coefficients: one thread per point, at most 1024 per subdomain");
    }
    // diagonal dominance (Section 2.1): d_p >= |cW| + |cE| + |cS| + |cN|, d_p > 0
    // (3D: checked above)
    if (d.dim != 3) {
        const int r0 = d.dim == 2 ? 1 : 0, r1 = d.dim == 2 ? d.ny : d.ny - 1;
        std::vector<double> hs, hc;
        if (d.sigma) {
            hs.resize((size_t)rows * d.ld);
            cudaError_t e = cudaMemcpy(hs.data(), d.sigma, hs.size() * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return seterr(HJ_ERR_CUDA, "reading sigma: %s", cudaGetErrorString(e));
        }
        const int planes = d.dim == 2 ? 4 : 2;
        const size_t ps = (size_t)rows * d.ld;
        if (d.coef) {
            hc.resize(ps * planes);
            cudaError_t e = cudaMemcpy(hc.data(), d.coef, hc.size() * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return seterr(HJ_ERR_CUDA, "reading coef: %s", cudaGetErrorString(e));
        }
        const double off_c = fabs(d.cW) + fabs(d.cE) + (d.dim == 2 ? fabs(d.cS) + fabs(d.cN) : 0.0);
        double worst = INFINITY, wd = 0.0, wo = 0.0;   // smallest d_p - sum |off|
        for (int j = r0; j <= r1; ++j)
            for (int i = 1; i <= d.nx; ++i) {
                const size_t q = (size_t)j * d.ld + i;
                const double dp = d.cD + d.sigma_const + (d.sigma ? hs[q] : 0.0);
                double off = off_c;
                if (d.coef) {
                    off = 0.0;
                    for (int m = 0; m < planes; ++m) off += fabs(hc[m * ps + q]);
                }
                if (!(dp > 0.0) || dp - off < worst) {
                    worst = dp > 0.0 ? dp - off : -INFINITY;
                    wd = dp;
                    wo = off;
                }
            }
        if (!(worst >= 0.0))
            return seterr(HJ_ERR_NOT_DIAG_DOMINANT, "diagonal %g < sum |off-diagonal| %g", wd, wo);
    }

    hj_handle *h = new hj_handle();
    h->d = d;
    h->p = p;
    h->ir = ir;
    h->rows = rows;
    h->esz = esz;
    h->grid_elems = (size_t)rows * d.ld * (d.dim == 3 ? (size_t)d.nz + 2 : 1);
    h->k3 = k3;
    h->grid_bytes = h->grid_elems * esz;
    h->fam_outer = p.precision == HJ_PREC_F32 ? FAM_F32 : FAM_F64;
    h->fam_inner = p.precision == HJ_PREC_BF16CORR_IR ? FAM_BF16 : FAM_F32;
    int st = HJ_OK;
#define HJ_FAIL(code, ...)              \
    do {                                \
        st = seterr(code, __VA_ARGS__); \
        hj_destroy(h);                  \
        return st;                      \
    } while (0)
#define HJ_ALLOC(ptr, bytes)                                                               \
    do {                                                                                   \
        if (dmalloc((void **)&(ptr), (bytes)) != cudaSuccess) {                         \
            cudaGetLastError();                                                            \
            HJ_FAIL(HJ_ERR_NO_MEMORY, "cudaMalloc of %zu bytes failed", (size_t)(bytes)); \
        }                                                                                  \
    } while (0)
    if (cudaGetDevice(&h->dev) != cudaSuccess) HJ_FAIL(HJ_ERR_CUDA, "no CUDA device");
    cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev);

    h->ld_in = ((long long)d.nx + 2 + 31) / 32 * 32;
    // 1D with fewer subdomains than SMs: a cycle is the latency of one
    // subdomain's k sweeps, and binary64 issues slowly per sub-partition, so
    // split each subdomain over as many warps as a built variant allows
    if (d.dim == 1 && p.tile_threads == 0 && p.method == HJ_METHOD_HIER) {
        const long long tiles = (long long)((d.nx + p.tile_x - 1) / p.tile_x) * d.ny;
        const int fam = ir ? h->fam_inner : h->fam_outer;
        if (tiles < h->nsm) {
            int n = 0, best = 0;
            const TileKernelInfo *k = family_tiles(fam, &n);
            for (int i = 0; i < n; ++i)
                if (k[i].dim == 1 && k[i].tx == p.tile_x) best = std::max(best, k[i].threads / k[i].tiles_per_cta);
            p.tile_threads = best;
            h->p.tile_threads = best;
        }
    }
    if (d.dim == 3) {
        // kernels picked above (k3) or the classic seven-point sweep
    } else if (ir) {
        h->k_inner = find_tile(h->fam_inner, d.dim, p.tile_x, p.tile_y, p.tile_threads);
        if (!h->k_inner)
            HJ_FAIL(HJ_ERR_UNSUPPORTED, "tile %dx%d (%d threads) not built for this precision", p.tile_x, p.tile_y,
                    p.tile_threads);
        if (d.dim == 2) h->p_inner = find_ppc(h->fam_inner, p.tile_x, p.tile_y, h->k_inner->threads, p.pipeline_stages);
    } else if (p.method == HJ_METHOD_CLASSIC) {
        h->k_classic = family_classic(h->fam_outer, d.dim);
    } else if (p.method == HJ_METHOD_MG) {
        // smoother, transfer and residual kernels live in hj_mg.cu
    } else {
        // (variable coefficients run their own thread-per-point kernel: any
        // subdomain of at most 1024 points)
        h->k_outer = d.coef ? nullptr : find_tile(h->fam_outer, d.dim, p.tile_x, p.tile_y, p.tile_threads);
        if (!h->k_outer && !d.coef)
            HJ_FAIL(HJ_ERR_UNSUPPORTED, "tile %dx%d (%d threads) not built for this precision", p.tile_x, p.tile_y,
                    p.tile_threads);
        if (d.dim == 2 && h->k_outer)
            h->p_outer = find_ppc(h->fam_outer, p.tile_x, p.tile_y, h->k_outer->threads, p.pipeline_stages);
    }
    if (p.pipeline == 1 && d.dim == 2 && p.method == HJ_METHOD_HIER && !(ir ? h->p_inner : h->p_outer))
        HJ_FAIL(HJ_ERR_UNSUPPORTED, "no pipelined kernel for tile %dx%d", p.tile_x, p.tile_y);
    // reduction workspace sized for the largest grid any kernel of this handle launches
    size_t maxb = (size_t)aux_max_blocks(d.dim, d.nx, d.ny);
    for (int fam = 0; fam < 3; ++fam) {
        int n = 0;
        const TileKernelInfo *k = family_tiles(fam, &n);
        for (int i = 0; i < n; ++i) {
            if (k[i].dim != d.dim) continue;
            dim3 g, b;
            geometry(h, &k[i], false, &g, &b);
            maxb = std::max(maxb, (size_t)g.x * g.y);
        }
    }
    if (d.dim == 3) {
        const long long gx = (d.nx + 31) / 32, gy = (d.ny + 7) / 8;
        maxb = std::max(maxb, (size_t)aux_max_blocks3(d.nx, d.ny, d.nz));
        maxb = std::max(maxb, (size_t)(gx * gy * d.nz));   // classic sweep
        if (k3) {
            const long long nsub = (long long)((d.nx + k3->tx - 1) / k3->tx) * ((d.ny + k3->ty - 1) / k3->ty) *
                                   ((d.nz + k3->tz - 1) / k3->tz);
            maxb = std::max(maxb, (size_t)((nsub + k3->nw - 1) / k3->nw));
        }
    }
    if (d.coef) {   // thread-per-point kernel: one block per subdomain
        const long long gx = (d.nx + p.tile_x - 1) / p.tile_x;
        maxb = std::max(maxb, (size_t)(d.dim == 2 ? gx * ((d.ny + p.tile_y - 1) / p.tile_y) : gx * d.ny));
    }
    h->max_blocks = maxb;
    h->max_groups = (maxb + kGroup - 1) / kGroup;
    HJ_ALLOC(h->ubuf, h->grid_bytes);
    if (d.coef && h->fam_outer == FAM_F32) {
        // -c/d per neighbour, 1/d and d per point, in binary32
        const int np = (d.dim == 2 ? 4 : 2) + 2;
        const long long ps = (long long)rows * d.ld;
        HJ_ALLOC(h->vcf, (size_t)np * ps * sizeof(float));
        if (cudaMemset(h->vcf, 0, (size_t)np * ps * sizeof(float)) != cudaSuccess ||
            launch_vc_prep(d.dim, d.coef, d.sigma, d.cD + d.sigma_const, d.ld, ps, d.nx, d.ny, h->vcf, 0) !=
                cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            HJ_FAIL(HJ_ERR_CUDA, "preparing variable coefficients");
    }
    HJ_ALLOC(h->partials, 2 * maxb * sizeof(double));
    HJ_ALLOC(h->gpart, 2 * h->max_groups * sizeof(double));
    HJ_ALLOC(h->gcnt, h->max_groups * sizeof(unsigned));
    HJ_ALLOC(h->fcnt, sizeof(unsigned));
    HJ_ALLOC(h->hist, kHistCap * sizeof(double));
    HJ_ALLOC(h->ctl, sizeof(Ctl));
    HJ_ALLOC(h->rstore, 2 * sizeof(double));
    if (cudaMemset(h->gcnt, 0, h->max_groups * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->fcnt, 0, sizeof(unsigned)) != cudaSuccess)
        HJ_FAIL(HJ_ERR_CUDA, "cudaMemset failed");
    if (cudaMallocHost((void **)&h->h_ctl, 2 * sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_ctl_init, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_hist, kHistCap * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_rstore, 2 * sizeof(double)) != cudaSuccess)
        HJ_FAIL(HJ_ERR_NO_MEMORY, "cudaMallocHost failed");
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->evs[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->evs[1], cudaEventDisableTiming) != cudaSuccess)
        HJ_FAIL(HJ_ERR_CUDA, "stream/event creation failed");

    if (p.method == HJ_METHOD_MG) {
        st = mg_setup(h, mg_levels);
        if (st != HJ_OK) {
            hj_destroy(h);
            return st;
        }
    }
    const double dconst = d.cD + d.sigma_const;
    const int r0 = d.dim == 2 ? 1 : 0;
    if (ir) {
        const bool bf16 = h->fam_inner == FAM_BF16;
        const size_t nin = (size_t)rows * h->ld_in;
        HJ_ALLOC(h->r32, nin * sizeof(float));
        HJ_ALLOC(h->dA, nin * (bf16 ? 2 : 4));
        HJ_ALLOC(h->dB, nin * (bf16 ? 2 : 4));
        if (cudaMemset(h->r32, 0, nin * sizeof(float)) != cudaSuccess ||
            cudaMemset(h->dA, 0, nin * (bf16 ? 2 : 4)) != cudaSuccess ||
            cudaMemset(h->dB, 0, nin * (bf16 ? 2 : 4)) != cudaSuccess)
            HJ_FAIL(HJ_ERR_CUDA, "cudaMemset failed");
        if (d.sigma) {
            HJ_ALLOC(h->dinv32, nin * sizeof(float));
            cudaMemset(h->dinv32, 0, nin * sizeof(float));
            if (launch_make_dinv_box(d.sigma, dconst, d.ld, h->ld_in, r0, d.ny, 1, d.nx, FAM_F32, h->dinv32, 0) !=
                cudaSuccess)
                HJ_FAIL(HJ_ERR_CUDA, "dinv kernel failed");
        }
    } else if (d.sigma) {
        const size_t tsz = h->fam_outer == FAM_F64 ? 8 : 4;
        HJ_ALLOC(h->dinv_outer, h->grid_elems * tsz);
        cudaMemset(h->dinv_outer, 0, h->grid_elems * tsz);
        if (launch_make_dinv_box(d.sigma, dconst, d.ld, d.ld, r0, d.ny, 1, d.nx, h->fam_outer, h->dinv_outer, 0) !=
            cudaSuccess)
            HJ_FAIL(HJ_ERR_CUDA, "dinv kernel failed");
    }
    if (cudaDeviceSynchronize() != cudaSuccess) HJ_FAIL(HJ_ERR_CUDA, "create: %s", cudaGetErrorString(cudaGetLastError()));
#undef HJ_ALLOC
#undef HJ_FAIL
    *out = h;
    g_err[0] = 0;
    return HJ_OK;
}

int hj_solve(hj_handle *h, const void *f, void *u, hj_stream stream, hj_stats *stats) {
    if (!h) return seterr(HJ_ERR_INVALID_ARG, "handle is NULL");
    if (!f || !u) return seterr(HJ_ERR_INVALID_ARG, "f and u must be non-NULL");
    const double t0 = now_ms();
    cudaStream_t s = (cudaStream_t)stream;
    const bool fdev = is_device_ptr(f), udev = is_device_ptr(u);
    const void *fd = f;
    void *ud = u;
    if (!fdev || !udev) {
        if (!h->hf) CKR(dmalloc(&h->hf, h->grid_bytes));
        if (!h->hu) CKR(dmalloc(&h->hu, h->grid_bytes));
        if (!fdev) {
            CKR(cudaMemcpyAsync(h->hf, f, h->grid_bytes, cudaMemcpyHostToDevice, s));
            fd = h->hf;
        }
        if (!udev) {
            CKR(cudaMemcpyAsync(h->hu, u, h->grid_bytes, cudaMemcpyHostToDevice, s));
            ud = h->hu;
        }
    }
    CKS(check_ptr(h, fd, "f"));
    CKS(check_ptr(h, ud, "u"));
    int st = h->ir                          ? solve_ir(h, (const double *)fd, (double *)ud, false, s, stats)
             : h->p.method == HJ_METHOD_MG ? solve_mg(h, fd, ud, s, stats)
                                           : solve_plain(h, fd, ud, false, s, stats);
    if (!udev && (st == HJ_OK || st == HJ_ERR_NOT_CONVERGED || st == HJ_ERR_DIVERGED)) {
        CKR(cudaMemcpyAsync(u, ud, h->grid_bytes, cudaMemcpyDeviceToHost, s));
        CKR(cudaStreamSynchronize(s));
    }
    fill_stats_config(h, stats, t0);
    return st;
}

int hj_residual(hj_handle *h, const void *f, const void *u, double *abs_l2, double *rel_l2, hj_stream stream) {
    if (!h) return seterr(HJ_ERR_INVALID_ARG, "handle is NULL");
    CKS(check_ptr(h, f, "f"));
    CKS(check_ptr(h, u, "u"));
    double rr = 0, ff = 0;
    CKS(residual_of(h, f, u, false, &rr, &ff, (cudaStream_t)stream));
    const double a = sqrt(rr);
    if (abs_l2) *abs_l2 = a;
    if (rel_l2) *rel_l2 = ff > 0 ? a / sqrt(ff) : a;
    return HJ_OK;
}

int hj_solve_adjoint(hj_handle *h, const void *g, const void *u, void *dl_df, void *dl_dsigma, hj_stream stream,
                     hj_stats *stats) {
    if (!h) return seterr(HJ_ERR_INVALID_ARG, "handle is NULL");
    if (h->d.coef) return seterr(HJ_ERR_UNSUPPORTED, "the adjoint is built for constant neighbour coefficients");
    if (h->d.dim == 3) return seterr(HJ_ERR_UNSUPPORTED, "the adjoint is built for 1D and 2D");
    if (h->p.method == HJ_METHOD_MG) return seterr(HJ_ERR_UNSUPPORTED, "the adjoint runs hierarchical cycles, not V-cycles");
    CKS(check_ptr(h, g, "g"));
    CKS(check_ptr(h, u, "u"));
    CKS(check_ptr(h, dl_df, "dl_df"));
    if (dl_dsigma) CKS(check_ptr(h, dl_dsigma, "dl_dsigma"));
    const double t0 = now_ms();
    cudaStream_t s = (cudaStream_t)stream;
    // lambda_0 = 0 with a zero ghost ring (homogeneous Dirichlet data of the adjoint)
    CKR(cudaMemsetAsync(dl_df, 0, h->grid_bytes, s));
    int st = h->ir ? solve_ir(h, (const double *)g, (double *)dl_df, true, s, stats)
                   : solve_plain(h, g, dl_df, true, s, stats);
    if (st != HJ_OK && st != HJ_ERR_NOT_CONVERGED) return st;
    if (dl_dsigma) {
        CKR(cudaMemsetAsync(dl_dsigma, 0, h->grid_elems * sizeof(double), s));
        CKR(launch_grad_sigma_ex(h->d.dim, h->d.dtype == HJ_F64, dl_df, u, (double *)dl_dsigma, h->d.ld, h->d.nx,
                                 h->d.ny, 0, s));
        CKR(cudaStreamSynchronize(s));
    }
    fill_stats_config(h, stats, t0);
    return st;
}



}  // extern "C"
