// hj_autotune.cu -- picks the subdomain shape (and with it the threads per
// subdomain) and the subiteration count k for a problem by measurement.
//
// k trades on-chip work against halo staleness (Section 3.3: small k keeps the
// halos fresh, large k saves global passes), and the best value depends on the
// tile shape, the stencil and the GPU, so it is measured rather than guessed.
// For every candidate (tile, k):
//   * contraction rho per cycle: start from the lowest discrete sine mode with
//     f = 0 and zero Dirichlet data (the slowest-converging error component),
//     run 128 cycles and take the mean rate over the last 32 (earlier windows
//     are biased by the transient at subdomain edges: the residual may even
//     grow during the first cycles);
//   * time per cycle t: CUDA events around the same run (graph path with the
//     fused residual, as a real solve runs);
//   * predicted time to the tolerance: ln(tol) / ln(rho) * t.
// The candidate with the smallest prediction wins.  Where the TMA-pipelined
// kernel runs the cycles (large 2D grids), its launch shape is tuned next
// (tune_launch: threads per subdomain, copy stages, CTAs per SM by measured
// time per cycle); autotune = 3 tunes only that.  Results are cached per
// process and, if HJ_AUTOTUNE_CACHE names a file, in that file (one line per
// key: "key tile_x tile_y threads k overlap").
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hj_runtime.cuh"

using namespace hj;

namespace {

template <typename T>
__global__ void fill_mode_kernel(T *u, long long ld, int nx, int ny, int dim) {
    const long long n = (long long)(dim == 2 ? ny + 2 : ny) * ld;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % ld);
        const long long j = q / ld;
        double v = 0.0;
        if (i >= 1 && i <= nx) {
            const double sx = sinpi((double)i / (nx + 1));
            if (dim == 2) {
                if (j >= 1 && j <= ny) v = sx * sinpi((double)j / (ny + 1));
            } else {
                v = sx;
            }
        }
        u[q] = (T)v;
    }
}

std::mutex g_mu;
std::map<std::string, std::vector<int>> g_cache;
bool g_loaded = false;

std::string make_key(const hj_desc &d, int precision, double tol) {
    char buf[512];
    snprintf(buf, sizeof(buf), "v2_d%d_n%dx%d_p%d_c%.9g,%.9g,%.9g,%.9g,%.9g_s%.9g_sig%d_tol%.3g", d.dim, d.nx, d.ny,
             precision, d.cW, d.cE, d.cS, d.cN, d.cD, d.sigma_const, d.sigma ? 1 : 0, tol);
    return buf;
}

// One line per key: "key v0 v1 v2 v3 v4"; lines that do not parse are skipped.
void load_cache_file() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("HJ_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    char line[768], key[512];
    int v[5];
    while (fgets(line, sizeof(line), fp))
        if (sscanf(line, "%511s %d %d %d %d %d", key, &v[0], &v[1], &v[2], &v[3], &v[4]) == 6)
            g_cache[key] = {v[0], v[1], v[2], v[3], v[4]};
    fclose(fp);
}

void store_cache_file(const std::string &key, const std::vector<int> &v) {
    const char *path = getenv("HJ_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s %d %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3], v[4]);
    fclose(fp);
}

// Scratch copy of a problem in the tuned precision (same stencil and sigma).
struct Scratch {
    void *u = nullptr, *f = nullptr;
    double *sig = nullptr;
    hj_desc td;
    long long ld = 0;
    int esz = 4;
    ~Scratch() {
        if (u) dfree(u);
        if (f) dfree(f);
        if (sig) dfree(sig);
    }
    int init(const hj_desc &d, int prec) {
        esz = prec == HJ_PREC_F64 ? 8 : 4;
        ld = ((long long)d.nx + 2 + 31) / 32 * 32;
        const int rows = d.dim == 2 ? d.ny + 2 : d.ny;
        const size_t bytes = (size_t)rows * ld * esz;
        if (dmalloc(&u, bytes) != cudaSuccess || dmalloc(&f, bytes) != cudaSuccess) {
            cudaGetLastError();
            return seterr(HJ_ERR_NO_MEMORY, "autotune scratch");
        }
        td = d;
        td.ld = ld;
        td.dtype = prec == HJ_PREC_F64 ? HJ_F64 : HJ_F32;
        if (d.sigma) {
            if (dmalloc((void **)&sig, (size_t)rows * ld * 8) != cudaSuccess ||
                cudaMemcpy2D(sig, ld * 8, d.sigma, d.ld * 8, (size_t)(d.nx + 2) * 8, rows, cudaMemcpyDeviceToDevice) !=
                    cudaSuccess) {
                cudaGetLastError();
                return seterr(HJ_ERR_NO_MEMORY, "autotune sigma copy");
            }
            td.sigma = sig;
        }
        if (cudaMemset(f, 0, bytes) != cudaSuccess) return seterr(HJ_ERR_CUDA, "autotune memset");
        return HJ_OK;
    }
};

constexpr int kCyc = 128;   // cycles per measurement
constexpr int kWin = 32;    // contraction measured over the last kWin cycles

// Run kCyc cycles of (tile, threads, k) from the lowest sine mode with f = 0.
// *rho: contraction per cycle over the second half; *ms: time of the kCyc
// cycles without the closing residual pass.  fixed: time fixed cycles instead
// (no residual, no rho).
bool measure(Scratch &sc, int prec, int tx, int ty, int th, int k, const hj_params &base, double *rho, double *ms,
             int ovl = 0) {
    hj_params tp;
    hj_default_params(&tp);
    tp.tile_x = tx;
    tp.tile_y = ty;
    tp.tile_threads = th;
    tp.pipeline_stages = base.pipeline_stages;
    tp.k = k;
    tp.precision = prec;
    tp.tol = 0.0;
    tp.max_cycles = kCyc;
    tp.check_every = kCyc;
    tp.persistent = base.persistent;
    tp.pipeline = base.pipeline;
    // overlapping subdomains run on graphs of the one-CTA-per-subdomain kernels
    tp.overlap_x = ovl;
    tp.overlap_y = sc.td.dim == 2 ? ovl : 0;
    if (ovl > 0) {
        if (tp.persistent == 1) tp.persistent = -1;
        if (tp.pipeline == 1) tp.pipeline = -1;
    }
    hj_handle *h = nullptr;
    if (hj_create(&h, &sc.td, &tp) != HJ_OK) return false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double hist[kCyc + 1];
    double best = INFINITY, r = 1.0;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {   // the first run warms graphs and caches
        if (sc.esz == 8) fill_mode_kernel<double><<<256, 256>>>((double *)sc.u, sc.ld, sc.td.nx, sc.td.ny, sc.td.dim);
        else fill_mode_kernel<float><<<256, 256>>>((float *)sc.u, sc.ld, sc.td.nx, sc.td.ny, sc.td.dim);
        hj_stats st;
        memset(&st, 0, sizeof(st));
        st.history = hist;
        st.history_cap = kCyc + 1;
        cudaEventRecord(e0, 0);
        const int code = hj_solve(h, sc.f, sc.u, nullptr, &st);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        if (code != HJ_OK && code != HJ_ERR_NOT_CONVERGED) { ok = false; break; }
        float t = 0.f, tr = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        // the solve ends with one residual pass of the last iterate (it did not
        // converge at tol = 0): time it alone and subtract it
        cudaEventRecord(e0, 0);
        hj_residual(h, sc.f, sc.u, nullptr, nullptr, nullptr);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&tr, e0, e1);
        best = std::min(best, (double)std::max(t - tr, 1e-3f));
        if (st.history_len >= kCyc && hist[kCyc - 1 - kWin] > 0 && hist[kCyc - 1] > 0)
            r = pow(hist[kCyc - 1] / hist[kCyc - 1 - kWin], 1.0 / kWin);
    }
    hj_destroy(h);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    *rho = r;
    *ms = best;
    return ok && std::isfinite(best);
}

// Time per cycle of the pipelined kernel for one launch shape: threads per
// subdomain th, copy stages, CTAs per SM (0 = as many as fit); converging
// mode (fused residual, deferred fold) as a real solve runs.  Best of three
// runs after a warm-up, minus the closing residual pass.
bool measure_launch(Scratch &sc, int prec, int tx, int ty, int th, int stages, int cps, int k, double *us) {
    constexpr int kL = 48;   // cycles per run (a multiple of the pipelined graph period)
    hj_params tp;
    hj_default_params(&tp);
    tp.tile_x = tx;
    tp.tile_y = ty;
    tp.tile_threads = th;
    tp.pipeline_stages = stages;
    tp.ctas_per_sm = cps;
    tp.k = k;
    tp.precision = prec;
    tp.tol = 0.0;
    tp.max_cycles = kL;
    tp.check_every = kL;
    tp.persistent = 0;
    tp.pipeline = 1;
    hj_handle *h = nullptr;
    if (hj_create(&h, &sc.td, &tp) != HJ_OK) return false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = INFINITY;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {   // run 0 builds the graph and warms caches
        if (sc.esz == 8) fill_mode_kernel<double><<<256, 256>>>((double *)sc.u, sc.ld, sc.td.nx, sc.td.ny, sc.td.dim);
        else fill_mode_kernel<float><<<256, 256>>>((float *)sc.u, sc.ld, sc.td.nx, sc.td.ny, sc.td.dim);
        float t = 0.f, tr = 0.f;
        cudaEventRecord(e0, 0);
        const int code = hj_solve(h, sc.f, sc.u, nullptr, nullptr);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        if (code != HJ_OK && code != HJ_ERR_NOT_CONVERGED) { ok = false; break; }
        cudaEventElapsedTime(&t, e0, e1);
        cudaEventRecord(e0, 0);
        hj_residual(h, sc.f, sc.u, nullptr, nullptr, nullptr);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&tr, e0, e1);
        if (rep > 0) best = std::min(best, 1e3 * (double)std::max(t - tr, 1e-3f) / kL);
    }
    hj_destroy(h);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    *us = best;
    return ok && std::isfinite(best);
}

// Launch shape of the pipelined kernel for a fixed subdomain shape and k:
// which threads-per-subdomain variant, how many copy stages, how many CTAs per
// SM.  How many copies are in flight per SM decides how well HBM serves the
// staging pattern, and the best residency is not monotonic in the CTA count,
// so it is measured on the problem's own grid.  Leaves *p unchanged when the
// pipelined kernel would not run (1D, small grids, pipeline = 0).
int tune_launch(const hj_desc &d, hj_params *p) {
    if (d.dim != 2 || p->pipeline == 0 || p->method == HJ_METHOD_CLASSIC || p->overlap_x > 0 || p->overlap_y > 0)
        return HJ_OK;
    const bool ir = p->precision == HJ_PREC_F32_IR || p->precision == HJ_PREC_BF16CORR_IR;
    const int prec = ir ? HJ_PREC_F32 : p->precision;
    const int fam = prec == HJ_PREC_F64 ? FAM_F64 : FAM_F32;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (long long)((d.nx + p->tile_x - 1) / p->tile_x) * ((d.ny + p->tile_y - 1) / p->tile_y);
    if (p->pipeline == -1 && ntiles < 8LL * nsm) return HJ_OK;
    std::string key = make_key(d, p->precision, p->tol);
    {
        char extra[96];
        snprintf(extra, sizeof(extra), "_launch%dx%dt%dk%d", p->tile_x, p->tile_y, p->tile_threads, p->k);
        key += extra;
        std::lock_guard<std::mutex> lk(g_mu);
        load_cache_file();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            p->tile_threads = it->second[0];
            p->pipeline_stages = it->second[1];
            p->ctas_per_sm = it->second[2];
            return HJ_OK;
        }
    }
    int n = 0;
    const PpcKernelInfo *ks = fam == FAM_F64 ? ppc_kernels_f64(&n) : ppc_kernels_f32(&n);
    const bool sig = d.sigma != nullptr;
    Scratch sc;
    CKS(sc.init(d, prec));
    double best = INFINITY;
    int bth = p->tile_threads, bst = p->pipeline_stages, bcps = p->ctas_per_sm;
    for (int i = 0; i < n; ++i) {
        const PpcKernelInfo &e = ks[i];
        if (e.tx != p->tile_x || e.ty != p->tile_y) continue;
        if (p->tile_threads && e.threads != p->tile_threads) continue;
        // the same threads-per-subdomain variant must exist as a tile kernel
        int nt = 0;
        const TileKernelInfo *tk = fam == FAM_F64 ? tile_kernels_f64(&nt) : tile_kernels_f32(&nt);
        bool have = false;
        for (int j = 0; j < nt; ++j) have |= tk[j].dim == 2 && tk[j].tx == e.tx && tk[j].ty == e.ty && tk[j].threads == e.threads;
        if (!have) continue;
        PpcKernel fn = e.fn[sig][1];
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e.smem[sig]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, e.threads, e.smem[sig]) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            continue;
        }
        for (int c = occ; c >= std::max(1, occ / 2); --c) {
            double us = INFINITY;
            if (!measure_launch(sc, prec, e.tx, e.ty, e.threads, e.stages, c == occ ? 0 : c, p->k, &us)) continue;
            if (us < best) {
                best = us;
                bth = e.threads;
                bst = e.stages;
                bcps = c == occ ? 0 : c;
            }
        }
    }
    if (!std::isfinite(best)) return HJ_OK;   // nothing measurable: keep the defaults
    p->tile_threads = bth;
    p->pipeline_stages = bst;
    p->ctas_per_sm = bcps;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = {bth, bst, bcps, 0, 0};
        store_cache_file(key, g_cache[key]);
    }
    return HJ_OK;
}

}  // namespace

extern "C" int hj_autotune(const hj_desc *desc, hj_params *params, double *predicted_ms) {
    if (!desc || !params) return seterr(HJ_ERR_INVALID_ARG, "desc and params must be non-NULL");
    const hj_desc &d = *desc;
    if (d.dim != 1 && d.dim != 2) return seterr(HJ_ERR_UNSUPPORTED, "the autotuner covers 1D and 2D grids");
    if (d.coef) return seterr(HJ_ERR_UNSUPPORTED, "the autotuner covers constant neighbour coefficients");
    if (params->method == HJ_METHOD_MG) return seterr(HJ_ERR_UNSUPPORTED, "the autotuner tunes hierarchical cycles");
    if (params->autotune == 3) {
        // launch shape only: tile_x, tile_y and k are the caller's
        if (predicted_ms) *predicted_ms = -1.0;
        return tune_launch(d, params);
    }
    const bool ir = params->precision == HJ_PREC_F32_IR || params->precision == HJ_PREC_BF16CORR_IR;
    const int prec = ir ? HJ_PREC_F32 : params->precision;   // refinement: tune the binary32 inner cycles
    const double tol = ir ? params->tol : std::max(params->tol, 1e-12);
    std::string key = make_key(d, params->precision, tol);
    if (params->autotune == 2) {
        char extra[64];
        snprintf(extra, sizeof(extra), "_fixed%dx%dt%d", params->tile_x, params->tile_y, params->tile_threads);
        key += extra;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_cache_file();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            params->tile_x = it->second[0];
            params->tile_y = it->second[1];
            params->tile_threads = it->second[2];
            params->k = it->second[3];
            params->overlap_x = it->second[4];
            params->overlap_y = d.dim == 2 ? it->second[4] : 0;
            if (predicted_ms) *predicted_ms = -1.0;
            return tune_launch(d, params);
        }
    }
    Scratch sc;
    CKS(sc.init(d, prec));
    int xy[3 * 64];
    const int nshape = std::min(64, hj_tile_variants(d.dim, prec, xy, 64));
    const int ks[] = {4, 8, 16, 32, 64};
    const int os[] = {0, 2, 4, 8};   // overlapping points per side (Sections 3.4, 4.3)
    double best = INFINITY;
    int btx = params->tile_x, bty = params->tile_y, bth = params->tile_threads, bk = params->k, bo = 0;
    for (int si = 0; si < nshape; ++si) {
        const int tx = xy[3 * si], ty = xy[3 * si + 1], th = xy[3 * si + 2];
        // autotune == 2: the tile variant is fixed by the caller, tune k only
        if (params->autotune == 2 && (tx != params->tile_x || (d.dim == 2 && ty != params->tile_y) ||
                                      (params->tile_threads && th != params->tile_threads)))
            continue;
        // skip shapes far larger than the grid
        if (tx > 2 * std::max(d.nx, 32) || (d.dim == 2 && ty > 2 * std::max(d.ny, 8))) continue;
        const int tmin = d.dim == 2 ? std::min(tx, ty) : tx;
        for (int k : ks) {
            for (int o : os) {
                if (2 * o >= tmin) continue;
                double rho = 1.0, ms = INFINITY;
                if (!measure(sc, prec, tx, ty, th, k, *params, &rho, &ms, o)) continue;
                if (!(rho > 0.0 && rho < 1.0)) continue;
                const double pred = log(std::max(tol, 1e-300)) / log(rho) * (ms / kCyc);
                if (pred < best) {
                    best = pred;
                    btx = tx;
                    bty = ty;
                    bth = th;
                    bk = k;
                    bo = o;
                }
            }
        }
    }
    if (!std::isfinite(best)) return seterr(HJ_ERR_UNSUPPORTED, "autotune found no usable candidate");
    params->tile_x = btx;
    params->tile_y = d.dim == 2 ? bty : 1;
    params->tile_threads = bth;
    params->k = bk;
    params->overlap_x = bo;
    params->overlap_y = d.dim == 2 ? bo : 0;
    if (predicted_ms) *predicted_ms = best;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = {btx, bty, bth, bk, bo};
        store_cache_file(key, g_cache[key]);
    }
    return tune_launch(d, params);
}

namespace hj {

// Batched scheduler tuning.  In a batch, cycles are throughput-bound (all
// active problems share each launch), so a candidate's cost per point per
// cycle c(t, k) is measured on a throughput-sized synthetic grid, while its
// contraction rho(t, k) is measured on the largest problem of each size
// class.  The tile variant t (one per launch, persistent kernels only)
// minimises  sum_p points_p * cycles(rho_class(p)(t, k_class)) * c(t, k_class),
// with k per class chosen the same way.  cls[p] is the class of problem p.
int autotune_batched(const hj_desc *descs, int nprob, const std::vector<int> &cls, int ncls, hj_params *par,
                     std::vector<int> *kcls) {
    // per-process cache keyed by the whole batch description
    static std::mutex mu;
    static std::map<std::string, std::vector<int>> cache;
    std::string key;
    {
        char buf[128];
        snprintf(buf, sizeof(buf), "p%d_tol%.3g_a%d_t%dx%dt%d:", par->precision, par->tol, par->autotune,
                 par->tile_x, par->tile_y, par->tile_threads);
        key = buf;
        for (int i = 0; i < nprob; ++i) {
            snprintf(buf, sizeof(buf), "%dx%d,%.9g,%.9g;", descs[i].nx, descs[i].ny, descs[i].cD, descs[i].sigma_const);
            key += buf;
        }
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            par->tile_x = it->second[0];
            par->tile_y = it->second[1];
            par->tile_threads = it->second[2];
            kcls->assign(it->second.begin() + 3, it->second.end());
            return HJ_OK;
        }
    }
    const int fam = par->precision == HJ_PREC_BF16CORR_IR ? FAM_BF16 : FAM_F32;
    const int prec = HJ_PREC_F32;
    const double tol = par->tol;
    std::vector<int> rep(ncls, -1);
    std::vector<double> pts(ncls, 0.0);
    for (int i = 0; i < nprob; ++i) {
        const int c = cls[i];
        pts[c] += (double)descs[i].nx * descs[i].ny;
        if (rep[c] < 0 || (long long)descs[i].nx * descs[i].ny > (long long)descs[rep[c]].nx * descs[rep[c]].ny)
            rep[c] = i;
    }
    // throughput grid: Poisson 2048^2 with the largest problem's screening
    hj_desc big = descs[0];
    big.nx = big.ny = 2048;
    big.sigma = nullptr;
    Scratch thr;
    CKS(thr.init(big, prec));
    int xy[3 * 64];
    const int nv = std::min(64, hj_tile_variants(2, prec, xy, 64));
    const int ks[] = {4, 8, 16, 32, 64};
    const int nk = 5;
    double best = INFINITY;
    std::vector<int> bestk(ncls, par->k);
    int btx = par->tile_x, bty = par->tile_y, bth = par->tile_threads;
    std::vector<Scratch> reps(ncls);
    for (int c = 0; c < ncls; ++c)
        if (rep[c] >= 0) CKS(reps[c].init(descs[rep[c]], prec));
    hj_params thp = *par;
    thp.persistent = 0;   // fixed-cycle throughput of the tile code on a large grid
    thp.pipeline = 0;
    hj_params solo = *par;
    solo.persistent = 1;  // a problem alone: the latency floor of a persistent cycle
    for (int v = 0; v < nv; ++v) {
        const int tx = xy[3 * v], ty = xy[3 * v + 1], th = xy[3 * v + 2];
        if (!find_persist(fam, 2, tx, ty, th)) continue;
        if (par->autotune == 2 && (tx != par->tile_x || ty != par->tile_y || (par->tile_threads && th != par->tile_threads)))
            continue;
        // measured per class and k: cycles to tol and solo cycle time; per k: throughput cost per point
        std::vector<double> cyc(ncls * nk, INFINITY), tau(ncls * nk, INFINITY), theta(nk, INFINITY);
        for (int j = 0; j < nk; ++j) {
            double rho_t = 0.0, ms_thr = 0.0;
            if (measure(thr, prec, tx, ty, th, ks[j], thp, &rho_t, &ms_thr))
                theta[j] = ms_thr / kCyc / (2048.0 * 2048.0);
            for (int c = 0; c < ncls; ++c) {
                if (rep[c] < 0) continue;
                double rho = 1.0, ms = 0.0;
                if (!measure(reps[c], prec, tx, ty, th, ks[j], solo, &rho, &ms)) continue;
                if (!(rho > 0.0 && rho < 1.0)) continue;
                cyc[c * nk + j] = log(std::max(tol, 1e-300)) / log(rho);
                tau[c * nk + j] = ms / kCyc;
            }
        }
        // simulate the batch for every choice of k per class: all classes run
        // together; a cycle costs max(latency floor of the active classes,
        // active points x throughput cost); classes retire after their cycles
        std::vector<int> choice(ncls, 0);
        const int ncomb = (int)pow(nk, ncls);
        for (int comb = 0; comb < ncomb; ++comb) {
            int t = comb;
            for (int c = 0; c < ncls; ++c) { choice[c] = t % nk; t /= nk; }
            std::vector<std::pair<double, int>> ord;
            bool okc = true;
            for (int c = 0; c < ncls; ++c) {
                if (rep[c] < 0) continue;
                const double n = cyc[c * nk + choice[c]];
                if (!std::isfinite(n) || !std::isfinite(theta[choice[c]])) { okc = false; break; }
                ord.push_back({n, c});
            }
            if (!okc || ord.empty()) continue;
            std::sort(ord.begin(), ord.end());
            double total = 0.0, done = 0.0;
            for (size_t a2 = 0; a2 < ord.size(); ++a2) {
                double floor_t = 0.0, work = 0.0;
                for (size_t b2 = a2; b2 < ord.size(); ++b2) {
                    const int c = ord[b2].second;
                    floor_t = std::max(floor_t, tau[c * nk + choice[c]]);
                    work += pts[c] * theta[choice[c]];
                }
                total += (ord[a2].first - done) * std::max(floor_t, work);
                done = ord[a2].first;
            }
            if (total < best) {
                best = total;
                btx = tx;
                bty = ty;
                bth = th;
                for (int c = 0; c < ncls; ++c) bestk[c] = ks[choice[c]];
            }
        }
    }
    if (!std::isfinite(best)) return seterr(HJ_ERR_UNSUPPORTED, "batched autotune found no usable candidate");
    par->tile_x = btx;
    par->tile_y = bty;
    par->tile_threads = bth;
    *kcls = bestk;
    {
        std::vector<int> v = {btx, bty, bth};
        v.insert(v.end(), bestk.begin(), bestk.end());
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = v;
    }
    return HJ_OK;
}

}  // namespace hj
