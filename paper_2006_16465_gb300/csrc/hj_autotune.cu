// hj_autotune.cu -- picks the subdomain shape (and with it the threads per
// subdomain) and the subiteration count k for a problem by measurement.
//
// k trades on-chip work against halo staleness (Section 3.3: small k keeps the
// halos fresh, large k saves global passes), and the best value depends on the
// tile shape, the stencil and the GPU, so it is measured rather than guessed.
// For every candidate (tile, k):
//   * contraction rho per cycle: start from the lowest discrete sine mode with
//     f = 0 and zero Dirichlet data (the slowest-converging error component),
//     run C cycles and take rho = (||r_C|| / ||r_{C/2}||)^(2/C);
//   * time per cycle t: CUDA events around the same run (graph path with the
//     fused residual, as a real solve runs);
//   * predicted time to the tolerance: ln(tol) / ln(rho) * t.
// The candidate with the smallest prediction wins.  Results are cached per
// process and, if HJ_AUTOTUNE_CACHE names a file, in that file (one line per
// key: "key tile_x tile_y threads k").
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
    snprintf(buf, sizeof(buf), "d%d_n%dx%d_p%d_c%.9g,%.9g,%.9g,%.9g,%.9g_s%.9g_sig%d_tol%.3g", d.dim, d.nx, d.ny,
             precision, d.cW, d.cE, d.cS, d.cN, d.cD, d.sigma_const, d.sigma ? 1 : 0, tol);
    return buf;
}

void load_cache_file() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("HJ_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    char key[512];
    int tx, ty, th, k;
    while (fscanf(fp, "%511s %d %d %d %d", key, &tx, &ty, &th, &k) == 5) g_cache[key] = {tx, ty, th, k};
    fclose(fp);
}

void store_cache_file(const std::string &key, int tx, int ty, int th, int k) {
    const char *path = getenv("HJ_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s %d %d %d %d\n", key.c_str(), tx, ty, th, k);
    fclose(fp);
}

}  // namespace

extern "C" int hj_autotune(const hj_desc *desc, hj_params *params, double *predicted_ms) {
    if (!desc || !params) return seterr(HJ_ERR_INVALID_ARG, "desc and params must be non-NULL");
    const hj_desc &d = *desc;
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
            if (predicted_ms) *predicted_ms = -1.0;
            return HJ_OK;
        }
    }
    // scratch problem in the tuned precision, same stencil and sigma
    const int esz = prec == HJ_PREC_F64 ? 8 : 4;
    const long long ld = ((long long)d.nx + 2 + 31) / 32 * 32;
    const int rows = d.dim == 2 ? d.ny + 2 : d.ny;
    const size_t bytes = (size_t)rows * ld * esz;
    void *u = nullptr, *f = nullptr;
    double *sig = nullptr;
    auto cleanup = [&]() {
        if (u) cudaFree(u);
        if (f) cudaFree(f);
        if (sig) cudaFree(sig);
    };
    if (cudaMalloc(&u, bytes) != cudaSuccess || cudaMalloc(&f, bytes) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return seterr(HJ_ERR_NO_MEMORY, "autotune scratch");
    }
    hj_desc td = d;
    td.ld = ld;
    td.dtype = prec == HJ_PREC_F64 ? HJ_F64 : HJ_F32;
    if (d.sigma) {
        if (cudaMalloc((void **)&sig, (size_t)rows * ld * 8) != cudaSuccess ||
            cudaMemcpy2D(sig, ld * 8, d.sigma, d.ld * 8, (size_t)(d.nx + 2) * 8, rows, cudaMemcpyDeviceToDevice) !=
                cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return seterr(HJ_ERR_NO_MEMORY, "autotune sigma copy");
        }
        td.sigma = sig;
    }
    if (cudaMemset(f, 0, bytes) != cudaSuccess) {
        cleanup();
        return seterr(HJ_ERR_CUDA, "autotune memset");
    }
    // candidate (tile shape, threads per tile) variants
    int xy[3 * 64];
    const int nshape = std::min(64, hj_tile_variants(d.dim, prec, xy, 64));
    const int ks[] = {4, 8, 16, 32, 64};
    const int C = 24;
    double best = INFINITY;
    int btx = params->tile_x, bty = params->tile_y, bth = params->tile_threads, bk = params->k;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double hist[C + 1];
    for (int si = 0; si < nshape; ++si) {
        const int tx = xy[3 * si], ty = xy[3 * si + 1], th = xy[3 * si + 2];
        // autotune == 2: the tile variant is fixed by the caller, tune k only
        if (params->autotune == 2 && (tx != params->tile_x || (d.dim == 2 && ty != params->tile_y) ||
                                      (params->tile_threads && th != params->tile_threads)))
            continue;
        // skip shapes far larger than the grid
        if (tx > 2 * std::max(d.nx, 32) || (d.dim == 2 && ty > 2 * std::max(d.ny, 8))) continue;
        for (int k : ks) {
            hj_params tp;
            hj_default_params(&tp);
            tp.tile_x = tx;
            tp.tile_y = ty;
            tp.tile_threads = th;
            tp.pipeline_stages = params->pipeline_stages;
            tp.k = k;
            tp.precision = prec;
            tp.tol = 0.0;
            tp.max_cycles = C;
            tp.check_every = C;
            tp.persistent = params->persistent;
            tp.pipeline = params->pipeline;
            hj_handle *h = nullptr;
            if (hj_create(&h, &td, &tp) != HJ_OK) continue;
            double ms = INFINITY, rho = 1.0;
            for (int rep = 0; rep < 2; ++rep) {   // first run warms graphs and caches
                if (esz == 8) fill_mode_kernel<double><<<256, 256>>>((double *)u, ld, d.nx, d.ny, d.dim);
                else fill_mode_kernel<float><<<256, 256>>>((float *)u, ld, d.nx, d.ny, d.dim);
                hj_stats st;
                memset(&st, 0, sizeof(st));
                st.history = hist;
                st.history_cap = C + 1;
                cudaEventRecord(e0, 0);
                const int code = hj_solve(h, f, u, nullptr, &st);
                cudaEventRecord(e1, 0);
                cudaEventSynchronize(e1);
                if (code != HJ_OK && code != HJ_ERR_NOT_CONVERGED) break;
                float t = 0.f, tr = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                // the solve ends with one residual pass of the last iterate (it
                // did not converge at tol = 0): time it alone and subtract it
                cudaEventRecord(e0, 0);
                hj_residual(h, f, u, nullptr, nullptr, nullptr);
                cudaEventRecord(e1, 0);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&tr, e0, e1);
                ms = std::min(ms, (double)std::max(t - tr, 1e-3f));
                if (st.history_len >= C && hist[C / 2] > 0 && hist[C - 1] > 0)
                    rho = pow(hist[C - 1] / hist[C / 2], 1.0 / (C - 1 - C / 2));
            }
            hj_destroy(h);
            if (!(rho > 0.0 && rho < 1.0) || !std::isfinite(ms)) continue;
            const double pred = log(std::max(tol, 1e-300)) / log(rho) * (ms / C);
            if (pred < best) {
                best = pred;
                btx = tx;
                bty = ty;
                bth = th;
                bk = k;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    cudaGetLastError();
    if (!std::isfinite(best)) return seterr(HJ_ERR_UNSUPPORTED, "autotune found no usable candidate");
    params->tile_x = btx;
    params->tile_y = d.dim == 2 ? bty : 1;
    params->tile_threads = bth;
    params->k = bk;
    if (predicted_ms) *predicted_ms = best;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = {btx, bty, bth, bk};
        store_cache_file(key, btx, bty, bth, bk);
    }
    return HJ_OK;
}
