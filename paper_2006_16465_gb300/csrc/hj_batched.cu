// hj_batched.cu -- the persistent engine (one cooperative launch iterating many
// cycles of one or many problems) and hj_solve_batched, the batched scheduler:
// independent 2D problems of different sizes share every launch, and each
// retires on its own tolerance.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "hj_runtime.cuh"
#include "hj_persist_tma.cuh"

using namespace hj;

namespace hj {

int ensure_reduction(hj_handle *h, size_t blocks) {
    if (blocks <= h->max_blocks) return HJ_OK;
    const size_t groups = (blocks + kGroup - 1) / kGroup;
    cudaFree(h->partials);
    cudaFree(h->gpart);
    cudaFree(h->gcnt);
    h->partials = nullptr;
    h->gpart = nullptr;
    h->gcnt = nullptr;
    h->max_blocks = h->max_groups = 0;
    if (cudaMalloc((void **)&h->partials, 2 * blocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->gpart, 2 * groups * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->gcnt, groups * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return seterr(HJ_ERR_NO_MEMORY, "reduction workspace for %zu blocks", blocks);
    }
    CKR(cudaMemset(h->gcnt, 0, groups * sizeof(unsigned)));
    h->max_blocks = blocks;
    h->max_groups = groups;
    return HJ_OK;
}

int ensure_scratch(hj_handle *h, size_t bytes) {
    if (bytes <= h->pscratch_bytes) return HJ_OK;
    CKR(cudaDeviceSynchronize());
    if (h->pscratch) cudaFree(h->pscratch);
    if (h->h_pstage) cudaFreeHost(h->h_pstage);
    h->pscratch = nullptr;
    h->h_pstage = nullptr;
    h->pscratch_bytes = 0;
    if (cudaMalloc(&h->pscratch, bytes) != cudaSuccess || cudaMallocHost((void **)&h->h_pstage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return seterr(HJ_ERR_NO_MEMORY, "persistent scratch of %zu bytes", bytes);
    }
    h->pscratch_bytes = bytes;
    return HJ_OK;
}

// TMA-staged persistent kernels run unless pipeline = 0 (2D only).
bool persist_uses_tma(const hj_handle *h, const PersistKernelInfo *ki, bool sig) {
    return h->p.pipeline != 0 && ki && ki->dim == 2 && ki->tma_fn[sig] && ki->tma_one[sig];
}

namespace {
int capacity_of(hj_handle *h, const PersistKernelInfo *ki, bool sig, bool tma, int *ctas) {
    int occ = 0, occ1 = 0;
    if (tma) {
        const int smem = ki->tma_smem[sig];
        for (PersistKernel fn : {ki->tma_fn[sig], ki->tma_one[sig]})
            CKR(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki->tma_fn[sig], ki->threads, smem));
        CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, ki->tma_one[sig], ki->threads, smem));
    } else {
        CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki->fn[sig], ki->threads, 0));
        CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, ki->one[sig], ki->threads, 0));
    }
    *ctas = std::min(occ, occ1) * h->nsm;
    return HJ_OK;
}
}  // namespace

int persist_capacity(hj_handle *h, const PersistKernelInfo *ki, bool sig, int *ctas) {
    return capacity_of(h, ki, sig, persist_uses_tma(h, ki, sig), ctas);
}

namespace {
size_t al(size_t x) { return (x + 255) / 256 * 256; }

long long env_ll(const char *name, long long dflt) {
    const char *v = getenv(name);
    return v && *v ? atoll(v) : dflt;
}
}  // namespace

int run_persistent(hj_handle *h, const PersistKernelInfo *ki, bool sig, std::vector<PersistProblem> &probs,
                   cudaStream_t s, std::vector<ProbState> *out, PersistKernel classic, int fam) {
    const int nprob = (int)probs.size();
    bool tma = !classic && fam >= 0 && persist_uses_tma(h, ki, sig);
    // tensor maps of each problem's two iterate buffers, RHS and 1/d; arrays
    // the encoder rejects (alignment) run the plain-staging kernel instead
    std::vector<PersistMaps> maps;
    if (tma) {
        maps.resize(nprob);
        const int ssz = fam == FAM_F64 ? 8 : fam == FAM_BF16 ? 2 : 4;
        const int tsz = fam == FAM_F64 ? 8 : 4;
        for (int p = 0; p < nprob && tma; ++p) {
            const CycArgs &a = probs[p].a;
            PersistMaps &m = maps[p];
            memset(&m, 0, sizeof(m));
            const int cols = a.nx + 2, rows = a.ny + 2;
            tma = make_tmap(&m.mu[0], a.uin, tmap_type(fam, true), ssz, a.ld, cols, rows, ki->bwu, ki->ty + 2) &&
                  make_tmap(&m.mu[1], a.uout, tmap_type(fam, true), ssz, a.ld, cols, rows, ki->bwu, ki->ty + 2) &&
                  make_tmap(&m.mf, a.f, tmap_type(fam, false), tsz, a.ld, cols, rows, ki->bwf, ki->ty);
            if (tma && sig)
                tma = a.dinv && make_tmap(&m.md, a.dinv, tmap_type(fam, false), tsz, a.ld, cols, rows, ki->bwf, ki->ty);
        }
    }
    long long nitems = 0, max_iters = 1;
    for (auto &p : probs) {
        nitems += p.blocks;
        max_iters = std::max(max_iters, p.a.red.max_cycles + 1);
    }
    if (nitems > (1LL << 30)) return seterr(HJ_ERR_INVALID_ARG, "too many work items");
    // scratch layout
    const size_t o_probs = 0;
    const size_t o_state = al(o_probs + nprob * sizeof(CycArgs));
    const size_t o_iprob = al(o_state + nprob * sizeof(ProbState));
    const size_t o_iblk = al(o_iprob + nitems * sizeof(int));
    const size_t o_p0 = al(o_iblk + nitems * sizeof(int));
    const size_t o_pn = al(o_p0 + nprob * sizeof(int));
    const size_t o_ptx = al(o_pn + nprob * sizeof(int));
    const size_t o_part = al(o_ptx + nprob * sizeof(int));
    const size_t o_bar = al(o_part + 2 * nitems * sizeof(double));
    const size_t o_maps = al(o_bar + 4 * sizeof(unsigned));
    const size_t total = al(o_maps + (tma ? nprob * sizeof(PersistMaps) : 0));
    CKS(ensure_scratch(h, total));
    unsigned char *hb = h->h_pstage;
    unsigned char *db = (unsigned char *)h->pscratch;
    CycArgs *hp = (CycArgs *)(hb + o_probs);
    ProbState *hs = (ProbState *)(hb + o_state);
    int *hip = (int *)(hb + o_iprob), *hib = (int *)(hb + o_iblk);
    int *hp0 = (int *)(hb + o_p0), *hpn = (int *)(hb + o_pn), *hptx = (int *)(hb + o_ptx);
    long long it = 0;
    for (int p = 0; p < nprob; ++p) {
        hp[p] = probs[p].a;
        hs[p] = ProbState{-1, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
        hp0[p] = (int)it;
        hpn[p] = probs[p].blocks;
        hptx[p] = probs[p].blocks_x;
        for (int b = 0; b < probs[p].blocks; ++b, ++it) {
            hip[it] = p;
            hib[it] = b;
        }
    }
    if (tma) memcpy(hb + o_maps, maps.data(), nprob * sizeof(PersistMaps));
    unsigned *hbar = (unsigned *)(hb + o_bar);
    hbar[0] = hbar[1] = 0u;
    ((int *)hbar)[2] = nprob;   // active
    ((int *)hbar)[3] = 0;       // err
    CKR(cudaMemcpyAsync(db, hb, total, cudaMemcpyHostToDevice, s));
    PersistArgs P;
    memset(&P, 0, sizeof(P));
    P.probs = (const CycArgs *)(db + o_probs);
    P.state = (ProbState *)(db + o_state);
    P.item_prob = (const int *)(db + o_iprob);
    P.item_blk = (const int *)(db + o_iblk);
    P.prob_item0 = (const int *)(db + o_p0);
    P.prob_nitems = (const int *)(db + o_pn);
    P.prob_tiles_x = (const int *)(db + o_ptx);
    P.partial = (double *)(db + o_part);
    P.bar = (unsigned *)(db + o_bar);
    P.active = (int *)(db + o_bar) + 2;
    P.err = (int *)(db + o_bar) + 3;
    P.nprob = nprob;
    P.nitems = (int)nitems;
    P.max_iters = max_iters;
    // bounded barrier waits: 4 s by default (test hooks may shorten them and
    // make one CTA leave early, so that the timeout path runs without a fault)
    P.timeout_ns = (unsigned long long)env_ll("HJ_TEST_BARRIER_TIMEOUT_NS", 4000000000LL);
    P.skip_barrier_cta = (int)env_ll("HJ_TEST_SKIP_BARRIER_CTA", -1);
    P.maps = tma ? (const PersistMaps *)(db + o_maps) : nullptr;
    P.spin_limit = 1LL << 26;
    int cap = 0, threads = 256;
    if (classic) {
        int occ = 0;
        CKR(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, classic, 256, 0));
        cap = occ * h->nsm;
    } else {
        CKS(capacity_of(h, ki, sig, tma, &cap));
        threads = ki->threads;
    }
    if (cap < 1) return seterr(HJ_ERR_UNSUPPORTED, "persistent kernel does not fit on an SM");
    const int grid = (int)std::min<long long>(nitems, cap);
    void *args[] = {&P};
    // one problem: one grid barrier per cycle; several: two (reduce, then retire)
    const void *fn = classic ? (const void *)classic
                     : tma ? (nprob == 1 ? (const void *)ki->tma_one[sig] : (const void *)ki->tma_fn[sig])
                           : (nprob == 1 ? (const void *)ki->one[sig] : (const void *)ki->fn[sig]);
    CKR(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, tma ? ki->tma_smem[sig] : 0, s));
    CKR(cudaMemcpyAsync(hb + o_state, db + o_state, nprob * sizeof(ProbState), cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(hb + o_bar, db + o_bar, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev, s));
    CKR(cudaEventSynchronize(h->ev));
    if (((int *)hbar)[3]) return seterr(HJ_ERR_TIMEOUT, "a bounded grid-barrier wait expired");
    out->assign(hs, hs + nprob);
    for (int p = 0; p < nprob; ++p)
        if ((*out)[p].done < 0) return seterr(HJ_ERR_CUDA, "persistent launch ended with problem %d active", p);
    return HJ_OK;
}

}  // namespace hj

// ===========================================================================
// hj_solve_batched
// ===========================================================================
namespace {

struct BProb;

}  // namespace

namespace {

struct BProb {
    hj_desc d;
    int rows;
    long long ld_in;
    size_t nin;              // rows * ld_in
    const double *f;
    double *u;               // caller's iterate
    double *u2;              // second binary64 buffer
    float *r32;              // binary32 residual (inner RHS)
    void *dA, *dB;           // correction buffers
    double *cur, *other;
    float *dinv;             // per-point 1/d in binary32 (some problem of the batch has sigma)
    double r0, rn;
    bool active;
    long long inner_cycles;
};

// transpose: the adjoint operator A^T (cW <-> cE, cS <-> cN)
CycArgs prob_args(const hj_desc &d, const hj_params &p, bool transpose = false) {
    CycArgs a;
    memset(&a, 0, sizeof(a));
    a.ld = d.ld;
    a.nx = d.nx;
    a.ny = d.ny;
    a.k = p.k;
    a.cW = transpose ? d.cE : d.cW;
    a.cE = transpose ? d.cW : d.cE;
    a.cS = transpose ? d.cN : d.cS;
    a.cN = transpose ? d.cS : d.cN;
    a.dconst = d.cD + d.sigma_const;
    a.invd = 1.0 / a.dconst;
    a.fW = (float)a.cW; a.fE = (float)a.cE; a.fS = (float)a.cS; a.fN = (float)a.cN;
    a.gW = (float)(-a.cW * a.invd); a.gE = (float)(-a.cE * a.invd);
    a.gS = (float)(-a.cS * a.invd); a.gN = (float)(-a.cN * a.invd);
    a.finvd = (float)a.invd;
    a.fdconst = (float)a.dconst;
    return a;
}

int validate_desc(const hj_desc &d, int i) {
    if (d.dim != 2) return seterr(HJ_ERR_INVALID_ARG, "problem %d: batched solves are 2D", i);
    if (d.nx < 1 || d.ny < 1 || d.ny > 524280) return seterr(HJ_ERR_INVALID_ARG, "problem %d: bad size", i);
    if (d.dtype != HJ_F64) return seterr(HJ_ERR_INVALID_ARG, "problem %d: batched solves take binary64 arrays", i);
    if (d.coef) return seterr(HJ_ERR_UNSUPPORTED, "problem %d: batched solves take constant neighbour coefficients", i);
    if (d.ld < (long long)d.nx + 2 || (d.ld * 8) % 16) return seterr(HJ_ERR_INVALID_ARG, "problem %d: bad ld", i);
    if (d.sigma && ((uintptr_t)d.sigma & 15)) return seterr(HJ_ERR_INVALID_ARG, "problem %d: sigma not aligned", i);
    const double off = fabs(d.cW) + fabs(d.cE) + fabs(d.cS) + fabs(d.cN);
    double dd = d.cD + d.sigma_const;
    if (d.sigma) {
        // smallest per-point screening (read once per distinct sigma array)
        static thread_local const double *last = nullptr;
        static thread_local double last_min = 0.0;
        if (d.sigma != last) {
            std::vector<double> hs((size_t)(d.ny + 2) * d.ld);
            if (cudaMemcpy(hs.data(), d.sigma, hs.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                return seterr(HJ_ERR_CUDA, "problem %d: reading sigma", i);
            double m = INFINITY;
            for (int j = 1; j <= d.ny; ++j)
                for (int x = 1; x <= d.nx; ++x) m = std::min(m, hs[(size_t)j * d.ld + x]);
            last = d.sigma;
            last_min = m;
        }
        dd += last_min;
    }
    if (!(dd > 0.0) || dd < off) return seterr(HJ_ERR_NOT_DIAG_DOMINANT, "problem %d: not diagonally dominant", i);
    return HJ_OK;
}

}  // namespace

int batched_core(hj_handle *h, int nprob, const hj_desc *descs, const void *const *f, void *const *u,
                 hj_stream stream, hj_stats *stats, long long *cycles_out, bool transpose) {
    if (!h) return seterr(HJ_ERR_INVALID_ARG, "handle is NULL");
    if (nprob < 1 || !descs || !f || !u) return seterr(HJ_ERR_INVALID_ARG, "nprob, descs, f, u");
    if (!h->ir) return seterr(HJ_ERR_UNSUPPORTED, "batched solves use HJ_PREC_F32_IR or HJ_PREC_BF16CORR_IR");
    cudaStream_t s = (cudaStream_t)stream;
    hj_params par = h->p;
    const int fam = h->fam_inner;
    for (int i = 0; i < nprob; ++i) CKS(validate_desc(descs[i], i));
    // autotune: one tile variant for the launch and k per size class (largest
    // side up to 128, 256, 384, beyond), by the batched cost model
    std::vector<int> kprob(nprob, par.k);
    if (par.autotune == 1 || par.autotune == 2) {
        std::vector<int> cls(nprob);
        for (int i = 0; i < nprob; ++i) {
            const int m = std::max(descs[i].nx, descs[i].ny);
            cls[i] = m <= 128 ? 0 : m <= 256 ? 1 : m <= 384 ? 2 : 3;
        }
        std::vector<int> kc;
        CKS(autotune_batched(descs, nprob, cls, 4, &par, &kc));
        for (int i = 0; i < nprob; ++i) kprob[i] = kc[cls[i]];
    }
    const PersistKernelInfo *ki = find_persist(fam, 2, par.tile_x, par.tile_y, par.tile_threads);
    if (!ki) return seterr(HJ_ERR_UNSUPPORTED, "no persistent kernel for tile %dx%d", par.tile_x, par.tile_y);
    const bool bf16 = fam == FAM_BF16;
    const size_t dsz = bf16 ? 2 : 4;
    bool sig_any = false;
    for (int i = 0; i < nprob; ++i) sig_any |= descs[i].sigma != nullptr;
    std::vector<BProb> P(nprob);
    size_t arena = 0, maxaux = 0;
    for (int i = 0; i < nprob; ++i) {
        if (!f[i] || !u[i] || ((uintptr_t)f[i] & 15) || ((uintptr_t)u[i] & 15))
            return seterr(HJ_ERR_INVALID_ARG, "problem %d: f/u NULL or not 16-byte aligned", i);
        BProb &b = P[i];
        b.d = descs[i];
        b.rows = b.d.ny + 2;
        b.ld_in = ((long long)b.d.nx + 2 + 31) / 32 * 32;
        b.nin = (size_t)b.rows * b.ld_in;
        b.f = (const double *)f[i];
        b.u = (double *)u[i];
        arena += ((size_t)b.rows * b.d.ld * 8 + 255) / 256 * 256;    // u2
        arena += (b.nin * 4 + 255) / 256 * 256;                       // r32
        arena += 2 * ((b.nin * dsz + 255) / 256 * 256);               // dA, dB
        if (sig_any) arena += (b.nin * 4 + 255) / 256 * 256;          // per-point 1/d (binary32)
        maxaux = std::max(maxaux, (size_t)aux_max_blocks(2, b.d.nx, b.d.ny));
    }
    CKS(ensure_reduction(h, maxaux));
    if (arena > h->barena_bytes) {
        CKR(cudaDeviceSynchronize());
        if (h->barena) cudaFree(h->barena);
        h->barena = nullptr;
        h->barena_bytes = 0;
        if (cudaMalloc(&h->barena, arena) != cudaSuccess) {
            cudaGetLastError();
            return seterr(HJ_ERR_NO_MEMORY, "batched workspace of %zu bytes", arena);
        }
        h->barena_bytes = arena;
    }
    if (h->nrs < (size_t)nprob) {
        if (h->rs) cudaFree(h->rs);
        if (h->h_rs) cudaFreeHost(h->h_rs);
        h->rs = nullptr;
        h->h_rs = nullptr;
        h->nrs = 0;
        if (cudaMalloc((void **)&h->rs, nprob * sizeof(double)) != cudaSuccess ||
            cudaMallocHost((void **)&h->h_rs, nprob * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return seterr(HJ_ERR_NO_MEMORY, "batched norms");
        }
        h->nrs = nprob;
    }
    unsigned char *ap = (unsigned char *)h->barena;
    for (auto &b : P) {
        b.u2 = (double *)ap; ap += ((size_t)b.rows * b.d.ld * 8 + 255) / 256 * 256;
        b.r32 = (float *)ap; ap += (b.nin * 4 + 255) / 256 * 256;
        b.dA = ap; ap += (b.nin * dsz + 255) / 256 * 256;
        b.dB = ap; ap += (b.nin * dsz + 255) / 256 * 256;
        b.dinv = nullptr;
        if (sig_any) {
            b.dinv = (float *)ap; ap += (b.nin * 4 + 255) / 256 * 256;
            CKR(cudaMemsetAsync(b.dinv, 0, b.nin * 4, s));
            CKR(launch_make_dinv_box(b.d.sigma, b.d.cD + b.d.sigma_const, b.d.ld, b.ld_in, 1, b.d.ny, 1, b.d.nx,
                                     FAM_F32, b.dinv, s));
        }
        CKR(cudaMemcpyAsync(b.u2, b.u, (size_t)b.rows * b.d.ld * 8, cudaMemcpyDeviceToDevice, s));
        CKR(cudaMemsetAsync(b.r32, 0, b.nin * 4, s));
        CKR(cudaMemsetAsync(b.dB, 0, b.nin * dsz, s));
        b.cur = b.u;
        b.other = b.u2;
        b.active = true;
        b.inner_cycles = 0;
    }
    auto norms = [&](bool update, const std::vector<int> &act, const std::vector<ProbState> *st) -> int {
        for (size_t j = 0; j < act.size(); ++j) {
            BProb &b = P[act[j]];
            const CycArgs g = prob_args(b.d, par, transpose);
            RedArgs red;
            memset(&red, 0, sizeof(red));
            red.partials = h->partials; red.gpart = h->gpart; red.gcnt = h->gcnt; red.fcnt = h->fcnt;
            red.out = h->rs + act[j];
            red.mode = RED_STORE;
            red.scale = 1.0;
            if (!update) {
                CKR(launch_residual_ex(2, 1, b.f, b.cur, b.d.sigma, b.d.ld, b.ld_in, b.d.nx, b.d.ny, g.cW, g.cE,
                                       g.cS, g.cN, g.dconst, 0, b.r32, red, s));
            } else {
                const void *dsel = ((*st)[j].done & 1) ? b.dB : b.dA;
                CKR(launch_update_residual_ex(2, b.f, b.cur, dsel, bf16 ? 1 : 0, b.other, b.d.sigma, b.r32, b.d.ld,
                                              b.ld_in, b.d.nx, b.d.ny, g.cW, g.cE, g.cS, g.cN, g.dconst, red, s));
                std::swap(b.cur, b.other);
            }
        }
        CKR(cudaMemcpyAsync(h->h_rs, h->rs, nprob * sizeof(double), cudaMemcpyDeviceToHost, s));
        CKR(cudaEventRecord(h->ev, s));
        CKR(cudaEventSynchronize(h->ev));
        for (int i : act) P[i].rn = sqrt(h->h_rs[i]);
        return HJ_OK;
    };
    std::vector<int> act;
    for (int i = 0; i < nprob; ++i) act.push_back(i);
    CKS(norms(false, act, nullptr));
    for (auto &b : P) b.r0 = b.rn;
    int o = 0, status = HJ_OK;
    long long total_inner = 0;
    for (;; ++o) {
        std::vector<int> next;
        for (int i : act) {
            BProb &b = P[i];
            if (!std::isfinite(b.rn)) { status = HJ_ERR_DIVERGED; b.active = false; continue; }
            if (b.rn <= par.tol * b.r0) { b.active = false; continue; }
            next.push_back(i);
        }
        act.swap(next);
        if (act.empty()) break;
        if (o >= par.max_outer) { status = HJ_ERR_NOT_CONVERGED; break; }
        std::vector<PersistProblem> pp;
        for (int i : act) {
            BProb &b = P[i];
            CKR(cudaMemsetAsync(b.dA, 0, b.nin * dsz, s));
            PersistProblem q;
            q.a = prob_args(b.d, par, transpose);
            q.a.k = kprob[i];
            q.a.ld = b.ld_in;
            q.a.f = b.r32;
            q.a.uin = b.dA;
            q.a.uout = b.dB;
            q.a.dinv = b.dinv;
            q.a.red.tol = par.inner_tol;
            q.a.red.max_cycles = par.inner_max_cycles;
            // the per-point-diagonal kernel forms r itself; the constant-diagonal one forms (u' - u)
            q.a.red.scale = sig_any ? 1.0 : q.a.dconst * q.a.dconst;
            q.a.red.stall_window = par.inner_stall;
            q.a.red.stall_rtol = 1e-3;
            q.blocks_x = (b.d.nx + ki->tx - 1) / ki->tx;
            q.blocks = q.blocks_x * ((b.d.ny + ki->ty - 1) / ki->ty);
            pp.push_back(q);
        }
        std::vector<ProbState> st;
        CKS(run_persistent(h, ki, sig_any, pp, s, &st, nullptr, fam));
        for (size_t j = 0; j < act.size(); ++j) {
            P[act[j]].inner_cycles += st[j].done;
            total_inner += st[j].done;
        }
        CKS(norms(true, act, &st));
    }
    for (auto &b : P)
        if (b.cur != b.u) CKR(cudaMemcpyAsync(b.u, b.cur, (size_t)b.rows * b.d.ld * 8, cudaMemcpyDeviceToDevice, s));
    CKR(cudaStreamSynchronize(s));
    if (cycles_out)
        for (int i = 0; i < nprob; ++i) cycles_out[i] = P[i].inner_cycles;
    if (stats) {
        double r0 = 0, rn = 0;
        for (auto &b : P) {
            r0 = std::max(r0, b.r0 > 0 ? 1.0 : 0.0);
            rn = std::max(rn, b.r0 > 0 ? b.rn / b.r0 : 0.0);
        }
        stats->cycles = total_inner;
        stats->cycles_launched = total_inner;
        stats->inner_cycles = total_inner;
        stats->outer_steps = o;
        stats->res0 = r0;
        stats->res_final = rn;
        stats->rel_final = rn;   // worst relative residual over the batch
        stats->history_len = 0;
        stats->tile_x = ki->tx;
        stats->tile_y = ki->ty;
        stats->tile_threads = ki->threads;
        stats->k = *std::max_element(kprob.begin(), kprob.end());
        stats->persistent = 1;
    }
    if (status == HJ_ERR_DIVERGED) return seterr(HJ_ERR_DIVERGED, "a problem of the batch diverged");
    if (status == HJ_ERR_NOT_CONVERGED)
        return seterr(HJ_ERR_NOT_CONVERGED, "%zu problems not converged after %d outer steps", act.size(), o);
    return HJ_OK;
}

extern "C" int hj_solve_batched(hj_handle *h, int nprob, const hj_desc *descs, const void *const *f, void *const *u,
                                hj_stream stream, hj_stats *stats, long long *cycles_out) {
    return batched_core(h, nprob, descs, f, u, stream, stats, cycles_out, false);
}

extern "C" int hj_solve_adjoint_batched(hj_handle *h, int nrhs, const void *const *g, const void *const *u,
                                        void *const *dl_df, void *dl_dsigma, hj_stream stream, hj_stats *stats) {
    if (!h) return seterr(HJ_ERR_INVALID_ARG, "handle is NULL");
    if (nrhs < 1 || !g || !u || !dl_df) return seterr(HJ_ERR_INVALID_ARG, "nrhs, g, u, dl_df");
    if (h->d.dim != 2) return seterr(HJ_ERR_UNSUPPORTED, "batched adjoint solves are 2D");
    cudaStream_t s = (cudaStream_t)stream;
    for (int b = 0; b < nrhs; ++b) {
        if (!g[b] || !u[b] || !dl_df[b] || ((uintptr_t)g[b] & 15) || ((uintptr_t)u[b] & 15) || ((uintptr_t)dl_df[b] & 15))
            return seterr(HJ_ERR_INVALID_ARG, "rhs %d: pointers NULL or not 16-byte aligned", b);
        // lambda_0 = 0 with a zero ghost ring (homogeneous Dirichlet data of the adjoint)
        CKR(cudaMemsetAsync(dl_df[b], 0, h->grid_bytes, s));
    }
    std::vector<hj_desc> descs(nrhs, h->d);
    const int st = batched_core(h, nrhs, descs.data(), g, dl_df, stream, stats, nullptr, true);
    if (st != HJ_OK && st != HJ_ERR_NOT_CONVERGED) return st;
    if (dl_dsigma) {
        if ((uintptr_t)dl_dsigma & 15) return seterr(HJ_ERR_INVALID_ARG, "dl_dsigma not 16-byte aligned");
        CKR(cudaMemsetAsync(dl_dsigma, 0, h->grid_elems * sizeof(double), s));
        for (int b = 0; b < nrhs; ++b)
            CKR(launch_grad_sigma_ex(2, 1, dl_df[b], u[b], (double *)dl_dsigma, h->d.ld, h->d.nx, h->d.ny, 1, s));
        CKR(cudaStreamSynchronize(s));
    }
    return st;
}
