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
    dfree(h->partials);
    dfree(h->gpart);
    dfree(h->gcnt);
    h->partials = nullptr;
    h->gpart = nullptr;
    h->gcnt = nullptr;
    h->max_blocks = h->max_groups = 0;
    if (dmalloc((void **)&h->partials, 2 * blocks * sizeof(double)) != cudaSuccess ||
        dmalloc((void **)&h->gpart, 2 * groups * sizeof(double)) != cudaSuccess ||
        dmalloc((void **)&h->gcnt, groups * sizeof(unsigned)) != cudaSuccess) {
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
    if (h->pscratch) dfree(h->pscratch);
    if (h->h_pstage) cudaFreeHost(h->h_pstage);
    h->pscratch = nullptr;
    h->h_pstage = nullptr;
    h->pscratch_bytes = 0;
    if (dmalloc(&h->pscratch, bytes) != cudaSuccess || cudaMallocHost((void **)&h->h_pstage, bytes) != cudaSuccess) {
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

// One persistent launch: its arguments, staged in the handle's persistent
// scratch (pinned host copy hb, device copy db), and the kernel's shape.
struct PersistLaunch {
    PersistArgs P;
    const void *fn = nullptr;
    int grid = 0, threads = 256, smem = 0;
    unsigned char *hb = nullptr, *db = nullptr;
    size_t o_state = 0, o_bar = 0, total = 0;
};

// Lay out and upload the arguments of a persistent launch over probs: the
// per-problem cycle arguments and state, the (problem, block) items, the
// partials, the barrier words, the work queue (rebuilt by the first barrier
// of a multi-problem launch) and, for TMA staging, each problem's tensor maps.
int persist_setup(hj_handle *h, const PersistKernelInfo *ki, bool sig, std::vector<PersistProblem> &probs,
                  cudaStream_t s, PersistKernel classic, int fam, PersistLaunch *L) {
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
    const size_t o_q = al(o_bar + 4 * sizeof(unsigned));          // head, count, changed, (pad)
    const size_t o_qitems = al(o_q + 4 * sizeof(int) + 2 * sizeof(long long));
    const size_t o_qoff = al(o_qitems + nitems * sizeof(int));
    const size_t o_ppts = al(o_qoff + nprob * sizeof(int));
    const size_t o_maps = al(o_ppts + nprob * sizeof(long long));
    const size_t total = al(o_maps + (tma ? nprob * sizeof(PersistMaps) : 0));
    CKS(ensure_scratch(h, total));
    unsigned char *hb = h->h_pstage;
    unsigned char *db = (unsigned char *)h->pscratch;
    CycArgs *hp = (CycArgs *)(hb + o_probs);
    ProbState *hs = (ProbState *)(hb + o_state);
    int *hip = (int *)(hb + o_iprob), *hib = (int *)(hb + o_iblk);
    int *hp0 = (int *)(hb + o_p0), *hpn = (int *)(hb + o_pn), *hptx = (int *)(hb + o_ptx);
    long long *hpts = (long long *)(hb + o_ppts);
    long long it = 0;
    for (int p = 0; p < nprob; ++p) {
        hp[p] = probs[p].a;
        hs[p] = ProbState{-1, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
        hp0[p] = (int)it;
        hpn[p] = probs[p].blocks;
        hptx[p] = probs[p].blocks_x;
        hpts[p] = (long long)probs[p].a.nx * probs[p].a.ny;
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
    int *hq = (int *)(hb + o_q);
    hq[0] = 0;                  // head
    hq[1] = 0;                  // count
    hq[2] = 1;                  // changed: the first barrier builds the queue
    hq[3] = 0;
    CKR(cudaMemcpyAsync(db, hb, total, cudaMemcpyHostToDevice, s));
    PersistArgs &P = L->P;
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
    P.q_head = (int *)(db + o_q);
    P.q_count = (int *)(db + o_q) + 1;
    P.q_changed = (int *)(db + o_q) + 2;
    P.q_points = (long long *)(db + o_q + 4 * sizeof(int));
    P.q_items = (int *)(db + o_qitems);
    P.q_off = (int *)(db + o_qoff);
    P.prob_points = (const long long *)(db + o_ppts);
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
    L->grid = (int)std::min<long long>(nitems, cap);
    L->threads = threads;
    L->smem = tma ? ki->tma_smem[sig] : 0;
    // one problem: one grid barrier per cycle; several: two (reduce, then
    // retire and rebuild the work queue)
    L->fn = classic ? (const void *)classic
            : tma ? (nprob == 1 ? (const void *)ki->tma_one[sig] : (const void *)ki->tma_fn[sig])
                  : (nprob == 1 ? (const void *)ki->one[sig] : (const void *)ki->fn[sig]);
    L->hb = hb;
    L->db = db;
    L->o_state = o_state;
    L->o_bar = o_bar;
    L->total = total;
    return HJ_OK;
}

int persist_launch(const PersistLaunch &L, cudaStream_t s) {
    void *args[] = {const_cast<PersistArgs *>(&L.P)};
    CKR(cudaLaunchCooperativeKernel(L.fn, dim3(L.grid), dim3(L.threads), args, L.smem, s));
    return HJ_OK;
}

int run_persistent(hj_handle *h, const PersistKernelInfo *ki, bool sig, std::vector<PersistProblem> &probs,
                   cudaStream_t s, std::vector<ProbState> *out, PersistKernel classic, int fam) {
    PersistLaunch L;
    CKS(persist_setup(h, ki, sig, probs, s, classic, fam, &L));
    const int nprob = (int)probs.size();
    CKS(persist_launch(L, s));
    CKR(cudaMemcpyAsync(L.hb + L.o_state, L.db + L.o_state, nprob * sizeof(ProbState), cudaMemcpyDeviceToHost, s));
    CKR(cudaMemcpyAsync(L.hb + L.o_bar, L.db + L.o_bar, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev, s));
    CKR(cudaEventSynchronize(h->ev));
    if (((int *)(L.hb + L.o_bar))[3]) return seterr(HJ_ERR_TIMEOUT, "a bounded grid-barrier wait expired");
    const ProbState *hs = (const ProbState *)(L.hb + L.o_state);
    out->assign(hs, hs + nprob);
    for (int p = 0; p < nprob; ++p)
        if ((*out)[p].done < 0) return seterr(HJ_ERR_CUDA, "persistent launch ended with problem %d active", p);
    return HJ_OK;
}

}  // namespace hj

// ===========================================================================
// hj_solve_batched
// ===========================================================================
namespace hj {
namespace bsched {

// ---------------------------------------------------------------------------
// Device side of the refinement loop over a batch.  Every problem has binary64
// iterate buffers u[0] (the caller's) and u[1], a binary32 residual r32 (the
// inner right-hand side), two correction buffers d[0], d[1] and an outer state.
// One refinement step is, for the problems still refining:
//   zero d[0]; inner cycles A d = r32 (the persistent launch, d[0] -> d[1] ...);
//   u[cur ^ 1] = u[cur] + d, r = f - A u[cur ^ 1] (binary64), ||r||;
//   retire the problem once ||r|| <= tol ||r_0|| (or if it diverged).
// The same kernels run every step (problems that retired return at once), so
// a step is one CUDA graph.
// ---------------------------------------------------------------------------
struct BDev {
    const double *f;
    double *u[2];
    float *r32;
    void *d[2];
    const double *sigma;
    long long ld, ld_in;      // pitch of f, u, sigma; pitch of r32 and d
    int nx, ny;
    double cW, cE, cS, cN, dconst;
    int aux0, naux;           // first aux item (block of 32 x 8 interior points) and count
};

struct BOuter {
    double r0, rn;            // ||f - A u_0||, ||f - A u|| of the current iterate
    long long inner;          // inner cycles so far
    int active;               // still refining
    int cur;                  // buffer holding the iterate
    int status;               // HJ_OK / HJ_ERR_DIVERGED
    int outer;                // refinement steps taken
};

struct BatchArgs {
    const BDev *prob;
    BOuter *outer;
    ProbState *state;         // the inner engine's per-problem state
    int *inner_active;        // the inner engine's count of active problems
    int *q_changed;           // the inner engine's queue: rebuild at the next launch
    const int *aux_prob;      // per aux item: its problem
    double *aux_part;         // per aux item: its share of ||r||^2
    int *count;               // problems still refining (read by the host)
    int nprob, naux;
    double tol;
    DbgWord *dbg;             // debug builds: the index-check word
};

__device__ __forceinline__ bool aux_point(const BDev &b, int a, int &i, int &j) {
    const int bxn = (b.nx + 31) / 32;
    const int blk = a - b.aux0;
    i = 1 + (blk % bxn) * 32 + (int)threadIdx.x;
    j = 1 + (blk / bxn) * 8 + (int)threadIdx.y;
    return i <= b.nx && j <= b.ny;
}

// zero d[0] on the interior of every refining problem (the ghost ring of the
// corrections is zero from the start and never written)
template <typename DS>
__global__ void __launch_bounds__(256) batch_zero_kernel(const BatchArgs A) {
    for (int a = blockIdx.x; a < A.naux; a += gridDim.x) {
        const int p = A.aux_prob[a];
        if (!A.outer[p].active) continue;
        const BDev b = A.prob[p];
        int i, j;
        const bool pt = aux_point(b, a, i, j);
        const long long q2 = (long long)j * b.ld_in + i;
        if (pt && HJ_IN(A.dbg, q2, (long long)(b.ny + 2) * b.ld_in, 60)) ((DS *)b.d[0])[q2] = DS(0.0f);
    }
}

template <typename DS>
__device__ __forceinline__ double corr(const DS *p) { return (double)(float)*p; }

// INIT: r = f - A u[cur] for every problem; else u[cur ^ 1] = u[cur] + d and
// r = f - A u[cur ^ 1] for the refining problems (d = the inner solve's last
// buffer, by the parity of its cycle count).  r goes to r32 and each aux
// item's ||r||^2 share to aux_part (fixed order within the item).
template <typename DS, bool INIT>
__global__ void __launch_bounds__(256) batch_residual_kernel(const BatchArgs A) {
    __shared__ double s_w[8];
    for (int a = blockIdx.x; a < A.naux; a += gridDim.x) {
        const int p = A.aux_prob[a];
        const BOuter o = A.outer[p];
        if (!INIT && !o.active) continue;
        const BDev b = A.prob[p];
        int i, j;
        double rr = 0.0;
        const bool pt = aux_point(b, a, i, j);
        const long long q = (long long)j * b.ld + i, q2 = (long long)j * b.ld_in + i;
        if (pt && HJ_IN(A.dbg, q + b.ld, (long long)(b.ny + 2) * b.ld, 61) &&
            HJ_IN(A.dbg, q - b.ld, (long long)(b.ny + 2) * b.ld, 61) &&
            HJ_IN(A.dbg, q2 + b.ld_in, (long long)(b.ny + 2) * b.ld_in, 62) &&
            HJ_IN(A.dbg, q2 - b.ld_in, (long long)(b.ny + 2) * b.ld_in, 62)) {
            const double *u = b.u[o.cur];
            double uc = u[q], uW = u[q - 1], uE = u[q + 1], uS = u[q - b.ld], uN = u[q + b.ld];
            if constexpr (!INIT) {
                const DS *d = (const DS *)b.d[A.state[p].done & 1];
                uc = __dadd_rn(uc, corr(d + q2));
                uW = __dadd_rn(uW, corr(d + q2 - 1));
                uE = __dadd_rn(uE, corr(d + q2 + 1));
                uS = __dadd_rn(uS, corr(d + q2 - b.ld_in));
                uN = __dadd_rn(uN, corr(d + q2 + b.ld_in));
                b.u[o.cur ^ 1][q] = uc;
            }
            const double dg = b.sigma ? __dadd_rn(b.dconst, b.sigma[q]) : b.dconst;
            double r = fma(-dg, uc, b.f[q]);
            r = fma(-b.cW, uW, r);
            r = fma(-b.cE, uE, r);
            r = fma(-b.cS, uS, r);
            r = fma(-b.cN, uN, r);
            b.r32[q2] = (float)r;
            rr = r * r;
        }
        rr = warp_sum(rr);
        const int w = (threadIdx.y * 32 + threadIdx.x) >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) s_w[w] = rr;
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += s_w[k];
            A.aux_part[a] = t;
        }
    }
}

// One CTA: ||r|| of every refining problem (its aux shares in a fixed order),
// retirement, and the inner engine's state for the next step.
template <bool INIT>
__global__ void __launch_bounds__(1024) batch_finalize_kernel(const BatchArgs A) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int mine = 0;
    for (int p = w; p < A.nprob; p += nw) {
        BOuter o = A.outer[p];
        if (o.active) {
            const BDev &b = A.prob[p];
            double s = 0.0;
            for (int k = lane; k < b.naux; k += 32) s += A.aux_part[b.aux0 + k];
            s = warp_sum(s);
            const double rn = sqrt(s);
            if (INIT) {
                o.r0 = rn;
            } else {
                o.inner += A.state[p].done;
                o.cur ^= 1;
                o.outer += 1;
            }
            o.rn = rn;
            if (!isfinite(rn)) {
                o.status = HJ_ERR_DIVERGED;
                o.active = 0;
            } else if (rn <= A.tol * o.r0) {
                o.active = 0;
            }
        }
        if (lane == 0) {
            A.outer[p] = o;
            // the inner engine's state: refining problems start afresh,
            // the others are left out of the work queue
            ProbState &st = A.state[p];
            st = ProbState{o.active ? -1 : 0, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
            mine += o.active;
        }
    }
    __shared__ int s_n[32];
    mine = __reduce_add_sync(0xffffffffu, mine);
    if (lane == 0) s_n[w] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < nw; ++k) n += s_n[k];
        *A.count = n;
        *A.inner_active = n;
        *A.q_changed = 1;
    }
}

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
    float *dinv;             // per-point 1/d in binary32 (some problem of the batch has sigma)
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
    a.dbg = debug_word();
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

// grid-stride launch shape of the batch kernels
dim3 batch_grid(int naux, int nsm) { return dim3((unsigned)std::max(1, std::min(naux, 8 * nsm))); }

}  // namespace bsched
}  // namespace hj

using namespace hj::bsched;

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
    size_t arena = 0;
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
    }
    if (arena > h->barena_bytes) {
        CKR(cudaDeviceSynchronize());
        if (h->barena) dfree(h->barena);
        h->barena = nullptr;
        h->barena_bytes = 0;
        if (dmalloc(&h->barena, arena) != cudaSuccess) {
            cudaGetLastError();
            return seterr(HJ_ERR_NO_MEMORY, "batched workspace of %zu bytes", arena);
        }
        h->barena_bytes = arena;
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
        CKR(cudaMemsetAsync(b.dA, 0, b.nin * dsz, s));
        CKR(cudaMemsetAsync(b.dB, 0, b.nin * dsz, s));
    }
    // the inner engine over every problem of the batch (its work queue holds
    // the items of the problems still refining)
    std::vector<PersistProblem> pp(nprob);
    for (int i = 0; i < nprob; ++i) {
        BProb &b = P[i];
        PersistProblem &q = pp[i];
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
    }
    PersistLaunch L;
    CKS(persist_setup(h, ki, sig_any, pp, s, nullptr, fam, &L));
    // batch metadata: per-problem buffers, outer state, aux items, the host
    // word and the per-cycle log
    const long long logcap = (stats && (stats->cycle_ms || stats->cycle_points)) ? std::max(0LL, stats->cycle_cap) : 0;
    long long naux = 0;
    std::vector<BDev> hd(nprob);
    for (int i = 0; i < nprob; ++i) {
        const BProb &b = P[i];
        const CycArgs g = prob_args(b.d, par, transpose);
        BDev &x = hd[i];
        x.f = b.f;
        x.u[0] = b.u;
        x.u[1] = b.u2;
        x.r32 = b.r32;
        x.d[0] = b.dA;
        x.d[1] = b.dB;
        x.sigma = b.d.sigma;
        x.ld = b.d.ld;
        x.ld_in = b.ld_in;
        x.nx = b.d.nx;
        x.ny = b.d.ny;
        x.cW = g.cW; x.cE = g.cE; x.cS = g.cS; x.cN = g.cN; x.dconst = g.dconst;
        x.aux0 = (int)naux;
        x.naux = ((b.d.nx + 31) / 32) * ((b.d.ny + 7) / 8);
        naux += x.naux;
    }
    if (naux > (1LL << 30)) return seterr(HJ_ERR_INVALID_ARG, "batch too large");
    const size_t m_prob = 0;
    const size_t m_outer = al(m_prob + nprob * sizeof(BDev));
    const size_t m_auxp = al(m_outer + nprob * sizeof(BOuter));
    const size_t m_part = al(m_auxp + naux * sizeof(int));
    const size_t m_word = al(m_part + naux * sizeof(double));
    const size_t m_tlog = al(m_word + 4 * sizeof(long long));
    const size_t m_total = al(m_tlog + (logcap > 0 ? 2 * (logcap + 1) * sizeof(unsigned long long) : 0));
    if (m_total > h->bmeta_bytes) {
        CKR(cudaDeviceSynchronize());
        if (h->bmeta) dfree(h->bmeta);
        if (h->h_bmeta) cudaFreeHost(h->h_bmeta);
        h->bmeta = nullptr;
        h->h_bmeta = nullptr;
        h->bmeta_bytes = 0;
        if (dmalloc(&h->bmeta, m_total) != cudaSuccess ||
            cudaMallocHost((void **)&h->h_bmeta, m_total) != cudaSuccess) {
            cudaGetLastError();
            return seterr(HJ_ERR_NO_MEMORY, "batch metadata of %zu bytes", m_total);
        }
        h->bmeta_bytes = m_total;
    }
    unsigned char *hm = h->h_bmeta, *dm = (unsigned char *)h->bmeta;
    memcpy(hm + m_prob, hd.data(), nprob * sizeof(BDev));
    BOuter *ho = (BOuter *)(hm + m_outer);
    for (int i = 0; i < nprob; ++i) ho[i] = BOuter{0.0, 0.0, 0, 1, 0, HJ_OK, 0};
    int *hauxp = (int *)(hm + m_auxp);
    for (int i = 0; i < nprob; ++i)
        for (int a = 0; a < hd[i].naux; ++a) hauxp[hd[i].aux0 + a] = i;
    long long *hword = (long long *)(hm + m_word);
    hword[0] = hword[1] = hword[2] = hword[3] = 0;
    CKR(cudaMemcpyAsync(dm, hm, m_word + 4 * sizeof(long long), cudaMemcpyHostToDevice, s));
    if (logcap > 0) {
        L.P.tlog = (unsigned long long *)(dm + m_tlog);
        L.P.tlog_n = (long long *)(dm + m_word) + 1;
        L.P.tlog_cap = logcap + 1;
    }
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    B.prob = (const BDev *)(dm + m_prob);
    B.outer = (BOuter *)(dm + m_outer);
    B.state = L.P.state;
    B.inner_active = L.P.active;
    B.q_changed = L.P.q_changed;
    B.aux_prob = (const int *)(dm + m_auxp);
    B.aux_part = (double *)(dm + m_part);
    B.count = (int *)(dm + m_word);
    B.nprob = nprob;
    B.naux = (int)naux;
    B.tol = par.tol;
    B.dbg = debug_word();
    const dim3 bg = batch_grid((int)naux, h->nsm), bb(32, 8);
    int *hcount = (int *)hword;
    // ||r_0|| of every problem, r32 = r_0; the problems already within tol retire
    batch_residual_kernel<float, true><<<bg, bb, 0, s>>>(B);
    batch_finalize_kernel<true><<<1, 1024, 0, s>>>(B);
    CKR(cudaGetLastError());
    CKR(cudaMemcpyAsync(hcount, B.count, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev, s));
    CKR(cudaEventSynchronize(h->ev));
    // one refinement step: zero the corrections, the persistent inner launch,
    // the binary64 update and residual, the retirement decisions, the count
    auto step = [&](cudaStream_t st) -> int {
        if (bf16) batch_zero_kernel<__nv_bfloat16><<<bg, bb, 0, st>>>(B);
        else batch_zero_kernel<float><<<bg, bb, 0, st>>>(B);
        CKS(persist_launch(L, st));
        if (bf16) batch_residual_kernel<__nv_bfloat16, false><<<bg, bb, 0, st>>>(B);
        else batch_residual_kernel<float, false><<<bg, bb, 0, st>>>(B);
        batch_finalize_kernel<false><<<1, 1024, 0, st>>>(B);
        CKR(cudaGetLastError());
        CKR(cudaMemcpyAsync(hcount, B.count, sizeof(int), cudaMemcpyDeviceToHost, st));
        CKR(cudaMemcpyAsync(hcount + 1, L.P.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        return HJ_OK;
    };
    int o = 0, graphed = 0;
    hcount[1] = 0;
    cudaGraphExec_t gexec = nullptr;
    if (hcount[0] > 0) {
        // capture the step once; replay it while problems are refining
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int cs = step(h->cap);
            const cudaError_t ee = cudaStreamEndCapture(h->cap, &graph);
            if (cs == HJ_OK && ee == cudaSuccess && graph &&
                cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess)
                graphed = 1;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
        }
    }
    while (hcount[0] > 0 && o < par.max_outer) {
        if (graphed) CKR(cudaGraphLaunch(gexec, s));
        else CKS(step(s));
        CKR(cudaEventRecord(h->ev, s));
        CKR(cudaEventSynchronize(h->ev));
        ++o;
        if (hcount[1]) {
            if (gexec) cudaGraphExecDestroy(gexec);
            return seterr(HJ_ERR_TIMEOUT, "a bounded grid-barrier wait expired");
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    // results: iterates held in the second buffer go back to the caller's
    CKR(cudaMemcpyAsync(hm, dm, m_word + 4 * sizeof(long long), cudaMemcpyDeviceToHost, s));
    if (logcap > 0)
        CKR(cudaMemcpyAsync(hm + m_tlog, dm + m_tlog, 2 * (logcap + 1) * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
    CKR(cudaEventRecord(h->ev, s));
    CKR(cudaEventSynchronize(h->ev));
    int status = HJ_OK, left = 0;
    long long total_inner = 0;
    double worst = 0.0, any_r0 = 0.0;
    for (int i = 0; i < nprob; ++i) {
        const BOuter &x = ho[i];
        if (x.r0 > 0) any_r0 = 1.0;
        if (x.cur) CKR(cudaMemcpyAsync(P[i].u, P[i].u2, (size_t)P[i].rows * P[i].d.ld * 8, cudaMemcpyDeviceToDevice, s));
        if (x.status == HJ_ERR_DIVERGED) status = HJ_ERR_DIVERGED;
        left += x.active;
        total_inner += x.inner;
        worst = std::max(worst, x.r0 > 0 ? x.rn / x.r0 : 0.0);
        if (cycles_out) cycles_out[i] = x.inner;
    }
    if (status == HJ_OK && left > 0) status = HJ_ERR_NOT_CONVERGED;
    CKR(cudaStreamSynchronize(s));
    if (stats) {
        stats->cycles = total_inner;
        stats->cycles_launched = total_inner;
        stats->inner_cycles = total_inner;
        stats->outer_steps = o;
        stats->res0 = any_r0;
        stats->res_final = worst;
        stats->rel_final = worst;   // worst relative residual over the batch
        stats->history_len = 0;
        stats->tile_x = ki->tx;
        stats->tile_y = ki->ty;
        stats->tile_threads = ki->threads;
        stats->k = *std::max_element(kprob.begin(), kprob.end());
        stats->persistent = 1;
        stats->graphed = graphed;
        stats->cycle_len = 0;
        if (logcap > 0) {
            // entry n: the time a barrier released (a launch's first barrier, or
            // the one ending a batch cycle) and the points active in the cycle
            // that follows it; a launch's last entry has none active, and the
            // interval after it (the binary64 step between launches) is skipped
            const unsigned long long *tl = (const unsigned long long *)(hm + m_tlog);
            const long long nlog = std::min<long long>(hword[1], logcap + 1);
            long long out = 0;
            for (long long n = 0; n + 1 < nlog && out < logcap; ++n) {
                if (tl[2 * n + 1] == 0) continue;
                const double ms = (double)(tl[2 * (n + 1)] - tl[2 * n]) * 1e-6;
                if (stats->cycle_ms) stats->cycle_ms[out] = ms;
                if (stats->cycle_points) stats->cycle_points[out] = (long long)tl[2 * n + 1];
                ++out;
            }
            stats->cycle_len = out;
        }
    }
    if (status == HJ_ERR_DIVERGED) return seterr(HJ_ERR_DIVERGED, "a problem of the batch diverged");
    if (status == HJ_ERR_NOT_CONVERGED)
        return seterr(HJ_ERR_NOT_CONVERGED, "%d problems not converged after %d outer steps", left, o);
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
