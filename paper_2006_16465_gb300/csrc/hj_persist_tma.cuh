// hj_persist_tma.cuh -- persistent multi-cycle kernels (hj_persist.cuh) whose
// CTAs stage subdomains with TMA and prefetch: while a CTA sweeps one work
// item in registers, the copy engine brings the next item's iterate box
// (subdomain + halo), RHS box (and 1/d box) into shared memory.
//
// Same cycle structure, barriers, reductions and stopping rules as the
// plain persistent kernels; only the staging differs (TMA boxes instead of
// predicated global loads, zero fill beyond the grid either way), so the
// iterates are identical.  Each problem has tensor maps of its two iterate
// buffers, its RHS and its 1/d in device memory (PersistMaps).
//
// Ordering: within a launch, cycle c's stores (generic proxy) are read by
// cycle c+1's copies (async proxy).  Every thread fences its stores towards
// the async proxy before the grid barrier, and the thread that issues copies
// fences again after it; the barrier orders the CTAs.  Every mbarrier wait
// is bounded: on expiry the CTA records HJ_ERR_TIMEOUT, waits (bounded) for
// its copy in flight and returns; the other CTAs then leave at the barrier.
#pragma once

#include "hj_persist.cuh"
#include "hj_tma.cuh"

namespace hj {

struct PersistMaps {
    CUtensorMap mu[2];   // iterate buffers b0 (cycle even) and b1 (cycle odd), box (bwu, TY + 2)
    CUtensorMap mf;      // right-hand side, box (bwf, TY)
    CUtensorMap md;      // per-point 1/d, box (bwf, TY); sigma only
};

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ONE: single problem (one barrier per cycle, every CTA reduces all partials
// itself, as persist2d_one_kernel); else many problems (reduce, then retire).
// Batched four-warp kernels with a sigma field are held to three CTAs per SM
// (at most 168 registers instead of about 220): measured 3.5 % faster on 16
// 1024^2 sigma-field problems.  The others keep the compiler's choice (a
// minimum of 0 CTAs leaves it as without one; an explicit 1 let the compiler
// take more registers, and the constant-sigma batched kernel held to three
// CTAs was slower).
template <typename S, typename T, int C, int R, int NW, int H, bool EXACT, bool SIG, bool ONE>
__global__ void __launch_bounds__(32 * NW, (NW == 4 && SIG && !ONE) ? 3 : 0) persist2d_tma_kernel(const PersistArgs P) {
    using L = PpcLayout<S, T, C, R, NW, H, SIG, 1>;
    constexpr int TX = L::TX, TY = L::TY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t *bar = (uint64_t *)(smem + L::BAR_OFF);
    T *xbuf = (T *)(smem + L::XB_OFF);
    S *su = (S *)smem;
    T *sf = (T *)(smem + L::UB_AL);
    T *sd = (T *)(smem + L::UB_AL + L::FB_AL);
    const int tid = threadIdx.x;
    const int band = band_of_lane<R, H>();
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    OneState ls{-1, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
    unsigned nwait = 0;   // copies waited for (mbarrier phase parity)
    // cycle index of problem p (every active problem advances once per cycle)
    auto cycle_of = [&](int p) -> long long {
        if constexpr (ONE) return ls.cycle;
        else return ((volatile ProbState *)P.state + p)->cycle;
    };
    // Items: ONE walks the problem's items with a static stride; otherwise
    // the work queue hands them out (qi = queue entry, item = its number),
    // one ahead, so that the next box is in flight while the current one
    // sweeps.  An entry at or beyond the cycle's count means no more work.
    __shared__ int s_first, s_next;
    int cnt = P.nitems;
    auto take = [&](int from_static) -> int {
        if constexpr (ONE) return from_static < P.nitems ? from_static : P.nitems;
        else return atomicAdd(P.q_head, 1);
    };
    auto item_of = [&](int qi) -> int {
        if constexpr (ONE) return qi;
        else return __ldcg(P.q_items + qi);
    };
    auto issue = [&](int item) {
        const int p = P.item_prob[item];
        const PersistMaps &m = P.maps[p];
        const int blk = P.item_blk[item], tx = P.prob_tiles_x[p];
        const int bx = blk % tx, by = blk / tx;
        mbar_expect_tx(bar, L::TX_BYTES);
        tma_load_2d(su, &m.mu[cycle_of(p) & 1], bar, bx * TX, by * TY);
        tma_load_2d(sf, &m.mf, bar, bx * TX, by * TY + 1);
        if constexpr (SIG) tma_load_2d(sd, &m.md, bar, bx * TX, by * TY + 1);
    };
    if constexpr (!ONE) {
        // the queue of the first cycle is built behind a barrier
        if (!grid_barrier_queue(P)) return;
    }
    for (long long it = 0; it < P.max_iters; ++it) {
        const int parity = (int)(it & 1);
        if constexpr (!ONE) cnt = *(volatile int *)P.q_count;
        if (tid == 0) s_first = take(blockIdx.x);
        __syncthreads();
        int i = s_first;
        if (tid == 0 && i < cnt) {
            fence_proxy_async_global();
            issue(item_of(i));
        }
        while (i < cnt) {
            if (tid == 0) s_next = take(i + gridDim.x);
            bool ok = true;
            long long spins = 0;
            while (!mbar_try_wait(bar, nwait & 1u)) {
                if (++spins > P.spin_limit) { ok = false; break; }
            }
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicExch(P.err, HJ_ERR_TIMEOUT);
                    long long sp = 0;
                    while (!mbar_try_wait(bar, nwait & 1u) && ++sp <= P.spin_limit) {
                    }
                }
                __syncthreads();
                return;
            }
            ++nwait;
            const int item = item_of(i);
            if (!HJ_IN(P.probs[0].dbg, item, P.nitems, 51)) break;
            const int p = P.item_prob[item];
            CycArgs a = P.probs[p];
            if (cycle_of(p) & 1) {
                const void *t = a.uin;
                a.uin = a.uout;
                a.uout = const_cast<void *>(t);
            }
            const int blk = P.item_blk[item], tx = P.prob_tiles_x[p];
            const int x0 = 1 + (blk % tx) * TX, y0 = 1 + (blk / tx) * TY, yb = y0 + band * R;
            const Coef<T> kc = make_coef<T>(a);
            Tile2D<T, C, R, SIG> t;
            stage2d_smem<S, T, C, R, H, EXACT, SIG>(t, kc, su, sf, sd, L::BWU, L::BWF, band * R,
                                                    L::UB / (int)sizeof(S), L::FB / (int)sizeof(T), a.dbg);
            __syncthreads();   // every thread is done with the boxes (and s_next is published)
            const int nxt = s_next;
            if (tid == 0 && nxt < cnt) {
                fence_proxy_async_smem();
                issue(item_of(nxt));
            }
            typename std::conditional<EXACT, double, T>::type acc;
            if (x0 + TX - 1 <= a.nx && y0 + TY - 1 <= a.ny) {
                acc = sweeps2d<T, C, R, NW, H, EXACT, SIG, true, false>(t, kc, a.k, x0, yb, a.nx, a.ny, xbuf,
                                                                        Own{0, 0, 0, 0}, a.dbg);
                store2d<S, T, C, R, H, SIG, false>(t, a, x0, yb);
            } else {
                acc = sweeps2d<T, C, R, NW, H, EXACT, SIG, true, true>(t, kc, a.k, x0, yb, a.nx, a.ny, xbuf,
                                                                       Own{0, 0, 0, 0}, a.dbg);
                store2d<S, T, C, R, H, SIG, true>(t, a, x0, yb);
            }
            const double s = cta_sum(acc);
            const size_t pi = (size_t)parity * P.nitems + item;
            if (tid == 0 && HJ_IN(a.dbg, pi, 2 * (long long)P.nitems, 50)) P.partial[pi] = s;
            i = nxt;
        }
        fence_proxy_async_global();   // this cycle's stores, before the next cycle's copies
        if ((int)blockIdx.x == P.skip_barrier_cta) return;
        if (!grid_barrier(P)) return;
        if constexpr (ONE) {
            if (one_decide(P, ls, parity, P.nitems)) return;
        } else {
            if (threadIdx.x < 32) {
                for (int p = blockIdx.x; p < P.nprob; p += gridDim.x)
                    if (((volatile ProbState *)P.state + p)->done < 0) retire_check(P, p, parity);
            }
            if (!grid_barrier_queue(P)) return;
            if (*(volatile int *)P.active <= 0) return;
        }
    }
}

}  // namespace hj

#define HJ_KP2D(S, T, C, R, NW, H, EX)                                                                    \
    {2, 32 * (C) / (H), (R) * (NW) * (H), 32 * (NW), 1,                                                  \
     {hj::persist2d_kernel<S, T, C, R, NW, H, EX, false>, hj::persist2d_kernel<S, T, C, R, NW, H, EX, true>}, \
     {hj::persist2d_one_kernel<S, T, C, R, NW, H, EX, false>, hj::persist2d_one_kernel<S, T, C, R, NW, H, EX, true>}, \
     {hj::persist2d_tma_kernel<S, T, C, R, NW, H, EX, false, false>,                                    \
      hj::persist2d_tma_kernel<S, T, C, R, NW, H, EX, true, false>},                                    \
     {hj::persist2d_tma_kernel<S, T, C, R, NW, H, EX, false, true>,                                     \
      hj::persist2d_tma_kernel<S, T, C, R, NW, H, EX, true, true>},                                     \
     {hj::PpcLayout<S, T, C, R, NW, H, false, 1>::SMEM, hj::PpcLayout<S, T, C, R, NW, H, true, 1>::SMEM},  \
     hj::PpcLayout<S, T, C, R, NW, H, false, 1>::BWU, hj::PpcLayout<S, T, C, R, NW, H, false, 1>::BWF}
