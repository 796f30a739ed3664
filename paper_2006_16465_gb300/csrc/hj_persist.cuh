// hj_persist.cuh -- persistent multi-cycle kernel: one cooperative launch runs
// the cycles of one or many problems until each meets its tolerance.
//
// Work items are (problem, block) pairs, numbered problem by problem.  With
// many problems (the batched scheduler) the CTAs are fed by a device work
// queue: a compacted list of the items of the problems still active, handed
// out by an atomic head, so a CTA never visits an item of a retired problem
// and uneven item costs balance themselves.  A cycle is:
//   phase A  CTAs take items from the queue; each runs one hierarchical cycle
//            of its tile (stage u_c + halo, k subiterations, write u_{c+1})
//            and stores its share of ||f - A u_c||^2 under the item's own
//            number (so the sums below do not depend on which CTA ran it);
//   barrier  (grid-wide, bounded)
//   phase B  CTA b reduces problems b, b + G, ... in a fixed order, records
//            ||r_c||, and retires the problem when it meets its tolerance
//            (its iterate u_c is still intact in buffer c mod 2), diverges, or
//            reaches its cycle cap;
//   barrier  (grid-wide, bounded): the last CTA to arrive rebuilds the queue
//            if a problem retired, resets its head and logs the cycle's end
//            time; stop when no problem is active.
// Problems of different sizes, stencils, k and tolerances share the launch.
// Single-problem launches keep a static stride over the problem's items.
// Every barrier wait is bounded by wall time (%globaltimer); on expiry the
// kernel records HJ_ERR_TIMEOUT in the error word and every CTA returns.
#pragma once

#include "hj_cycle.cuh"

namespace hj {

struct ProbState {
    int done;           // -1 while active; else index of the returned iterate
    int status;         // HJ_OK / HJ_ERR_DIVERGED / HJ_ERR_NOT_CONVERGED
    long long cycle;    // cycles completed
    double res2_0;      // ||r_0||^2
    double res2_last;   // ||r_c||^2 of the last reduced cycle
    double res2_mark;   // stagnation rule state
    long long mark_cycle;
};

struct PersistMaps;   // hj_persist_tma.cuh: per-problem tensor maps

struct PersistArgs {
    const CycArgs *probs;    // per problem: f, b0 (=uin), b1 (=uout), dinv, geometry, k, coefficients,
                             // red.tol, red.max_cycles, red.scale
    ProbState *state;        // per problem
    const int *item_prob;    // per item: problem index
    const int *item_blk;     // per item: block index within the problem (bx + tiles_x * by)
    const int *prob_item0;   // per problem: first item index (items of a problem are contiguous)
    const int *prob_nitems;  // per problem: number of items
    const int *prob_tiles_x; // per problem: blocks along x
    double *partial;         // [2][nitems]
    unsigned *bar;           // [0] arrival count, [1] generation (zero before launch)
    int *active;             // number of active problems (set before launch)
    int *err;                // error word
    int nprob, nitems;
    long long max_iters;     // cap on cycles in this launch
    unsigned long long timeout_ns;
    int skip_barrier_cta;    // test hook: this CTA leaves before the first barrier (-1 = none)
    const PersistMaps *maps; // per problem (TMA-staging kernels only)
    long long spin_limit;    // polls of an mbarrier before giving up (TMA-staging kernels)
    // work queue of the multi-problem kernels
    int *q_head;             // next queue entry to hand out this cycle
    int *q_items;            // [nitems] item numbers of the active problems, problem by problem
    int *q_count;            // entries in q_items
    int *q_changed;          // a problem retired: rebuild before the next cycle
    int *q_off;              // [nprob] scratch of the rebuild: first entry of each problem, -1 if retired
    const long long *prob_points;   // per problem: interior points
    long long *q_points;     // interior points of the active problems
    // per-cycle log (nullable): [2 * n] = end time (ns), [2 * n + 1] = active points of the next cycle
    unsigned long long *tlog;
    long long *tlog_n;
    long long tlog_cap;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Returns
// false if the wait expired or another CTA already recorded an error.
__device__ __forceinline__ bool grid_barrier(const PersistArgs &P) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = P.bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(P.bar, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(P.bar, 0u);
            __threadfence();
            atomicAdd(P.bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == gen) {
                if (*(volatile int *)P.err) { ok = 0; break; }
                if (global_ns() - t0 > P.timeout_ns) {
                    atomicExch(P.err, HJ_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && (*(volatile int *)P.err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// Rebuild the work queue from the problems still active (whole CTA; run by
// the last CTA to reach a grid barrier while the others wait in it), reset
// the head and log the time.  Problems keep their order and each problem's
// items stay contiguous, so consecutive CTAs take neighbouring subdomains.
__device__ __forceinline__ void queue_rebuild(const PersistArgs &P) {
    // every thread takes the same branch: the flag is read once, before warp 0 clears it
    __shared__ int s_changed;
    if (threadIdx.x == 0) s_changed = *(volatile int *)P.q_changed;
    __syncthreads();
    if (s_changed) {
        const int lane = threadIdx.x & 31;
        if (threadIdx.x < 32) {
            int base = 0;
            long long pts = 0;
            for (int p0 = 0; p0 < P.nprob; p0 += 32) {
                const int p = p0 + lane;
                const bool act = p < P.nprob && ((volatile ProbState *)P.state + p)->done < 0;
                const int n = act ? P.prob_nitems[p] : 0;
                int x = n;   // inclusive scan over the warp
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (p < P.nprob) P.q_off[p] = act ? base + x - n : -1;
                double dp = act ? (double)P.prob_points[p] : 0.0;
                pts += (long long)warp_sum(dp);
                base += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) {
                *P.q_count = base;
                *P.q_points = pts;
                *(volatile int *)P.q_changed = 0;
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < P.nprob; p += blockDim.x) {
            const int off = P.q_off[p];
            if (off < 0) continue;
            const int i0 = P.prob_item0[p], n = P.prob_nitems[p];
            for (int b = 0; b < n; ++b) P.q_items[off + b] = i0 + b;
        }
    }
    if (threadIdx.x == 0) {
        *P.q_head = 0;
        if (P.tlog) {
            const long long n = *P.tlog_n;
            if (n < P.tlog_cap) {
                P.tlog[2 * n] = global_ns();
                P.tlog[2 * n + 1] = (unsigned long long)*P.q_points;
            }
            *P.tlog_n = n + 1;
        }
    }
}

// Grid barrier whose last CTA to arrive rebuilds the work queue before it
// releases the others (same bounded waits and error word as grid_barrier).
__device__ __forceinline__ bool grid_barrier_queue(const PersistArgs &P) {
    __syncthreads();
    __shared__ int s_last, s_ok;
    __shared__ unsigned s_gen;
    if (threadIdx.x == 0) {
        s_gen = *(volatile unsigned *)(P.bar + 1);
        __threadfence();
        s_last = atomicAdd(P.bar, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    int ok = 1;
    if (s_last) {
        __threadfence();
        queue_rebuild(P);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(P.bar, 0u);
            __threadfence();
            atomicAdd(P.bar + 1, 1u);
        }
    } else if (threadIdx.x == 0) {
        volatile unsigned *vgen = P.bar + 1;
        const unsigned long long t0 = global_ns();
        while (*vgen == s_gen) {
            if (*(volatile int *)P.err) { ok = 0; break; }
            if (global_ns() - t0 > P.timeout_ns) {
                atomicExch(P.err, HJ_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_ok = ok && (*(volatile int *)P.err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename A>
__device__ __forceinline__ double cta_sum(A acc) {
    __shared__ double s_w[32];
    double v;
    if constexpr (std::is_same<A, float>::value) v = (double)warp_sum_f(acc);
    else v = warp_sum(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += s_w[i];
    return s;
}

// Phase B for problem p (run by warp 0 of one CTA).
__device__ __forceinline__ void retire_check(const PersistArgs &P, int p, int parity) {
    const int lane = threadIdx.x & 31;
    const int i0 = P.prob_item0[p], n = P.prob_nitems[p];
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += __ldcg(&P.partial[(size_t)parity * P.nitems + i0 + i]);
    s = warp_sum(s);
    if (lane == 0) {
        volatile ProbState *st = P.state + p;
        const RedArgs &r = P.probs[p].red;
        const double res2 = s * r.scale;
        const long long c = st->cycle;
        if (r.hist) r.hist[c & (kHistCap - 1)] = res2;
        if (c == 0) st->res2_0 = res2;
        const double r0 = sqrt(c == 0 ? res2 : st->res2_0);
        const double rc = sqrt(res2);
        st->res2_last = res2;
        int retire = 1;
        if (!isfinite(rc)) {
            st->status = HJ_ERR_DIVERGED;
            st->done = (int)c;
        } else if (rc <= r.tol * r0) {
            st->done = (int)c;
        } else if (stalled(r, c, res2, &st->res2_mark, &st->mark_cycle)) {
            st->done = (int)c;
        } else if (c + 1 >= r.max_cycles) {
            st->status = HJ_ERR_NOT_CONVERGED;
            st->done = (int)(c + 1);
        } else {
            retire = 0;
        }
        st->cycle = c + 1;
        if (retire) {
            atomicSub(P.active, 1);
            if (P.q_changed) *(volatile int *)P.q_changed = 1;
        }
    }
}

template <typename S, typename T, int C, int R, int NW, int H, bool EXACT, bool SIG>
__global__ void __launch_bounds__(32 * NW) persist2d_kernel(const PersistArgs P) {
    constexpr int TX = 32 * C / H, TY = R * NW * H;
    constexpr int XB = NW > 1 ? 2 * NW * 2 * TX : 1;
    __shared__ T xbuf[XB];
    __shared__ int s_take;
    // the queue of the first cycle is built behind a barrier
    if (!grid_barrier_queue(P)) return;
    for (long long it = 0; it < P.max_iters; ++it) {
        const int parity = (int)(it & 1);
        const int cnt = *(volatile int *)P.q_count;
        for (;;) {
            if (threadIdx.x == 0) s_take = atomicAdd(P.q_head, 1);
            __syncthreads();
            const int qi = s_take;
            if (qi >= cnt) break;
            const int item = __ldcg(P.q_items + qi);
            if (!HJ_IN(P.probs[0].dbg, item, P.nitems, 51)) break;
            const int p = P.item_prob[item];
            CycArgs a = P.probs[p];
            volatile ProbState *st = P.state + p;
            if (st->cycle & 1) {
                const void *t = a.uin;
                a.uin = a.uout;
                a.uout = const_cast<void *>(t);
            }
            const int blk = P.item_blk[item], tx = P.prob_tiles_x[p];
            const int x0 = 1 + (blk % tx) * TX, y0 = 1 + (blk / tx) * TY;
            typename std::conditional<EXACT, double, T>::type acc;
            if (x0 + TX - 1 <= a.nx && y0 + TY - 1 <= a.ny)
                acc = tile2d<S, T, C, R, NW, H, EXACT, SIG, true, false>(a, x0, y0, xbuf);
            else
                acc = tile2d<S, T, C, R, NW, H, EXACT, SIG, true, true>(a, x0, y0, xbuf);
            const double s = cta_sum(acc);
            if (threadIdx.x == 0) P.partial[(size_t)parity * P.nitems + item] = s;
        }
        if ((int)blockIdx.x == P.skip_barrier_cta) return;
        if (!grid_barrier(P)) return;
        if (threadIdx.x < 32) {
            for (int p = blockIdx.x; p < P.nprob; p += gridDim.x)
                if (((volatile ProbState *)P.state + p)->done < 0) retire_check(P, p, parity);
        }
        if (!grid_barrier_queue(P)) return;
        if (*(volatile int *)P.active <= 0) return;
    }
}

template <typename S, typename T, int C, int WPT, int WPB, bool EXACT, bool SIG>
__global__ void __launch_bounds__(32 * WPT * WPB) persist1d_kernel(const PersistArgs P) {
    constexpr int TX = 32 * C * WPT;
    __shared__ Xchg1D<T, WPT> xb;
    for (long long it = 0; it < P.max_iters; ++it) {
        const int parity = (int)(it & 1);
        for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
            const int p = P.item_prob[item];
            volatile ProbState *st = P.state + p;
            if (st->done >= 0) continue;
            CycArgs a = P.probs[p];
            if (st->cycle & 1) {
                const void *t = a.uin;
                a.uin = a.uout;
                a.uout = const_cast<void *>(t);
            }
            const int blk = P.item_blk[item], bxn = P.prob_tiles_x[p];
            const int x0 = 1 + ((blk % bxn) * WPB + (int)(threadIdx.x >> 5) / WPT) * TX;
            const int row = blk / bxn;
            typename std::conditional<EXACT, double, T>::type acc = 0;
            if (x0 <= a.nx) {
                if (x0 + TX - 1 <= a.nx) acc = tile1d<S, T, C, WPT, EXACT, SIG, true, false>(a, x0, row, xb);
                else acc = tile1d<S, T, C, WPT, EXACT, SIG, true, true>(a, x0, row, xb);
            }
            const double s = cta_sum(acc);
            if (threadIdx.x == 0) P.partial[(size_t)parity * P.nitems + item] = s;
        }
        if ((int)blockIdx.x == P.skip_barrier_cta) return;
        if (!grid_barrier(P)) return;
        if (threadIdx.x < 32) {
            for (int p = blockIdx.x; p < P.nprob; p += gridDim.x)
                if (((volatile ProbState *)P.state + p)->done < 0) retire_check(P, p, parity);
        }
        if (!grid_barrier(P)) return;
        if (*(volatile int *)P.active <= 0) return;
    }
}

// Single-problem variant with ONE grid barrier per cycle: after the barrier
// every CTA sums all partials of the cycle in the same fixed order, so every
// CTA reaches the same stopping decision on its own; CTA 0 publishes the
// state and the residual history.  Partials are double-buffered by cycle
// parity, so a CTA that runs ahead cannot overwrite values another CTA is
// still summing.
struct OneState {
    int done, status;
    long long cycle;
    double res2_0, res2_last, mark;
    long long mark_c;
};

// count: partials written per cycle (one per item, or one per CTA)
__device__ __forceinline__ bool one_decide(const PersistArgs &P, OneState &ls, int parity, int count) {
    const int lane = threadIdx.x & 31;
    __shared__ OneState s_ls;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = lane; i < count; i += 32) s += __ldcg(&P.partial[(size_t)parity * P.nitems + i]);
        s = warp_sum(s);
        if (lane == 0) {
            const RedArgs &r = P.probs[0].red;
            const double res2 = s * r.scale;
            const long long c = ls.cycle;
            if (blockIdx.x == 0 && r.hist) r.hist[c & (kHistCap - 1)] = res2;
            if (c == 0) ls.res2_0 = res2;
            const double r0 = sqrt(ls.res2_0), rc = sqrt(res2);
            ls.res2_last = res2;
            if (!isfinite(rc)) {
                ls.status = HJ_ERR_DIVERGED;
                ls.done = (int)c;
            } else if (rc <= r.tol * r0) {
                ls.done = (int)c;
            } else if (stalled(r, c, res2, &ls.mark, &ls.mark_c)) {
                ls.done = (int)c;
            } else if (c + 1 >= r.max_cycles) {
                ls.status = HJ_ERR_NOT_CONVERGED;
                ls.done = (int)(c + 1);
            }
            ls.cycle = c + 1;
            s_ls = ls;
            if (blockIdx.x == 0 && ls.done >= 0) {
                ProbState *st = P.state;
                st->status = ls.status;
                st->cycle = ls.cycle;
                st->res2_0 = ls.res2_0;
                st->res2_last = ls.res2_last;
                __threadfence();
                st->done = ls.done;
            }
        }
    }
    __syncthreads();
    ls = s_ls;
    return ls.done >= 0;
}

template <typename S, typename T, int C, int R, int NW, int H, bool EXACT, bool SIG>
__global__ void __launch_bounds__(32 * NW) persist2d_one_kernel(const PersistArgs P) {
    constexpr int TX = 32 * C / H, TY = R * NW * H;
    constexpr int XB = NW > 1 ? 2 * NW * 2 * TX : 1;
    __shared__ T xbuf[XB];
    OneState ls{-1, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
    const int tx = P.prob_tiles_x[0];
    for (long long it = 0; it < P.max_iters; ++it) {
        const int parity = (int)(it & 1);
        CycArgs a = P.probs[0];
        if (ls.cycle & 1) {
            const void *t = a.uin;
            a.uin = a.uout;
            a.uout = const_cast<void *>(t);
        }
        for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
            const int x0 = 1 + (item % tx) * TX, y0 = 1 + (item / tx) * TY;
            typename std::conditional<EXACT, double, T>::type acc;
            if (x0 + TX - 1 <= a.nx && y0 + TY - 1 <= a.ny)
                acc = tile2d<S, T, C, R, NW, H, EXACT, SIG, true, false>(a, x0, y0, xbuf);
            else
                acc = tile2d<S, T, C, R, NW, H, EXACT, SIG, true, true>(a, x0, y0, xbuf);
            const double s = cta_sum(acc);
            if (threadIdx.x == 0) P.partial[(size_t)parity * P.nitems + item] = s;
        }
        if ((int)blockIdx.x == P.skip_barrier_cta) return;
        if (!grid_barrier(P)) return;
        if (one_decide(P, ls, parity, P.nitems)) return;
    }
}

template <typename S, typename T, int C, int WPT, int WPB, bool EXACT, bool SIG>
__global__ void __launch_bounds__(32 * WPT * WPB) persist1d_one_kernel(const PersistArgs P) {
    constexpr int TX = 32 * C * WPT;
    __shared__ Xchg1D<T, WPT> xb;
    OneState ls{-1, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
    const int bxn = P.prob_tiles_x[0];
    for (long long it = 0; it < P.max_iters; ++it) {
        const int parity = (int)(it & 1);
        CycArgs a = P.probs[0];
        if (ls.cycle & 1) {
            const void *t = a.uin;
            a.uin = a.uout;
            a.uout = const_cast<void *>(t);
        }
        for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
            const int x0 = 1 + ((item % bxn) * WPB + (int)(threadIdx.x >> 5) / WPT) * TX;
            const int row = item / bxn;
            typename std::conditional<EXACT, double, T>::type acc = 0;
            if (x0 <= a.nx) {
                if (x0 + TX - 1 <= a.nx) acc = tile1d<S, T, C, WPT, EXACT, SIG, true, false>(a, x0, row, xb);
                else acc = tile1d<S, T, C, WPT, EXACT, SIG, true, true>(a, x0, row, xb);
            }
            const double s = cta_sum(acc);
            if (threadIdx.x == 0) P.partial[(size_t)parity * P.nitems + item] = s;
        }
        if ((int)blockIdx.x == P.skip_barrier_cta) return;
        if (!grid_barrier(P)) return;
        if (one_decide(P, ls, parity, P.nitems)) return;
    }
}

// Classic global-memory Jacobi (Section 3.2) as one persistent launch for a
// single problem: every grid-wide sweep is one cycle of the loop above, with
// a grid barrier between sweeps instead of a kernel boundary (the grid-sync
// variant of the classic baseline).  Items are blocks of 32 x 8 points (2D)
// or 256 points of one row (1D), one thread per point.
template <typename S, typename T, int D, bool EXACT, bool SIG>
__device__ __forceinline__ typename std::conditional<EXACT, double, T>::type classic_block(const CycArgs &a,
                                                                                           int item) {
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    const Coef<T> kc = make_coef<T>(a);
    const S *__restrict__ uin = (const S *)a.uin;
    int i, j;
    if constexpr (D == 2) {
        const int bxn = (a.nx + 31) / 32;
        i = 1 + (item % bxn) * 32 + (threadIdx.x & 31);
        j = 1 + (item / bxn) * 8 + (threadIdx.x >> 5);
        if (i > a.nx || j > a.ny) return acc;
    } else {
        const int bxn = (a.nx + 255) / 256;
        i = 1 + (item % bxn) * 256 + threadIdx.x;
        j = item / bxn;
        if (i > a.nx) return acc;
    }
    const long long q = (long long)j * a.ld + i;
    const T old = ld_s<S, T>(uin + q);
    const T W = ld_s<S, T>(uin + q - 1), E = ld_s<S, T>(uin + q + 1);
    const T Sv = D == 2 ? ld_s<S, T>(uin + q - a.ld) : (T)0, Nv = D == 2 ? ld_s<S, T>(uin + q + a.ld) : (T)0;
    const T fv = __ldg((const T *)a.f + q);
    const T iv = SIG ? __ldg((const T *)a.dinv + q) : (T)0;
    const T g = (EXACT || SIG) ? fv : fv * kc.invd;
    T res = 0;
    const T nv = point_update<T, EXACT, SIG, D == 2, true>(kc, g, iv, W, E, Sv, Nv, old, res);
    st_s<S, T>((S *)a.uout + q, nv);
    return (Acc)res * (Acc)res;
}

template <typename S, typename T, int D, bool EXACT, bool SIG>
__global__ void __launch_bounds__(256) persist_classic_one_kernel(const PersistArgs P) {
    OneState ls{-1, HJ_OK, 0, 0.0, 0.0, 0.0, 0};
    for (long long it = 0; it < P.max_iters; ++it) {
        const int parity = (int)(it & 1);
        CycArgs a = P.probs[0];
        if (ls.cycle & 1) {
            const void *t = a.uin;
            a.uin = a.uout;
            a.uout = const_cast<void *>(t);
        }
        typename std::conditional<EXACT, double, T>::type acc = 0;
        for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) acc += classic_block<S, T, D, EXACT, SIG>(a, item);
        const double s = cta_sum(acc);
        if (threadIdx.x == 0) P.partial[(size_t)parity * P.nitems + blockIdx.x] = s;
        if ((int)blockIdx.x == P.skip_barrier_cta) return;
        if (!grid_barrier(P)) return;
        if (one_decide(P, ls, parity, gridDim.x)) return;
    }
}

typedef void (*PersistKernel)(PersistArgs);

struct PersistKernelInfo {
    int dim, tx, ty, threads, tiles_per_cta;
    PersistKernel fn[2];      // [sig]  many problems, two barriers per cycle
    PersistKernel one[2];     // [sig]  one problem, one barrier per cycle
    // TMA-staged variants (2D; null otherwise) and their dynamic shared memory
    PersistKernel tma_fn[2], tma_one[2];
    int tma_smem[2];
    int bwu, bwf;             // box widths (elements) of the iterate / RHS boxes
};

// Grid-sync classic baseline, one problem ([dim - 1][sig]).
struct PersistClassicInfo {
    PersistKernel fn[2][2];
};

}  // namespace hj

#define HJ_KPC(S, T, EX) \
    {{{hj::persist_classic_one_kernel<S, T, 1, EX, false>, hj::persist_classic_one_kernel<S, T, 1, EX, true>}, \
      {hj::persist_classic_one_kernel<S, T, 2, EX, false>, hj::persist_classic_one_kernel<S, T, 2, EX, true>}}}
#define HJ_KP1D(S, T, C, WPT, WPB, EX) \
    {1, 32 * (C) * (WPT), 1, 32 * (WPT) * (WPB), (WPB), \
     {hj::persist1d_kernel<S, T, C, WPT, WPB, EX, false>, hj::persist1d_kernel<S, T, C, WPT, WPB, EX, true>}, \
     {hj::persist1d_one_kernel<S, T, C, WPT, WPB, EX, false>, hj::persist1d_one_kernel<S, T, C, WPT, WPB, EX, true>}, \
     {nullptr, nullptr}, {nullptr, nullptr}, {0, 0}, 0, 0}
