// hj_tma.cuh -- TMA-pipelined cycle kernel for grids much larger than the
// number of resident CTAs.
//
// One CTA per resident slot walks a static list of tiles (t = blockIdx.x +
// i * gridDim.x, row-major so that neighbouring tiles run together and halo
// re-reads hit L2).  A single thread issues cp.async.bulk.tensor copies of the
// next NST tiles' iterate box (tile + halo) and RHS box into shared memory,
// completing on an mbarrier, while the warps sweep the current tile in
// registers; the interior goes back to HBM with plain coalesced stores from
// registers.  The residual of the whole CTA's tiles becomes one partial per
// CTA, folded by the next launch (no atomics or fences at the kernel's end).
// Every wait on an mbarrier is bounded; on expiry the kernel records the
// error in the control block, drains its own copies (bounded) and returns.
#pragma once

#include <cuda.h>

#include "hj_cycle.cuh"

namespace hj {

struct PpcArgs {
    CUtensorMap mu;   // iterate u_c (storage type), box (bwu, TY + 2)
    CUtensorMap mf;   // right-hand side (compute type), box (bwf, TY)
    CUtensorMap md;   // per-point 1/d (compute type), box (bwf, TY); sigma only
    CycArgs a;
    int tiles_x, ntiles;
    int tiles_y;            // 3D kernel: subdomains along y (the tile index is x fastest, then y, then z)
    long long spin_limit;   // polls of an mbarrier before giving up
    // Fused residual (deferred fold): this launch writes one partial of
    // ||f - A u_c||^2 per CTA into part_w; the last CTA of the next launch
    // folds them (part_r there) into the control block.  parity = launch
    // index mod 2 selects the launch's fold_only flag.
    double *part_w;
    const double *part_r;
    int parity;
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <typename S, typename T, int C, int R, int NW, int H, bool SIG, int NST>
struct PpcLayout {
    static constexpr int TX = 32 * C / H, TY = R * NW * H;
    static constexpr int BWU = round_up(TX + 2, 16 / (int)sizeof(S));   // box width, 16-byte multiple
    static constexpr int BWF = round_up(TX + 2, 16 / (int)sizeof(T));
    static constexpr int UB = BWU * (TY + 2) * (int)sizeof(S);
    static constexpr int FB = BWF * TY * (int)sizeof(T);
    static constexpr int UB_AL = round_up(UB, 128), FB_AL = round_up(FB, 128);
    static constexpr int STAGE = UB_AL + FB_AL + (SIG ? FB_AL : 0);
    static constexpr int TX_BYTES = UB + FB + (SIG ? FB : 0);
    static constexpr int BAR_OFF = NST * STAGE;
    static constexpr int XB_OFF = round_up(BAR_OFF + 8 * NST, 128);
    static constexpr int XB_BYTES = NW > 1 ? 2 * NW * 2 * TX * (int)sizeof(T) : 0;
    static constexpr int SMEM = XB_OFF + XB_BYTES + 128;   // + room to align the base to 128 bytes
};

// Deferred fold of the pipelined kernel's residual (deferred_fold_parts over
// the previous launch's one partial per CTA).
__device__ __forceinline__ void deferred_fold(const PpcArgs &P) {
    deferred_fold_parts(P.a.red, P.part_r, (int)gridDim.x, P.parity);
}

template <typename S, typename T, int C, int R, int NW, int H, bool EXACT, bool SIG, bool RES, int NST>
__global__ void __launch_bounds__(32 * NW) ppc2d_kernel(const __grid_constant__ PpcArgs P) {
    using L = PpcLayout<S, T, C, R, NW, H, SIG, NST>;
    constexpr int TX = L::TX, TY = L::TY;
    const CycArgs &a = P.a;
    const bool reducer = blockIdx.x == gridDim.x - 1;
    if constexpr (RES) {
        volatile Ctl *ctl = a.red.ctl;
        if (ctl->done >= 0) return;
        if (ctl->fold_only[P.parity]) {
            if (reducer && threadIdx.x < 32) deferred_fold(P);
            return;
        }
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // copy destinations must be 128-byte aligned: align the dynamic base explicitly
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t *bars = (uint64_t *)(smem + L::BAR_OFF);
    T *xbuf = (T *)(smem + L::XB_OFF);
    const int tid = threadIdx.x;
    const int band = band_of_lane<R, H>();
    const int mine = (P.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    auto su = [&](int s) { return (S *)(smem + s * L::STAGE); };
    auto sf = [&](int s) { return (T *)(smem + s * L::STAGE + L::UB_AL); };
    auto sd = [&](int s) { return (T *)(smem + s * L::STAGE + L::UB_AL + L::FB_AL); };
    auto issue = [&](int s, int tile) {
        const int bx = tile % P.tiles_x, by = tile / P.tiles_x;
        mbar_expect_tx(&bars[s], L::TX_BYTES);
        tma_load_2d(su(s), &P.mu, &bars[s], bx * TX, by * TY);
        tma_load_2d(sf(s), &P.mf, &bars[s], bx * TX, by * TY + 1);
        if constexpr (SIG) tma_load_2d(sd(s), &P.md, &bars[s], bx * TX, by * TY + 1);
    };
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int i = 0; i < NST && i < mine; ++i) issue(i, blockIdx.x + i * gridDim.x);
    }
    // the last CTA has the fewest tiles when the grid does not divide them:
    // it folds the previous launch's residual while its first copies land
    if constexpr (RES) {
        if (reducer && tid < 32) deferred_fold(P);
    }
    const Coef<T> kc = make_coef<T>(a);
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    int i = 0;
    bool failed = false;
    for (; i < mine; ++i) {
        const int s = i % NST;
        const unsigned ph = (unsigned)(i / NST) & 1u;
        bool ok = true;
        long long spins = 0;
        while (!mbar_try_wait(&bars[s], ph)) {
            if (++spins > P.spin_limit) { ok = false; break; }
        }
        if (__syncthreads_or(!ok)) { failed = true; break; }
        const int tile = blockIdx.x + i * gridDim.x;
        const int bx = tile % P.tiles_x, by = tile / P.tiles_x;
        const int x0 = 1 + bx * TX, y0 = 1 + by * TY, yb = y0 + band * R;
        Tile2D<T, C, R, SIG> t;
        stage2d_smem<S, T, C, R, H, EXACT, SIG>(t, kc, su(s), sf(s), sd(s), L::BWU, L::BWF, band * R,
                                                L::UB / (int)sizeof(S), L::FB / (int)sizeof(T), a.dbg);
        __syncthreads();   // every thread is done with stage s
        if (tid == 0 && i + NST < mine) {
            fence_proxy_async_smem();
            issue(s, blockIdx.x + (i + NST) * gridDim.x);
        }
        const bool full = (x0 + TX - 1 <= a.nx) && (y0 + TY - 1 <= a.ny);
        if (full) {
            acc += sweeps2d<T, C, R, NW, H, EXACT, SIG, RES, false>(t, kc, a.k, x0, yb, a.nx, a.ny, xbuf, Own{0, 0, 0, 0},
                                                                    a.dbg);
            store2d<S, T, C, R, H, SIG, false>(t, a, x0, yb);
        } else {
            acc += sweeps2d<T, C, R, NW, H, EXACT, SIG, RES, true>(t, kc, a.k, x0, yb, a.nx, a.ny, xbuf, Own{0, 0, 0, 0},
                                                                   a.dbg);
            store2d<S, T, C, R, H, SIG, true>(t, a, x0, yb);
        }
    }
    if (failed) {
        // record the expiry, drain this CTA's copies in flight (bounded), return
        if (tid == 0) {
            atomicExch(a.err, HJ_ERR_TIMEOUT);
            for (int j = i; j < mine && j < i + NST; ++j) {
                const int s = j % NST;
                const unsigned ph = (unsigned)(j / NST) & 1u;
                long long spins = 0;
                while (!mbar_try_wait(&bars[s], ph) && ++spins <= P.spin_limit) {
                }
            }
        }
        __syncthreads();
        return;
    }
    if constexpr (RES) write_cta_partial<NW>(P.part_w + blockIdx.x, acc);
}

}  // namespace hj

#define HJ_KPPC(S, T, C, R, NW, H, EX, NST)                                                                \
    {32 * (C) / (H), (R) * (NW) * (H), 32 * (NW), (NST), hj::PpcLayout<S, T, C, R, NW, H, false, NST>::SMEM,    \
     hj::PpcLayout<S, T, C, R, NW, H, true, NST>::SMEM,                                                      \
     hj::PpcLayout<S, T, C, R, NW, H, false, NST>::BWU, hj::PpcLayout<S, T, C, R, NW, H, false, NST>::BWF,   \
     {{hj::ppc2d_kernel<S, T, C, R, NW, H, EX, false, false, NST>, hj::ppc2d_kernel<S, T, C, R, NW, H, EX, false, true, NST>}, \
      {hj::ppc2d_kernel<S, T, C, R, NW, H, EX, true, false, NST>, hj::ppc2d_kernel<S, T, C, R, NW, H, EX, true, true, NST>}}}
