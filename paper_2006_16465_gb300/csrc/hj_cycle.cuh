// hj_cycle.cuh -- hierarchical Jacobi cycle kernels (templates).
//
// One cycle (Sections 3.3 and 4.1): every subdomain (tile) stages its interior
// plus a one-point halo from the iterate u_c, runs k Jacobi subiterations with
// the halo frozen, and writes its interior into the other buffer u_{c+1}.
//
// GB300 mapping (differs from the paper's one-thread-per-point shared-memory
// kernel, which targets a 48 KB/SM Volta):
//   * a 2D tile of TX x TY = (32*C/H) x (R*NW*H) points is one CTA of NW warps;
//     each warp owns H bands of R rows, and a lane owns C consecutive columns
//     of its band (the layout is spelled out above Tile2D below);
//   * the tile and its halo go into registers, straight from HBM with
//     coalesced row loads or from a shared-memory box filled by TMA;
//   * the k subiterations run entirely in registers: N/S neighbours are the
//     thread's own registers, W/E neighbours arrive by warp shuffle, the frozen
//     halo column sits in registers of the first and last lane of each row,
//     the two bands of a warp swap their edge rows by shuffle, and only the
//     edge rows of each warp go through a ping-pong shared-memory buffer (one
//     barrier per subiteration, none when NW = 1);
//   * binary32 lanes with an even number of columns update them partly in
//     packed pairs (fma.rn.f32x2: two independent round-to-nearest operations)
//     and fold the frozen halo's contribution into the right-hand-side term
//     once per cycle, so their sweeps carry no halo selects;
//   * the residual ||f - A u_c||^2 of the staged input is formed in the first
//     subiteration (r_p = d_p (u'_p - u_p)) and reduced deterministically
//     (warp butterfly, CTA, two-level grid) inside the same launch.
// The two containers of the paper's listing become the register state plus the
// separate global output buffer: the result equals the container rule exactly.
#pragma once

#include "hj_internal.cuh"

namespace hj {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct Coef {
    T cW, cE, cS, cN;   // raw stencil (exact / sigma paths)
    T bW, bE, bS, bN;   // -c * (1/d) for the constant-diagonal fast path
    T invd, dconst;
};

template <typename T>
__device__ __forceinline__ Coef<T> make_coef(const CycArgs &a);
template <>
__device__ __forceinline__ Coef<double> make_coef<double>(const CycArgs &a) {
    Coef<double> k;
    k.cW = a.cW; k.cE = a.cE; k.cS = a.cS; k.cN = a.cN;
    k.bW = k.bE = k.bS = k.bN = 0.0;   // unused: binary64 kernels take the exact path
    k.invd = a.invd;
    k.dconst = a.dconst;
    return k;
}
template <>
__device__ __forceinline__ Coef<float> make_coef<float>(const CycArgs &a) {
    Coef<float> k;
    k.cW = a.fW; k.cE = a.fE; k.cS = a.fS; k.cN = a.fN;
    k.bW = a.gW; k.bE = a.gE; k.bS = a.gS; k.bN = a.gN;
    k.invd = a.finvd;
    k.dconst = a.fdconst;
    return k;
}

// One Jacobi point update.
//  EXACT (binary64): acc = cW*W; acc += cE*E; [acc += cS*S; acc += cN*N;]
//                    u' = (f - acc) * (1/d), every operation rounded separately.
//  fast, constant d: u' = bW W + bE E + bS S + bN N + f/d as a fused chain.
//  fast, per-point d: u' = (f - cW W - cE E - cS S - cN N) * (1/d_p).
// If WANT_RES, res receives f - (A u)_p of the *old* value (unscaled by d for
// the fast constant-d path, where the caller multiplies the sum by d^2).
template <typename T, bool EXACT, bool SIG, bool D2, bool WANT_RES>
__device__ __forceinline__ T point_update(const Coef<T> &k, T g, T iv, T W, T E, T S, T N, T old, T &res) {
    if constexpr (EXACT) {
        double acc = __dmul_rn(k.cW, W);
        acc = __dadd_rn(acc, __dmul_rn(k.cE, E));
        if constexpr (D2) {
            acc = __dadd_rn(acc, __dmul_rn(k.cS, S));
            acc = __dadd_rn(acc, __dmul_rn(k.cN, N));
        }
        const double t = __dsub_rn(g, acc);
        const double inv = SIG ? (double)iv : (double)k.invd;
        if constexpr (WANT_RES) {
            const double dp = SIG ? __drcp_rn(iv) : (double)k.dconst;
            res = (T)__dsub_rn(t, __dmul_rn(dp, old));
        }
        return (T)__dmul_rn(t, inv);
    } else if constexpr (SIG) {
        T t = g;
        t = fma(-k.cW, W, t);
        t = fma(-k.cE, E, t);
        if constexpr (D2) {
            t = fma(-k.cS, S, t);
            t = fma(-k.cN, N, t);
        }
        const T nv = t * iv;
        if constexpr (WANT_RES) res = (nv - old) * ((T)1 / iv);
        return nv;
    } else {
        T t = g;
        if constexpr (D2) {
            t = fma(k.bN, N, t);
            t = fma(k.bS, S, t);
        }
        t = fma(k.bE, E, t);
        t = fma(k.bW, W, t);
        if constexpr (WANT_RES) res = t - old;
        return t;
    }
}

// ---------------------------------------------------------------------------
// 2D tile: register state, staging (from global memory or from a TMA-filled
// shared box), the k subiterations, and the write-back.
//
// A CTA of NW warps owns a TX x TY tile with TX = L*C, L = 32/H lanes per row,
// TY = R*NW*H.  Each warp holds H bands of R rows (H = 1, 2 or 4): lane l belongs
// to band hb = l / L of its warp and owns the C consecutive columns
// x0 + (l % L)*C ... of that band's rows; band b = w*H + hb starts at row
// y0 + b*R.  Two (four) bands per warp let a 32-wide tile give every lane two
// (four) neighbouring columns, whose updates then run as packed binary32
// pairs; the more columns a lane owns, the fewer shuffles and halo selects
// each point update carries.
// ---------------------------------------------------------------------------
template <typename T, int C, int R, bool SIG>
struct Tile2D {
    T v[R][C];                       // band values (current iterate)
    T g[R][C];                       // RHS term: f (exact / sigma) or f/d (fast)
    T dv[SIG ? R : 1][SIG ? C : 1];  // per-point 1/d_p
    T hx[R];                         // frozen halo column: first lane of a row -> W, last -> E
    T top[C], bot[C];                // row above / below the band
};

template <typename T, bool EXACT, bool SIG>
__device__ __forceinline__ T rhs_term(const Coef<T> &kc, T fv) {
    if constexpr (EXACT || SIG) return fv;
    else return fv * kc.invd;
}

// Band of this lane within its CTA and its first row.
template <int R, int H>
__device__ __forceinline__ int band_of_lane() {
    return (int)(threadIdx.x >> 5) * H + (int)(threadIdx.x & 31) / (32 / H);
}

// Stage from global memory with predicated loads (zero beyond the ghost ring).
template <typename S, typename T, int C, int R, int H, bool EXACT, bool SIG, bool PART>
__device__ __forceinline__ void stage2d_global(Tile2D<T, C, R, SIG> &t, const CycArgs &a, const Coef<T> &kc,
                                               const int x0, const int yb) {
    constexpr int L = 32 / H, TX = L * C;
    const int li = (threadIdx.x & 31) % L;
    const int xl = x0 + li * C;
    const long long ld = a.ld;
    const int nx = a.nx, ny = a.ny;
    const S *__restrict__ uin = (const S *)a.uin;
    const T *__restrict__ f = (const T *)a.f;
    const T *__restrict__ dinv = (const T *)a.dinv;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = yb + r;
        const bool rowok = !PART || row <= ny + 1;
        const bool rowin = !PART || row <= ny;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = xl + c;
            const long long q = (long long)row * ld + col;
            const bool ok = rowok && (!PART || col <= nx + 1) && HJ_IN(a.dbg, q, grid_elems2d(a), 1);
            const bool in = rowin && (!PART || col <= nx) && HJ_IN(a.dbg, q, grid_elems2d(a), 2);
            t.v[r][c] = ok ? ld_s<S, T>(uin + q) : (T)0;
            t.g[r][c] = rhs_term<T, EXACT, SIG>(kc, in ? __ldg(f + q) : (T)0);
            if constexpr (SIG) t.dv[r][c] = in ? __ldg(dinv + q) : (T)0;
        }
        const int hcol = (li == 0) ? x0 - 1 : x0 + TX;
        const long long hq = (long long)row * ld + hcol;
        const bool hok = (li == 0 || li == L - 1) && rowok && (!PART || hcol <= nx + 1) &&
                         HJ_IN(a.dbg, hq, grid_elems2d(a), 3);
        t.hx[r] = hok ? ld_s<S, T>(uin + hq) : (T)0;
    }
    const int rt = yb - 1, rb = yb + R;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = xl + c;
        const bool okc = !PART || col <= nx + 1;
        const long long qt = (long long)rt * ld + col, qb = (long long)rb * ld + col;
        t.top[c] = (okc && (!PART || rt <= ny + 1) && HJ_IN(a.dbg, qt, grid_elems2d(a), 4)) ? ld_s<S, T>(uin + qt) : (T)0;
        t.bot[c] = (okc && (!PART || rb <= ny + 1) && HJ_IN(a.dbg, qb, grid_elems2d(a), 5)) ? ld_s<S, T>(uin + qb) : (T)0;
    }
}

template <typename S, typename T> __device__ __forceinline__ T sm_s(const S *p) { return (T)*p; }
template <> __device__ __forceinline__ float sm_s<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}

// Stage from shared-memory boxes filled by TMA.  su: (TY+2) rows of the
// iterate starting at (x0-1, y0-1); sf / sd: TY rows of f / (1/d) starting at
// (x0-1, y0); all with row pitch bw elements.  Out-of-bounds box elements
// were zero-filled by the copy engine, exactly like the predicated path.
// Four binary32 columns per lane: the lane's columns 1 + 4 li .. 4 + 4 li of a
// box row straddle the 16-byte chunks at 4 li and 4 li + 4, so two 16-byte
// shared loads give them together with the W and E neighbours (the halo
// column for the first and last lane of a row).  The L = 8 lanes of a band
// read 8 consecutive chunks, one bank each: no conflicts.
__device__ __forceinline__ void lds_row4(const float *row, const int li, float (&v)[4], float &w, float &e) {
    const float4 a = *(const float4 *)(row + 4 * li);
    const float4 b = *(const float4 *)(row + 4 * li + 4);
    w = a.x;
    v[0] = a.y;
    v[1] = a.z;
    v[2] = a.w;
    v[3] = b.x;
    e = b.y;
}

// nu, nf: elements of the iterate box and of the RHS (1/d) box, for the
// index checks of debug builds (dbg: their device word)
template <typename S, typename T, int C, int R, int H, bool EXACT, bool SIG>
__device__ __forceinline__ void stage2d_smem(Tile2D<T, C, R, SIG> &t, const Coef<T> &kc, const S *su, const T *sf,
                                             const T *sd, const int bwu, const int bwf, const int band_row0,
                                             const int nu = 1 << 30, const int nf = 1 << 30,
                                             DbgWord *dbg = nullptr) {
    constexpr int L = 32 / H, TX = L * C;
    const int li = (threadIdx.x & 31) % L;
    (void)nu; (void)nf; (void)dbg;
    if constexpr (C == 4 && std::is_same<S, float>::value && std::is_same<T, float>::value) {
        // box pitches are multiples of 16 bytes and the boxes 128-byte aligned
        float w = 0.f, e = 0.f, tmp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int sr = band_row0 + r;
            if (HJ_IN(dbg, (sr + 1) * bwu + 4 * li + 7, nu, 11)) lds_row4(su + (sr + 1) * bwu, li, t.v[r], w, e);
            t.hx[r] = (li == 0) ? w : e;
            if (HJ_IN(dbg, sr * bwf + 4 * li + 7, nf, 12)) lds_row4(sf + sr * bwf, li, tmp, w, e);
#pragma unroll
            for (int c = 0; c < 4; ++c) t.g[r][c] = rhs_term<T, EXACT, SIG>(kc, tmp[c]);
            if constexpr (SIG) {
                if (HJ_IN(dbg, sr * bwf + 4 * li + 7, nf, 13)) lds_row4(sd + sr * bwf, li, t.dv[SIG ? r : 0], w, e);
            }
        }
        if (HJ_IN(dbg, band_row0 * bwu + 4 * li + 7, nu, 14)) lds_row4(su + band_row0 * bwu, li, t.top, w, e);
        if (HJ_IN(dbg, (band_row0 + R + 1) * bwu + 4 * li + 7, nu, 15))
            lds_row4(su + (band_row0 + R + 1) * bwu, li, t.bot, w, e);
        return;
    }
    const int xc = 1 + li * C;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int sr = band_row0 + r;   // tile-interior row index
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int iu = (sr + 1) * bwu + xc + c, jf = sr * bwf + xc + c;
            t.v[r][c] = HJ_IN(dbg, iu, nu, 11) ? sm_s<S, T>(su + iu) : (T)0;
            t.g[r][c] = rhs_term<T, EXACT, SIG>(kc, HJ_IN(dbg, jf, nf, 12) ? sf[jf] : (T)0);
            if constexpr (SIG) t.dv[r][c] = HJ_IN(dbg, jf, nf, 13) ? sd[jf] : (T)0;
        }
        const int ih = (sr + 1) * bwu + ((li == 0) ? 0 : TX + 1);
        t.hx[r] = HJ_IN(dbg, ih, nu, 14) ? sm_s<S, T>(su + ih) : (T)0;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int it = band_row0 * bwu + xc + c, ib = (band_row0 + R + 1) * bwu + xc + c;
        t.top[c] = HJ_IN(dbg, it, nu, 15) ? sm_s<S, T>(su + it) : (T)0;
        t.bot[c] = HJ_IN(dbg, ib, nu, 15) ? sm_s<S, T>(su + ib) : (T)0;
    }
}

// m ? x : y for a per-lane mask m (all ones or zero), as bitwise operations:
// the halo and band selects below differ between the lanes of a warp on
// every row, and as masks they stay single instructions, never branches.
__device__ __forceinline__ float mask_sel(unsigned m, float x, float y) {
    return __uint_as_float((__float_as_uint(x) & m) | (__float_as_uint(y) & ~m));
}
__device__ __forceinline__ double mask_sel(unsigned m, double x, double y) {
    const unsigned long long mm = (unsigned long long)(int)m;   // sign-extended: all ones or zero
    return __longlong_as_double((long long)(((unsigned long long)__double_as_longlong(x) & mm) |
                                            ((unsigned long long)__double_as_longlong(y) & ~mm)));
}
__device__ __forceinline__ unsigned lane_mask(bool b) { return b ? 0xffffffffu : 0u; }

// Packed binary32 pairs (fma/mul .f32x2: two independent round-to-nearest
// operations, so a pair gives exactly the two scalar results).
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long p, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// k subiterations on registers.  Returns this thread's share of
// ||f - A u_c||^2 (unscaled by d^2 on the fast constant-diagonal path).
// Points a subdomain owns (overlapping subdomains write back and count in the
// residual only these): columns [xlo, xhi], rows [ylo, yhi].
struct Own {
    int xlo, xhi, ylo, yhi;
};

// Binary32 path for lanes of an even number of columns (constant or per-point
// diagonal, full tiles), with the frozen halo folded into the right-hand-side
// term.  Within a cycle the halo of a subdomain does not change, so its
// weighted contribution to the updates along the subdomain's edge is a
// constant: it is added to g once, before the first subiteration, and the
// edge lanes then weight what they receive by shuffle (a point of another row,
// or their own) with a zero coefficient.  No halo select is left in the sweeps.
// A point update is the sum g + kW W + kE E + kS S + kN N (times 1/d_p on the
// per-point path) taken in a fixed order: the two horizontal neighbours first
// (E then W in even columns of the subdomain, W then E in odd ones), then S,
// then N; the last two steps are packed pairs (fma.rn.f32x2: two independent
// round-to-nearest operations) whose results are the next pair of iterate
// registers.  The order depends only on the point's place in the subdomain, so
// every lane layout of a subdomain (two columns per lane in two bands, four in
// four bands, one to eight warps) gives the same values bit for bit.  Per row
// and lane of two columns: two shuffles, two scalar and three packed
// multiply-adds.
template <int C, int R, int NW, int H, bool SIG, bool RES, bool OVL>
__device__ __forceinline__ float sweeps2d_fold(Tile2D<float, C, R, SIG> &t, const Coef<float> &kc, const int k,
                                               const int x0, const int yb, float *xbuf, const Own own,
                                               DbgWord *dbg) {
    (void)dbg; (void)own; (void)x0; (void)yb;
    static_assert(C % 2 == 0, "packed pairs of columns");
    constexpr int L = 32 / H, TX = L * C;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int li = lane % L, hb = lane / L, band = w * H + hb;
    const int xl = x0 + li * C;
    // neighbour weights: -c_X / d (constant diagonal) or -c_X (per-point 1/d, applied last)
    const float kW = SIG ? -kc.cW : kc.bW, kE = SIG ? -kc.cE : kc.bE;
    const float kS = SIG ? -kc.cS : kc.bS, kN = SIG ? -kc.cN : kc.bN;
    const bool wl = li == 0, el = li == L - 1, tb = band == 0, bb = band == NW * H - 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        t.g[r][0] = fmaf(wl ? kW : 0.f, t.hx[r], t.g[r][0]);
        t.g[r][C - 1] = fmaf(el ? kE : 0.f, t.hx[r], t.g[r][C - 1]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        t.g[0][c] = fmaf(tb ? kS : 0.f, t.top[c], t.g[0][c]);
        t.g[R - 1][c] = fmaf(bb ? kN : 0.f, t.bot[c], t.g[R - 1][c]);
    }
    // weights of the shuffled W / E values and of the band's outer rows
    const float kWs = wl ? 0.f : kW, kEs = el ? 0.f : kE;
    const float kS0 = tb ? 0.f : kS, kNR = bb ? 0.f : kN;
    const unsigned long long kS2 = pk2(kS, kS), kN2 = pk2(kN, kN), kS02 = pk2(kS0, kS0), kNR2 = pk2(kNR, kNR);
    const unsigned long long kWE = pk2(kWs, kEs);
    const unsigned m_top = lane_mask(hb > 0);
    float acc = 0.f;
    auto sweep = [&](auto first_tag) {
        constexpr bool FIRST = decltype(first_tag)::value;
        float prev[C];
#pragma unroll
        for (int c = 0; c < C; ++c) prev[c] = t.top[c];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float cur[C], a[C];
#pragma unroll
            for (int c = 0; c < C; ++c) cur[c] = t.v[r][c];
            const float sW = __shfl_up_sync(FULL, cur[C - 1], 1);
            const float sE = __shfl_down_sync(FULL, cur[0], 1);
            const unsigned long long cN2 = (r == R - 1) ? kNR2 : kN2, cS2 = (r == 0) ? kS02 : kS2;
            // horizontal neighbours: even column E then W, odd column W then E
            if constexpr (C == 2) {
                a[0] = fmaf(kE, cur[1], t.g[r][0]);
                a[1] = fmaf(kW, cur[0], t.g[r][1]);
                upk2(ffma2(kWE, pk2(sW, sE), pk2(a[0], a[1])), a[0], a[1]);
            } else {
#pragma unroll
                for (int c = 0; c < C; c += 2) {
                    a[c] = fmaf(kE, cur[c + 1], t.g[r][c]);
                    a[c] = (c == 0) ? fmaf(kWs, sW, a[c]) : fmaf(kW, cur[c > 0 ? c - 1 : 0], a[c]);
                    a[c + 1] = fmaf(kW, cur[c], t.g[r][c + 1]);
                    a[c + 1] = (c + 2 == C) ? fmaf(kEs, sE, a[c + 1]) : fmaf(kE, cur[c + 2 < C ? c + 2 : 0], a[c + 1]);
                }
            }
            // then S and N as packed pairs
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                const float N0 = (r == R - 1) ? t.bot[c] : t.v[r < R - 1 ? r + 1 : 0][c];
                const float N1 = (r == R - 1) ? t.bot[c + 1] : t.v[r < R - 1 ? r + 1 : 0][c + 1];
                unsigned long long p = ffma2(cS2, pk2(prev[c], prev[c + 1]), pk2(a[c], a[c + 1]));
                p = ffma2(cN2, pk2(N0, N1), p);
                upk2(p, a[c], a[c + 1]);
            }
            if constexpr (SIG) {
#pragma unroll
                for (int c = 0; c < C; c += 2)
                    upk2(fmul2(pk2(a[c], a[c + 1]), pk2(t.dv[SIG ? r : 0][SIG ? c : 0], t.dv[SIG ? r : 0][SIG ? c + 1 : 0])),
                         a[c], a[c + 1]);
            }
            if constexpr (FIRST && RES) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    float rc = a[c] - cur[c];
                    if constexpr (SIG) rc = rc * (1.f / t.dv[SIG ? r : 0][SIG ? c : 0]);
                    if constexpr (OVL) {
                        if (!(yb + r >= own.ylo && yb + r <= own.yhi && xl + c >= own.xlo && xl + c <= own.xhi))
                            rc = 0.f;
                    }
                    acc += rc * rc;
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                t.v[r][c] = a[c];
                prev[c] = cur[c];
            }
        }
    };
    int par = 0;
    // the rows next to each band become the neighbouring bands' values of the
    // previous subiteration; the frozen edges of the subdomain carry zero
    // weights, so what lands there does not matter
    auto exchange = [&]() {
        if constexpr (H == 2) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float recv = __shfl_xor_sync(FULL, mask_sel(m_top, t.v[0][c], t.v[R - 1][c]), 16);
                t.top[c] = recv;
                t.bot[c] = recv;
            }
        } else if constexpr (H == 4) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                t.top[c] = __shfl_up_sync(FULL, t.v[R - 1][c], L);
                t.bot[c] = __shfl_down_sync(FULL, t.v[0][c], L);
            }
        }
        if constexpr (NW > 1) {
            constexpr int NX = 2 * NW * 2 * TX;
            (void)NX;   // read by the index checks of debug builds
            const int o = par * (NW * 2 * TX);
            float *buf = xbuf + o;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int i0 = (w * 2 + 0) * TX + li * C + c, i1 = (w * 2 + 1) * TX + li * C + c;
                if (hb == 0 && HJ_IN(dbg, o + i0, NX, 16)) buf[i0] = t.v[0][c];
                if (hb == H - 1 && HJ_IN(dbg, o + i1, NX, 16)) buf[i1] = t.v[R - 1][c];
            }
            __syncthreads();
            if (w > 0 && hb == 0) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int i = ((w - 1) * 2 + 1) * TX + li * C + c;
                    if (HJ_IN(dbg, o + i, NX, 17)) t.top[c] = buf[i];
                }
            }
            if (w < NW - 1 && hb == H - 1) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int i = ((w + 1) * 2 + 0) * TX + li * C + c;
                    if (HJ_IN(dbg, o + i, NX, 17)) t.bot[c] = buf[i];
                }
            }
            par ^= 1;
        }
    };
    sweep(std::integral_constant<bool, true>());
    for (int s = 1; s < k; ++s) {
        exchange();
        sweep(std::integral_constant<bool, false>());
    }
    return acc;
}

template <typename T, int C, int R, int NW, int H, bool EXACT, bool SIG, bool RES, bool PART, bool OVL = false>
__device__ __forceinline__ typename std::conditional<EXACT, double, T>::type
sweeps2d(Tile2D<T, C, R, SIG> &t, const Coef<T> &kc, const int k, const int x0, const int yb, const int nx,
         const int ny, T *xbuf, const Own own = Own{0, 0, 0, 0}, DbgWord *dbg = nullptr) {
    (void)dbg;
    static_assert(H == 1 || H == 2 || H == 4, "one, two or four bands per warp");
    constexpr int L = 32 / H, TX = L * C;
    constexpr bool PACK = std::is_same<T, float>::value && !EXACT && (C % 2 == 0) && !PART;
    if constexpr (PACK) {
        return sweeps2d_fold<C, R, NW, H, SIG, RES, OVL>(t, kc, k, x0, yb, xbuf, own, dbg);
    } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int li = lane % L, hb = lane / L;
    const int xl = x0 + li * C;
    const unsigned m_first = lane_mask(li == 0), m_last = lane_mask(li == L - 1);   // halo lanes of a row
    const unsigned m_top = lane_mask(hb > 0), m_bot = lane_mask(hb < H - 1);         // bands with a band above / below
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    auto sweep = [&](auto first_tag) {
        constexpr bool FIRST = decltype(first_tag)::value;
        T prev[C];
#pragma unroll
        for (int c = 0; c < C; ++c) prev[c] = t.top[c];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T cur[C];
#pragma unroll
            for (int c = 0; c < C; ++c) cur[c] = t.v[r][c];
            const T left = mask_sel(m_first, t.hx[r], __shfl_up_sync(FULL, cur[C - 1], 1));
            const T right = mask_sel(m_last, t.hx[r], __shfl_down_sync(FULL, cur[0], 1));
            {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const T W = (c == 0) ? left : cur[c > 0 ? c - 1 : 0];
                    const T E = (c == C - 1) ? right : cur[c < C - 1 ? c + 1 : 0];
                    const T Sv = prev[c];
                    const T Nv = (r == R - 1) ? t.bot[c] : t.v[r < R - 1 ? r + 1 : 0][c];
                    T res = 0;
                    T nv = point_update<T, EXACT, SIG, true, FIRST && RES>(
                        kc, t.g[r][c], SIG ? t.dv[SIG ? r : 0][SIG ? c : 0] : (T)0, W, E, Sv, Nv, cur[c], res);
                    if constexpr (PART) {
                        const bool act = (yb + r <= ny) && (xl + c <= nx);
                        nv = act ? nv : cur[c];
                        if (!act) res = 0;
                    }
                    if constexpr (OVL && FIRST && RES) {
                        if (!(yb + r >= own.ylo && yb + r <= own.yhi && xl + c >= own.xlo && xl + c <= own.xhi))
                            res = 0;
                    }
                    if constexpr (FIRST && RES) acc += (Acc)res * (Acc)res;
                    t.v[r][c] = nv;
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) prev[c] = cur[c];
        }
    };
    int par = 0;
    // before each subiteration after the first: the rows next to each band
    // become the neighbouring bands' values of the previous subiteration
    // (v: the registers holding that subiteration's values)
    auto exchange = [&](T (&v)[R][C]) {
        if constexpr (H == 2) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const T send = mask_sel(m_top, v[0][c], v[R - 1][c]);
                const T recv = __shfl_xor_sync(FULL, send, 16);
                t.top[c] = mask_sel(m_top, recv, t.top[c]);
                t.bot[c] = mask_sel(m_bot, recv, t.bot[c]);
            }
        } else if constexpr (H == 4) {
            // band hb's top row is band hb-1's last row (L lanes down), its
            // bottom row band hb+1's first row (L lanes up)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const T up = __shfl_up_sync(FULL, v[R - 1][c], L);
                const T dn = __shfl_down_sync(FULL, v[0][c], L);
                t.top[c] = mask_sel(m_top, up, t.top[c]);
                t.bot[c] = mask_sel(m_bot, dn, t.bot[c]);
            }
        }
        if constexpr (NW > 1) {
            // two parities of NW x 2 edge rows of TX points
            constexpr int NX = 2 * NW * 2 * TX;
            (void)NX;   // read by the index checks of debug builds
            const int o = par * (NW * 2 * TX);
            T *buf = xbuf + o;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int i0 = (w * 2 + 0) * TX + li * C + c, i1 = (w * 2 + 1) * TX + li * C + c;
                if (hb == 0 && HJ_IN(dbg, o + i0, NX, 16)) buf[i0] = v[0][c];
                if (hb == H - 1 && HJ_IN(dbg, o + i1, NX, 16)) buf[i1] = v[R - 1][c];
            }
            __syncthreads();
            if (w > 0 && hb == 0) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int i = ((w - 1) * 2 + 1) * TX + li * C + c;
                    if (HJ_IN(dbg, o + i, NX, 17)) t.top[c] = buf[i];
                }
            }
            if (w < NW - 1 && hb == H - 1) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int i = ((w + 1) * 2 + 0) * TX + li * C + c;
                    if (HJ_IN(dbg, o + i, NX, 17)) t.bot[c] = buf[i];
                }
            }
            par ^= 1;
        }
    };
    sweep(std::integral_constant<bool, true>());
    for (int s = 1; s < k; ++s) {
        exchange(t.v);
        sweep(std::integral_constant<bool, false>());
    }
    return acc;
    }
}

// Write the band's interior points into u_{c+1}.
template <typename S, typename T, int C, int R, int H, bool SIG, bool PART, bool OVL = false>
__device__ __forceinline__ void store2d(const Tile2D<T, C, R, SIG> &t, const CycArgs &a, const int x0,
                                        const int yb, const Own own = Own{0, 0, 0, 0}) {
    const int li = (threadIdx.x & 31) % (32 / H);
    const int xl = x0 + li * C;
    S *__restrict__ uout = (S *)a.uout;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = yb + r;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int col = xl + c;
            bool w = !PART || (row <= a.ny && col <= a.nx);
            if constexpr (OVL) w = w && row >= own.ylo && row <= own.yhi && col >= own.xlo && col <= own.xhi;
            const long long q = (long long)row * a.ld + col;
            if (w && HJ_IN(a.dbg, q, grid_elems2d(a), 10)) st_s<S, T>(uout + q, t.v[r][c]);
        }
    }
}

template <typename S, typename T, int C, int R, int NW, int H, bool EXACT, bool SIG, bool RES, bool PART,
          bool OVL = false>
__device__ __forceinline__ typename std::conditional<EXACT, double, T>::type
tile2d(const CycArgs &a, const int x0, const int y0, T *xbuf, const Own own = Own{0, 0, 0, 0}) {
    const int yb = y0 + band_of_lane<R, H>() * R;
    const Coef<T> kc = make_coef<T>(a);
    Tile2D<T, C, R, SIG> t;
    stage2d_global<S, T, C, R, H, EXACT, SIG, PART>(t, a, kc, x0, yb);
    auto acc = sweeps2d<T, C, R, NW, H, EXACT, SIG, RES, PART, OVL>(t, kc, a.k, x0, yb, a.nx, a.ny, xbuf, own, a.dbg);
    store2d<S, T, C, R, H, SIG, PART, OVL>(t, a, x0, yb, own);
    return acc;
}

// One partial of the CTA's residual share, written without atomics to *slot:
// the next launch reads it after this kernel has completed.
template <int NW, typename A>
__device__ __forceinline__ void write_cta_partial(double *slot, A acc) {
    double v;
    if constexpr (std::is_same<A, float>::value) v = (double)warp_sum_f(acc);
    else v = warp_sum((double)acc);
    if constexpr (NW == 1) {
        if (threadIdx.x == 0) *slot = v;
    } else {
        __shared__ double s_w[NW];
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) t += s_w[w];
            *slot = t;
        }
    }
}

// OVL: overlapping subdomains (Sections 3.4, 4.3): block (bx, by) is subdomain
// (bx, by) of a.jx x a.jy, placed and owning points as subdomain_span says.
// RES with a.part_w set: the deferred fold (one partial per CTA, folded by the
// next launch's last CTA) instead of the grid reduction at the launch's end.
template <typename S, typename T, int C, int R, int NW, int H, bool EXACT, bool SIG, bool RES, bool OVL = false>
__global__ void __launch_bounds__(32 * NW) hier2d_kernel(const CycArgs a) {
    const int nblk = (int)(gridDim.x * gridDim.y), bid = (int)(blockIdx.y * gridDim.x + blockIdx.x);
    if constexpr (RES) {
        volatile Ctl *ctl = a.red.ctl;
        if (ctl->done >= 0) return;
        if (a.part_w) {
            const bool reducer = bid == nblk - 1;
            if (ctl->fold_only[a.parity]) {
                if (reducer && threadIdx.x < 32) deferred_fold_parts(a.red, a.part_r, nblk, a.parity);
                return;
            }
            if (reducer && threadIdx.x < 32) deferred_fold_parts(a.red, a.part_r, nblk, a.parity);
        }
    }
    constexpr int TX = 32 * C / H, TY = R * NW * H;
    constexpr int XB = NW > 1 ? 2 * NW * 2 * TX : 1;
    __shared__ T xbuf[XB];
    int x0 = 1 + blockIdx.x * TX, y0 = 1 + blockIdx.y * TY;
    Own own{0, 0, 0, 0};
    if constexpr (OVL) {
        const Span sx = subdomain_span(blockIdx.x, a.jx, a.nx, TX, a.ox);
        const Span sy = subdomain_span(blockIdx.y, a.jy, a.ny, TY, a.oy);
        x0 = sx.start;
        y0 = sy.start;
        own = Own{sx.lo, sx.hi, sy.lo, sy.hi};
    }
    const bool full = (x0 + TX - 1 <= a.nx) && (y0 + TY - 1 <= a.ny);
    typename std::conditional<EXACT, double, T>::type acc;
    if (full) acc = tile2d<S, T, C, R, NW, H, EXACT, SIG, RES, false, OVL>(a, x0, y0, xbuf, own);
    else acc = tile2d<S, T, C, R, NW, H, EXACT, SIG, RES, true, OVL>(a, x0, y0, xbuf, own);
    if constexpr (RES) {
        if (a.part_w) write_cta_partial<NW>(a.part_w + bid, acc);
        else reduce_grid_acc(a.red, acc);
    }
}

// ---------------------------------------------------------------------------
// 1D tile: a subdomain of TX = 32*C*WPT points of one row (the independent
// copies of Section 3.5, one row per blockIdx.y) is swept by WPT warps; warp
// q of it owns the 32*C points starting at x0 + q*32*C, lane l the C
// consecutive points from there + l*C.  Neighbouring warps swap their edge
// points through a double-buffered shared array (one barrier per
// subiteration); with WPT > 1 binary64 updates run on WPT sub-partitions at
// once.  A CTA holds WPB subdomains side by side (WPB > 1 only with WPT = 1,
// so that no barrier sits in a branch that differs between subdomains).
// ---------------------------------------------------------------------------
template <typename T, int WPT>
struct Xchg1D {
    T e[2][WPT > 1 ? WPT : 1][2];   // [parity][warp][first, last]
};

template <typename S, typename T, int C, int WPT, bool EXACT, bool SIG, bool RES, bool PART, bool OVL = false>
__device__ __forceinline__ typename std::conditional<EXACT, double, T>::type
tile1d(const CycArgs &a, const int x0, const int row, Xchg1D<T, WPT> &xb, const int own_lo = 0, const int own_hi = 0) {
    constexpr int TX = 32 * C * WPT;
    const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) % WPT;
    const int xl = x0 + q * 32 * C + lane * C;
    const long long ld = a.ld;
    const int nx = a.nx;
    const long long rb = (long long)row * ld;
    const S *__restrict__ uin = (const S *)a.uin;
    const T *__restrict__ f = (const T *)a.f;
    const T *__restrict__ dinv = (const T *)a.dinv;
    const Coef<T> kc = make_coef<T>(a);
    T v[C], g[C], dv[SIG ? C : 1];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = xl + c;
        const bool ok = (!PART || col <= nx + 1) && HJ_IN(a.dbg, rb + col, grid_elems1d(a), 30);
        const bool in = (!PART || col <= nx) && HJ_IN(a.dbg, rb + col, grid_elems1d(a), 31);
        v[c] = ok ? ld_s<S, T>(uin + rb + col) : (T)0;
        const T fv = in ? __ldg(f + rb + col) : (T)0;
        if constexpr (SIG) {
            dv[c] = in ? __ldg(dinv + rb + col) : (T)0;
            g[c] = fv;
        } else if constexpr (EXACT) {
            g[c] = fv;
        } else {
            g[c] = fv * kc.invd;
        }
    }
    // frozen halo: first lane of warp 0 (W) and last lane of the last warp (E)
    const bool wl = lane == 0 && q == 0, el = lane == 31 && q == WPT - 1;
    const int hcol = wl ? x0 - 1 : x0 + TX;
    const bool hok = (wl || el) && (!PART || hcol <= nx + 1) && HJ_IN(a.dbg, rb + hcol, grid_elems1d(a), 32);
    const T hx = hok ? ld_s<S, T>(uin + rb + hcol) : (T)0;

    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    int par = 0;
    auto sweep = [&](auto first_tag) {
        constexpr bool FIRST = decltype(first_tag)::value;
        T cur[C];
#pragma unroll
        for (int c = 0; c < C; ++c) cur[c] = v[c];
        T left = __shfl_up_sync(FULL, cur[C - 1], 1);
        T right = __shfl_down_sync(FULL, cur[0], 1);
        if constexpr (WPT > 1) {
            // the neighbouring warps' edge points of the previous subiterate
            if (lane == 0) xb.e[par][q][0] = cur[0];
            if (lane == 31) xb.e[par][q][1] = cur[C - 1];
            __syncthreads();
            if (lane == 0 && q > 0) left = xb.e[par][q - 1][1];
            if (lane == 31 && q < WPT - 1) right = xb.e[par][q + 1][0];
            par ^= 1;
        }
        if (wl) left = hx;
        if (el) right = hx;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const T W = (c == 0) ? left : cur[c > 0 ? c - 1 : 0];
            const T E = (c == C - 1) ? right : cur[c < C - 1 ? c + 1 : 0];
            T res = 0;
            T nv = point_update<T, EXACT, SIG, false, FIRST && RES>(kc, g[c], SIG ? dv[SIG ? c : 0] : (T)0,
                                                                    W, E, (T)0, (T)0, cur[c], res);
            if constexpr (PART) {
                const bool act = xl + c <= nx;
                nv = act ? nv : cur[c];
                if (!act) res = 0;
            }
            if constexpr (OVL && FIRST && RES) {
                if (!(xl + c >= own_lo && xl + c <= own_hi)) res = 0;
            }
            if constexpr (FIRST && RES) acc += (Acc)res * (Acc)res;
            v[c] = nv;
        }
    };
    sweep(std::integral_constant<bool, true>());
    for (int s = 1; s < a.k; ++s) sweep(std::integral_constant<bool, false>());

    S *__restrict__ uout = (S *)a.uout;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = xl + c;
        bool w = !PART || col <= nx;
        if constexpr (OVL) w = w && col >= own_lo && col <= own_hi;
        if (w && HJ_IN(a.dbg, rb + col, grid_elems1d(a), 33)) st_s<S, T>(uout + rb + col, v[c]);
    }
    return acc;
}

template <typename S, typename T, int C, int WPT, int WPB, bool EXACT, bool SIG, bool RES, bool OVL = false>
__global__ void __launch_bounds__(32 * WPT * WPB) hier1d_kernel(const CycArgs a) {
    static_assert(WPT == 1 || WPB == 1, "several subdomains per CTA only with one warp each");
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    constexpr int TX = 32 * C * WPT;
    __shared__ Xchg1D<T, WPT> xb;
    const int j = blockIdx.x * WPB + (int)(threadIdx.x >> 5) / WPT;   // subdomain along the row
    int x0 = 1 + j * TX, lo = 0, hi = 0;
    bool here = x0 <= a.nx;
    if constexpr (OVL) {
        here = j < a.jx;
        if (here) {
            const Span sp = subdomain_span(j, a.jx, a.nx, TX, a.ox);
            x0 = sp.start;
            lo = sp.lo;
            hi = sp.hi;
        }
    }
    const int row = blockIdx.y;
    typename std::conditional<EXACT, double, T>::type acc = 0;
    // with WPT > 1, the subdomain is uniform across the CTA and the whole CTA
    // takes the same branch; with WPB > 1 the branches hold no barrier
    if (here) {
        if (x0 + TX - 1 <= a.nx) acc = tile1d<S, T, C, WPT, EXACT, SIG, RES, false, OVL>(a, x0, row, xb, lo, hi);
        else acc = tile1d<S, T, C, WPT, EXACT, SIG, RES, true, OVL>(a, x0, row, xb, lo, hi);
    }
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

// ---------------------------------------------------------------------------
// Variable neighbour coefficients (the general tridiagonal a_i, d_i, c_i of
// Section 3 and its 2D analogue): one thread per point, the subdomain plus its
// halo in two shared-memory containers used in turn (the paper's own kernel
// layout, Appendix A), one barrier per subiteration.  A thread keeps its
// point's coefficients in registers.  blockDim = (tile_x, tile_y) in 2D,
// (tile_x) in 1D with one copy per blockIdx.y.
//   binary64: acc = cW*uW; acc += cE*uE; [acc += cS*uS; acc += cN*uN;]
//             u' = (f - acc) * (1/d_p), d_p = dconst + sigma_p, each operation
//             rounded separately (the oracle's order); 1/d_p comes from the
//             handle's dinv plane when sigma is a field;
//   binary32: u' = f/d + (-cN/d) uN + (-cS/d) uS + (-cE/d) uE + (-cW/d) uW as a
//             fused chain from precomputed per-point factors.
// ---------------------------------------------------------------------------
template <typename S, typename T, int DIM, bool EXACT, bool RES>
__global__ void __launch_bounds__(1024, 2) vc_kernel(const CycArgs a) {
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    extern __shared__ __align__(16) unsigned char vc_smem[];
    const int TX = blockDim.x, TY = DIM == 2 ? blockDim.y : 1;
    const int lw = TX + 2, lh = DIM == 2 ? TY + 2 : 1;
    T *buf0 = (T *)vc_smem, *buf1 = buf0 + lw * lh;
    const int tx = threadIdx.x, ty = DIM == 2 ? threadIdx.y : 0;
    const int i = 1 + blockIdx.x * TX + tx;
    const int j = DIM == 2 ? 1 + blockIdx.y * TY + ty : blockIdx.y;
    const int nx = a.nx, ny = a.ny;
    const long long ld = a.ld;
    const bool in = i <= nx && (DIM == 1 || j <= ny);
    const S *__restrict__ uin = (const S *)a.uin;
    const T *__restrict__ f = (const T *)a.f;
    const int me = (ty + (DIM == 2 ? 1 : 0)) * lw + tx + 1;
    auto ld_u = [&](int jj, int ii) -> T {
        const bool ok = ii <= nx + 1 && (DIM == 1 || jj <= ny + 1);
        return ok ? ld_s<S, T>(uin + (long long)jj * ld + ii) : (T)0;
    };
    // Every global load first (the point, the halo cells next to it, f and
    // the point's factors), then the shared-memory stores: one round of
    // memory latency per subdomain instead of one per kind of operand.
    const T v0 = ld_u(j, i);
    const T hw = tx == 0 ? ld_u(j, i - 1) : (T)0;
    const T he = tx == TX - 1 ? ld_u(j, i + 1) : (T)0;
    T hs = 0, hn = 0;
    if constexpr (DIM == 2) {
        hs = ty == 0 ? ld_u(j - 1, i) : (T)0;
        hn = ty == TY - 1 ? ld_u(j + 1, i) : (T)0;
    }
    const long long q = (long long)j * ld + i;
    const long long ps = a.vcs;
    T cw = 0, ce = 0, cs = 0, cn = 0, g = 0, dpt = 0, iv = 0;
    if (in) {
        if constexpr (EXACT) {
            const double *__restrict__ c = (const double *)a.vc;
            cw = __ldg(c + q);
            ce = __ldg(c + ps + q);
            if constexpr (DIM == 2) {
                cs = __ldg(c + 2 * ps + q);
                cn = __ldg(c + 3 * ps + q);
            }
            // 1/d_p from the handle's plane (the same correctly rounded
            // reciprocal of dconst + sigma_p): binary64 arithmetic is the
            // scarce resource here, bytes are not
            if constexpr (RES) dpt = a.vsig ? __dadd_rn(a.dconst, __ldg(a.vsig + q)) : a.dconst;
            iv = a.dinv ? __ldg((const double *)a.dinv + q) : __drcp_rn(a.dconst);
            g = __ldg(f + q);
        } else {
            const float *__restrict__ c = (const float *)a.vc;
            constexpr int NP = DIM == 2 ? 4 : 2;   // planes before 1/d and d
            cw = __ldg(c + q);
            ce = __ldg(c + ps + q);
            if constexpr (DIM == 2) {
                cs = __ldg(c + 2 * ps + q);
                cn = __ldg(c + 3 * ps + q);
            }
            iv = __ldg(c + NP * ps + q);
            if constexpr (RES) dpt = __ldg(c + (NP + 1) * ps + q);
            g = __ldg(f + q) * iv;
        }
    }
    buf0[me] = v0;
    buf1[me] = v0;
    if (tx == 0) { buf0[me - 1] = hw; buf1[me - 1] = hw; }
    if (tx == TX - 1) { buf0[me + 1] = he; buf1[me + 1] = he; }
    if constexpr (DIM == 2) {
        if (ty == 0) { buf0[me - lw] = hs; buf1[me - lw] = hs; }
        if (ty == TY - 1) { buf0[me + lw] = hn; buf1[me + lw] = hn; }
    }
    __syncthreads();
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    for (int s = 0; s < a.k; ++s) {
        const T *src = (s & 1) ? buf1 : buf0;
        T *dst = (s & 1) ? buf0 : buf1;
        if (in) {
            const T old = src[me], W = src[me - 1], E = src[me + 1];
            const T Sv = DIM == 2 ? src[me - lw] : (T)0, Nv = DIM == 2 ? src[me + lw] : (T)0;
            T nv, res = 0;
            if constexpr (EXACT) {
                double t = __dmul_rn(cw, W);
                t = __dadd_rn(t, __dmul_rn(ce, E));
                if constexpr (DIM == 2) {
                    t = __dadd_rn(t, __dmul_rn(cs, Sv));
                    t = __dadd_rn(t, __dmul_rn(cn, Nv));
                }
                const double tt = __dsub_rn(g, t);
                nv = __dmul_rn(tt, iv);
                if (RES && s == 0) res = __dsub_rn(tt, __dmul_rn(dpt, old));
            } else {
                T t = g;
                if constexpr (DIM == 2) {
                    t = fma(cn, Nv, t);
                    t = fma(cs, Sv, t);
                }
                t = fma(ce, E, t);
                t = fma(cw, W, t);
                nv = t;
                if (RES && s == 0) res = (t - old) * dpt;
            }
            if constexpr (RES) acc += (Acc)res * (Acc)res;
            dst[me] = nv;
        }
        __syncthreads();
    }
    if (in) st_s<S, T>((S *)a.uout + q, ((a.k & 1) ? buf1 : buf0)[me]);
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

// ---------------------------------------------------------------------------
// Classic global-memory Jacobi (Section 3.2): one sweep per launch, every
// point reads u_c only and writes u_{c+1}.  Same update arithmetic and fused
// residual as the cycle kernels.
//
// HBM-bound (12 B per point in binary32, 24 B in binary64), so the layout is
// chosen for bytes in flight: a CTA of 32 x 8 threads covers a block of
// 32*V columns x 8*R rows (classic2d_block_cols/rows); a thread owns one
// 16-byte vector of V = 16 / sizeof(S) columns (ghost columns included, so
// every vector starts on a 16-byte boundary) for R consecutive rows, issues
// the R + 2 iterate rows and R right-hand-side rows as vector loads before it
// computes anything, keeps the vertical neighbours in registers, and takes the
// horizontal ones from its neighbouring lanes by shuffle (the two columns just
// outside the warp's segment by scalar loads).  Ghost and padding columns in
// a vector are stored back unchanged.
// ---------------------------------------------------------------------------
template <typename S, typename T>
__device__ __forceinline__ void ld_vec16(const S *p, T (&out)[16 / sizeof(S)]) {
    constexpr int V = 16 / (int)sizeof(S);
    const uint4 raw = __ldg((const uint4 *)p);
    S tmp[V];
    memcpy(tmp, &raw, 16);
#pragma unroll
    for (int c = 0; c < V; ++c) out[c] = sm_s<S, T>(&tmp[c]);
}

// V values of the compute type (16 bytes or, for bfloat16 storage, 32)
template <typename T, int V>
__device__ __forceinline__ void ld_vecT(const T *p, T (&out)[V]) {
    static_assert((V * sizeof(T)) % 16 == 0, "whole 16-byte chunks");
#pragma unroll
    for (int q = 0; q < (int)(V * sizeof(T)) / 16; ++q) {
        const uint4 raw = __ldg((const uint4 *)p + q);
        memcpy(&out[q * 16 / sizeof(T)], &raw, 16);
    }
}

template <typename S, typename T>
__device__ __forceinline__ void st_vec16(S *p, const T (&v)[16 / sizeof(S)]) {
    constexpr int V = 16 / (int)sizeof(S);
    S tmp[V];
#pragma unroll
    for (int c = 0; c < V; ++c) st_s<S, T>(&tmp[c], v[c]);
    uint4 raw;
    memcpy(&raw, tmp, 16);
    *(uint4 *)p = raw;
}

template <typename S, typename T, bool EXACT, bool SIG, bool RES>
__global__ void __launch_bounds__(256) classic2d_kernel(const CycArgs a) {
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    constexpr int V = 16 / (int)sizeof(S);
    constexpr int R = kClassicRows;
    constexpr int BX = 32 * V, BY = 8 * R;
    const long long ld = a.ld;
    const int nx = a.nx, ny = a.ny;
    const int bxn = (nx + 2 + BX - 1) / BX;
    const long long nb = (long long)bxn * ((ny + BY - 1) / BY);
    const Coef<T> kc = make_coef<T>(a);
    const S *__restrict__ uin = (const S *)a.uin;
    const T *__restrict__ f = (const T *)a.f;
    const T *__restrict__ dinv = (const T *)a.dinv;
    S *__restrict__ uout = (S *)a.uout;
    const int lane = threadIdx.x;
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const int c0 = (int)(b % bxn) * BX + lane * V;               // first column of this lane's vector
        const int j0 = 1 + (int)(b / bxn) * BY + (int)threadIdx.y * R;   // first row (warp-uniform)
        if (j0 > ny) continue;
        const bool colok = c0 <= nx + 1;
        T u[R + 2][V], g[R][V];
        T dv[SIG ? R : 1][SIG ? V : 1];
        T hw[R], he[R];
        // every load first: iterate rows j0-1 .. j0+R, RHS (and 1/d) rows j0 .. j0+R-1,
        // and the columns just outside the warp's segment
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            const int row = j0 - 1 + r;
            if (colok && row <= ny + 1 && HJ_IN(a.dbg, (long long)row * ld + c0 + V - 1, grid_elems2d(a), 20)) {
                ld_vec16<S, T>(uin + (long long)row * ld + c0, u[r]);
            } else {
#pragma unroll
                for (int c = 0; c < V; ++c) u[r][c] = (T)0;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = j0 + r;
            const long long q = (long long)row * ld + c0;
            if (colok && row <= ny && HJ_IN(a.dbg, q + V - 1, grid_elems2d(a), 21)) {
                ld_vecT<T, V>(f + q, g[r]);
                if constexpr (SIG) ld_vecT<T, V>(dinv + q, dv[r]);
            } else {
#pragma unroll
                for (int c = 0; c < V; ++c) {
                    g[r][c] = (T)0;
                    if constexpr (SIG) dv[r][c] = (T)0;
                }
            }
            hw[r] = (lane == 0 && c0 >= 1 && row <= ny && HJ_IN(a.dbg, q - 1, grid_elems2d(a), 22)) ? ld_s<S, T>(uin + q - 1)
                                                                                            : (T)0;
            he[r] = (lane == 31 && c0 + V <= nx + 1 && row <= ny && HJ_IN(a.dbg, q + V, grid_elems2d(a), 23))
                        ? ld_s<S, T>(uin + q + V) : (T)0;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = j0 + r;
            T left = __shfl_up_sync(FULL, u[r + 1][V - 1], 1);
            T right = __shfl_down_sync(FULL, u[r + 1][0], 1);
            if (lane == 0) left = hw[r];
            if (lane == 31) right = he[r];
            T out[V];
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const int col = c0 + c;
                const T W = c == 0 ? left : u[r + 1][c > 0 ? c - 1 : 0];
                const T E = c == V - 1 ? right : u[r + 1][c < V - 1 ? c + 1 : 0];
                const T gv = (EXACT || SIG) ? g[r][c] : g[r][c] * kc.invd;
                T res = 0;
                const T nv = point_update<T, EXACT, SIG, true, RES>(kc, gv, SIG ? dv[SIG ? r : 0][SIG ? c : 0] : (T)0,
                                                                    W, E, u[r][c], u[r + 2][c], u[r + 1][c], res);
                const bool in = col >= 1 && col <= nx;
                out[c] = in ? nv : u[r + 1][c];
                if constexpr (RES) {
                    if (in) acc += (Acc)res * (Acc)res;
                }
            }
            if (colok && row <= ny && HJ_IN(a.dbg, (long long)row * ld + c0 + V - 1, grid_elems2d(a), 24))
                st_vec16<S, T>(uout + (long long)row * ld + c0, out);
        }
    }
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

template <typename S, typename T, bool EXACT, bool SIG, bool RES>
__global__ void __launch_bounds__(256) classic1d_kernel(const CycArgs a) {
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    const int bxn = (a.nx + 255) / 256;
    const long long nb = (long long)bxn * a.ny;
    const Coef<T> kc = make_coef<T>(a);
    const S *__restrict__ uin = (const S *)a.uin;
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const int i = 1 + (int)(b % bxn) * 256 + threadIdx.x;
        const int row = (int)(b / bxn);
        if (i > a.nx) continue;
        const long long q = (long long)row * a.ld + i;
        const T old = ld_s<S, T>(uin + q);
        const T W = ld_s<S, T>(uin + q - 1), E = ld_s<S, T>(uin + q + 1);
        const T fv = __ldg((const T *)a.f + q);
        const T iv = SIG ? __ldg((const T *)a.dinv + q) : (T)0;
        const T g = (EXACT || SIG) ? fv : fv * kc.invd;
        T res = 0;
        const T nv = point_update<T, EXACT, SIG, false, RES>(kc, g, iv, W, E, (T)0, (T)0, old, res);
        st_s<S, T>((S *)a.uout + q, nv);
        acc += (Acc)res * (Acc)res;
    }
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

}  // namespace hj

// Registry entry helpers ------------------------------------------------------
#define HJ_K2D(S, T, C, R, NW, H, EX)                                                                \
    {2, 32 * (C) / (H), (R) * (NW) * (H), 32 * (NW), 1,                                               \
     {{hj::hier2d_kernel<S, T, C, R, NW, H, EX, false, false>,                                        \
       hj::hier2d_kernel<S, T, C, R, NW, H, EX, false, true>},                                        \
      {hj::hier2d_kernel<S, T, C, R, NW, H, EX, true, false>, hj::hier2d_kernel<S, T, C, R, NW, H, EX, true, true>}}, \
     {{hj::hier2d_kernel<S, T, C, R, NW, H, EX, false, false, true>,                                  \
       hj::hier2d_kernel<S, T, C, R, NW, H, EX, false, true, true>},                                  \
      {hj::hier2d_kernel<S, T, C, R, NW, H, EX, true, false, true>,                                   \
       hj::hier2d_kernel<S, T, C, R, NW, H, EX, true, true, true>}}}
#define HJ_K1D(S, T, C, WPT, WPB, EX)                                                                \
    {1, 32 * (C) * (WPT), 1, 32 * (WPT) * (WPB), (WPB),                                              \
     {{hj::hier1d_kernel<S, T, C, WPT, WPB, EX, false, false>,                                       \
       hj::hier1d_kernel<S, T, C, WPT, WPB, EX, false, true>},                                       \
      {hj::hier1d_kernel<S, T, C, WPT, WPB, EX, true, false>, hj::hier1d_kernel<S, T, C, WPT, WPB, EX, true, true>}}, \
     {{hj::hier1d_kernel<S, T, C, WPT, WPB, EX, false, false, true>,                                 \
       hj::hier1d_kernel<S, T, C, WPT, WPB, EX, false, true, true>},                                 \
      {hj::hier1d_kernel<S, T, C, WPT, WPB, EX, true, false, true>,                                  \
       hj::hier1d_kernel<S, T, C, WPT, WPB, EX, true, true, true>}}}
#define HJ_KC2D(S, T, EX)                                                                             \
    {2, 32, 8, 256, 1,                                                                               \
     {{hj::classic2d_kernel<S, T, EX, false, false>, hj::classic2d_kernel<S, T, EX, false, true>},   \
      {hj::classic2d_kernel<S, T, EX, true, false>, hj::classic2d_kernel<S, T, EX, true, true>}},     \
     {{nullptr, nullptr}, {nullptr, nullptr}}}
#define HJ_KC1D(S, T, EX)                                                                             \
    {1, 256, 1, 256, 1,                                                                              \
     {{hj::classic1d_kernel<S, T, EX, false, false>, hj::classic1d_kernel<S, T, EX, false, true>},   \
      {hj::classic1d_kernel<S, T, EX, true, false>, hj::classic1d_kernel<S, T, EX, true, true>}},     \
     {{nullptr, nullptr}, {nullptr, nullptr}}}
#define HJ_KVC(S, T, EX)                                                                              \
    {{{hj::vc_kernel<S, T, 1, EX, false>, hj::vc_kernel<S, T, 1, EX, true>},                          \
      {hj::vc_kernel<S, T, 2, EX, false>, hj::vc_kernel<S, T, 2, EX, true>}}}
