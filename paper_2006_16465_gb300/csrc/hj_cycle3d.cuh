// hj_cycle3d.cuh -- the 3D seven-point extension of the hierarchical cycle
// (the paper's 2D stencil of Section 4 plus a bottom (z - 1) and a top (z + 1)
// neighbour; subdomains of TX x TY x TZ points, Section 4.1 carried to 3D).
//
// Layout of one subdomain in a warp (no shared-memory containers):
//   * LX lanes span x (TX = LX), LY = 32 / LX lane groups span y, and every
//     lane holds RY consecutive rows x RZ planes of its x column in registers:
//     TY = LY * RY, TZ = RZ;
//   * x neighbours come from lane shuffles within the LX-lane segment; the
//     two edge lanes of a segment hold the x-halo column in registers;
//   * y neighbours are registers of the same lane, or the neighbouring lane
//     group's edge row (one shuffle pair per plane), or the frozen y-halo rows;
//   * z neighbours are registers: the sweep walks the planes in order and keeps
//     the old values of the previous plane, the z-halo planes are frozen.
// Each warp owns one subdomain; a CTA holds NW independent warps.  Points
// beyond the grid (ragged last subdomains) keep their staged values, so the
// ghost value at nx + 1 (ny + 1, nz + 1) is the frozen neighbour of the last
// interior point, as in the oracle's truncated subdomain.
//
// Arithmetic per point update:
//   binary64: acc = cW*W; acc += cE*E; acc += cS*S; acc += cN*N; acc += cB*B;
//             acc += cT*T; u' = (f - acc) * (1/d), each operation rounded once
//             (the oracle's order, so the GPU matches it bitwise);
//   binary32: u' = f/d + bT T + bB B + bN N + bS S + bE E + bW W (b = -c/d) as a
//             fused chain.
#pragma once

#include "hj_tma.cuh"

namespace hj {

template <typename T>
struct Coef3 {
    T cW, cE, cS, cN, cB, cT;   // stencil (exact path)
    T bW, bE, bS, bN, bB, bT;   // -c/d (binary32 path)
    T invd, dconst;
};

template <typename T>
__device__ __forceinline__ Coef3<T> make_coef3(const CycArgs &a);
template <>
__device__ __forceinline__ Coef3<double> make_coef3<double>(const CycArgs &a) {
    Coef3<double> k;
    k.cW = a.cW; k.cE = a.cE; k.cS = a.cS; k.cN = a.cN; k.cB = a.cB; k.cT = a.cT;
    k.bW = k.bE = k.bS = k.bN = k.bB = k.bT = 0.0;
    k.invd = a.invd;
    k.dconst = a.dconst;
    return k;
}
template <>
__device__ __forceinline__ Coef3<float> make_coef3<float>(const CycArgs &a) {
    Coef3<float> k;
    k.cW = a.fW; k.cE = a.fE; k.cS = a.fS; k.cN = a.fN; k.cB = a.fB; k.cT = a.fT;
    k.bW = a.gW; k.bE = a.gE; k.bS = a.gS; k.bN = a.gN; k.bB = a.gB; k.bT = a.gT;
    k.invd = a.finvd;
    k.dconst = a.fdconst;
    return k;
}

// One seven-point update.  g: f (binary64) or f/d (binary32).  res receives
// f - (A u)_p of the old value (binary32: divided by d; the caller scales the
// reduced sum by d^2).
template <typename T, bool EXACT, bool WANT_RES>
__device__ __forceinline__ T point_update3(const Coef3<T> &k, T g, T W, T E, T S, T N, T B, T Tp, T old,
                                           T &res) {
    if constexpr (EXACT) {
        double acc = __dmul_rn(k.cW, W);
        acc = __dadd_rn(acc, __dmul_rn(k.cE, E));
        acc = __dadd_rn(acc, __dmul_rn(k.cS, S));
        acc = __dadd_rn(acc, __dmul_rn(k.cN, N));
        acc = __dadd_rn(acc, __dmul_rn(k.cB, B));
        acc = __dadd_rn(acc, __dmul_rn(k.cT, Tp));
        const double t = __dsub_rn(g, acc);
        if constexpr (WANT_RES) res = (T)__dsub_rn(t, __dmul_rn(k.dconst, old));
        return (T)__dmul_rn(t, k.invd);
    } else {
        T t = g;
        t = fma(k.bT, Tp, t);
        t = fma(k.bB, B, t);
        t = fma(k.bN, N, t);
        t = fma(k.bS, S, t);
        t = fma(k.bE, E, t);
        t = fma(k.bW, W, t);
        if constexpr (WANT_RES) res = t - old;
        return t;
    }
}

template <typename S, typename T, int LX, int RY, int RZ, int NW, bool EXACT, bool RES>
__global__ void __launch_bounds__(32 * NW) hier3d_kernel(const CycArgs a) {
    constexpr int LY = 32 / LX, TX = LX, TY = LY * RY, TZ = RZ;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(LX == 8 || LX == 16 || LX == 32, "LX lanes per x segment");
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = lane % LX, gy = lane / LX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nbx = (nx + TX - 1) / TX, nby = (ny + TY - 1) / TY, nbz = (nz + TZ - 1) / TZ;
    const long long nsub = (long long)nbx * nby * nbz;
    const long long sub = (long long)blockIdx.x * NW + warp;
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    if (sub < nsub) {   // warp-uniform
        const int bx = (int)(sub % nbx);
        const int by = (int)((sub / nbx) % nby);
        const int bz = (int)(sub / ((long long)nbx * nby));
        const int x0 = 1 + bx * TX, y0 = 1 + by * TY, z0 = 1 + bz * TZ;
        const int x = x0 + lx, yl = y0 + gy * RY;   // this lane's column and first row
        const long long ld = a.ld, ps = a.ps;
        const S *__restrict__ uin = (const S *)a.uin;
        const T *__restrict__ f = (const T *)a.f;
        const Coef3<T> kc = make_coef3<T>(a);
        // every point of the subdomain inside the grid (so its halo is inside
        // the ghost shell): one base pointer, fixed offsets, no checks
        const bool full = x0 + TX - 1 <= nx && y0 + TY - 1 <= ny && z0 + TZ - 1 <= nz;   // warp-uniform
        // stage: u, f/d, the y- and z-halo values and, on the two edge lanes of
        // each x segment, the x-halo column (xh: W on lane 0, E on lane LX-1)
        T u[RY][RZ], g[RY][RZ], sS[RZ], sN[RZ], hB[RY], hT[RY], xh[RY][RZ];
        const int xo = lx == 0 ? -1 : (lx == LX - 1 ? 1 : 0);   // x-halo offset of this lane (0: none)
        if (full) {
            const long long o = (long long)z0 * ps + (long long)yl * ld + x;
            const S *bu = uin + o;
            const T *bf = f + o;
#pragma unroll
            for (int z = 0; z < RZ; ++z) {
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const long long d = z * ps + r * ld;
                    u[r][z] = ld_s<S, T>(bu + d);
                    const T fv = __ldg(bf + d);
                    g[r][z] = EXACT ? fv : fv * kc.invd;
                    xh[r][z] = xo ? ld_s<S, T>(bu + d + xo) : (T)0;
                }
                sS[z] = gy == 0 ? ld_s<S, T>(bu + z * ps - ld) : (T)0;
                sN[z] = gy == LY - 1 ? ld_s<S, T>(bu + z * ps + RY * ld) : (T)0;
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                hB[r] = ld_s<S, T>(bu - ps + r * ld);
                hT[r] = ld_s<S, T>(bu + TZ * ps + r * ld);
            }
        } else {
            auto ld_u = [&](int xx, int yy, int zz) -> T {
                const bool ok = xx <= nx + 1 && yy <= ny + 1 && zz <= nz + 1;
                return ok ? ld_s<S, T>(uin + (long long)zz * ps + (long long)yy * ld + xx) : (T)0;
            };
#pragma unroll
            for (int z = 0; z < RZ; ++z) {
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const int yy = yl + r, zz = z0 + z;
                    u[r][z] = ld_u(x, yy, zz);
                    const bool in = x <= nx && yy <= ny && zz <= nz;
                    const T fv = in ? __ldg(f + (long long)zz * ps + (long long)yy * ld + x) : (T)0;
                    g[r][z] = EXACT ? fv : fv * kc.invd;
                    xh[r][z] = xo ? ld_u(x + xo, yy, zz) : (T)0;
                }
                sS[z] = gy == 0 ? ld_u(x, y0 - 1, z0 + z) : (T)0;
                sN[z] = gy == LY - 1 ? ld_u(x, y0 + TY, z0 + z) : (T)0;
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                hB[r] = ld_u(x, yl + r, z0 - 1);
                hT[r] = ld_u(x, yl + r, z0 + TZ);
            }
        }
        for (int s = 0; s < a.k; ++s) {
            T prev[RY];   // old values of the plane below
#pragma unroll
            for (int r = 0; r < RY; ++r) prev[r] = hB[r];
#pragma unroll
            for (int z = 0; z < RZ; ++z) {
                T up = sS[z], dn = sN[z];
                if constexpr (LY > 1) {
                    const T a_up = __shfl_up_sync(FULL, u[RY - 1][z], LX);
                    const T a_dn = __shfl_down_sync(FULL, u[0][z], LX);
                    if (gy > 0) up = a_up;
                    if (gy < LY - 1) dn = a_dn;
                }
                T nv[RY];
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const T c = u[r][z];
                    T Wv = __shfl_up_sync(FULL, c, 1, LX);
                    T Ev = __shfl_down_sync(FULL, c, 1, LX);
                    if (lx == 0) Wv = xh[r][z];
                    if (lx == LX - 1) Ev = xh[r][z];
                    const T Sv = r > 0 ? u[r - 1][z] : up;
                    const T Nv = r < RY - 1 ? u[r + 1][z] : dn;
                    const T Tv = z < RZ - 1 ? u[r][z + 1] : hT[r];
                    T res = 0;
                    const T v = point_update3<T, EXACT, RES>(kc, g[r][z], Wv, Ev, Sv, Nv, prev[r], Tv, c, res);
                    const bool in = full || (x <= nx && yl + r <= ny && z0 + z <= nz);
                    nv[r] = in ? v : c;
                    if constexpr (RES) {
                        if (s == 0 && in) acc += (Acc)res * (Acc)res;
                    }
                }
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    prev[r] = u[r][z];
                    u[r][z] = nv[r];
                }
            }
        }
        // write back this lane's interior points
        S *uo = (S *)a.uout;
        if (full) {
            S *bo = uo + (long long)z0 * ps + (long long)yl * ld + x;
#pragma unroll
            for (int z = 0; z < RZ; ++z)
#pragma unroll
                for (int r = 0; r < RY; ++r) st_s<S, T>(bo + z * ps + r * ld, u[r][z]);
        } else {
#pragma unroll
            for (int z = 0; z < RZ; ++z)
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const int yy = yl + r, zz = z0 + z;
                    if (x <= nx && yy <= ny && zz <= nz)
                        st_s<S, T>(uo + (long long)zz * ps + (long long)yy * ld + x, u[r][z]);
                }
        }
    }
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

// ---------------------------------------------------------------------------
// Binary32 variant with two x columns per lane (LX lanes span TX = 2 LX
// columns, LY = 32 / LX lane groups span y with RY rows each, RZ planes per
// lane): half the x shuffles of the one-column kernel, and the frozen halo
// folded into the right-hand-side term once per cycle, as in the 2D binary32
// sweeps.  Within a cycle the halo does not change, so its weighted
// contribution to the updates next to the subdomain's faces is added to
// g = f/d before the first subiteration; the lanes on an x or y face then
// weight what they receive by shuffle (their own value) with zero, and the
// first and last planes drop their B and T terms.  A point update is
// g + bW W + bE E + bS S + bN N + bB B + bT T in the order: the horizontal
// pair (E then W in even columns of the subdomain, W then E in odd ones), then
// S, N, B, T as packed pairs (fma.rn.f32x2, two independent round-to-nearest
// operations).  Per pair of points: two x shuffles, two scalar and five packed
// multiply-adds.
// ---------------------------------------------------------------------------
// Register state of one subdomain in the two-column layout, and the steps
// every binary32 3D kernel applies to it once a stager has filled it: u and
// f (in g), and the frozen halo values the lane needs (x column: W on the
// first lane of a segment, E on the last; y row: S on the first lane group,
// N on the last; the planes below and above).
template <int LX, int RY, int RZ>
struct Pk3 {
    static constexpr int LY = 32 / LX, TX = 2 * LX, TY = LY * RY, TZ = RZ;
    float u[RY][RZ][2], g[RY][RZ][2];
    float xh[RY][RZ], hy[RZ][2], hb[RY][2], ht[RY][2];
};

// g = f/d plus the weighted frozen halo: x faces, y faces, z faces.
template <int LX, int RY, int RZ>
__device__ __forceinline__ void pk3_fold(Pk3<LX, RY, RZ> &t, const Coef3<float> &kc, bool wl, bool el, bool sl,
                                         bool nl) {
#pragma unroll
    for (int z = 0; z < RZ; ++z) {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
#pragma unroll
            for (int c = 0; c < 2; ++c) t.g[r][z][c] *= kc.invd;
            t.g[r][z][0] = fmaf(wl ? kc.bW : 0.f, t.xh[r][z], t.g[r][z][0]);
            t.g[r][z][1] = fmaf(el ? kc.bE : 0.f, t.xh[r][z], t.g[r][z][1]);
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            t.g[0][z][c] = fmaf(sl ? kc.bS : 0.f, t.hy[z][c], t.g[0][z][c]);
            t.g[RY - 1][z][c] = fmaf(nl ? kc.bN : 0.f, t.hy[z][c], t.g[RY - 1][z][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            t.g[r][0][c] = fmaf(kc.bB, t.hb[r][c], t.g[r][0][c]);
            t.g[r][RZ - 1][c] = fmaf(kc.bT, t.ht[r][c], t.g[r][RZ - 1][c]);
        }
    }
}

// k subiterations; returns the lane's share of ||f - A u||^2 / d^2 of the
// staged iterate (RES).  PART: points beyond the grid keep their values.
template <int LX, int RY, int RZ, bool RES, bool PART>
__device__ __forceinline__ float pk3_sweeps(Pk3<LX, RY, RZ> &t, const Coef3<float> &kc, int k, bool wl, bool el,
                                            bool sl, bool nl, int x, int yl, int z0, int nx, int ny, int nz) {
    constexpr int LY = 32 / LX;
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned long long kWE = pk2(wl ? 0.f : kc.bW, el ? 0.f : kc.bE);
    const unsigned long long kS2 = pk2(kc.bS, kc.bS), kN2 = pk2(kc.bN, kc.bN);
    const unsigned long long kS02 = pk2(sl ? 0.f : kc.bS, sl ? 0.f : kc.bS);
    const unsigned long long kNl2 = pk2(nl ? 0.f : kc.bN, nl ? 0.f : kc.bN);
    const unsigned long long kB2 = pk2(kc.bB, kc.bB), kT2 = pk2(kc.bT, kc.bT);
    float acc = 0.f;
#pragma unroll 1
    for (int s = 0; s < k; ++s) {
        float prev[RY][2];   // old values of the plane below
#pragma unroll
        for (int z = 0; z < RZ; ++z) {
            float up[2], dn[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                up[c] = __shfl_up_sync(FULL, t.u[RY - 1][z][c], LX);
                dn[c] = __shfl_down_sync(FULL, t.u[0][z][c], LX);
            }
            float nv[RY][2];
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const float c0 = t.u[r][z][0], c1 = t.u[r][z][1];
                const float sW = __shfl_up_sync(FULL, c1, 1, LX);
                const float sE = __shfl_down_sync(FULL, c0, 1, LX);
                const float a0 = fmaf(kc.bE, c1, t.g[r][z][0]);
                const float a1 = fmaf(kc.bW, c0, t.g[r][z][1]);
                unsigned long long p = ffma2(kWE, pk2(sW, sE), pk2(a0, a1));
                if (r > 0) p = ffma2(kS2, pk2(t.u[r > 0 ? r - 1 : 0][z][0], t.u[r > 0 ? r - 1 : 0][z][1]), p);
                else p = ffma2(kS02, pk2(up[0], up[1]), p);
                if (r < RY - 1)
                    p = ffma2(kN2, pk2(t.u[r < RY - 1 ? r + 1 : 0][z][0], t.u[r < RY - 1 ? r + 1 : 0][z][1]), p);
                else p = ffma2(kNl2, pk2(dn[0], dn[1]), p);
                if (z > 0) p = ffma2(kB2, pk2(prev[r][0], prev[r][1]), p);
                if (z < RZ - 1)
                    p = ffma2(kT2, pk2(t.u[r][z < RZ - 1 ? z + 1 : 0][0], t.u[r][z < RZ - 1 ? z + 1 : 0][1]), p);
                float n0, n1;
                upk2(p, n0, n1);
                bool in0 = true, in1 = true;
                if constexpr (PART) {
                    const bool iyz = yl + r <= ny && z0 + z <= nz;
                    in0 = iyz && x <= nx;
                    in1 = iyz && x + 1 <= nx;
                    n0 = in0 ? n0 : c0;
                    n1 = in1 ? n1 : c1;
                }
                if constexpr (RES) {
                    if (s == 0) {
                        const float r0 = in0 ? n0 - c0 : 0.f, r1 = in1 ? n1 - c1 : 0.f;
                        acc += r0 * r0;
                        acc += r1 * r1;
                    }
                }
                nv[r][0] = n0;
                nv[r][1] = n1;
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    prev[r][c] = t.u[r][z][c];
                    t.u[r][z][c] = nv[r][c];
                }
            }
        }
    }
    (void)LY;
    return acc;
}

// Write back the lane's interior points.
template <int LX, int RY, int RZ>
__device__ __forceinline__ void pk3_store(const Pk3<LX, RY, RZ> &t, float *uo, long long ld, long long ps, bool full,
                                          int x, int yl, int z0, int nx, int ny, int nz) {
#pragma unroll
    for (int z = 0; z < RZ; ++z)
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int yy = yl + r, zz = z0 + z;
                if (full || (x + c <= nx && yy <= ny && zz <= nz))
                    uo[(long long)zz * ps + (long long)yy * ld + x + c] = t.u[r][z][c];
            }
}

template <int LX, int RY, int RZ, int NW, bool RES>
__global__ void __launch_bounds__(32 * NW, 3) hier3d_pk_kernel(const CycArgs a) {
    using P3 = Pk3<LX, RY, RZ>;
    constexpr int LY = P3::LY, TX = P3::TX, TY = P3::TY, TZ = P3::TZ;
    static_assert(LX == 4 || LX == 8 || LX == 16, "LX lanes of two columns per x segment");
    static_assert(LY > 1, "the first and last lane groups are different groups");
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = lane % LX, gy = lane / LX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nbx = (nx + TX - 1) / TX, nby = (ny + TY - 1) / TY, nbz = (nz + TZ - 1) / TZ;
    const long long nsub = (long long)nbx * nby * nbz;
    const long long sub = (long long)blockIdx.x * NW + warp;
    float acc = 0.f;
    if (sub < nsub) {   // warp-uniform
        const int bx = (int)(sub % nbx);
        const int by = (int)((sub / nbx) % nby);
        const int bz = (int)(sub / ((long long)nbx * nby));
        const int x0 = 1 + bx * TX, y0 = 1 + by * TY, z0 = 1 + bz * TZ;
        const int x = x0 + 2 * lx, yl = y0 + gy * RY;   // this lane's first column and first row
        const long long ld = a.ld, ps = a.ps;
        const float *__restrict__ uin = (const float *)a.uin;
        const float *__restrict__ f = (const float *)a.f;
        const Coef3<float> kc = make_coef3<float>(a);
        const bool full = x0 + TX - 1 <= nx && y0 + TY - 1 <= ny && z0 + TZ - 1 <= nz;   // warp-uniform
        const bool wl = lx == 0, el = lx == LX - 1, sl = gy == 0, nl = gy == LY - 1;
        P3 t;
        // stage from global memory.  A subdomain inside the grid loads from one
        // base pointer at fixed offsets; a ragged one checks every load: points
        // beyond the grid read the ghost value (x, y or z = n + 1) or zero, and
        // keep it.  Inside the grid every address within one point of the
        // subdomain is in the ghost shell, so no load needs a lane condition
        // and all of them are in flight before the first use.
        auto stage = [&](auto part_tag) {
            constexpr bool PART = decltype(part_tag)::value;
            const long long o = (long long)z0 * ps + (long long)yl * ld + x;
            const float *bu = uin + o, *bf = f + o;
            // offset (dx, row dy, plane dz) from this lane's first point
            auto ldu = [&](int dx, int dy, int dz) -> float {
                if constexpr (PART) {
                    if (x + dx > nx + 1 || yl + dy > ny + 1 || z0 + dz > nz + 1) return 0.f;
                }
                return ld_s<float, float>(bu + (long long)dz * ps + (long long)dy * ld + dx);
            };
            // the same load where p holds, zero elsewhere, as a predicated
            // instruction (no branch, so it is issued with the others; the
            // lanes that skip it keep the rows it touches, and so its L1
            // wavefronts, to the ones that are needed)
            auto ld_pred = [&](bool p, int dx, int dy, int dz) -> float {
                if constexpr (PART) {
                    if (x + dx > nx + 1 || yl + dy > ny + 1 || z0 + dz > nz + 1) p = false;
                }
                float v = 0.f;
                const float *q = bu + (long long)dz * ps + (long long)dy * ld + dx;
                asm volatile("{\n\t.reg .pred pp;\n\tsetp.ne.b32 pp, %2, 0;\n\t@pp ld.global.nc.f32 %0, [%1];\n\t}"
                             : "+f"(v)
                             : "l"(q), "r"((int)p));
                return v;
            };
            const int xo = wl ? -1 : 2, yo = sl ? -1 : RY;
#pragma unroll
            for (int z = 0; z < RZ; ++z) {
#pragma unroll
                for (int r = 0; r < RY; ++r) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        t.u[r][z][c] = ldu(c, r, z);
                        const bool in = !PART || (x + c <= nx && yl + r <= ny && z0 + z <= nz);
                        t.g[r][z][c] = in ? __ldg(bf + (long long)z * ps + (long long)r * ld + c) : 0.f;
                    }
                    t.xh[r][z] = ld_pred(wl || el, xo, r, z);
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) t.hy[z][c] = ld_pred(sl || nl, c, yo, z);
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    t.hb[r][c] = ldu(c, r, -1);
                    t.ht[r][c] = ldu(c, r, TZ);
                }
            }
        };
        if (full) stage(std::integral_constant<bool, false>());
        else stage(std::integral_constant<bool, true>());
        pk3_fold<LX, RY, RZ>(t, kc, wl, el, sl, nl);
        if (full) acc = pk3_sweeps<LX, RY, RZ, RES, false>(t, kc, a.k, wl, el, sl, nl, x, yl, z0, nx, ny, nz);
        else acc = pk3_sweeps<LX, RY, RZ, RES, true>(t, kc, a.k, wl, el, sl, nl, x, yl, z0, nx, ny, nz);
        pk3_store<LX, RY, RZ>(t, (float *)a.uout, ld, ps, full, x, yl, z0, nx, ny, nz);
    }
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

// ---------------------------------------------------------------------------
// TMA-pipelined binary32 variant for grids much larger than the resident CTAs
// (the 3D counterpart of ppc2d_kernel).  One warp per CTA walks a static list
// of subdomains (t = blockIdx.x + i gridDim.x, x fastest); one lane issues
// cp.async.bulk.tensor copies of the next subdomain's iterate box (subdomain
// + halo) and RHS box into shared memory, completing on an mbarrier, while
// the warp sweeps the current one in registers (the two-column layout of
// hier3d_pk_kernel, from the same steps).  The boxes start at x0 - 1 = bx TX,
// a 16-byte boundary, and are BX = TX + 2 rounded up to four values wide;
// elements beyond the tensor (the ghost shell) read as zero, as the checked
// loads of the one-warp kernel do.  The residual is one partial per CTA,
// folded by the next launch (the deferred fold of the 2D pipelined kernel).
// Every wait on the mbarrier is bounded; on expiry the kernel records the
// error, waits (bounded) for its copy in flight and returns.
// ---------------------------------------------------------------------------
template <int LX, int RY, int RZ>
struct Ppc3Layout {
    static constexpr int LY = 32 / LX, TX = 2 * LX, TY = LY * RY, TZ = RZ;
    static constexpr int BX = round_up(TX + 2, 4);   // box width (iterate and RHS), 16-byte multiple
    static constexpr int UB = BX * (TY + 2) * (TZ + 2) * 4, FB = BX * TY * TZ * 4;
    static constexpr int UB_AL = round_up(UB, 128), FB_AL = round_up(FB, 128);
    static constexpr int TX_BYTES = UB + FB;
    static constexpr int BAR_OFF = UB_AL + FB_AL;
    static constexpr int SMEM = BAR_OFF + 8 + 128;   // + room to align the base to 128 bytes
};

template <int LX, int RY, int RZ, bool RES>
__global__ void __launch_bounds__(32) ppc3d_kernel(const __grid_constant__ PpcArgs P) {
    using L = Ppc3Layout<LX, RY, RZ>;
    using P3 = Pk3<LX, RY, RZ>;
    constexpr int LY = L::LY, TX = L::TX, TY = L::TY, TZ = L::TZ, BX = L::BX;
    static_assert(LY > 1, "the first and last lane groups are different groups");
    const CycArgs &a = P.a;
    const bool reducer = blockIdx.x == gridDim.x - 1;
    if constexpr (RES) {
        volatile Ctl *ctl = a.red.ctl;
        if (ctl->done >= 0) return;
        if (ctl->fold_only[P.parity]) {
            if (reducer) deferred_fold(P);
            return;
        }
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float *su = (float *)smem, *sf = (float *)(smem + L::UB_AL);
    uint64_t *bar = (uint64_t *)(smem + L::BAR_OFF);
    const int lane = threadIdx.x;
    const int lx = lane % LX, gy = lane / LX;
    const bool wl = lx == 0, el = lx == LX - 1, sl = gy == 0, nl = gy == LY - 1;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int txs = P.tiles_x, tys = P.tiles_y;
    const int mine = (P.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    auto issue = [&](int tile) {
        const int bx = tile % txs, by = (tile / txs) % tys, bz = tile / (txs * tys);
        mbar_expect_tx(bar, L::TX_BYTES);
        tma_load_3d(su, &P.mu, bar, bx * TX, by * TY, bz * TZ);
        tma_load_3d(sf, &P.mf, bar, bx * TX, by * TY + 1, bz * TZ + 1);
    };
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (lane == 0 && mine > 0) issue(blockIdx.x);
    // the last CTA has the fewest subdomains when the grid does not divide
    // them: it folds the previous launch's residual while its first copy lands
    if constexpr (RES) {
        if (reducer) deferred_fold(P);
    }
    const Coef3<float> kc = make_coef3<float>(a);
    const long long ld = a.ld, ps = a.ps;
    float acc = 0.f;
    int i = 0;
    bool failed = false;
    for (; i < mine; ++i) {
        bool ok = true;
        long long spins = 0;
        while (!mbar_try_wait(bar, (unsigned)i & 1u)) {
            if (++spins > P.spin_limit) { ok = false; break; }
        }
        if (__syncthreads_or(!ok)) { failed = true; break; }
        const int tile = blockIdx.x + i * gridDim.x;
        const int bx = tile % txs, by = (tile / txs) % tys, bz = tile / (txs * tys);
        const int x0 = 1 + bx * TX, y0 = 1 + by * TY, z0 = 1 + bz * TZ;
        const int x = x0 + 2 * lx, yl = y0 + gy * RY;
        const bool full = x0 + TX - 1 <= nx && y0 + TY - 1 <= ny && z0 + TZ - 1 <= nz;
        // stage from the boxes: iterate box element (X, Y, Z) relative to
        // (x0 - 1, y0 - 1, z0 - 1), RHS box element relative to (x0 - 1, y0, z0)
        P3 t;
        {
            const int cx = 1 + 2 * lx, ry = gy * RY;
            auto U = [&](int X, int Y, int Z) -> float { return su[(Z * (TY + 2) + Y) * BX + X]; };
            const int xo = wl ? 0 : cx + 2, yo = sl ? 0 : ry + RY + 1;
#pragma unroll
            for (int z = 0; z < RZ; ++z) {
#pragma unroll
                for (int r = 0; r < RY; ++r) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        t.u[r][z][c] = U(cx + c, ry + r + 1, z + 1);
                        const bool in = full || (x + c <= nx && yl + r <= ny && z0 + z <= nz);
                        t.g[r][z][c] = in ? sf[(z * TY + ry + r) * BX + cx + c] : 0.f;
                    }
                    t.xh[r][z] = U(xo, ry + r + 1, z + 1);
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) t.hy[z][c] = U(cx + c, yo, z + 1);
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    t.hb[r][c] = U(cx + c, ry + r + 1, 0);
                    t.ht[r][c] = U(cx + c, ry + r + 1, TZ + 1);
                }
            }
        }
        __syncthreads();   // every lane is done with the boxes
        if (lane == 0 && i + 1 < mine) {
            fence_proxy_async_smem();
            issue(blockIdx.x + (i + 1) * gridDim.x);
        }
        pk3_fold<LX, RY, RZ>(t, kc, wl, el, sl, nl);
        if (full) acc += pk3_sweeps<LX, RY, RZ, RES, false>(t, kc, a.k, wl, el, sl, nl, x, yl, z0, nx, ny, nz);
        else acc += pk3_sweeps<LX, RY, RZ, RES, true>(t, kc, a.k, wl, el, sl, nl, x, yl, z0, nx, ny, nz);
        pk3_store<LX, RY, RZ>(t, (float *)a.uout, ld, ps, full, x, yl, z0, nx, ny, nz);
    }
    if (failed) {
        // record the expiry, wait (bounded) for the copy in flight, return
        if (lane == 0) {
            atomicExch(a.err, HJ_ERR_TIMEOUT);
            long long spins = 0;
            while (!mbar_try_wait(bar, (unsigned)i & 1u) && ++spins <= P.spin_limit) {
            }
        }
        __syncthreads();
        return;
    }
    if constexpr (RES) write_cta_partial<1>(P.part_w + blockIdx.x, acc);
}

// ---------------------------------------------------------------------------
// Prefetching variant: persistent warps walk subdomains (warp g takes
// g, g + G, g + 2G, ... for G warps in the grid), and while a warp sweeps one
// subdomain in registers, cp.async copies the next one's box (subdomain +
// halo, (TX+2) x (TY+2) x (TZ+2) values) and its f (TX x TY x TZ) into the
// warp's shared buffers.  The sweep and its arithmetic are those of
// hier3d_kernel, so the iterates are identical.  A box row starts at
// x0 - 1 = bx TX, a multiple of 8 elements, in a row of pitch ld (a multiple
// of 32 elements), so each row is copied as 16-byte chunks plus one chunk
// for its last two elements; the part of a chunk beyond the ghost shell is
// zero-filled without being read (cp.async's source size).
// ---------------------------------------------------------------------------
// copy `bytes` (<= BYTES) of src and zero-fill the rest of the BYTES at dst
template <int BYTES>
__device__ __forceinline__ void cp_async_part(void *dst, const void *src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(bytes)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T, int LX, int RY, int RZ>
struct Pf3Layout {
    static constexpr int LY = 32 / LX, TX = LX, TY = LY * RY, TZ = RZ;
    static constexpr int EPC = 16 / (int)sizeof(T);            // elements per 16-byte chunk
    static constexpr int BX = TX + 2 * (EPC > 2 ? 2 : 1);      // box row pitch: 16-byte multiple, >= TX + 2
    static constexpr int BYR = TY + 2, BZ = TZ + 2;
    static constexpr int BOX = BX * BYR * BZ, FBOX = (TX + EPC) * TY * TZ, XH = 2 * TY * TZ;
    static constexpr int PER_WARP = BOX + FBOX + XH;           // elements (a 16-byte multiple)
    static constexpr int RCH = TX / EPC;                       // full chunks per row
    static_assert(TX % EPC == 0 && (BX * (int)sizeof(T)) % 16 == 0 && (PER_WARP * (int)sizeof(T)) % 16 == 0,
                  "16-byte rows");
};

template <typename S, typename T, int LX, int RY, int RZ, int NW, bool EXACT, bool RES>
__global__ void __launch_bounds__(32 * NW) hier3d_pf_kernel(const CycArgs a) {
    using L = Pf3Layout<T, LX, RY, RZ>;
    constexpr int LY = L::LY, TX = L::TX, TY = L::TY, TZ = L::TZ, BX = L::BX, BYR = L::BYR;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(sizeof(S) == sizeof(T), "binary32 or binary64 storage");
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    extern __shared__ __align__(16) unsigned char pf3_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *box = (T *)pf3_smem + (size_t)warp * L::PER_WARP;
    T *fbox = box + L::BOX;
    T *xh = fbox + L::FBOX;
    const int lx = lane % LX, gy = lane / LX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nbx = (nx + TX - 1) / TX, nby = (ny + TY - 1) / TY, nbz = (nz + TZ - 1) / TZ;
    const long long nsub = (long long)nbx * nby * nbz;
    const long long G = (long long)gridDim.x * NW;
    const long long ld = a.ld, ps = a.ps;
    const S *__restrict__ uin = (const S *)a.uin;
    const T *__restrict__ f = (const T *)a.f;
    const Coef3<T> kc = make_coef3<T>(a);
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    // origin (x0 - 1, y0 - 1, z0 - 1) of subdomain sub's box
    auto origin = [&](long long sub, int &bx0, int &by0, int &bz0) {
        bx0 = (int)(sub % nbx) * TX;
        by0 = (int)((sub / nbx) % nby) * TY;
        bz0 = (int)(sub / ((long long)nbx * nby)) * TZ;
    };
    constexpr int EPC = L::EPC, RCH = L::RCH, ES = (int)sizeof(T);
    // bytes of a chunk of EPC elements starting at global x = gx that lie
    // at or below x = xmax (0 if none)
    auto part = [&](int gx, int n, int xmax) -> int {
        const int m = xmax - gx + 1;
        return (m <= 0 ? 0 : (m >= n ? n : m)) * ES;
    };
    auto prefetch = [&](long long sub) {
        int bx0, by0, bz0;
        origin(sub, bx0, by0, bz0);
        // u box: rows (yy, zz) of TX + 2 elements from x = bx0: RCH 16-byte
        // chunks and a tail chunk holding x = bx0 + TX and bx0 + TX + 1
        constexpr int RQ = RCH + 1, NQ = BYR * L::BZ * RQ;
        for (int q = lane; q < NQ; q += 32) {
            const int j = q % RQ, rho = q / RQ, yy = rho % BYR, zz = rho / BYR;
            const int gyy = by0 + yy, gz = bz0 + zz, gx = bx0 + j * EPC;
            const bool row_ok = gyy <= ny + 1 && gz <= nz + 1;
            const int bytes = row_ok ? part(gx, j < RCH ? EPC : 2, nx + 1) : 0;
            const S *src = uin + (bytes ? (long long)gz * ps + (long long)gyy * ld + gx : 0);
            T *dst = box + rho * BX + j * EPC;
            if (j < RCH) cp_async_part<16>(dst, src, bytes);
            else cp_async_part<2 * sizeof(T)>(dst, src, bytes);
        }
        // f box: TX x TY x TZ interior values, RCH chunks per row from x0 = bx0 + 1
        // (not 16-byte aligned: element-sized copies would be too many, so the
        // row is fetched from bx0, whose chunk 0 carries x0 - 1 .. x0 + EPC - 2,
        // into a scratch row pitch of TX + EPC and read at offset 1)
        for (int q = lane; q < TY * TZ * (RCH + 1); q += 32) {
            const int j = q % (RCH + 1), rho = q / (RCH + 1), yy = rho % TY, zz = rho / TY;
            const int gyy = by0 + 1 + yy, gz = bz0 + 1 + zz, gx = bx0 + j * EPC;
            const bool row_ok = gyy <= ny && gz <= nz;
            const int bytes = row_ok ? part(gx, EPC, nx) : 0;
            const T *src = f + (bytes ? (long long)gz * ps + (long long)gyy * ld + gx : 0);
            cp_async_part<16>(fbox + rho * (TX + EPC) + j * EPC, src, bytes);
        }
        cp_async_commit();
    };
    long long sub = (long long)blockIdx.x * NW + warp;
    if (sub < nsub) prefetch(sub);
    for (; sub < nsub; sub += G) {   // warp-uniform
        cp_async_wait_all();
        __syncwarp();
        int bx0, by0, bz0;
        origin(sub, bx0, by0, bz0);
        const int x0 = bx0 + 1, y0 = by0 + 1, z0 = bz0 + 1;
        const int x = x0 + lx, yl = y0 + gy * RY;
        T u[RY][RZ], g[RY][RZ], sS[RZ], sN[RZ], hB[RY], hT[RY];
        auto B = [&](int zz, int yy, int xx) -> T { return box[(zz * BYR + yy) * BX + xx]; };
#pragma unroll
        for (int z = 0; z < RZ; ++z) {
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                u[r][z] = B(z + 1, gy * RY + r + 1, lx + 1);
                const T fv = fbox[(z * TY + gy * RY + r) * (TX + EPC) + lx + 1];
                g[r][z] = EXACT ? fv : fv * kc.invd;
            }
            sS[z] = B(z + 1, 0, lx + 1);
            sN[z] = B(z + 1, TY + 1, lx + 1);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            hB[r] = B(0, gy * RY + r + 1, lx + 1);
            hT[r] = B(TZ + 1, gy * RY + r + 1, lx + 1);
        }
        for (int t = lane; t < TY * TZ; t += 32) {
            const int yy = t % TY, zz = t / TY;
            xh[t] = B(zz + 1, yy + 1, 0);
            xh[TY * TZ + t] = B(zz + 1, yy + 1, TX + 1);
        }
        __syncwarp();
        // the box is in registers (and xh): copy the next subdomain in
        if (sub + G < nsub) prefetch(sub + G);
        const bool full = x0 + TX - 1 <= nx && y0 + TY - 1 <= ny && z0 + TZ - 1 <= nz;
        for (int s = 0; s < a.k; ++s) {
            T prev[RY];
#pragma unroll
            for (int r = 0; r < RY; ++r) prev[r] = hB[r];
#pragma unroll
            for (int z = 0; z < RZ; ++z) {
                T up = sS[z], dn = sN[z];
                if constexpr (LY > 1) {
                    const T a_up = __shfl_up_sync(FULL, u[RY - 1][z], LX);
                    const T a_dn = __shfl_down_sync(FULL, u[0][z], LX);
                    if (gy > 0) up = a_up;
                    if (gy < LY - 1) dn = a_dn;
                }
                T nv[RY];
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const T c = u[r][z];
                    T Wv = __shfl_up_sync(FULL, c, 1, LX);
                    T Ev = __shfl_down_sync(FULL, c, 1, LX);
                    const int hy = gy * RY + r + TY * z;
                    if (lx == 0) Wv = xh[hy];
                    if (lx == LX - 1) Ev = xh[TY * TZ + hy];
                    const T Sv = r > 0 ? u[r - 1][z] : up;
                    const T Nv = r < RY - 1 ? u[r + 1][z] : dn;
                    const T Tv = z < RZ - 1 ? u[r][z + 1] : hT[r];
                    T res = 0;
                    const T v = point_update3<T, EXACT, RES>(kc, g[r][z], Wv, Ev, Sv, Nv, prev[r], Tv, c, res);
                    const bool in = full || (x <= nx && yl + r <= ny && z0 + z <= nz);
                    nv[r] = in ? v : c;
                    if constexpr (RES) {
                        if (s == 0 && in) acc += (Acc)res * (Acc)res;
                    }
                }
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    prev[r] = u[r][z];
                    u[r][z] = nv[r];
                }
            }
        }
        S *uo = (S *)a.uout;
#pragma unroll
        for (int z = 0; z < RZ; ++z)
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int yy = yl + r, zz = z0 + z;
                if (x <= nx && yy <= ny && zz <= nz)
                    st_s<S, T>(uo + (long long)zz * ps + (long long)yy * ld + x, u[r][z]);
            }
        __syncwarp();   // every lane is done with xh before the next staging
    }
    cp_async_wait_all();
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

// Classic global-memory Jacobi in 3D (Section 3.2's comparator with the
// seven-point stencil): one thread per point, block (32, 8), one z plane per
// blockIdx.z.  Same update arithmetic and fused residual as hier3d_kernel.
template <typename S, typename T, bool EXACT, bool RES>
__global__ void __launch_bounds__(256) classic3d_kernel(const CycArgs a) {
    if constexpr (RES) {
        if (*(volatile int *)&a.red.ctl->done >= 0) return;
    }
    const int x = 1 + blockIdx.x * 32 + threadIdx.x;
    const int y = 1 + blockIdx.y * 8 + threadIdx.y;
    const int z = 1 + blockIdx.z;
    typedef typename std::conditional<EXACT, double, T>::type Acc;
    Acc acc = 0;
    if (x <= a.nx && y <= a.ny) {
        const long long ld = a.ld, ps = a.ps;
        const long long q = (long long)z * ps + (long long)y * ld + x;
        const S *__restrict__ uin = (const S *)a.uin;
        const Coef3<T> kc = make_coef3<T>(a);
        const T old = ld_s<S, T>(uin + q);
        const T W = ld_s<S, T>(uin + q - 1), E = ld_s<S, T>(uin + q + 1);
        const T Sv = ld_s<S, T>(uin + q - ld), Nv = ld_s<S, T>(uin + q + ld);
        const T B = ld_s<S, T>(uin + q - ps), Tv = ld_s<S, T>(uin + q + ps);
        const T fv = __ldg((const T *)a.f + q);
        const T g = EXACT ? fv : fv * kc.invd;
        T res = 0;
        const T nv = point_update3<T, EXACT, RES>(kc, g, W, E, Sv, Nv, B, Tv, old, res);
        st_s<S, T>((S *)a.uout + q, nv);
        acc += (Acc)res * (Acc)res;
    }
    if constexpr (RES) reduce_grid_acc(a.red, acc);
}

}  // namespace hj

// registry entry: tile (TX, TY, TZ), threads, warps per CTA, kernels without /
// with the fused residual, the prefetching kernels and their shared memory
#define HJ_K3D(S, T, LX, RY, RZ, NW, EX)                                                              \
    {(LX), (32 / (LX)) * (RY), (RZ), 32 * (NW), (NW),                                               \
     {hj::hier3d_kernel<S, T, LX, RY, RZ, NW, EX, false>, hj::hier3d_kernel<S, T, LX, RY, RZ, NW, EX, true>}, \
     {hj::hier3d_pf_kernel<S, T, LX, RY, RZ, NW, EX, false>,                                         \
      hj::hier3d_pf_kernel<S, T, LX, RY, RZ, NW, EX, true>},                                         \
     (int)((NW) * hj::Pf3Layout<T, LX, RY, RZ>::PER_WARP * sizeof(T)), {nullptr, nullptr}, 0, 0}

// binary32 entry of the same TX x TY x TZ shape: the two-column kernel, whose
// LX / 2 lanes span x with RY / 2 rows per lane group, the one-column
// prefetching kernel, and the TMA-pipelined two-column kernel with its
// resident CTAs per SM (CPS, measured per shape: more copies in flight slowed
// the 16-wide boxes sharply)
#define HJ_K3D_F32(LX, RY, RZ, NW, CPS)                                                              \
    {(LX), (32 / (LX)) * (RY), (RZ), 32 * (NW), (NW),                                               \
     {hj::hier3d_pk_kernel<(LX) / 2, (RY) / 2, RZ, NW, false>, hj::hier3d_pk_kernel<(LX) / 2, (RY) / 2, RZ, NW, true>}, \
     {hj::hier3d_pf_kernel<float, float, LX, RY, RZ, NW, false, false>,                              \
      hj::hier3d_pf_kernel<float, float, LX, RY, RZ, NW, false, true>},                              \
     (int)((NW) * hj::Pf3Layout<float, LX, RY, RZ>::PER_WARP * sizeof(float)),                       \
     {hj::ppc3d_kernel<(LX) / 2, (RY) / 2, RZ, false>, hj::ppc3d_kernel<(LX) / 2, (RY) / 2, RZ, true>},  \
     hj::Ppc3Layout<(LX) / 2, (RY) / 2, RZ>::SMEM, (CPS)}

// the same without the pipelined kernel (8-wide boxes: 48-byte rows, which
// the copy engine moves too slowly to gain on the one-warp kernel)
#define HJ_K3D_F32_NOPPC(LX, RY, RZ, NW)                                                             \
    {(LX), (32 / (LX)) * (RY), (RZ), 32 * (NW), (NW),                                               \
     {hj::hier3d_pk_kernel<(LX) / 2, (RY) / 2, RZ, NW, false>, hj::hier3d_pk_kernel<(LX) / 2, (RY) / 2, RZ, NW, true>}, \
     {hj::hier3d_pf_kernel<float, float, LX, RY, RZ, NW, false, false>,                              \
      hj::hier3d_pf_kernel<float, float, LX, RY, RZ, NW, false, true>},                              \
     (int)((NW) * hj::Pf3Layout<float, LX, RY, RZ>::PER_WARP * sizeof(float)), {nullptr, nullptr}, 0, 0}
