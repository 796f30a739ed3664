// hj_mg.cu -- hierarchical Jacobi as the smoother of a geometric multigrid
// V-cycle (the use the paper's conclusion names; the V-cycle is the textbook
// one of the multigrid tutorial it cites).
//
// Levels: level 0 is the caller's 2D grid; level l + 1 halves the interior
// ((n - 1) / 2 points per axis, coarse point (I, J) on fine point (2I, 2J)),
// and its operator rediscretises the stencil on the doubled spacing (every
// h^-2 coefficient divided by 4, sigma_const kept).
//
// Kernels (one launch each, all captured in one CUDA graph per handle):
//   * mg_smooth_kernel: one weighted hierarchical cycle, a thread per point of
//     up to four rows, the subdomain plus halo in two shared-memory
//     containers, k damped Jacobi subiterations u' = u + omega (jac - u)
//     with the halo frozen;
//   * mg_restrict_kernel: the fine residual f - A u at the nine fine points
//     around each coarse point, full-weighted into the coarse right-hand side
//     (fused, no residual array), and the coarse correction set to zero;
//   * mg_prolong_kernel: u + bilinear interpolation of the coarse correction,
//     one thread per coarse cell writing the 2 x 2 fine points inside it.
// The graph also holds the residual norm of the level-0 iterate and its copy
// to pinned host memory, so a V-cycle costs one graph launch and one wait.
//
// Binary64 evaluates every sum in the oracle's order with separately rounded
// operations (no fused multiply-add), so the GPU V-cycle equals the oracle's
// bit for bit; binary32 uses fused chains.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "hj_runtime.cuh"

namespace hj {

namespace {

struct MgXferArgs {
    const void *f;       // fine right-hand side (restriction)
    const void *u;       // fine iterate (restriction: input; prolongation: u_in)
    void *uout;          // prolongation output (may equal u)
    void *fc;            // coarse right-hand side (restriction output)
    void *ec;            // coarse correction (restriction: zeroed; prolongation: input)
    long long ld, ldc;
    int nx, ny, ncx, ncy;
    double d, cW, cE, cS, cN;
};

// What a smoothing launch stages besides its level's iterate and RHS:
//   MG_PLAIN:    u and f of the level;
//   MG_RESTRICT: the level's first smoothing after the restriction: the RHS is
//                the full-weighted fine residual (x: the finer level), formed
//                here and also stored as the level's f, and the iterate (the
//                coarse correction) starts at zero;
//   MG_PROLONG:  the level's first smoothing after the coarse solve: the
//                iterate is u + the bilinear interpolation of the coarse
//                correction (x: this level as the fine one), formed here for
//                the subdomain and its halo.
enum MgStage { MG_PLAIN = 0, MG_RESTRICT = 1, MG_PROLONG = 2 };

struct MgSmoothArgs {
    const void *f;
    const void *uin;
    void *uout;
    long long ld;
    int nx, ny, k, stage;   // stage: MgStage (the kernel instance is chosen by it)
    double cW, cE, cS, cN, invd, omega;
    float fW, fE, fS, fN, finvd, fomega;   // binary32: -c/d, 1/d, omega
    MgXferArgs x;                          // MG_RESTRICT / MG_PROLONG
};

template <typename T>
__device__ __forceinline__ T ld_g(const T *p) {
    return __ldg(p);
}

// f - A u at fine index q, in the oracle's order (binary64) or fused (binary32)
template <typename T, bool EXACT>
__device__ __forceinline__ T mg_resid(const MgXferArgs &x, const T *u, const T *f, long long q) {
    if constexpr (EXACT) {
        double au = __dmul_rn(x.d, u[q]);
        au = __dadd_rn(au, __dmul_rn(x.cW, u[q - 1]));
        au = __dadd_rn(au, __dmul_rn(x.cE, u[q + 1]));
        au = __dadd_rn(au, __dmul_rn(x.cS, u[q - x.ld]));
        au = __dadd_rn(au, __dmul_rn(x.cN, u[q + x.ld]));
        return __dsub_rn(f[q], au);
    } else {
        T r = fmaf(-(T)x.d, u[q], f[q]);
        r = fmaf(-(T)x.cW, u[q - 1], r);
        r = fmaf(-(T)x.cE, u[q + 1], r);
        r = fmaf(-(T)x.cS, u[q - x.ld], r);
        r = fmaf(-(T)x.cN, u[q + x.ld], r);
        return r;
    }
}

// The full-weighted fine residual at coarse point (I, J): the restriction.
template <typename T, bool EXACT>
__device__ __forceinline__ T restrict_at(const MgXferArgs &x, int I, int J) {
    const T *u = (const T *)x.u, *f = (const T *)x.f;
    const long long q = 2LL * J * x.ld + 2LL * I, ld = x.ld;
    const T r00 = mg_resid<T, EXACT>(x, u, f, q);
    if constexpr (EXACT) {
        double s1 = __dadd_rn(mg_resid<T, EXACT>(x, u, f, q - 1), mg_resid<T, EXACT>(x, u, f, q + 1));
        s1 = __dadd_rn(s1, mg_resid<T, EXACT>(x, u, f, q - ld));
        s1 = __dadd_rn(s1, mg_resid<T, EXACT>(x, u, f, q + ld));
        double s2 = __dadd_rn(mg_resid<T, EXACT>(x, u, f, q - ld - 1), mg_resid<T, EXACT>(x, u, f, q - ld + 1));
        s2 = __dadd_rn(s2, mg_resid<T, EXACT>(x, u, f, q + ld - 1));
        s2 = __dadd_rn(s2, mg_resid<T, EXACT>(x, u, f, q + ld + 1));
        double t = __dmul_rn(4.0, r00);
        t = __dadd_rn(t, __dmul_rn(2.0, s1));
        t = __dadd_rn(t, s2);
        return __dmul_rn(t, 0.0625);
    } else {
        const T s1 = (mg_resid<T, EXACT>(x, u, f, q - 1) + mg_resid<T, EXACT>(x, u, f, q + 1)) +
                     (mg_resid<T, EXACT>(x, u, f, q - ld) + mg_resid<T, EXACT>(x, u, f, q + ld));
        const T s2 = (mg_resid<T, EXACT>(x, u, f, q - ld - 1) + mg_resid<T, EXACT>(x, u, f, q - ld + 1)) +
                     (mg_resid<T, EXACT>(x, u, f, q + ld - 1) + mg_resid<T, EXACT>(x, u, f, q + ld + 1));
        return (4.0f * r00 + 2.0f * s1 + s2) * 0.0625f;
    }
}

// Bilinear interpolation of the coarse correction: a fine point between four
// coarse points (both indices odd), between two (one odd), or on one.
template <typename T, bool EXACT>
__device__ __forceinline__ T avg2(T x, T y) {
    if constexpr (EXACT) return __dmul_rn(__dadd_rn(x, y), 0.5);
    else return (x + y) * (T)0.5;
}

template <typename T, bool EXACT>
__device__ __forceinline__ T avg4(T e00, T e10, T e01, T e11) {
    if constexpr (EXACT) {
        double t = __dadd_rn(e00, e10);
        t = __dadd_rn(t, e01);
        t = __dadd_rn(t, e11);
        return __dmul_rn(t, 0.25);
    } else {
        return ((e00 + e10) + (e01 + e11)) * (T)0.25;
    }
}

// The correction at interior fine point (i, j); coarse point (I, J) lies on
// fine point (2I, 2J), and the coarse ghost ring holds zeros.  Columns
// i >> 1 and (i + 1) >> 1 are the two coarse columns around an odd i and both
// the one under an even i (rows likewise); the value for each parity of i is
// formed and one is selected, so neighbouring lanes (alternating parities) do
// not diverge.  Each value is the prolongation kernel's formula for its parity.
template <typename T, bool EXACT>
__device__ __forceinline__ T prolong_at(const MgXferArgs &x, int i, int j) {
    const T *e = (const T *)x.ec;
    const long long ldc = x.ldc;
    const int cl = i >> 1, cr = (i + 1) >> 1;
    const bool odd_i = i & 1;
    const T *r0 = e + (long long)(j >> 1) * ldc;
    if (j & 1) {
        const T *r1 = r0 + ldc;
        const T e00 = r0[cl], e10 = r0[cr], e01 = r1[cl], e11 = r1[cr];
        const T vo = avg4<T, EXACT>(e00, e10, e01, e11), ve = avg2<T, EXACT>(e00, e01);
        return odd_i ? vo : ve;
    }
    const T e00 = r0[cl], e10 = r0[cr];
    const T vo = avg2<T, EXACT>(e00, e10);
    return odd_i ? vo : e00;
}

// RPT rows per thread: thread (tx, ty) of a (TX, BY) block owns rows
// ty + m BY (m < RPT) of a TX x (BY RPT) subdomain, so each thread keeps RPT
// independent loads of u and f in flight (one point per thread leaves too
// few bytes in flight per SM to cover HBM latency).
template <typename T, bool EXACT, int RPT, int STAGE>
__global__ void __launch_bounds__(1024 / RPT, (RPT == 1 && STAGE == MG_PLAIN) ? 2 : 1)
    mg_smooth_kernel(const MgSmoothArgs a) {
    extern __shared__ __align__(16) unsigned char mg_smem[];
    const int TX = blockDim.x, BY = blockDim.y, TY = BY * RPT, lw = TX + 2, lh = TY + 2;
    T *buf0 = (T *)mg_smem, *buf1 = buf0 + lw * lh;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = 1 + blockIdx.x * TX + tx, j0 = 1 + blockIdx.y * TY;
    const int nx = a.nx, ny = a.ny;
    const long long ld = a.ld;
    const T *__restrict__ u = (const T *)a.uin;
    constexpr int stage = STAGE;
    auto ld_u = [&](int jj, int ii) -> T {
        if (ii > nx + 1 || jj > ny + 1 || stage == MG_RESTRICT) return (T)0;
        T v = ld_g(u + (long long)jj * ld + ii);
        if (stage == MG_PROLONG && ii >= 1 && ii <= nx && jj >= 1 && jj <= ny) {
            const T c = prolong_at<T, EXACT>(a.x, ii, jj);
            v = EXACT ? (T)__dadd_rn(v, c) : v + c;
        }
        return v;
    };
    // every global load first, then the shared-memory stores
    T v0[RPT], hw[RPT], he[RPT], g[RPT];
    bool in[RPT];
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        const int j = j0 + ty + m * BY;
        in[m] = i <= nx && j <= ny;
        v0[m] = ld_u(j, i);
        hw[m] = tx == 0 ? ld_u(j, i - 1) : (T)0;
        he[m] = tx == TX - 1 ? ld_u(j, i + 1) : (T)0;
        T fv = (T)0;
        if (in[m]) {
            if (stage == MG_RESTRICT) {
                fv = restrict_at<T, EXACT>(a.x, i, j);
                ((T *)a.x.fc)[(long long)j * ld + i] = fv;
            } else {
                fv = ld_g((const T *)a.f + (long long)j * ld + i);
            }
        }
        g[m] = EXACT ? fv : fv * (T)a.finvd;
    }
    const T hs = ty == 0 ? ld_u(j0 - 1, i) : (T)0;
    const T hn = ty == BY - 1 ? ld_u(j0 + TY, i) : (T)0;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        const int me = (ty + m * BY + 1) * lw + tx + 1;
        buf0[me] = v0[m];
        buf1[me] = v0[m];
        if (tx == 0) { buf0[me - 1] = hw[m]; buf1[me - 1] = hw[m]; }
        if (tx == TX - 1) { buf0[me + 1] = he[m]; buf1[me + 1] = he[m]; }
    }
    if (ty == 0) { buf0[tx + 1] = hs; buf1[tx + 1] = hs; }
    if (ty == BY - 1) { buf0[(TY + 1) * lw + tx + 1] = hn; buf1[(TY + 1) * lw + tx + 1] = hn; }
    __syncthreads();
    for (int s = 0; s < a.k; ++s) {
        const T *src = (s & 1) ? buf1 : buf0;
        T *dst = (s & 1) ? buf0 : buf1;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            if (!in[m]) continue;
            const int me = (ty + m * BY + 1) * lw + tx + 1;
            const T old = src[me];
            const T W = src[me - 1], E = src[me + 1], Sv = src[me - lw], Nv = src[me + lw];
            T nv;
            if constexpr (EXACT) {
                double acc = __dmul_rn(a.cW, W);
                acc = __dadd_rn(acc, __dmul_rn(a.cE, E));
                acc = __dadd_rn(acc, __dmul_rn(a.cS, Sv));
                acc = __dadd_rn(acc, __dmul_rn(a.cN, Nv));
                const double jac = __dmul_rn(__dsub_rn(g[m], acc), a.invd);
                nv = __dadd_rn(old, __dmul_rn(a.omega, __dsub_rn(jac, old)));
            } else {
                T t = g[m];
                t = fmaf(a.fN, Nv, t);
                t = fmaf(a.fS, Sv, t);
                t = fmaf(a.fE, E, t);
                t = fmaf(a.fW, W, t);
                nv = fmaf(a.fomega, t - old, old);
            }
            dst[me] = nv;
        }
        __syncthreads();
    }
    const T *fin = (a.k & 1) ? buf1 : buf0;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        const int j = j0 + ty + m * BY;
        if (in[m]) ((T *)a.uout)[(long long)j * ld + i] = fin[(ty + m * BY + 1) * lw + tx + 1];
    }
}

template <typename T, bool EXACT>
__global__ void __launch_bounds__(256) mg_restrict_kernel(const MgXferArgs x) {
    const int I = 1 + blockIdx.x * 32 + threadIdx.x, J = 1 + blockIdx.y * 8 + threadIdx.y;
    if (I > x.ncx || J > x.ncy) return;
    const long long qc = (long long)J * x.ldc + I;
    ((T *)x.fc)[qc] = restrict_at<T, EXACT>(x, I, J);
    ((T *)x.ec)[qc] = (T)0;
}

// One thread per coarse cell (a, b), a in [0, ncx], b in [0, ncy]: the fine
// points (2a+1 | 2a+2, 2b+1 | 2b+2) inside it, each with the oracle's formula
// for its parity; a warp writes coalesced pairs of every fine row.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(256) mg_prolong_kernel(const MgXferArgs x) {
    const int ca = blockIdx.x * 32 + threadIdx.x, cb = blockIdx.y * 8 + threadIdx.y;
    if (ca > x.ncx || cb > x.ncy) return;
    const T *e = (const T *)x.ec;
    const long long r0 = (long long)cb * x.ldc, r1 = r0 + x.ldc;
    const T e00 = e[r0 + ca], e10 = e[r0 + ca + 1], e01 = e[r1 + ca], e11 = e[r1 + ca + 1];
    const int i1 = 2 * ca + 1, j1 = 2 * cb + 1;
    const bool xe = ca < x.ncx, ye = cb < x.ncy;   // the even column / row exists
    const T *ui = (const T *)x.u;
    T *uo = (T *)x.uout;
    auto put = [&](int ii, int jj, T v) {
        const long long q = (long long)jj * x.ld + ii;
        const T un = ui[q];
        uo[q] = EXACT ? (T)__dadd_rn(un, v) : un + v;
    };
    put(i1, j1, avg4<T, EXACT>(e00, e10, e01, e11));             // (odd, odd)
    if (xe) put(i1 + 1, j1, avg2<T, EXACT>(e10, e11));          // (even, odd)
    if (ye) put(i1, j1 + 1, avg2<T, EXACT>(e01, e11));          // (odd, even)
    if (xe && ye) put(i1 + 1, j1 + 1, e11);                     // (even, even)
}

MgSmoothArgs smooth_args(const MgLevel &L, const void *f, const void *uin, void *uout, int k, double omega,
                         double sigma_const) {
    MgSmoothArgs a;
    memset(&a, 0, sizeof(a));
    a.f = f;
    a.uin = uin;
    a.uout = uout;
    a.ld = L.ld;
    a.nx = L.nx;
    a.ny = L.ny;
    a.k = k;
    a.stage = MG_PLAIN;
    a.cW = L.cW; a.cE = L.cE; a.cS = L.cS; a.cN = L.cN;
    a.invd = 1.0 / (L.cD + sigma_const);
    a.omega = omega;
    a.fW = (float)(-L.cW * a.invd); a.fE = (float)(-L.cE * a.invd);
    a.fS = (float)(-L.cS * a.invd); a.fN = (float)(-L.cN * a.invd);
    a.finvd = (float)a.invd;
    a.fomega = (float)omega;
    return a;
}

// Launch one smoothing cycle on level l (buffer cur -> 1 - cur); tile tx x ty.
// x: the transfer a MG_RESTRICT / MG_PROLONG launch forms while staging.
void launch_smooth(hj_handle *h, int l, int cur, int tx, int ty, int k, double omega, cudaStream_t s,
                   int stage = MG_PLAIN, const MgXferArgs *x = nullptr) {
    const MgLevel &L = h->mg[l];
    void *buf[2] = {L.a, L.b};
    MgSmoothArgs a = smooth_args(L, L.f, buf[cur], buf[1 - cur], k, omega, h->d.sigma_const);
    if (x) {
        a.stage = stage;
        a.x = *x;
    }
    // rows per thread: 4 (or 2) when the subdomain height allows, 1 otherwise
    const int rpt = (ty % 4 == 0 && ty >= 8) ? 4 : (ty % 2 == 0 && ty >= 4) ? 2 : 1;
    const dim3 block(tx, ty / rpt), grid((L.nx + tx - 1) / tx, (L.ny + ty - 1) / ty);
    const bool f64 = h->fam_outer == FAM_F64;
    const int smem = 2 * (tx + 2) * (ty + 2) * (f64 ? 8 : 4);
#define HJ_MG_SMOOTH(T, EX, ST)                                                            \
    do {                                                                                   \
        if (rpt == 4) mg_smooth_kernel<T, EX, 4, ST><<<grid, block, smem, s>>>(a);         \
        else if (rpt == 2) mg_smooth_kernel<T, EX, 2, ST><<<grid, block, smem, s>>>(a);    \
        else mg_smooth_kernel<T, EX, 1, ST><<<grid, block, smem, s>>>(a);                  \
    } while (0)
#define HJ_MG_SMOOTH_ST(T, EX)                                        \
    do {                                                              \
        if (a.stage == MG_RESTRICT) HJ_MG_SMOOTH(T, EX, MG_RESTRICT); \
        else if (a.stage == MG_PROLONG) HJ_MG_SMOOTH(T, EX, MG_PROLONG); \
        else HJ_MG_SMOOTH(T, EX, MG_PLAIN);                           \
    } while (0)
    if (f64) HJ_MG_SMOOTH_ST(double, true);
    else HJ_MG_SMOOTH_ST(float, false);
#undef HJ_MG_SMOOTH_ST
#undef HJ_MG_SMOOTH
}

MgXferArgs xfer_args(const hj_handle *h, int l) {
    const MgLevel &F = h->mg[l], &Cc = h->mg[l + 1];
    MgXferArgs x;
    memset(&x, 0, sizeof(x));
    x.ld = F.ld;
    x.ldc = Cc.ld;
    x.nx = F.nx; x.ny = F.ny;
    x.ncx = Cc.nx; x.ncy = Cc.ny;
    x.d = F.cD + h->d.sigma_const;
    x.cW = F.cW; x.cE = F.cE; x.cS = F.cS; x.cN = F.cN;
    return x;
}

// Levels up to this many points fold the transfers into their smoothing
// launches (record_level).
constexpr long long kMgFuseMaxPoints = 512LL * 512;

void launch_restrict(const hj_handle *h, const MgXferArgs &x, int ncx, int ncy, cudaStream_t s) {
    const dim3 g((ncx + 31) / 32, (ncy + 7) / 8), b(32, 8);
    if (h->fam_outer == FAM_F64) mg_restrict_kernel<double, true><<<g, b, 0, s>>>(x);
    else mg_restrict_kernel<float, false><<<g, b, 0, s>>>(x);
}

// The V-cycle below level l, starting from buffer cur of level l; returns the
// buffer that holds the level's result.  rin: the restriction from the finer
// level, still to be formed (by this level's first smoothing launch, or by a
// restriction launch when the level starts without one); null at level 0.
//
// Launch count: on levels of a few hundred thousand points or fewer a launch
// costs its fixed latency (a few microseconds) whatever its size, so there the
// transfers are folded into the launches next to them where the result is the
// same: the restriction into the coarse level's first smoothing (which forms
// the coarse RHS for its subdomain while staging, stores it for the level's
// later launches, and starts from a zero correction, as the restriction sets
// it) and the prolongation into the fine level's first post-smoothing (which
// stages u + P e for its subdomain and halo).  On larger levels the separate
// transfer kernels stay: they form each value once with coalesced accesses,
// where a smoothing launch would recompute the halo's.  The coarsest level's
// cycles are always one launch (one subdomain whose halo is the level's fixed
// zero boundary, so c cycles of k subiterations are c k subiterations).
int record_level(hj_handle *h, int l, int cur, cudaStream_t s, const MgXferArgs *rin) {
    const hj_params &p = h->p;
    const int levels = (int)h->mg.size();
    const MgLevel &L = h->mg[l];
    if (l == levels - 1) {
        if (p.mg_coarse_cycles <= 0) {
            if (rin) launch_restrict(h, *rin, L.nx, L.ny, s);
            return cur;
        }
        if (l > 0) {
            launch_smooth(h, l, cur, L.nx, L.ny, p.mg_coarse_k * p.mg_coarse_cycles, 1.0, s, MG_RESTRICT, rin);
            return cur ^ 1;
        }
        for (int c = 0; c < p.mg_coarse_cycles; ++c) {
            launch_smooth(h, l, cur, L.nx, L.ny, p.mg_coarse_k, 1.0, s);
            cur ^= 1;
        }
        return cur;
    }
    const bool small = (long long)L.nx * L.ny <= kMgFuseMaxPoints;
    const MgXferArgs *pending = rin;
    if (pending && (!small || p.mg_pre == 0)) {
        launch_restrict(h, *pending, L.nx, L.ny, s);
        pending = nullptr;
    }
    for (int c = 0; c < p.mg_pre; ++c) {
        launch_smooth(h, l, cur, p.tile_x, p.tile_y, p.k, p.mg_omega, s, MG_RESTRICT, pending);
        pending = nullptr;
        cur ^= 1;
    }
    MgXferArgs x = xfer_args(h, l);
    const MgLevel &Cc = h->mg[l + 1];
    x.f = L.f;
    x.u = cur ? L.b : L.a;
    x.fc = Cc.f;
    x.ec = Cc.a;
    const int ce = record_level(h, l + 1, 0, s, &x);
    x.ec = ce ? Cc.b : Cc.a;
    x.u = cur ? L.b : L.a;
    // level 0 must end in buffer a (the graph is replayed from there): when
    // pre + post is odd, a prolongation launch writes the other buffer
    const bool flip = l == 0 && ((p.mg_pre + p.mg_post) & 1);
    const bool fuse = small && p.mg_post > 0 && !flip;
    if (!fuse) {
        x.uout = flip ? (cur ? L.a : L.b) : const_cast<void *>(x.u);
        const dim3 g((Cc.nx + 1 + 31) / 32, (Cc.ny + 1 + 7) / 8), b(32, 8);   // coarse cells 0..ncx x 0..ncy
        if (h->fam_outer == FAM_F64) mg_prolong_kernel<double, true><<<g, b, 0, s>>>(x);
        else mg_prolong_kernel<float, false><<<g, b, 0, s>>>(x);
        if (flip) cur ^= 1;
    }
    for (int c = 0; c < p.mg_post; ++c) {
        launch_smooth(h, l, cur, p.tile_x, p.tile_y, p.k, p.mg_omega, s, MG_PROLONG, (fuse && c == 0) ? &x : nullptr);
        cur ^= 1;
    }
    return cur;
}

RedArgs store_red(const hj_handle *h) {
    RedArgs r;
    memset(&r, 0, sizeof(r));
    r.partials = h->partials;
    r.gpart = h->gpart;
    r.gcnt = h->gcnt;
    r.fcnt = h->fcnt;
    r.hist = h->hist;
    r.out = h->rstore;
    r.ctl = h->ctl;
    r.mode = RED_STORE;
    r.scale = 1.0;
    return r;
}

// ||f - A u||^2 of the level-0 buffer a into pinned host memory (h_rstore).
cudaError_t record_residual(hj_handle *h, cudaStream_t s) {
    const MgLevel &L = h->mg[0];
    const hj_desc &d = h->d;
    cudaError_t e = launch_residual_ex(2, d.dtype == HJ_F64, L.f, L.a, nullptr, d.ld, d.ld, d.nx, d.ny, d.cW, d.cE,
                                       d.cS, d.cN, d.cD + d.sigma_const, 0, nullptr, store_red(h), s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(h->h_rstore, h->rstore, sizeof(double), cudaMemcpyDeviceToHost, s);
}

}  // namespace

int mg_levels_of(int nx, int ny) {
    int L = 1;
    while (nx > 1 && ny > 1 && (nx & 1) && (ny & 1)) {
        nx = (nx - 1) / 2;
        ny = (ny - 1) / 2;
        ++L;
    }
    return L;
}

int mg_setup(hj_handle *h, int levels) {
    const hj_desc &d = h->d;
    const size_t esz = h->esz;
    h->mg.resize(levels);
    int nx = d.nx, ny = d.ny;
    double cW = d.cW, cE = d.cE, cS = d.cS, cN = d.cN, cD = d.cD;
    size_t total = 0;
    for (int l = 0; l < levels; ++l) {
        MgLevel &L = h->mg[l];
        L.nx = nx;
        L.ny = ny;
        L.ld = l == 0 ? d.ld : ((long long)nx + 2 + 31) / 32 * 32;
        L.cW = cW; L.cE = cE; L.cS = cS; L.cN = cN; L.cD = cD;
        total += 3 * (size_t)(ny + 2) * L.ld * esz;
        nx = (nx - 1) / 2;
        ny = (ny - 1) / 2;
        cW /= 4.0; cE /= 4.0; cS /= 4.0; cN /= 4.0; cD /= 4.0;
    }
    if (dmalloc(&h->mg_arena, total) != cudaSuccess) {
        cudaGetLastError();
        return seterr(HJ_ERR_NO_MEMORY, "cudaMalloc of %zu bytes failed (multigrid levels)", total);
    }
    CKR(cudaMemset(h->mg_arena, 0, total));
    unsigned char *p = (unsigned char *)h->mg_arena;
    for (int l = 0; l < levels; ++l) {
        MgLevel &L = h->mg[l];
        const size_t b = (size_t)(L.ny + 2) * L.ld * esz;
        L.a = p; p += b;
        L.b = p; p += b;
        L.f = p; p += b;
    }
    return HJ_OK;
}

// V-cycles until ||r_c|| <= tol ||r_0|| (or fixed_cycles V-cycles), u in/out.
int solve_mg(hj_handle *h, const void *f, void *u, cudaStream_t s, hj_stats *st) {
    const MgLevel &L0 = h->mg[0];
    CKR(cudaMemcpyAsync(L0.a, u, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    CKR(cudaMemcpyAsync(L0.b, u, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    CKR(cudaMemcpyAsync(L0.f, f, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    // one graph per kind of run: a converging run's V-cycle ends with the
    // level-0 residual norm (binary64 arithmetic, a large share of a binary32
    // V-cycle on this part's FP64 pipe) and its copy to pinned host memory; a
    // fixed-cycle run reads no residual, so its V-cycle has neither
    const long long fixed = h->p.fixed_cycles;
    cudaGraphExec_t &exec = fixed > 0 ? h->mg_exec_fixed : h->mg_exec;
    if (!exec) {
        cudaGraph_t graph;
        CKR(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        const int fin = record_level(h, 0, 0, h->cap, nullptr);
        cudaError_t le = cudaGetLastError();
        if (le == cudaSuccess && fixed <= 0) le = record_residual(h, h->cap);
        cudaError_t ee = cudaStreamEndCapture(h->cap, &graph);
        if (le != cudaSuccess) return seterr(HJ_ERR_CUDA, "multigrid capture: %s", cudaGetErrorString(le));
        if (ee != cudaSuccess) return seterr(HJ_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
        if (fin != 0) {
            cudaGraphDestroy(graph);
            return seterr(HJ_ERR_CUDA, "internal: V-cycle does not end in the level-0 buffer");
        }
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            exec = nullptr;
            return seterr(HJ_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        }
    }
    long long c = 0, hl = 0;
    bool stalled = false;
    int status = HJ_OK;
    double r0 = -1.0, rc = -1.0;
    if (fixed > 0) {
        for (c = 0; c < fixed; ++c) CKR(cudaGraphLaunch(exec, s));
    } else {
        CKR(record_residual(h, s));
        CKR(cudaStreamSynchronize(s));
        r0 = rc = sqrt(std::max(h->h_rstore[0], 0.0));
        status = HJ_ERR_NOT_CONVERGED;
        // the last kStall + 1 residuals: a V-cycle contracts by a fixed factor
        // until the storage precision's floor (binary32 u: about eps |u| / h^2
        // relative), so a drop of less than 1 % over kStall V-cycles ends the solve
        constexpr int kStall = 4;
        double ring[kStall + 1];
        for (;;) {
            if (st && st->history && hl < st->history_cap) st->history[hl++] = rc;
            ring[c % (kStall + 1)] = rc;
            if (!std::isfinite(rc)) { status = HJ_ERR_DIVERGED; break; }
            if (rc <= h->p.tol * r0) { status = HJ_OK; break; }
            if (c >= h->p.max_cycles) break;
            if (c >= kStall && rc > 0.99 * ring[(c - kStall) % (kStall + 1)]) { stalled = true; break; }
            CKR(cudaGraphLaunch(exec, s));
            CKR(cudaStreamSynchronize(s));
            rc = sqrt(std::max(h->h_rstore[0], 0.0));
            ++c;
        }
    }
    CKR(cudaMemcpyAsync(u, L0.a, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
    CKR(cudaStreamSynchronize(s));
    if (st) {
        st->cycles = c;
        st->cycles_launched = c;
        st->inner_cycles = 0;
        st->outer_steps = 0;
        st->res0 = r0;
        st->res_final = rc;
        st->rel_final = r0 > 0 ? rc / r0 : 0.0;
        st->history_len = hl;
        st->persistent = 0;
    }
    if (status == HJ_ERR_DIVERGED) return seterr(HJ_ERR_DIVERGED, "residual became non-finite at V-cycle %lld", c);
    if (status == HJ_ERR_NOT_CONVERGED)
        return seterr(HJ_ERR_NOT_CONVERGED, "tolerance %g not met after %lld V-cycles (rel %g%s)", h->p.tol, c,
                      r0 > 0 ? rc / r0 : 0.0, stalled ? "; the residual stopped falling" : "");
    return HJ_OK;
}

}  // namespace hj
