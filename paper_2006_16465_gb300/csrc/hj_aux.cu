// hj_aux.cu -- grid-wide helper kernels: binary64 residual (with optional
// ||f|| and binary32 copy of r for refinement), the fused refinement update
// u_{o+1} = u_o + d with the next residual, the adjoint gradient
// dL/dsigma = -lambda * u, and the per-point inverse diagonal.
#include <algorithm>

#include "hj_internal.cuh"

namespace hj {

namespace {

// r_p = f_p - (A u)_p in binary64 as a fused multiply-add chain,
// r = f - d u - cW uW - cE uE - cS uS - cN uN (binary64 throughput is low on
// this part; the residual needs no particular rounding order, only binary64).
template <bool D2>
__device__ __forceinline__ double resid_exact(double f, double d, double u, double uW, double uE, double uS,
                                              double uN, double cW, double cE, double cS, double cN) {
    double r = fma(-d, u, f);
    r = fma(-cW, uW, r);
    r = fma(-cE, uE, r);
    if (D2) {
        r = fma(-cS, uS, r);
        r = fma(-cN, uN, r);
    }
    return r;
}

// Binary32 -> binary64 by integer operations: the conversion instruction runs
// on this part's narrow FP64 pipe, which the residual's multiply-adds already
// saturate.  A normal binary32 value becomes the binary64 value with the same
// sign, the exponent re-biased (127 -> 1023) and the 23 fraction bits at the
// top of the 52 (exact, like the conversion); zeros keep their sign; subnormal,
// infinite and NaN inputs (rare) take the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned b = __float_as_uint(x), a = b & 0x7fffffffu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if (a - 0x00800000u < 0x7f000000u)   // exponent field in [1, 254]
        return __longlong_as_double((long long)(sign | ((unsigned long long)a + (896ull << 23)) << 29));
    if (a == 0) return __longlong_as_double((long long)sign);
    return (double)x;
}
template <typename T> __device__ __forceinline__ double to_f64(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return f32_to_f64(x); }

struct AuxArgs {
    const void *f;        // user dtype
    const void *u;        // user dtype
    const void *d;        // refinement correction (float or bf16), nullable
    void *uout;           // refinement: u + d (binary64)
    const double *sigma;  // nullable
    float *r32;           // nullable: binary32 copy of r (interior; ghosts untouched)
    long long ld;         // pitch of f, u, uout, sigma
    long long ld2;        // pitch of r32 and d
    int nx, ny;
    double cW, cE, cS, cN, dconst;
    RedArgs red;
    const double *coef;   // nullable: per-point W, E[, S, N] coefficient planes, cps apart
    long long cps;
};

// Grid-stride walk over blocks of points: 2D blocks of 32 x 8 points (one
// thread each, x fastest), 1D blocks of 256 points of one row.  The grid is
// bounded (a few CTAs per SM), so every CTA reduces its sums once.
template <int D> struct AuxGeom;
template <> struct AuxGeom<2> {
    static __device__ __forceinline__ long long nblocks(int nx, int ny) {
        return (long long)((nx + 31) / 32) * ((ny + 7) / 8);
    }
    static __device__ __forceinline__ bool idx(int nx, int ny, long long b, int &i, int &j) {
        const int bxn = (nx + 31) / 32;
        i = 1 + (int)(b % bxn) * 32 + (int)threadIdx.x;
        j = 1 + (int)(b / bxn) * 8 + (int)threadIdx.y;
        return i <= nx && j <= ny;
    }
};
template <> struct AuxGeom<1> {
    static __device__ __forceinline__ long long nblocks(int nx, int ny) { return (long long)((nx + 255) / 256) * ny; }
    static __device__ __forceinline__ bool idx(int nx, int ny, long long b, int &i, int &j) {
        const int bxn = (nx + 255) / 256;
        i = 1 + (int)(b % bxn) * 256 + (int)threadIdx.x;
        j = (int)(b / bxn);
        return i <= nx;
    }
};

template <typename T, int D, bool WITH_F>
__global__ void __launch_bounds__(256) residual_kernel(const AuxArgs a) {
    int i, j;
    double rr = 0.0, ff = 0.0;
    const long long nb = AuxGeom<D>::nblocks(a.nx, a.ny);
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        if (!AuxGeom<D>::idx(a.nx, a.ny, b, i, j)) continue;
        const T *u = (const T *)a.u;
        const long long q = (long long)j * a.ld + i;
        const double fv = to_f64<T>(((const T *)a.f)[q]);
        const double d = a.sigma ? __dadd_rn(a.dconst, a.sigma[q]) : a.dconst;
        double cW = a.cW, cE = a.cE, cS = a.cS, cN = a.cN;
        if (a.coef) {
            cW = a.coef[q];
            cE = a.coef[a.cps + q];
            if (D == 2) {
                cS = a.coef[2 * a.cps + q];
                cN = a.coef[3 * a.cps + q];
            }
        }
        const double r = resid_exact<D == 2>(fv, d, to_f64<T>(u[q]), to_f64<T>(u[q - 1]), to_f64<T>(u[q + 1]),
                                             D == 2 ? to_f64<T>(u[q - a.ld]) : 0.0,
                                             D == 2 ? to_f64<T>(u[q + a.ld]) : 0.0, cW, cE, cS, cN);
        rr += r * r;
        ff += fv * fv;
        if (a.r32) a.r32[(long long)j * a.ld2 + i] = (float)r;
    }
    if (WITH_F) {
        const double vals[2] = {rr, ff};
        reduce_grid<2>(a.red, vals);
    } else {
        const double vals[1] = {rr};
        reduce_grid<1>(a.red, vals);
    }
}

// Binary32 factors of the variable-coefficient kernels from the caller's
// binary64 coefficients: planes -cW/d, -cE/d[, -cS/d, -cN/d], 1/d, d with
// d_p = dconst + sigma_p (each computed in binary64, then rounded once).
template <int D>
__global__ void __launch_bounds__(256) vc_prep_kernel(const double *coef, const double *sigma, double dconst,
                                                     long long ld, long long ps, int nx, int ny, float *out) {
    int i, j;
    const long long nb = AuxGeom<D>::nblocks(nx, ny);
    constexpr int NP = D == 2 ? 4 : 2;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        if (!AuxGeom<D>::idx(nx, ny, b, i, j)) continue;
        const long long q = (long long)j * ld + i;
        const double d = sigma ? __dadd_rn(dconst, sigma[q]) : dconst;
        const double iv = __drcp_rn(d);
        for (int m = 0; m < NP; ++m) out[m * ps + q] = (float)(-coef[m * ps + q] * iv);
        out[NP * ps + q] = (float)iv;
        out[(NP + 1) * ps + q] = (float)d;
    }
}

template <typename DS>
__device__ __forceinline__ double ld_corr(const DS *p) { return f32_to_f64(__ldg(p)); }
template <>
__device__ __forceinline__ double ld_corr<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return f32_to_f64(__bfloat162float(__ldg(p)));
}

// u_out = u_in + d on interior points, and r = f - A u_out (binary64) with its
// binary32 copy and ||r||^2.  Neighbour values of u_out are re-formed from
// u_in and d (d is zero on the ghost ring), so no point reads a value that
// another thread is writing.
template <typename DS, int D>
__global__ void __launch_bounds__(256) update_residual_kernel(const AuxArgs a) {
    int i, j;
    double rr = 0.0;
    const long long nb = AuxGeom<D>::nblocks(a.nx, a.ny);
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        if (!AuxGeom<D>::idx(a.nx, a.ny, b, i, j)) continue;
        const double *u = (const double *)a.u;
        const DS *dd = (const DS *)a.d;
        const long long q = (long long)j * a.ld + i;
        const long long q2 = (long long)j * a.ld2 + i;
        const double uc = __dadd_rn(u[q], ld_corr<DS>(dd + q2));
        const double uW = __dadd_rn(u[q - 1], ld_corr<DS>(dd + q2 - 1));
        const double uE = __dadd_rn(u[q + 1], ld_corr<DS>(dd + q2 + 1));
        double uS = 0.0, uN = 0.0;
        if (D == 2) {
            uS = __dadd_rn(u[q - a.ld], ld_corr<DS>(dd + q2 - a.ld2));
            uN = __dadd_rn(u[q + a.ld], ld_corr<DS>(dd + q2 + a.ld2));
        }
        ((double *)a.uout)[q] = uc;
        const double fv = ((const double *)a.f)[q];
        const double d = a.sigma ? __dadd_rn(a.dconst, a.sigma[q]) : a.dconst;
        const double r = resid_exact<D == 2>(fv, d, uc, uW, uE, uS, uN, a.cW, a.cE, a.cS, a.cN);
        rr += r * r;
        a.r32[q2] = (float)r;
    }
    const double vals[1] = {rr};
    reduce_grid<1>(a.red, vals);
}

// dL/dsigma_p = -lambda_p u_p (accumulate != 0: added to dsig, for a batch of
// right-hand sides sharing sigma)
template <typename T, int D>
__global__ void __launch_bounds__(256) grad_sigma_kernel(const T *lam, const T *u, double *dsig, long long ld,
                                                         int nx, int ny, int accumulate) {
    int i, j;
    const long long nb = AuxGeom<D>::nblocks(nx, ny);
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        if (!AuxGeom<D>::idx(nx, ny, b, i, j)) continue;
        const long long q = (long long)j * ld + i;
        // separately rounded (no contraction into an FMA), so a batch's sum equals
        // the sum of the per-right-hand-side gradients bit for bit
        const double g = -__dmul_rn((double)lam[q], (double)u[q]);
        dsig[q] = accumulate ? __dadd_rn(dsig[q], g) : g;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) make_dinv_kernel(const double *sigma, double dconst, long long ld,
                                                       long long ld2, int rows, int cols, T *dinv) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int j = blockIdx.y;
    if (i < cols && j < rows)
        dinv[(long long)j * ld2 + i] = (T)__drcp_rn(__dadd_rn(dconst, sigma ? sigma[(long long)j * ld + i] : 0.0));
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

// bounded grid: at most 8 CTAs of 256 threads per SM
dim3 aux_grid(int dim, int nx, int ny) {
    const long long nb = dim == 2 ? (long long)((nx + 31) / 32) * ((ny + 7) / 8)
                                  : (long long)((nx + 255) / 256) * ny;
    return dim3((unsigned)std::min<long long>(nb, 8LL * sm_count()));
}
dim3 aux_block(int dim) { return dim == 2 ? dim3(32, 8) : dim3(256); }

}  // namespace

// rows/cols: the index box of interior points, in grid coordinates
cudaError_t launch_make_dinv_box(const double *sigma, double dconst, long long ld, long long ld2, int row0, int rows,
                                 int col0, int cols, int family, void *dinv, cudaStream_t s) {
    const size_t off = (size_t)row0 * ld + col0, off2 = (size_t)row0 * ld2 + col0;
    const double *sg = sigma ? sigma + off : nullptr;
    dim3 grid((cols + 255) / 256, rows);
    if (family == FAM_F64)
        make_dinv_kernel<double><<<grid, 256, 0, s>>>(sg, dconst, ld, ld2, rows, cols, (double *)dinv + off2);
    else
        make_dinv_kernel<float><<<grid, 256, 0, s>>>(sg, dconst, ld, ld2, rows, cols, (float *)dinv + off2);
    return cudaGetLastError();
}

cudaError_t launch_residual_ex(int dim, int user_f64, const void *f, const void *u, const double *sigma,
                               long long ld, long long ld2, int nx, int ny, double cW, double cE, double cS,
                               double cN, double dconst, int with_fnorm, float *r32, RedArgs red, cudaStream_t s,
                               const double *coef, long long cps) {
    AuxArgs a = {};
    a.f = f; a.u = u; a.sigma = sigma; a.r32 = r32; a.ld = ld; a.ld2 = ld2; a.nx = nx; a.ny = ny;
    a.cW = cW; a.cE = cE; a.cS = cS; a.cN = cN; a.dconst = dconst; a.red = red;
    a.coef = coef; a.cps = cps;
    const dim3 g = aux_grid(dim, nx, ny), b = aux_block(dim);
#define HJ_RES_LAUNCH(T, D)                                                              \
    do {                                                                                 \
        if (with_fnorm) residual_kernel<T, D, true><<<g, b, 0, s>>>(a);                 \
        else residual_kernel<T, D, false><<<g, b, 0, s>>>(a);                           \
    } while (0)
    if (user_f64) {
        if (dim == 2) HJ_RES_LAUNCH(double, 2); else HJ_RES_LAUNCH(double, 1);
    } else {
        if (dim == 2) HJ_RES_LAUNCH(float, 2); else HJ_RES_LAUNCH(float, 1);
    }
#undef HJ_RES_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_update_residual_ex(int dim, const double *f, const double *uin, const void *d, int d_bf16,
                                      double *uout, const double *sigma, float *r32, long long ld, long long ld2,
                                      int nx, int ny, double cW, double cE, double cS, double cN, double dconst,
                                      RedArgs red, cudaStream_t s) {
    AuxArgs a = {};
    a.f = f; a.u = uin; a.d = d; a.uout = uout; a.sigma = sigma; a.r32 = r32; a.ld = ld; a.ld2 = ld2;
    a.nx = nx; a.ny = ny;
    a.cW = cW; a.cE = cE; a.cS = cS; a.cN = cN; a.dconst = dconst; a.red = red;
    const dim3 g = aux_grid(dim, nx, ny), b = aux_block(dim);
    if (d_bf16) {
        if (dim == 2) update_residual_kernel<__nv_bfloat16, 2><<<g, b, 0, s>>>(a);
        else update_residual_kernel<__nv_bfloat16, 1><<<g, b, 0, s>>>(a);
    } else {
        if (dim == 2) update_residual_kernel<float, 2><<<g, b, 0, s>>>(a);
        else update_residual_kernel<float, 1><<<g, b, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_sigma_ex(int dim, int user_f64, const void *lam, const void *u, double *dsig, long long ld,
                                 int nx, int ny, int accumulate, cudaStream_t s) {
    const dim3 g = aux_grid(dim, nx, ny), b = aux_block(dim);
    if (user_f64) {
        if (dim == 2) grad_sigma_kernel<double, 2><<<g, b, 0, s>>>((const double *)lam, (const double *)u, dsig, ld, nx, ny, accumulate);
        else grad_sigma_kernel<double, 1><<<g, b, 0, s>>>((const double *)lam, (const double *)u, dsig, ld, nx, ny, accumulate);
    } else {
        if (dim == 2) grad_sigma_kernel<float, 2><<<g, b, 0, s>>>((const float *)lam, (const float *)u, dsig, ld, nx, ny, accumulate);
        else grad_sigma_kernel<float, 1><<<g, b, 0, s>>>((const float *)lam, (const float *)u, dsig, ld, nx, ny, accumulate);
    }
    return cudaGetLastError();
}

cudaError_t launch_vc_prep(int dim, const double *coef, const double *sigma, double dconst, long long ld,
                           long long ps, int nx, int ny, float *out, cudaStream_t s) {
    const dim3 g = aux_grid(dim, nx, ny), b = aux_block(dim);
    if (dim == 2) vc_prep_kernel<2><<<g, b, 0, s>>>(coef, sigma, dconst, ld, ps, nx, ny, out);
    else vc_prep_kernel<1><<<g, b, 0, s>>>(coef, sigma, dconst, ld, ps, nx, ny, out);
    return cudaGetLastError();
}

namespace {
// ||f - A u||^2 (and ||f||^2) of the seven-point operator over the interior:
// blocks of 32 x 8 points of one plane, grid-stride, deterministic reduction
// (binary64 accumulation in a fixed order per CTA, fixed-order grid fold).
template <typename T, bool WITH_F>
__global__ void __launch_bounds__(256) residual3d_kernel(const T *f, const T *u, long long ld, long long ps, int nx,
                                                        int ny, int nz, double cW, double cE, double cS, double cN,
                                                        double cB, double cT, double dconst, RedArgs red) {
    const int bxn = (nx + 31) / 32, byn = (ny + 7) / 8;
    const long long nb = (long long)bxn * byn * nz;
    double rr = 0.0, ff = 0.0;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const int i = 1 + (int)(b % bxn) * 32 + (int)threadIdx.x;
        const int j = 1 + (int)((b / bxn) % byn) * 8 + (int)threadIdx.y;
        const int z = 1 + (int)(b / ((long long)bxn * byn));
        if (i > nx || j > ny) continue;
        const long long q = (long long)z * ps + (long long)j * ld + i;
        const double fv = to_f64<T>(f[q]);
        double r = fma(-dconst, to_f64<T>(u[q]), fv);
        r = fma(-cW, to_f64<T>(u[q - 1]), r);
        r = fma(-cE, to_f64<T>(u[q + 1]), r);
        r = fma(-cS, to_f64<T>(u[q - ld]), r);
        r = fma(-cN, to_f64<T>(u[q + ld]), r);
        r = fma(-cB, to_f64<T>(u[q - ps]), r);
        r = fma(-cT, to_f64<T>(u[q + ps]), r);
        rr += r * r;
        ff += fv * fv;
    }
    if (WITH_F) {
        const double vals[2] = {rr, ff};
        reduce_grid<2>(red, vals);
    } else {
        const double vals[1] = {rr};
        reduce_grid<1>(red, vals);
    }
}

dim3 aux_grid3(int nx, int ny, int nz) {
    const long long nb = (long long)((nx + 31) / 32) * ((ny + 7) / 8) * nz;
    return dim3((unsigned)std::min<long long>(nb, 8LL * sm_count()));
}
}  // namespace

cudaError_t launch_residual3d(int user_f64, const void *f, const void *u, long long ld, long long ps, int nx,
                              int ny, int nz, double cW, double cE, double cS, double cN, double cB, double cT,
                              double dconst, int with_fnorm, RedArgs red, cudaStream_t s) {
    const dim3 g = aux_grid3(nx, ny, nz), b(32, 8);
#define HJ_R3(T, F)                                                                                                residual3d_kernel<T, F><<<g, b, 0, s>>>((const T *)f, (const T *)u, ld, ps, nx, ny, nz, cW, cE, cS, cN, cB,                                             cT, dconst, red)
    if (user_f64) {
        if (with_fnorm) HJ_R3(double, true); else HJ_R3(double, false);
    } else {
        if (with_fnorm) HJ_R3(float, true); else HJ_R3(float, false);
    }
#undef HJ_R3
    return cudaGetLastError();
}

int aux_max_blocks3(int nx, int ny, int nz) { return (int)aux_grid3(nx, ny, nz).x; }

int aux_max_blocks(int dim, int nx, int ny) {
    const dim3 g = aux_grid(dim, nx, ny);
    return (int)(g.x * g.y);
}

int aux_sm_count() { return sm_count(); }

}  // namespace hj
