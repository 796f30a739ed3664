// hj_noalloc.cu -- hj_cycles_noalloc: hierarchical (or classic) Jacobi cycles
// that allocate no memory at all.
//
// Who needs it: callers that must not allocate device memory at the point
// where they run cycles, for example
//   * services that reserve their whole device-memory budget at start-up and
//     forbid allocation afterwards (predictable latency, no fragmentation);
//   * real-time loops, where cudaMalloc's latency and the device-wide
//     synchronisation it may imply are not acceptable;
//   * callers whose device memory is owned by another allocator or capped.
// hj_create is not usable there: it allocates the handle's workspace (the
// second iterate buffer, reduction buffers, graphs).  This entry point takes
// the one piece of scratch the cycle kernels need -- the buffer that holds
// u_{c+1} while u_c is read -- from a static device array compiled into the
// library, and launches the kernels directly (no graph, no handle).
//
// The array (kNoAllocBytes) exists once per GPU that loads the library and
// lives until the process exits.  Its device address is obtained with
// cudaGetSymbolAddress the first time the entry point runs on a device, with
// that device current, so that first call should come before any stream
// capture; in host code the array's name is only a host-side stand-in and
// must never be passed to a kernel.  The address is cached per device
// together with the id of the CUDA context it belongs to: after
// cudaDeviceReset (a new primary context) the next call looks it up again,
// and that call too should come before any stream capture.  Every call shares the array
// and it keeps the last call's contents: each call first copies the caller's
// u (ghost ring included) into it, so nothing stale is ever read.  Calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and corrupt each other's results.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "hj_runtime.cuh"

using namespace hj;

namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;   // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
struct ScratchSlot {
    unsigned long long ctx_id;   // id of the context the address belongs to (0: none yet)
    void *addr;
};
ScratchSlot g_slot[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (cuCtxGetId, through
// the runtime's driver entry points: the library does not link libcuda), or 0
// if no context is current yet.  Ids are never reused within a process, so a
// context created after cudaDeviceReset never matches a cached address.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool queried = false;
    if (!queried) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_cuCtxGetCurrent_v4000)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
        queried = true;
    }
    CUcontext c = nullptr;
    if (!get_cur || get_cur(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    if (!get_id || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id + 1;   // keep 0 for "no context"
}

// Device address of the static scratch array on the current device: looked up
// on the first call per device, and again whenever the device's context has
// changed since (cudaDeviceReset).
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return seterr(HJ_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return seterr(HJ_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchSlot &sl = g_slot[dev];
    const unsigned long long id = current_context_id();
    if (!sl.addr || id == 0 || sl.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // makes the device's context current if none is
        if (e != cudaSuccess || !p)
            return seterr(HJ_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
        sl.addr = p;
        sl.ctx_id = current_context_id();
    }
    *out = sl.addr;
    return HJ_OK;
}

const TileKernelInfo *pick(int fam, int dim, int tx, int ty, bool classic) {
    int n = 0;
    const TileKernelInfo *k = classic ? (fam == FAM_F64 ? classic_kernels_f64(&n) : classic_kernels_f32(&n))
                                      : (fam == FAM_F64 ? tile_kernels_f64(&n) : tile_kernels_f32(&n));
    for (int i = 0; i < n; ++i)
        if (k[i].dim == dim && (classic || (k[i].tx == tx && (dim == 1 || k[i].ty == ty)))) return &k[i];
    return nullptr;
}

}  // namespace

extern "C" int hj_cycles_noalloc(const hj_desc *desc, const hj_params *params, const void *f, void *u,
                                 hj_stream stream) {
    if (!desc || !params || !f || !u) return seterr(HJ_ERR_INVALID_ARG, "desc, params, f and u must be non-NULL");
    const hj_desc &d = *desc;
    const hj_params &p = *params;
    if (d.dim != 1 && d.dim != 2) return seterr(HJ_ERR_INVALID_ARG, "dim must be 1 or 2");
    if (d.nx < 1 || d.ny < 1) return seterr(HJ_ERR_INVALID_ARG, "nx, ny must be >= 1");
    if (d.dtype != HJ_F64 && d.dtype != HJ_F32) return seterr(HJ_ERR_INVALID_ARG, "dtype must be HJ_F64 or HJ_F32");
    const size_t esz = d.dtype == HJ_F64 ? 8 : 4;
    if (d.ld < (long long)d.nx + 2 || (d.ld * (long long)esz) % 16)
        return seterr(HJ_ERR_INVALID_ARG, "ld must be >= nx + 2 with ld * element size a multiple of 16");
    if (d.dim == 1 && d.ny > 65535) return seterr(HJ_ERR_INVALID_ARG, "1D: at most 65535 rows");
    if (d.dim == 2 && (d.ny + 7) / 8 > 65535) return seterr(HJ_ERR_INVALID_ARG, "2D: ny must be <= 524280");
    if (d.sigma) return seterr(HJ_ERR_UNSUPPORTED, "per-point sigma needs workspace; use sigma_const or hj_create");
    if (d.coef) return seterr(HJ_ERR_UNSUPPORTED, "per-point neighbour coefficients need workspace; use hj_create");
    const bool f64 = p.precision == HJ_PREC_F64;
    if (!(f64 || p.precision == HJ_PREC_F32) || f64 != (d.dtype == HJ_F64))
        return seterr(HJ_ERR_INVALID_ARG, "precision must be HJ_PREC_F64 (binary64 data) or HJ_PREC_F32 (binary32 data)");
    if (p.method != HJ_METHOD_HIER && p.method != HJ_METHOD_CLASSIC) return seterr(HJ_ERR_INVALID_ARG, "unknown method");
    if (p.k < 1) return seterr(HJ_ERR_INVALID_ARG, "k must be >= 1");
    if (p.overlap_x > 0 || (d.dim == 2 && p.overlap_y > 0))
        return seterr(HJ_ERR_UNSUPPORTED, "hj_cycles_noalloc does not take overlapping subdomains");
    // the engines below need workspace or a handle: refuse them rather than ignore them
    if (p.in_place != 0) return seterr(HJ_ERR_UNSUPPORTED, "hj_cycles_noalloc: in_place must be 0");
    if (p.persistent == 1) return seterr(HJ_ERR_UNSUPPORTED, "hj_cycles_noalloc: persistent must not be 1");
    if (p.pipeline == 1) return seterr(HJ_ERR_UNSUPPORTED, "hj_cycles_noalloc: pipeline must not be 1");
    if (p.autotune != 0) return seterr(HJ_ERR_UNSUPPORTED, "hj_cycles_noalloc: autotune must be 0");
    if (p.fixed_cycles < 0) return seterr(HJ_ERR_INVALID_ARG, "fixed_cycles (the cycle count) must be >= 0");
    const double off = fabs(d.cW) + fabs(d.cE) + (d.dim == 2 ? fabs(d.cS) + fabs(d.cN) : 0.0);
    const double dc = d.cD + d.sigma_const;
    if (!(dc > 0.0) || dc < off) return seterr(HJ_ERR_NOT_DIAG_DOMINANT, "diagonal %g < sum |off-diagonal| %g", dc, off);
    const int rows = d.dim == 2 ? d.ny + 2 : d.ny;
    const size_t bytes = (size_t)rows * (size_t)d.ld * esz;
    if (bytes > kNoAllocBytes)
        return seterr(HJ_ERR_INVALID_ARG,
                      "grid needs %zu bytes of scratch (rows * ld * element size); hj_cycles_noalloc holds at "
                      "most %zu bytes (16 MiB): use hj_create/hj_solve for larger grids",
                      bytes, kNoAllocBytes);
    if (((uintptr_t)f & 15) || ((uintptr_t)u & 15)) return seterr(HJ_ERR_INVALID_ARG, "f and u must be 16-byte aligned");
    const bool classic = p.method == HJ_METHOD_CLASSIC;
    const TileKernelInfo *ki = pick(f64 ? FAM_F64 : FAM_F32, d.dim, p.tile_x, p.tile_y, classic);
    if (!ki) return seterr(HJ_ERR_UNSUPPORTED, "tile %dx%d not built for this precision", p.tile_x, p.tile_y);
    if (p.fixed_cycles == 0) return HJ_OK;

    void *scratch = nullptr;
    CKS(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    // the other iterate buffer starts as a copy of u: same ghost ring, and
    // nothing of an earlier call survives
    CKR(cudaMemcpyAsync(scratch, u, bytes, cudaMemcpyDeviceToDevice, s));

    CycArgs a;
    memset(&a, 0, sizeof(a));
    a.f = f;
    a.ld = d.ld;
    a.nx = d.nx;
    a.ny = d.ny;
    a.k = p.k;
    a.cW = d.cW;
    a.cE = d.cE;
    a.cS = d.dim == 2 ? d.cS : 0.0;
    a.cN = d.dim == 2 ? d.cN : 0.0;
    a.dconst = dc;
    a.invd = 1.0 / dc;
    a.fW = (float)a.cW; a.fE = (float)a.cE; a.fS = (float)a.cS; a.fN = (float)a.cN;
    a.gW = (float)(-a.cW * a.invd); a.gE = (float)(-a.cE * a.invd);
    a.gS = (float)(-a.cS * a.invd); a.gN = (float)(-a.cN * a.invd);
    a.finvd = (float)a.invd;
    a.fdconst = (float)a.dconst;

    dim3 grid, block;
    if (classic) {
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const long long nb = d.dim == 2 ? classic2d_blocks(d.nx, d.ny, (int)esz)
                                        : (long long)((d.nx + 255) / 256) * d.ny;
        grid = dim3((unsigned)std::min<long long>(nb, 8LL * nsm));
        block = d.dim == 2 ? dim3(32, 8) : dim3(256);
    } else if (d.dim == 2) {
        grid = dim3((d.nx + ki->tx - 1) / ki->tx, (d.ny + ki->ty - 1) / ki->ty);
        block = dim3(ki->threads);
    } else {
        const int tiles = (d.nx + ki->tx - 1) / ki->tx;
        grid = dim3((tiles + ki->tiles_per_cta - 1) / ki->tiles_per_cta, d.ny);
        block = dim3(ki->threads);
    }
    CycKernel fn = ki->fn[0][0];   // no per-point sigma, no residual: no reduction scratch needed
    for (long long c = 0; c < p.fixed_cycles; ++c) {
        a.uin = (c & 1) ? scratch : u;
        a.uout = (c & 1) ? u : scratch;
        fn<<<grid, block, 0, s>>>(a);
    }
    CKR(cudaGetLastError());
    if (p.fixed_cycles & 1) CKR(cudaMemcpyAsync(u, scratch, bytes, cudaMemcpyDeviceToDevice, s));
    return HJ_OK;
}
