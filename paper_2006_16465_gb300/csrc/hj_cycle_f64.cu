// Binary64 cycle kernels (exact evaluation order, no fused multiply-add).
#include "hj_cycle.cuh"
#include "hj_tma.cuh"

namespace hj {

static const TileKernelInfo k_tiles[] = {
    HJ_K2D(double, double, 1, 16, 2, 1, true),   // 32 x 32
    HJ_K2D(double, double, 1, 16, 1, 1, true),   // 32 x 16
    HJ_K2D(double, double, 1, 8, 1, 1, true),    // 32 x 8
    HJ_K2D(double, double, 1, 16, 4, 1, true),   // 32 x 64
    HJ_K2D(double, double, 2, 8, 4, 1, true),    // 64 x 32
    HJ_K2D(double, double, 2, 8, 8, 1, true),    // 64 x 64
    HJ_K1D(double, double, 1, 1, 4, true),    // 32
    HJ_K1D(double, double, 2, 1, 4, true),    // 64
    HJ_K1D(double, double, 1, 2, 1, true),    // 64, 2 warps
    HJ_K1D(double, double, 4, 1, 4, true),    // 128
    HJ_K1D(double, double, 2, 2, 1, true),    // 128, 2 warps
    HJ_K1D(double, double, 1, 4, 1, true),    // 128, 4 warps
    HJ_K1D(double, double, 8, 1, 4, true),    // 256
    HJ_K1D(double, double, 4, 2, 1, true),    // 256, 2 warps
    HJ_K1D(double, double, 2, 4, 1, true),    // 256, 4 warps
    HJ_K1D(double, double, 1, 8, 1, true),    // 256, 8 warps
};
static const TileKernelInfo k_classic[] = {HJ_KC2D(double, double, true), HJ_KC1D(double, double, true)};

const TileKernelInfo *tile_kernels_f64(int *n) { *n = sizeof(k_tiles) / sizeof(k_tiles[0]); return k_tiles; }
const TileKernelInfo *classic_kernels_f64(int *n) { *n = 2; return k_classic; }

static const PpcKernelInfo k_ppc[] = {
    HJ_KPPC(double, double, 1, 16, 2, 1, true, 2),   // 32 x 32
    HJ_KPPC(double, double, 1, 16, 1, 1, true, 2),   // 32 x 16
    HJ_KPPC(double, double, 1, 8, 1, 1, true, 2),   // 32 x 8
    HJ_KPPC(double, double, 1, 16, 4, 1, true, 2),   // 32 x 64
    HJ_KPPC(double, double, 2, 8, 4, 1, true, 2),   // 64 x 32
    HJ_KPPC(double, double, 2, 8, 8, 1, true, 2),   // 64 x 64
};
const PpcKernelInfo *ppc_kernels_f64(int *n) { *n = sizeof(k_ppc) / sizeof(k_ppc[0]); return k_ppc; }

static const VcKernelInfo k_vc = HJ_KVC(double, double, true);
const VcKernelInfo *vc_kernels_f64() { return &k_vc; }

}  // namespace hj
