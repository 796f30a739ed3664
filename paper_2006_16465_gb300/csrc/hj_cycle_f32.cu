// Binary32 cycle kernels (fused multiply-add chains).
#include "hj_persist.cuh"

namespace hj {

static const TileKernelInfo k_tiles[] = {
    HJ_K2D(float, float, 2, 16, 1, 2, false),    // 32 x 32
    HJ_K2D(float, float, 2, 8, 2, 2, false),     // 32 x 32, two warps
    HJ_K2D(float, float, 2, 8, 1, 2, false),     // 32 x 16
    HJ_K2D(float, float, 2, 4, 1, 2, false),     // 32 x 8
    HJ_K2D(float, float, 2, 16, 2, 2, false),    // 32 x 64
    HJ_K2D(float, float, 2, 16, 2, 1, false),    // 64 x 32
    HJ_K2D(float, float, 2, 16, 4, 1, false),    // 64 x 64
    HJ_K2D(float, float, 4, 8, 4, 1, false),     // 128 x 32
    HJ_K2D(float, float, 4, 8, 8, 1, false),     // 128 x 64
    HJ_K1D(float, float, 1, 4, false),        // 32
    HJ_K1D(float, float, 2, 4, false),        // 64
    HJ_K1D(float, float, 4, 4, false),        // 128
    HJ_K1D(float, float, 8, 4, false),        // 256
};
static const TileKernelInfo k_classic[] = {HJ_KC2D(float, float, false), HJ_KC1D(float, float, false)};

const TileKernelInfo *tile_kernels_f32(int *n) { *n = sizeof(k_tiles) / sizeof(k_tiles[0]); return k_tiles; }
const TileKernelInfo *classic_kernels_f32(int *n) { *n = 2; return k_classic; }

static const PersistKernelInfo k_persist[] = {
    HJ_KP2D(float, float, 2, 16, 1, 2, false),
    HJ_KP2D(float, float, 2, 8, 2, 2, false),
    HJ_KP2D(float, float, 2, 8, 1, 2, false),
    HJ_KP2D(float, float, 2, 4, 1, 2, false),
    HJ_KP2D(float, float, 2, 16, 2, 1, false),
    HJ_KP2D(float, float, 2, 16, 4, 1, false),
    HJ_KP2D(float, float, 4, 8, 8, 1, false),
    HJ_KP1D(float, float, 1, 4, false),
    HJ_KP1D(float, float, 2, 4, false),
    HJ_KP1D(float, float, 4, 4, false),
    HJ_KP1D(float, float, 8, 4, false),
};
const PersistKernelInfo *persist_kernels_f32(int *n) { *n = sizeof(k_persist) / sizeof(k_persist[0]); return k_persist; }

static const PersistClassicInfo k_pclassic = HJ_KPC(float, float, false);
const PersistClassicInfo *persist_classic_f32() { return &k_pclassic; }

}  // namespace hj
