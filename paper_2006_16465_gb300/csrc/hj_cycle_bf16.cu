// Binary32 arithmetic on bfloat16-stored iterates (the refinement correction).
#include "hj_cycle.cuh"

namespace hj {

static const TileKernelInfo k_tiles[] = {
    HJ_K2D(__nv_bfloat16, float, 2, 16, 1, 2, false),    // 32 x 32
    HJ_K2D(__nv_bfloat16, float, 2, 8, 2, 2, false),     // 32 x 32, two warps
    HJ_K2D(__nv_bfloat16, float, 2, 4, 4, 2, false),     // 32 x 32, four warps
    HJ_K2D(__nv_bfloat16, float, 2, 2, 8, 2, false),     // 32 x 32, eight warps
    HJ_K2D(__nv_bfloat16, float, 2, 8, 1, 2, false),     // 32 x 16
    HJ_K2D(__nv_bfloat16, float, 2, 4, 1, 2, false),     // 32 x 8
    HJ_K2D(__nv_bfloat16, float, 2, 16, 2, 2, false),    // 32 x 64
    HJ_K2D(__nv_bfloat16, float, 2, 16, 2, 1, false),    // 64 x 32
    HJ_K2D(__nv_bfloat16, float, 2, 16, 4, 1, false),    // 64 x 64
    HJ_K2D(__nv_bfloat16, float, 4, 8, 4, 1, false),     // 128 x 32
    HJ_K2D(__nv_bfloat16, float, 4, 8, 8, 1, false),     // 128 x 64
    HJ_K1D(__nv_bfloat16, float, 1, 1, 4, false),    // 32
    HJ_K1D(__nv_bfloat16, float, 2, 1, 4, false),    // 64
    HJ_K1D(__nv_bfloat16, float, 1, 2, 1, false),    // 64, 2 warps
    HJ_K1D(__nv_bfloat16, float, 4, 1, 4, false),    // 128
    HJ_K1D(__nv_bfloat16, float, 2, 2, 1, false),    // 128, 2 warps
    HJ_K1D(__nv_bfloat16, float, 1, 4, 1, false),    // 128, 4 warps
    HJ_K1D(__nv_bfloat16, float, 8, 1, 4, false),    // 256
    HJ_K1D(__nv_bfloat16, float, 4, 2, 1, false),    // 256, 2 warps
    HJ_K1D(__nv_bfloat16, float, 2, 4, 1, false),    // 256, 4 warps
    HJ_K1D(__nv_bfloat16, float, 1, 8, 1, false),    // 256, 8 warps
};
static const TileKernelInfo k_classic[] = {HJ_KC2D(__nv_bfloat16, float, false), HJ_KC1D(__nv_bfloat16, float, false)};

const TileKernelInfo *tile_kernels_bf16(int *n) { *n = sizeof(k_tiles) / sizeof(k_tiles[0]); return k_tiles; }
const TileKernelInfo *classic_kernels_bf16(int *n) { *n = 2; return k_classic; }

}  // namespace hj
