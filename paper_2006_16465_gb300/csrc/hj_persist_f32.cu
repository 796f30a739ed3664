// Binary32: persistent cooperative cycle kernels (hj_persist.cuh,
// hj_persist_tma.cuh), in a
// translation unit of their own so that the library's kernels compile in
// parallel.
#include "hj_persist_tma.cuh"

namespace hj {

static const PersistKernelInfo k_persist[] = {
    HJ_KP2D(float, float, 2, 16, 1, 2, false),
    HJ_KP2D(float, float, 2, 8, 2, 2, false),
    HJ_KP2D(float, float, 2, 4, 4, 2, false),
    HJ_KP2D(float, float, 2, 2, 8, 2, false),
    HJ_KP2D(float, float, 2, 8, 1, 2, false),
    HJ_KP2D(float, float, 2, 4, 1, 2, false),
    HJ_KP2D(float, float, 2, 16, 2, 1, false),
    HJ_KP2D(float, float, 2, 16, 4, 1, false),
    HJ_KP2D(float, float, 4, 8, 8, 1, false),
    HJ_KP1D(float, float, 1, 1, 4, false),
    HJ_KP1D(float, float, 2, 1, 4, false),
    HJ_KP1D(float, float, 1, 2, 1, false),
    HJ_KP1D(float, float, 4, 1, 4, false),
    HJ_KP1D(float, float, 2, 2, 1, false),
    HJ_KP1D(float, float, 1, 4, 1, false),
    HJ_KP1D(float, float, 8, 1, 4, false),
    HJ_KP1D(float, float, 4, 2, 1, false),
    HJ_KP1D(float, float, 2, 4, 1, false),
    HJ_KP1D(float, float, 1, 8, 1, false),
};
const PersistKernelInfo *persist_kernels_f32(int *n) { *n = sizeof(k_persist) / sizeof(k_persist[0]); return k_persist; }

static const PersistClassicInfo k_pclassic = HJ_KPC(float, float, false);
const PersistClassicInfo *persist_classic_f32() { return &k_pclassic; }

}  // namespace hj
