// Binary64: persistent cooperative cycle kernels (hj_persist.cuh,
// hj_persist_tma.cuh), in a
// translation unit of their own so that the library's kernels compile in
// parallel.
#include "hj_persist_tma.cuh"

namespace hj {

static const PersistKernelInfo k_persist[] = {
    HJ_KP2D(double, double, 1, 16, 2, 1, true),
    HJ_KP2D(double, double, 1, 16, 1, 1, true),
    HJ_KP2D(double, double, 1, 8, 1, 1, true),
    HJ_KP2D(double, double, 2, 8, 4, 1, true),
    HJ_KP1D(double, double, 1, 1, 4, true),
    HJ_KP1D(double, double, 2, 1, 4, true),
    HJ_KP1D(double, double, 1, 2, 1, true),
    HJ_KP1D(double, double, 4, 1, 4, true),
    HJ_KP1D(double, double, 2, 2, 1, true),
    HJ_KP1D(double, double, 1, 4, 1, true),
    HJ_KP1D(double, double, 8, 1, 4, true),
    HJ_KP1D(double, double, 4, 2, 1, true),
    HJ_KP1D(double, double, 2, 4, 1, true),
    HJ_KP1D(double, double, 1, 8, 1, true),
};
const PersistKernelInfo *persist_kernels_f64(int *n) { *n = sizeof(k_persist) / sizeof(k_persist[0]); return k_persist; }

static const PersistClassicInfo k_pclassic = HJ_KPC(double, double, true);
const PersistClassicInfo *persist_classic_f64() { return &k_pclassic; }

}  // namespace hj
