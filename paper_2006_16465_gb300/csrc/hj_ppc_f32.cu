// Binary32: TMA-pipelined cycle kernels (hj_tma.cuh), in a translation
// unit of their own so that the library's kernels compile in parallel.
//
// For each subdomain shape the one-stage kernel comes first and is the
// default: the next tile's copy lands while the current tile sweeps in
// registers, which keeps few enough copies in flight per SM for HBM to serve
// them at full rate.  The two-stage kernel is kept for pipeline_stages = 2.
#include "hj_tma.cuh"

namespace hj {

static const PpcKernelInfo k_ppc[] = {
    HJ_KPPC(float, float, 2, 16, 1, 2, false, 1),   // 32 x 32, one stage (default)
    HJ_KPPC(float, float, 2, 16, 1, 2, false, 2),   // 32 x 32, two stages
    HJ_KPPC(float, float, 2, 8, 2, 2, false, 1),   // 32 x 32, two warps, one stage (default)
    HJ_KPPC(float, float, 2, 8, 2, 2, false, 2),   // 32 x 32, two warps, two stages
    HJ_KPPC(float, float, 2, 8, 1, 2, false, 1),   // 32 x 16, one stage (default)
    HJ_KPPC(float, float, 2, 8, 1, 2, false, 2),   // 32 x 16, two stages
    HJ_KPPC(float, float, 2, 4, 1, 2, false, 1),   // 32 x 8, one stage (default)
    HJ_KPPC(float, float, 2, 4, 1, 2, false, 2),   // 32 x 8, two stages
    HJ_KPPC(float, float, 2, 16, 2, 2, false, 1),   // 32 x 64, one stage (default)
    HJ_KPPC(float, float, 2, 16, 2, 2, false, 2),   // 32 x 64, two stages
    HJ_KPPC(float, float, 2, 16, 2, 1, false, 1),   // 64 x 32, one stage (default)
    HJ_KPPC(float, float, 2, 16, 2, 1, false, 2),   // 64 x 32, two stages
    HJ_KPPC(float, float, 2, 16, 4, 1, false, 1),   // 64 x 64, one stage (default)
    HJ_KPPC(float, float, 2, 16, 4, 1, false, 2),   // 64 x 64, two stages
    HJ_KPPC(float, float, 4, 8, 4, 1, false, 1),   // 128 x 32, one stage (default)
    HJ_KPPC(float, float, 4, 8, 4, 1, false, 2),   // 128 x 32, two stages
    HJ_KPPC(float, float, 4, 8, 8, 1, false, 1),   // 128 x 64, one stage (default)
    HJ_KPPC(float, float, 4, 8, 8, 1, false, 2),   // 128 x 64, two stages
};
const PpcKernelInfo *ppc_kernels_f32(int *n) { *n = sizeof(k_ppc) / sizeof(k_ppc[0]); return k_ppc; }

}  // namespace hj
