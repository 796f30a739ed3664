// hj_cycle3d.cu -- registries of the 3D seven-point kernels (hj_cycle3d.cuh).
//
// Shapes: LX lanes along x, 32 / LX lane groups along y with RY rows each,
// RZ planes per lane, four warps (four subdomains) per CTA.  Binary32 runs the
// same shapes with two columns per lane (LX / 2 lanes along x, RY / 2 rows
// per lane group); its prefetching variant keeps one column per lane.
//   binary32: 16 x 8 x 8 (default), 32 x 4 x 8, 8 x 8 x 8, 16 x 8 x 4, 32 x 8 x 4
//   binary64: 16 x 4 x 8 (default), 8 x 8 x 8, 32 x 2 x 8, 16 x 8 x 4
#include "hj_cycle3d.cuh"

namespace hj {

namespace {
const Tile3Info k3_f32[] = {
    HJ_K3D_F32(16, 4, 8, 4, 8),    // 16 x 8 x 8
    HJ_K3D_F32(32, 4, 8, 4, 0),    // 32 x 4 x 8
    HJ_K3D_F32_NOPPC(8, 2, 8, 4),  // 8 x 8 x 8
    HJ_K3D_F32(16, 4, 4, 4, 12),   // 16 x 8 x 4
    HJ_K3D_F32(32, 8, 4, 4, 0),    // 32 x 8 x 4
};
const Tile3Info k3_f64[] = {
    HJ_K3D(double, double, 16, 2, 8, 4, true),
    HJ_K3D(double, double, 8, 2, 8, 4, true),
    HJ_K3D(double, double, 32, 2, 8, 4, true),
    HJ_K3D(double, double, 16, 4, 4, 4, true),
};
}  // namespace

const Tile3Info *tiles3d_f64(int *n) {
    *n = (int)(sizeof(k3_f64) / sizeof(k3_f64[0]));
    return k3_f64;
}
const Tile3Info *tiles3d_f32(int *n) {
    *n = (int)(sizeof(k3_f32) / sizeof(k3_f32[0]));
    return k3_f32;
}

CycKernel classic3d_kernel_of(int fam, int res) {
    if (fam == FAM_F64) return res ? classic3d_kernel<double, double, true, true> : classic3d_kernel<double, double, true, false>;
    return res ? classic3d_kernel<float, float, false, true> : classic3d_kernel<float, float, false, false>;
}

}  // namespace hj
