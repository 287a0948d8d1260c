// hj_inst_f32_sn_hopf.cu -- float kernels of the smooth non-convex family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_sn_hopf(Registry &r)
{
    register_compute<float, HJ_FAM_SMOOTH_NONCONVEX, HJ_HOPF, 1, 2, 4, 5, 8, 10>(r);
    register_cert<float, HJ_FAM_SMOOTH_NONCONVEX, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
