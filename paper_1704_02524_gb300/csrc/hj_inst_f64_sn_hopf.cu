// hj_inst_f64_sn_hopf.cu -- double kernels of the smooth non-convex family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_sn_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_SMOOTH_NONCONVEX, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_SMOOTH_NONCONVEX, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
