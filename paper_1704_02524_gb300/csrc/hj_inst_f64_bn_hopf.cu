// hj_inst_f64_bn_hopf.cu -- double kernels of the bump-norm family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_bn_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_BUMP_NORM, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_BUMP_NORM, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
