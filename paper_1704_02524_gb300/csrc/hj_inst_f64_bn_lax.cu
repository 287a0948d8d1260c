// hj_inst_f64_bn_lax.cu -- double kernels of the bump-norm family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_bn_lax(Registry &r)
{
    register_compute<double, HJ_FAM_BUMP_NORM, HJ_LAX, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_BUMP_NORM, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
