// hj_inst_f32_bn_hopf.cu -- float kernels of the bump-norm family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_bn_hopf(Registry &r)
{
    register_compute<float, HJ_FAM_BUMP_NORM, HJ_HOPF, 1, 2, 4, 8>(r);
    register_cert<float, HJ_FAM_BUMP_NORM, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
