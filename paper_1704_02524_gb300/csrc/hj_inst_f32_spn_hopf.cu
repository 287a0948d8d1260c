// hj_inst_f32_spn_hopf.cu -- float kernels of the split-norm family (and of the bump norm,
// its one-block case), Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_spn_hopf(Registry &r)
{
    register_compute<float, HJ_FAM_SPLIT_NORM, HJ_HOPF, 1, 2, 4, 8>(r);
    register_cert<float, HJ_FAM_SPLIT_NORM, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
