// hj_inst_f64_spn_hopf.cu -- double kernels of the split-norm family (and of the bump norm,
// its one-block case), Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_spn_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_SPLIT_NORM, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_SPLIT_NORM, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
