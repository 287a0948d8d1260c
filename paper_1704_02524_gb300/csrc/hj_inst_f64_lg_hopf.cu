// hj_inst_f64_lg_hopf.cu -- double kernels of the time-dependent linear-game family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_lg_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_LINEAR_GAME, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_LINEAR_GAME, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
