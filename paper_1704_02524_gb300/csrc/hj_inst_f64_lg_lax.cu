// hj_inst_f64_lg_lax.cu -- double kernels of the time-dependent linear-game family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_lg_lax(Registry &r)
{
    register_compute<double, HJ_FAM_LINEAR_GAME, HJ_LAX, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_LINEAR_GAME, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
