// hj_inst_f32_lg_lax.cu -- float kernels of the time-dependent linear-game family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_lg_lax(Registry &r)
{
    register_compute<float, HJ_FAM_LINEAR_GAME, HJ_LAX, 1, 2, 4, 8>(r);
    register_cert<float, HJ_FAM_LINEAR_GAME, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
