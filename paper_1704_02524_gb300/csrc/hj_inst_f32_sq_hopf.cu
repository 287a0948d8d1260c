// hj_inst_f32_sq_hopf.cu -- float kernels of the speed-quadratic family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_sq_hopf(Registry &r)
{
    register_compute<float, HJ_FAM_SPEED_QUAD, HJ_HOPF, 1, 2, 4, 5, 8, 10>(r);
    register_cert<float, HJ_FAM_SPEED_QUAD, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
