// hj_inst_f32_qi_lax.cu -- float kernels of the quadratic isotropic family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_qi_lax(Registry &r)
{
    register_compute<float, HJ_FAM_QUAD_ISO, HJ_LAX, 1, 2, 4>(r);
    register_cert<float, HJ_FAM_QUAD_ISO, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
