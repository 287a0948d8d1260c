// hj_inst_f32_ev_lax.cu -- float kernels of the Evans-type non-convex family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_ev_lax(Registry &r)
{
    register_compute<float, HJ_FAM_EVANS, HJ_LAX, 1, 2, 4, 8>(r);
    register_cert<float, HJ_FAM_EVANS, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
