// hj_inst_f32_ev_hopf.cu -- float kernels of the Evans-type non-convex family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_ev_hopf(Registry &r)
{
    register_compute<float, HJ_FAM_EVANS, HJ_HOPF, 1, 2, 4, 8>(r);
    register_cert<float, HJ_FAM_EVANS, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
