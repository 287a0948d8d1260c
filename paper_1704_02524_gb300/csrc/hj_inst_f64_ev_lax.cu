// hj_inst_f64_ev_lax.cu -- double kernels of the Evans-type non-convex family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_ev_lax(Registry &r)
{
    register_compute<double, HJ_FAM_EVANS, HJ_LAX, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_EVANS, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
