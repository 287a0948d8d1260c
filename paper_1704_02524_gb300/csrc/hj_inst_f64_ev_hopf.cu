// hj_inst_f64_ev_hopf.cu -- double kernels of the Evans-type non-convex family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_ev_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_EVANS, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_EVANS, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
