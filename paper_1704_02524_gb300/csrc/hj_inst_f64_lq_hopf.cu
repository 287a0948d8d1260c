// hj_inst_f64_lq_hopf.cu -- double kernels of the linear-quadratic family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_lq_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_LINEAR_QUAD, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_LINEAR_QUAD, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
