// hj_inst_f64_ho_hopf.cu -- double kernels of the harmonic-oscillator family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_ho_hopf(Registry &r)
{
    register_compute<double, HJ_FAM_HARMONIC, HJ_HOPF, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_HARMONIC, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
