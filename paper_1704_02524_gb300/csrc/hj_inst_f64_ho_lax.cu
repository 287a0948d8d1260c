// hj_inst_f64_ho_lax.cu -- double kernels of the harmonic-oscillator family, Lax principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f64_ho_lax(Registry &r)
{
    register_compute<double, HJ_FAM_HARMONIC, HJ_LAX, 1, 2, 4>(r);
    register_cert<double, HJ_FAM_HARMONIC, HJ_LAX, 1, 2, 4>(r);
}
}  // namespace hjd
