// hj_inst_f32_ho_hopf.cu -- float kernels of the harmonic-oscillator family, Hopf principle.
#include "hj_inst.cuh"

namespace hjd {
void reg_f32_ho_hopf(Registry &r)
{
    register_compute<float, HJ_FAM_HARMONIC, HJ_HOPF, 1, 2, 4, 8>(r);
    register_cert<float, HJ_FAM_HARMONIC, HJ_HOPF, 1, 2, 4>(r);
}
}  // namespace hjd
