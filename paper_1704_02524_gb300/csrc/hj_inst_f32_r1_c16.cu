// hj_inst_f32_r1_c16.cu -- one-thread-per-pair kernels of the smooth non-convex family (Hopf), d <= 16.
#include "hj_r1_inst.cuh"

namespace hjd {
void reg_f32_r1_c16(Registry &r) { register_r1<16>(r); }
}  // namespace hjd
