// hj_inst_f32_r1_c32.cu -- one-thread-per-pair kernels of the smooth non-convex family (Hopf), d <= 32.
#include "hj_r1_inst.cuh"

namespace hjd {
void reg_f32_r1_c32(Registry &r) { register_r1<32>(r); }
}  // namespace hjd
