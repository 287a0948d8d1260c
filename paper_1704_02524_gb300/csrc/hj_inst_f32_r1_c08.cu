// hj_inst_f32_r1_c08.cu -- one-thread-per-pair kernels of the smooth non-convex family (Hopf), d <= 8.
#include "hj_r1_inst.cuh"

namespace hjd {
void reg_f32_r1_c08(Registry &r) { register_r1<8>(r); }
}  // namespace hjd
