// hj_inst_f32_r1_c04.cu -- one-thread-per-pair kernels of the smooth non-convex family (Hopf), d <= 4.
#include "hj_r1_inst.cuh"

namespace hjd {
void reg_f32_r1_c04(Registry &r) { register_r1<4>(r); }
}  // namespace hjd
