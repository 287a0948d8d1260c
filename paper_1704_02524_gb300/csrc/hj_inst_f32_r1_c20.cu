// hj_inst_f32_r1_c20.cu -- one-thread-per-pair kernels of the smooth non-convex family (Hopf), d <= 20.
#include "hj_r1_inst.cuh"

namespace hjd {
void reg_f32_r1_c20(Registry &r) { register_r1<20>(r); }
}  // namespace hjd
