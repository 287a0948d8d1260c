// hj_internal.h -- host-side registry of the instantiated kernels.
#pragma once

#include <cuda_runtime.h>

namespace hjd {

constexpr int MAXC = 10;  // largest components-per-thread instantiated
constexpr int R1_MAXD = 32;  // largest d of the one-thread-per-pair kernels (hj_r1.cuh)

using Launch = cudaError_t (*)(const void *args, int grid, cudaStream_t stream);

// Launchers of one (precision, family, principle, C) combination.  eval,
// grad, cd, gd and cg compute in the context precision; cert_* compute in FP64
// and read v in the context precision.
struct KSet {
    Launch eval = nullptr, grad = nullptr, cd = nullptr, gd = nullptr, cg = nullptr, cert_rows = nullptr,
           cert_pairs = nullptr, cert_final = nullptr;
    const void *f_eval = nullptr, *f_grad = nullptr, *f_cd = nullptr, *f_gd = nullptr, *f_cg = nullptr,
               *f_cert_rows = nullptr, *f_cert_pairs = nullptr, *f_cert_final = nullptr;
    // one-thread-per-pair sets only: the gradient descent with two lanes per
    // pair, for rounds too small to fill the GPU (lower latency per pair;
    // bit-identical results)
    Launch gd_lat = nullptr;
    const void *f_gd_lat = nullptr;
};

struct Registry {
    KSet k[2][9][2][MAXC + 1];  // [precision][family][principle][C]
    // one-thread-per-pair kernels of the smooth non-convex family, fp32,
    // Hopf principle, by padded dimension C (eval, grad, cd and gd only)
    KSet r1[R1_MAXD + 1];
};

Registry &registry();

}  // namespace hjd
