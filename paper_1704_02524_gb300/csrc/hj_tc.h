// hj_tc.h -- host interface of the tensor-core tile kernel of the
// linear-quadratic family (hj_tc.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "hj_device.cuh"
#include "hj_kernels.cuh"

namespace hjd {

enum { LQ_ROWS_EVAL = 0, LQ_ROWS_GRAD = 1, LQ_DESC = 2 };
constexpr size_t LQ_TC_SMEM_MAX = 220 * 1024;  // dynamic shared memory budget of one CTA
constexpr size_t LQ_TC_SMEM_MIN = 120 * 1024;  // requested at least, so one CTA (and one TMEM owner) per SM

// One tensor-core product of a pass: accumulator columns from dcol, A =
// stage-tile columns [acol, acol + K), B = the N x K matrix at byte offset
// boff of the pass's matrices (row pitch kw = K).
struct LqTcProd {
    int dcol, acol, K;
    uint32_t boff;
    int N, kw;
};

// Padded sizes of one problem: dp = d rounded up to 16, mp = m rounded up
// to 16; the stage tile has KZ = 2 dp + mp columns; two products per pass.
struct LqTcGeom {
    int d = 0, m = 0, dp = 0, mp = 0, KV = 0, KZ = 0;
    LqTcProd fwd[2], rev[2];
    size_t w_bytes = 0, z_bytes = 0, smem = 0;
};

struct LqTcArgs {
    int d, dp, m, mp, ld;
    int KV, KZ;
    LqTcProd fwd[2], rev[2];
    size_t w_bytes, z_bytes;
    const uint4 *wf_hi, *wf_lo, *wv_hi, *wv_lo;  // fixed matrices, core-matrix layout, bf16 hi/lo
    int principle, g_kind;
    const float *ga, *gs2, *gis2;                // initial-data vectors (zero padded)
    // rows mode
    long long n;
    const float *x, *t;
    const int32_t *nsteps;
    int n_default;
    const float *v;
    float *F, *grad;
    const int32_t *pidx;
    int pfilter;
    // descent mode (pair bookkeeping as in the lane-group descent kernel)
    DescArgs<float> D;
    int mode_desc;                               // DESC_GD or DESC_CG
    // per-CTA scratch
    float *vec;
    size_t vec_slot;
    float *ybuf;
    size_t ybuf_slot;
    int *err;
};

// True when the problem fits the tile kernel (d <= 64 after padding,
// shared memory within budget).
bool lq_tc_geometry(int d, int m, LqTcGeom *g);
// The forward and reverse matrices of a problem, split into bf16 hi/lo in the
// core-matrix layout (A: d x d row-major, B: d x m row-major).
void lq_tc_matrices(const LqTcGeom &g, const double *A, const double *B, std::vector<uint8_t> &wf_hi,
                    std::vector<uint8_t> &wf_lo, std::vector<uint8_t> &wv_hi, std::vector<uint8_t> &wv_lo);
size_t lq_tc_vec_slot(const LqTcGeom &g);   // floats of per-CTA vector scratch
size_t lq_tc_ybuf_slot(const LqTcGeom &g);  // floats of per-CTA stage-output scratch
cudaError_t lq_tc_launch(int mode, const LqTcArgs &a, int grid, size_t smem, cudaStream_t s);

}  // namespace hjd
