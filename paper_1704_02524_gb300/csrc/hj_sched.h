// hj_sched.h -- launchers of the bookkeeping kernels (hj_sched.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hjd {

struct SelectArgs {
    long long nq;
    const int32_t *pidx;
    int np;  // problems (a problem index outside [0, np) marks the query invalid)
    const int32_t *pg, *pt, *pd, *pprin;  // per problem: starts, trials (starts + reseed budget), d, principle
    int ld;
    const int32_t *pair_base;
    const double *pF;
    const uint8_t *pP, *flags;
    const void *vfin;
    int32_t *pair_slot, *pair_round, *trials, *qflags;
    int round, schedule;
    const int32_t *seg_begin;
    int32_t *wl_count, *wl;
    double *phi;
    void *v_out;
    int32_t *status;
    int32_t *best_pid;
};

cudaError_t launch_count(long long nq, const int32_t *pidx, const int32_t *pt, int32_t *starts, int32_t *pcount,
                         int np, int32_t *seg_begin, int32_t *wl_count, cudaStream_t s);
cudaError_t launch_scan(long long n, const int32_t *in, int32_t *out, int32_t *block_sums, cudaStream_t s);
// Longest-first order (by coarse-level iterations, descending) of problem
// p's work list into out (same segment); bins: LPT_BINS_HOST ints of scratch.
constexpr int LPT_BINS_HOST = 256;
cudaError_t launch_lpt_order(const int32_t *wl, const int32_t *seg_begin, const int32_t *wl_count, int p,
                             const int32_t *iters, int max_iters, int32_t *bins, int32_t *out, int grid,
                             cudaStream_t s);
cudaError_t launch_build_pairs(long long nq, const int32_t *pidx, int np, const int32_t *pg, const int32_t *pt,
                               const int32_t *pair_base, int32_t *pair_q, int32_t *pair_slot, int32_t *pair_round,
                               int32_t *trials, int32_t *qflags, const int32_t *seg_begin, int32_t *wl_count,
                               int32_t *wl, double *pF, uint8_t *pP, uint8_t *flags, cudaStream_t s);
cudaError_t launch_select(const SelectArgs &a, int prec, cudaStream_t s);
cudaError_t launch_guess(long long n, const long long *qid, const int32_t *slot, const int32_t *round,
                         const int32_t *pidx, int np, const int32_t *pd, int ld, unsigned long long seed, int dist, int prec,
                         void *v, cudaStream_t s);

}  // namespace hjd
