// hj_sched.cu -- bookkeeping kernels of hj_solve: pair layout, work lists,
// best-of-guesses with reseeding (Sec. 4.3 and Sec. 5), and the guesses
// entry point.  None of these touches the Hamiltonian.
#include <cstdint>

#include "hj.h"
#include "hj_device.cuh"
#include "hj_sched.h"

namespace hjd {

// A query's problem index, or -1 when it is outside [0, np) (such a query
// gets no starts and the status HJ_ST_NONFINITE).
__device__ __forceinline__ int problem_of(const int32_t *pidx, long long q, int np)
{
    const int p = pidx ? pidx[q] : 0;
    return (p >= 0 && p < np) ? p : -1;
}

// Pair entries per query (its trials: starts plus reseed budget) ->
// starts[q]; entries per problem accumulated in pcount.
__global__ void k_count(long long nq, const int32_t *pidx, int np, const int32_t *pt, int32_t *starts,
                        int32_t *pcount)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        const int p = problem_of(pidx, q, np);
        const int G = (p >= 0) ? pt[p] : 0;
        starts[q] = G;
        if (p >= 0) atomicAdd(pcount + p, G);
    }
}

// Exclusive prefix over problems; clears the work-list counters.
__global__ void k_problem_offsets(int np, const int32_t *pcount, int32_t *seg_begin, int32_t *wl_count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int p = 0; p < np; ++p) {
            seg_begin[p] = acc;
            acc += pcount[p];
            wl_count[p] = 0;
        }
        seg_begin[np] = acc;
    }
}

// Three-phase exclusive scan of int32 counts: per-block scans, a serial
// scan of the block totals, then the block offsets added back.
constexpr int SCAN_BLOCK = 1024;

__global__ void k_scan_blocks(long long n, const int32_t *in, int32_t *out, int32_t *block_sums)
{
    __shared__ int32_t sh[SCAN_BLOCK];
    long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int32_t v = (i < n) ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
        int32_t t = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;
    if (threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_sums(int nb, int32_t *block_sums)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t acc = 0;
        for (int b = 0; b < nb; ++b) {
            int32_t v = block_sums[b];
            block_sums[b] = acc;
            acc += v;
        }
    }
}

__global__ void k_scan_add(long long n, int32_t *out, const int32_t *block_sums)
{
    long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] += block_sums[blockIdx.x];
}

// Pair entries of every query: its pt[p] trials, of which the first pg[p]
// (slot s, round 0) go to its problem's work list for round 0; the rest are
// the reseed budget, assigned by k_select (their value NaN until they run).
__global__ void k_build_pairs(long long nq, const int32_t *pidx, int np, const int32_t *pg, const int32_t *pt,
                              const int32_t *pair_base, int32_t *pair_q, int32_t *pair_slot, int32_t *pair_round,
                              int32_t *trials, int32_t *qflags, const int32_t *seg_begin, int32_t *wl_count,
                              int32_t *wl, double *pF, uint8_t *pP, uint8_t *flags)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        const int p = problem_of(pidx, q, np);
        if (p < 0) {
            trials[q] = 0;
            qflags[q] = HJ_ST_NONFINITE;
            continue;
        }
        const int G = pg[p], T = pt[p];
        const int base = pair_base[q];
        const int pos = atomicAdd(wl_count + p, G);
        for (int s = 0; s < T; ++s) {
            const int pid = base + s;
            pair_q[pid] = (int32_t)q;
            if (s < G) {
                pair_slot[pid] = s;
                pair_round[pid] = 0;
                wl[seg_begin[p] + pos + s] = pid;
            } else {
                pair_slot[pid] = -1;
                pair_round[pid] = -1;
                pF[pid] = nan("");
                pP[pid] = 0;
                flags[pid] = 0;
            }
        }
        trials[q] = G;
        qflags[q] = 0;
    }
}

// Best of the trials run so far of each query, and after round 0 the
// reseed schedule (Sec. 4.3, Sec. 5): when some of the pg[p] starts failed
// the certificate, the query's whole remaining budget (pt[p] - pg[p]
// trials) runs in the next round, restart j drawing (q, S[j mod |S|],
// 1 + j / |S|) with S the failed slots in slot order.  Best: certified
// first, then the smallest value, ties to the lowest trial.  phi = F (Lax)
// or -G (Hopf) at the chosen trial (the FP64 value replaces it after the
// last round); best_pid records the trial.  After round 0 a query that was
// not reseeded is final and is left as it is.
template <typename T>
__global__ void k_select(long long nq, const int32_t *pidx, int np, const int32_t *pg, const int32_t *pt,
                         const int32_t *pd, const int32_t *pprin, int ld, const int32_t *pair_base, const double *pF,
                         const uint8_t *pP, const uint8_t *flags, const T *vfin, int32_t *pair_slot,
                         int32_t *pair_round, int32_t *trials, int32_t *qflags, int round, int schedule,
                         const int32_t *seg_begin, int32_t *wl_count, int32_t *wl, double *phi, T *v_out,
                         int32_t *status, int32_t *best_pid)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        const int p = problem_of(pidx, q, np);
        if (p < 0) {
            best_pid[q] = -1;
            phi[q] = nan("");
            status[q] = HJ_ST_NONFINITE;
            continue;
        }
        // after the reseed round only the reseeded queries change
        if (round > 0 && !(qflags[q] & HJ_ST_RESEEDED)) continue;
        const int G = pg[p], nt = pt[p], d = pd[p];
        const int base = pair_base[q];
        int best = -1, best_cert = 0, qf = qflags[q];
        for (int s = 0; s < nt; ++s) {
            const int pid = base + s;
            if (flags[pid] & 2) qf |= HJ_ST_NONFINITE;
            const double F = pF[pid];
            if (!isfinite(F)) continue;
            const int ok = pP[pid];
            if (ok && !best_cert) { best = s; best_cert = 1; continue; }
            if (ok != best_cert) continue;
            if (best < 0 || F < pF[base + best]) best = s;
        }
        int st = 0;
        if (best >= 0) {
            const int pid = base + best;
            const double F = pF[pid];
            phi[q] = (pprin[p] == HJ_HOPF) ? -F : F;
            for (int i = 0; i < d; ++i) v_out[q * ld + i] = vfin[(long long)pid * ld + i];
            if (best_cert) st |= HJ_ST_CERTIFIED;
            if (flags[pid] & 1) st |= HJ_ST_MAX_ITERS;
            best_pid[q] = pid;
        } else {
            best_pid[q] = -1;
            phi[q] = nan("");
            for (int i = 0; i < d; ++i) v_out[q * ld + i] = (T)nan("");
            st |= HJ_ST_NONFINITE;
        }
        if (schedule) {
            int nfail = 0;
            for (int s = 0; s < G; ++s) nfail += pP[base + s] ? 0 : 1;
            if (nfail > 0 && nt > G) {
                for (int j = 0; G + j < nt; ++j) {
                    int k = j % nfail, slot = 0;
                    for (int s = 0; s < G; ++s)
                        if (!pP[base + s] && k-- == 0) {
                            slot = s;
                            break;
                        }
                    const int pid = base + G + j;
                    pair_slot[pid] = slot;
                    pair_round[pid] = round + 1 + j / nfail;
                    const int pos = atomicAdd(wl_count + p, 1);
                    wl[seg_begin[p] + pos] = pid;
                }
                trials[q] = nt;
                qf |= HJ_ST_RESEEDED;
            }
        }
        qflags[q] = qf;
        status[q] = st | qf;
    }
}

// Longest-first order of one problem's work list for the fine level of a
// two-level descent: a persistent launch ends with the pairs it started last,
// so starting the long ones first shortens its tail (the classical
// longest-processing-time rule).  A pair's coarse-level iteration count is
// the predictor of its fine-level work at hand.  Counting sort over LPT_BINS
// bins, descending; the order within a bin is the atomics' and changes no
// result (each pair's arithmetic does not depend on where it runs).
constexpr int LPT_BINS = 256;

__device__ __forceinline__ int lpt_key(int it, int max_iters)
{
    const int m = max(max_iters, 1);
    const int c = min(max(it, 0), m);
    return LPT_BINS - 1 - (int)((long long)c * (LPT_BINS - 1) / m);
}

__global__ void k_lpt_hist(const int32_t *wl, const int32_t *seg_begin, const int32_t *wl_count, int p,
                           const int32_t *iters, int max_iters, int32_t *bins)
{
    __shared__ int32_t h[LPT_BINS];
    for (int i = threadIdx.x; i < LPT_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int n = wl_count[p], b = seg_begin[p];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&h[lpt_key(iters[wl[b + i]], max_iters)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < LPT_BINS; i += blockDim.x)
        if (h[i]) atomicAdd(bins + i, h[i]);
}

__global__ void k_lpt_offsets(int32_t *bins)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t acc = 0;
        for (int i = 0; i < LPT_BINS; ++i) {
            const int32_t c = bins[i];
            bins[i] = acc;
            acc += c;
        }
    }
}

__global__ void k_lpt_scatter(const int32_t *wl, const int32_t *seg_begin, const int32_t *wl_count, int p,
                              const int32_t *iters, int max_iters, int32_t *bins, int32_t *out)
{
    const int n = wl_count[p], b = seg_begin[p];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t pid = wl[b + i];
        out[b + atomicAdd(bins + lpt_key(iters[pid], max_iters), 1)] = pid;
    }
}

cudaError_t launch_lpt_order(const int32_t *wl, const int32_t *seg_begin, const int32_t *wl_count, int p,
                             const int32_t *iters, int max_iters, int32_t *bins, int32_t *out, int grid,
                             cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int32_t) * LPT_BINS, s);
    if (e != cudaSuccess) return e;
    k_lpt_hist<<<grid, 256, 0, s>>>(wl, seg_begin, wl_count, p, iters, max_iters, bins);
    k_lpt_offsets<<<1, 32, 0, s>>>(bins);
    k_lpt_scatter<<<grid, 256, 0, s>>>(wl, seg_begin, wl_count, p, iters, max_iters, bins, out);
    return cudaGetLastError();
}

// hj_guesses: the starts drawn by hj_solve, for testing.
template <typename T>
__global__ void k_guess(long long n, const long long *qid, const int32_t *slot, const int32_t *round,
                        const int32_t *pidx, int np, const int32_t *pd, int ld, unsigned long long seed, int dist, T *v)
{
    const long long total = n * ld;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / ld;
        const int i = (int)(e % ld);
        const int p = pidx ? pidx[r] : 0;
        if (p < 0 || p >= np) continue;  // rows of an unknown problem are left untouched
        const int d = pd[p];
        if (i < d) v[e] = start_component<T>(seed, qid[r], slot[r], round[r], i, dist);
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
static int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)g;
}

cudaError_t launch_count(long long nq, const int32_t *pidx, const int32_t *pt, int32_t *starts, int32_t *pcount,
                         int np, int32_t *seg_begin, int32_t *wl_count, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(pcount, 0, sizeof(int32_t) * np, s);
    if (e != cudaSuccess) return e;
    k_count<<<grid_for(nq, 256), 256, 0, s>>>(nq, pidx, np, pt, starts, pcount);
    k_problem_offsets<<<1, 1, 0, s>>>(np, pcount, seg_begin, wl_count);
    return cudaGetLastError();
}

cudaError_t launch_scan(long long n, const int32_t *in, int32_t *out, int32_t *block_sums, cudaStream_t s)
{
    int nb = (int)((n + SCAN_BLOCK - 1) / SCAN_BLOCK);
    if (nb < 1) nb = 1;
    k_scan_blocks<<<nb, SCAN_BLOCK, 0, s>>>(n, in, out, block_sums);
    k_scan_sums<<<1, 1, 0, s>>>(nb, block_sums);
    k_scan_add<<<nb, SCAN_BLOCK, 0, s>>>(n, out, block_sums);
    return cudaGetLastError();
}

cudaError_t launch_build_pairs(long long nq, const int32_t *pidx, int np, const int32_t *pg, const int32_t *pt,
                               const int32_t *pair_base, int32_t *pair_q, int32_t *pair_slot, int32_t *pair_round,
                               int32_t *trials, int32_t *qflags, const int32_t *seg_begin, int32_t *wl_count,
                               int32_t *wl, double *pF, uint8_t *pP, uint8_t *flags, cudaStream_t s)
{
    k_build_pairs<<<grid_for(nq, 256), 256, 0, s>>>(nq, pidx, np, pg, pt, pair_base, pair_q, pair_slot, pair_round,
                                                    trials, qflags, seg_begin, wl_count, wl, pF, pP, flags);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_select_t(const SelectArgs &a, cudaStream_t s)
{
    k_select<T><<<grid_for(a.nq, 128), 128, 0, s>>>(
        a.nq, a.pidx, a.np, a.pg, a.pt, a.pd, a.pprin, a.ld, a.pair_base, a.pF, a.pP, a.flags, (const T *)a.vfin,
        a.pair_slot, a.pair_round, a.trials, a.qflags, a.round, a.schedule, a.seg_begin, a.wl_count, a.wl, a.phi,
        (T *)a.v_out, a.status, a.best_pid);
    return cudaGetLastError();
}

cudaError_t launch_select(const SelectArgs &a, int prec, cudaStream_t s)
{
    return prec ? launch_select_t<double>(a, s) : launch_select_t<float>(a, s);
}

cudaError_t launch_guess(long long n, const long long *qid, const int32_t *slot, const int32_t *round,
                         const int32_t *pidx, int np, const int32_t *pd, int ld, unsigned long long seed, int dist,
                         int prec, void *v, cudaStream_t s)
{
    int g = grid_for(n * ld, 256);
    if (prec) k_guess<double><<<g, 256, 0, s>>>(n, qid, slot, round, pidx, np, pd, ld, seed, dist, (double *)v);
    else k_guess<float><<<g, 256, 0, s>>>(n, qid, slot, round, pidx, np, pd, ld, seed, dist, (float *)v);
    return cudaGetLastError();
}

}  // namespace hjd
