// hj_kernels.cuh -- templated kernels of the solver (instantiated per
// family and precision in hj_inst_*.cu) and the argument blocks they take.
#pragma once

#include "hj_device.cuh"

namespace hjd {

// Rows-mode arguments (hj_eval_functional / hj_grad / hj_certify).
template <typename T>
struct RowArgs {
    ProbDev<T> P;
    int tpp;
    long long n;
    const T *x;              // [n, ld]
    const T *t;              // [n]
    const int32_t *nsteps;   // [n] or null
    int n_default;
    const T *v;              // [n, ld]
    T *F;                    // [n] or null
    T *grad;                 // [n, ld] (gradient kernel)
    const int32_t *pidx;     // [n] or null: rows whose problem is not `pfilter` are skipped
    int pfilter;
    int quad, kahan, ck_interval;
};

// Certificate arguments: rows mode (pid = row) or pair mode (work list).
template <typename Tv>
struct CertArgs {
    ProbDev<double> P;
    int tpp;
    long long n;             // rows mode: number of rows
    const Tv *x;             // [nq, ld] (context precision)
    const Tv *t;
    const int32_t *nsteps;
    int n_default;
    const Tv *v;             // rows mode: [n, ld]; pair mode: per-pair v [npairs, ld]
    double *F;               // [n] / [npairs]
    double *resid;
    uint8_t *pass;
    double tol;
    const int32_t *pidx;
    int pfilter;
    int quad;
    // pair mode
    const int32_t *wl;       // work list
    const int32_t *seg_begin;
    const int32_t *wl_count;
    int problem;
    const int32_t *pair_q;
    // final mode: FP64 value at each query's chosen start
    const int32_t *best_pid;   // [nq], -1 when no start is usable
    double *phi;               // [nq]
};

// Descent arguments (always pair mode).
template <typename T>
struct DescArgs {
    ProbDev<T> P;
    int tpp;
    int problem;
    const T *x;
    const T *t;
    const int32_t *nsteps;
    long long q_begin;
    SolverDev S;
    const int32_t *wl;
    const int32_t *seg_begin;
    const int32_t *wl_count;
    int *cursor;
    const int32_t *pair_q, *pair_slot, *pair_round;
    T *vfin;                 // [npairs, ld]
    int32_t *iters;
    uint8_t *flags;          // bit0: iteration cap, bit1: non-finite
    // certificate at the final v in the kernel precision: F, residual and
    // pass (0/1), or pass = 2 with the pair appended to the FP64 list when
    // a binary32 residual falls inside [CERT_BAND_LO, CERT_BAND_HI] * tol
    double *pF, *pR;
    uint8_t *pP;
    int32_t *amb_wl, *amb_count;
    double tol;
    // coarse-to-fine as two launches per round: 0 the whole descent, 1 the
    // coarse level only (from the Philox start; writes v to vfin, no
    // certificate), 2 the fine level from the v in vfin
    int phase;
    unsigned long long *stats;  // [0] iterations [1] functional evals [2] gradients [3] forward RK4 steps
                                // [4] adjoint steps [5] pairs [6] sum of N over pairs
                                // [7] RK4 steps of the in-kernel certificate
    // one-thread-per-pair kernels: run only when the problem's work list
    // holds a number of pairs in [run_lo, run_hi) (read on the device), so
    // that a throughput and a latency variant can both be enqueued and the
    // one that fits the round's size does the work
    long long run_lo, run_hi;
};

constexpr int BLOCK = 128;
// Band around the certificate tolerance inside which a binary32 residual is
// re-checked in FP64.  Binary32 evaluation moves the residual of a given v by
// ~1e-6 absolute (the RK4 state after <= 256 steps), so a 5% band is at least
// 5x that for tolerances >= 1e-4 (50x at the default 1e-3); a wider band only
// sends more starts through the slow FP64 pipe.
constexpr double CERT_BAND_LO = 0.95, CERT_BAND_HI = 1.05;

template <typename T, int C>
__device__ __forceinline__ void load_row(const Grp &g, const T *row, int d, T *out)
{
#pragma unroll
    for (int k = 0; k < C; ++k) {
        int i = g.lane + k * g.tpp;
        out[k] = (i < d) ? row[i] : (T)0;
    }
}
template <typename T, int C>
__device__ __forceinline__ void store_row(const Grp &g, T *row, int d, const T *val)
{
#pragma unroll
    for (int k = 0; k < C; ++k) {
        int i = g.lane + k * g.tpp;
        if (i < d) row[i] = val[k];
    }
}

// ---------------------------------------------------------------------------
// Functional values at given (x, t, v) rows.
// ---------------------------------------------------------------------------
// Points tp.sh at the group's slice of the block's linear-quadratic scratch.
template <typename T, int C, int FAM>
__device__ __forceinline__ void bind_scratch(TP<T, C> &tp, T *sh, int tpp)
{
    if (FAM == HJ_FAM_LINEAR_QUAD) tp.sh = sh + (threadIdx.x & ~(tpp - 1)) * LqScratch<T, C, FAM>::N;
}

template <typename T, int C, int FAM, int PR>
__global__ void __launch_bounds__(BLOCK) k_eval(RowArgs<T> a)
{
    const Grp g = make_grp(a.tpp);
    TP<T, C> tp;
    tp.load(a.P, g);
    __shared__ T lq_sh[BLOCK * LqScratch<T, C, FAM>::N];
    bind_scratch<T, C, FAM>(tp, lq_sh, a.tpp);
    const long long groups = (long long)gridDim.x * (BLOCK / a.tpp);
    for (long long r = ((long long)blockIdx.x * BLOCK + threadIdx.x) / a.tpp; r < a.n; r += groups) {
        if (a.pidx && a.pidx[r] != a.pfilter) continue;
        const int N = a.nsteps ? a.nsteps[r] : a.n_default;
        T x[C], v[C], gam[C], p[C];
        load_row<T, C>(g, a.x + r * a.P.ld, a.P.d, x);
        load_row<T, C>(g, a.v + r * a.P.ld, a.P.d, v);
#pragma unroll
        for (int k = 0; k < C; ++k) { gam[k] = x[k]; p[k] = v[k]; }
        T F = functional<T, C, FAM, PR>(g, tp, a.P, a.quad, a.kahan, x, v, a.t[r], N, gam, p);
        if (g.lane == 0) a.F[r] = F;
    }
}

// ---------------------------------------------------------------------------
// Exact gradients at given rows.
// ---------------------------------------------------------------------------
template <typename T, int C, int FAM, int PR>
__global__ void __launch_bounds__(BLOCK) k_grad(RowArgs<T> a)
{
    const Grp g = make_grp(a.tpp);
    TP<T, C> tp;
    tp.load(a.P, g);
    __shared__ T lq_sh[BLOCK * LqScratch<T, C, FAM>::N];
    bind_scratch<T, C, FAM>(tp, lq_sh, a.tpp);
    T ck[MAX_CK * 2 * C];
    T seg[MAX_SEG * 2 * C];
    const long long groups = (long long)gridDim.x * (BLOCK / a.tpp);
    for (long long r = ((long long)blockIdx.x * BLOCK + threadIdx.x) / a.tpp; r < a.n; r += groups) {
        if (a.pidx && a.pidx[r] != a.pfilter) continue;
        const int N = a.nsteps ? a.nsteps[r] : a.n_default;
        T x[C], v[C], gr[C];
        load_row<T, C>(g, a.x + r * a.P.ld, a.P.d, x);
        load_row<T, C>(g, a.v + r * a.P.ld, a.P.d, v);
        T F = gradient<T, C, FAM, PR>(g, tp, a.P, a.quad, a.kahan, a.ck_interval, x, v, a.t[r], N, gr, ck, seg);
        store_row<T, C>(g, a.grad + r * a.P.ld, a.P.d, gr);
        if (a.F && g.lane == 0) a.F[r] = F;
    }
}

// ---------------------------------------------------------------------------
// Certificate of Sec. 4.3 in FP64 (and the FP64 functional value).
// ---------------------------------------------------------------------------
// MODE 0: rows (hj_certify); MODE 1: the pairs of a work list (starts whose
// binary32 residual was too close to the tolerance); MODE 2: the chosen
// start of every query, writing phi = F (Lax) or -G (Hopf).
template <typename Tv, int C, int FAM, int PR, int MODE>
__global__ void __launch_bounds__(BLOCK) k_cert(CertArgs<Tv> a)
{
    const Grp g = make_grp(a.tpp);
    TP<double, C> tp;
    tp.load(a.P, g);
    __shared__ double lq_sh[BLOCK * LqScratch<double, C, FAM>::N];
    bind_scratch<double, C, FAM>(tp, lq_sh, a.tpp);
    long long n, begin = 0;
    if (MODE == 1) {
        n = a.wl_count[a.problem];
        begin = a.seg_begin[a.problem];
    } else {
        n = a.n;
    }
    const long long groups = (long long)gridDim.x * (BLOCK / a.tpp);
    for (long long j = ((long long)blockIdx.x * BLOCK + threadIdx.x) / a.tpp; j < n; j += groups) {
        long long pid, q;
        if (MODE == 1) {
            pid = a.wl[begin + j];
            q = a.pair_q[pid];
        } else if (MODE == 2) {
            if (a.pidx && a.pidx[j] != a.pfilter) continue;
            q = j;
            pid = a.best_pid[j];
            if (pid < 0) continue;
        } else {
            if (a.pidx && a.pidx[j] != a.pfilter) continue;
            pid = j;
            q = j;
        }
        const int N = a.nsteps ? a.nsteps[q] : a.n_default;
        double x[C], v[C], gam[C], p[C];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            int i = g.lane + k * g.tpp;
            x[k] = (i < a.P.d) ? (double)a.x[q * a.P.ld + i] : 0.0;
            v[k] = (i < a.P.d) ? (double)a.v[pid * a.P.ld + i] : 0.0;
            gam[k] = x[k];
            p[k] = v[k];
        }
        double F = functional<double, C, FAM, PR>(g, tp, a.P, a.quad, 0, x, v, (double)a.t[q], N, gam, p);
        if (MODE == 2) {
            if (g.lane == 0) a.phi[q] = (PR == HJ_LAX) ? F : -F;
            continue;
        }
        double r = cert_residual<double, C, PR>(g, a.P, gam, p);
        if (g.lane == 0) {
            a.F[pid] = F;
            a.resid[pid] = r;
            a.pass[pid] = (r <= a.tol && isfinite(F)) ? 1 : 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent descent kernel.  Each lane group owns one (query, start) pair at
// a time: it draws the start (Philox), runs Algorithm 1 (cyclic coordinate
// descent with finite differences) or its gradient form with the adjoint
// gradient, and writes the final v.  The loop is organised per iteration so
// that every group of a warp executes the same iteration body together
// (the body has no data-dependent branches besides the RK4 step count); a
// group whose pair has finished takes the next pair from the problem's work
// list between iterations, so lanes never wait for a whole warp to drain.
// ---------------------------------------------------------------------------
// MODE: 0 cyclic coordinate descent with finite differences (Algorithm 1),
// 1 gradient descent, 2 conjugate-gradient descent (both with the adjoint).
constexpr int DESC_CD = 0, DESC_GD = 1, DESC_CG = 2;

// Resident blocks per SM the register allocation aims at: the adjoint
// descents keep more state per component, so fewer components per thread
// buy more resident warps (C <= 2: 5 blocks; C <= 5: 4, which costs the
// 5-component adjoint a 138-byte spill and is 3% faster than 3 blocks; else 3).
template <int C, int MODE>
constexpr int desc_min_blocks() { return MODE == DESC_CD ? 4 : (C <= 2 ? 5 : (C <= 5 ? 4 : 3)); }

template <typename T, int C, int FAM, int PR, int MODE>
__global__ void __launch_bounds__(BLOCK, (desc_min_blocks<C, MODE>())) k_desc(DescArgs<T> a)
{
    constexpr bool GD = MODE != DESC_CD;  // adjoint gradients (checkpoint storage)
    const Grp g = make_grp(a.tpp);
    TP<T, C> tp;
    tp.load(a.P, g);
    __shared__ T lq_sh[BLOCK * LqScratch<T, C, FAM>::N];
    bind_scratch<T, C, FAM>(tp, lq_sh, a.tpp);
    const int d = a.P.d;
    const long long n = a.wl_count[a.problem];
    const long long begin = a.seg_begin[a.problem];
    const int lead = (threadIdx.x & 31) & ~(a.tpp - 1);
    const T eps_stop = (T)a.S.eps;
    const T fd_h = (T)a.S.fd_h;
    const bool central = (a.S.grad != HJ_GRAD_FD_FORWARD);
    T ck[GD ? MAX_CK * 2 * C : 1];
    T seg[GD ? MAX_SEG * 2 * C : 1];
    unsigned long long n_it = 0, n_f = 0, n_g = 0, n_rk = 0, n_adj = 0, n_pairs = 0, n_sumN = 0, n_cert = 0;

    bool active = false, exhausted = false;
    long long pid = 0, q = 0;
    int N = 1, it = 0, count = 0, kper = 0, bad = 0;
    // the coarse launch descends on the N / coarse_div-step functional
    const bool coarse = (MODE != DESC_CD) && a.phase == 1;
    int Ncur = 1;
    T t = 0;
    T x[C], v[C], alpha[C], prev[C];
    // conjugate gradients: direction, phase (0: gradient at v, 1: probe),
    // probe length sigma and max|dir|
    T dir[MODE == DESC_CG ? C : 1];
    int phase = 0;
    T sig = 0, dn = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) { x[k] = 0; v[k] = 0; alpha[k] = 0; prev[k] = 0; }
#pragma unroll
    for (int k = 0; k < (MODE == DESC_CG ? C : 1); ++k) dir[k] = 0;

    for (;;) {
        // ---- refill: groups without a pair take the next one ----------------
        if (!active && !exhausted) {
            long long j = 0;
            if (g.lane == 0) j = atomicAdd(a.cursor + a.problem, 1);
            j = __shfl_sync(g.mask, j, lead);
            if (j >= n) {
                exhausted = true;
            } else {
                pid = a.wl[begin + j];
                q = a.pair_q[pid];
                const int slot = a.pair_slot[pid], round = a.pair_round[pid];
                N = a.nsteps ? a.nsteps[q] : a.S.n_default;
                t = a.t[q];
                load_row<T, C>(g, a.x + q * a.P.ld, d, x);
                if (a.phase == 2) load_row<T, C>(g, a.vfin + pid * a.P.ld, d, v);  // the coarse level's v
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    int i = g.lane + k * g.tpp;
                    if (a.phase != 2)
                        v[k] = (i < d) ? start_component<T>(a.S.seed, a.q_begin + q, slot, round, i, a.S.guess_dist)
                                       : (T)0;
                    alpha[k] = (T)a.S.step;
                    prev[k] = 0;
                }
                it = count = kper = bad = phase = 0;
                Ncur = coarse ? max(1, N / a.S.coarse_div) : N;
                active = true;
            }
        }
        if (!__any_sync(0xffffffffu, active)) break;
        if (!active) continue;

        // ---- one iteration ----------------------------------------------------
        bool stop = (it >= a.S.max_iters), conv = false;
        const T eps_lvl = coarse ? (T)a.S.coarse_eps : eps_stop;
        if (!stop) {
            if constexpr (MODE == DESC_CG) {
                // one gradient per pass: at v (phase 0) or at the probe v + sig dir
                T pt[C], gr[C];
#pragma unroll
                for (int k = 0; k < C; ++k) pt[k] = phase ? fma(sig, dir[k], v[k]) : v[k];
                gradient<T, C, FAM, PR>(g, tp, a.P, a.S.quad, a.S.kahan, a.S.ck_interval, x, pt, t, Ncur, gr, ck, seg);
                n_g++;
                n_rk += Ncur;
                n_adj += Ncur;
                if (phase == 0) {
                    // new direction (Polak-Ribiere+, restart when not descending)
                    if (it == 0) {
#pragma unroll
                        for (int k = 0; k < C; ++k) dir[k] = -gr[k];
                    } else {
                        T gg = 0, gy = 0;
#pragma unroll
                        for (int k = 0; k < C; ++k) {
                            gg = fma(prev[k], prev[k], gg);
                            gy = fma(gr[k], gr[k] - prev[k], gy);
                        }
                        gsum2(g, gg, gy);
                        const T beta = (gg > (T)0) ? fmax((T)0, gy / gg) : (T)0;
                        T gd = 0;
#pragma unroll
                        for (int k = 0; k < C; ++k) {
                            dir[k] = fma(beta, dir[k], -gr[k]);
                            gd = fma(gr[k], dir[k], gd);
                        }
                        if (gsum(g, gd) >= (T)0) {
#pragma unroll
                            for (int k = 0; k < C; ++k) dir[k] = -gr[k];
                        }
                    }
#pragma unroll
                    for (int k = 0; k < C; ++k) prev[k] = gr[k];
                    T n = 0;
#pragma unroll
                    for (int k = 0; k < C; ++k) n = fmax(n, fabs(dir[k]));
                    bool fin = true;
#pragma unroll
                    for (int k = 0; k < C; ++k) fin = fin && finite_(dir[k]);
                    n = gmax(g, fin ? n : (T)INFINITY);
                    if (!(n < (T)INFINITY)) { bad = 1; stop = true; }
                    else if (n == (T)0) { conv = stop = true; }
                    else { dn = n; sig = (T)a.S.step / n; phase = 1; }
                } else {
                    // secant line search along dir, then the move
                    T s0 = 0, s1 = 0;
#pragma unroll
                    for (int k = 0; k < C; ++k) {
                        s0 = fma(prev[k], dir[k], s0);
                        s1 = fma(gr[k], dir[k], s1);
                    }
                    gsum2(g, s0, s1);
                    const T curv = (s1 - s0) / sig;
                    T al = (curv > (T)0) ? -s0 / curv : sig;
                    const T cap = (T)a.S.step_max / dn;
                    if (al > cap) al = cap;
                    ++it;
                    if (!finite_(al)) { bad = 1; stop = true; }
                    else {
#pragma unroll
                        for (int k = 0; k < C; ++k) v[k] = fma(al, dir[k], v[k]);
                        if (al * dn < eps_lvl) conv = stop = true;
                        phase = 0;
                    }
                }
            } else if (GD) {
                T gr[C];
                gradient<T, C, FAM, PR>(g, tp, a.P, a.S.quad, a.S.kahan, a.S.ck_interval, x, v, t, Ncur, gr, ck, seg);
                n_g++;
                n_rk += Ncur;
                n_adj += Ncur;
                T big = 0;
                bool fin = true;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    if (a.S.adapt) {
                        T prod = gr[k] * prev[k];
                        if (prod < 0) alpha[k] *= (T)a.S.shrink;
                        else if (prod > 0) alpha[k] = fmin(alpha[k] * (T)a.S.grow, (T)a.S.step_max);
                    }
                    T st = alpha[k] * gr[k];
                    fin = fin && finite_(st);
                    v[k] -= st;
                    big = fmax(big, fabs(st));
                    prev[k] = gr[k];
                }
                big = gmax(g, fin ? big : (T)INFINITY);
                ++it;
                if (!(big < (T)INFINITY)) { bad = 1; stop = true; }
                if (a.S.halving_period > 0 && it % a.S.halving_period == 0) {
#pragma unroll
                    for (int k = 0; k < C; ++k) alpha[k] *= (T)0.5;
                }
                if (big < eps_lvl) conv = stop = true;
            } else {
                const int jc = it % d;
                const int owner = jc % a.tpp, comp = jc / a.tpp;
                const bool mine = (g.lane == owner);
                T gam[C], p[C], vp[C];
                // F(v + h e_j)
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    vp[k] = v[k] + ((mine && k == comp) ? fd_h : (T)0);
                    gam[k] = x[k];
                    p[k] = vp[k];
                }
                T Fp = functional<T, C, FAM, PR>(g, tp, a.P, a.S.quad, a.S.kahan, x, vp, t, N, gam, p);
                // F(v - h e_j) (central) or F(v) (forward)
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    vp[k] = v[k] - ((central && mine && k == comp) ? fd_h : (T)0);
                    gam[k] = x[k];
                    p[k] = vp[k];
                }
                T Fm = functional<T, C, FAM, PR>(g, tp, a.P, a.S.quad, a.S.kahan, x, vp, t, N, gam, p);
                n_f += 2;
                n_rk += 2 * N;
                T dj = central ? (Fp - Fm) / ((T)2 * fd_h) : (Fp - Fm) / fd_h;
                T st = 0;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    if (mine && k == comp) {
                        if (a.S.adapt) {
                            T prod = dj * prev[k];
                            if (prod < 0) alpha[k] *= (T)a.S.shrink;
                            else if (prod > 0) alpha[k] = fmin(alpha[k] * (T)a.S.grow, (T)a.S.step_max);
                            prev[k] = dj;
                        }
                        st = alpha[k] * dj;
                        v[k] -= st;
                    }
                }
                st = __shfl_sync(g.mask, st, lead + owner);
                ++it;
                if (!finite_(st)) { bad = 1; stop = true; }
                // steps 3-4 of Algorithm 1: reset on a move > eps, count a move < eps
                if (fabs(st) > eps_stop) count = 0;
                else if (fabs(st) < eps_stop) ++count;
                if (a.S.halving_period > 0 && ++kper == a.S.halving_period) {
                    kper = 0;
#pragma unroll
                    for (int k = 0; k < C; ++k) alpha[k] *= (T)0.5;
                }
                if (count >= d) conv = stop = true;
            }
            if (it >= a.S.max_iters) stop = true;
        }
        // ---- finished pair: certificate at the final v, then write it out -----
        if (stop && a.phase == 1) {
            // coarse level done: hand v to the fine launch
            n_it += it;
            store_row<T, C>(g, a.vfin + pid * a.P.ld, d, v);
            if (g.lane == 0) {
                a.iters[pid] = it;
                a.flags[pid] = (uint8_t)(bad << 1);
            }
            active = false;
        } else if (stop) {
            const int cap = (!conv && !bad) ? 1 : 0;
            n_it += it;
            n_pairs++;
            n_sumN += N;
            T gam[C], p[C];
#pragma unroll
            for (int k = 0; k < C; ++k) { gam[k] = x[k]; p[k] = v[k]; }
            const T F = functional<T, C, FAM, PR>(g, tp, a.P, a.S.quad, a.S.kahan, x, v, t, N, gam, p);
            const T r = cert_residual<T, C, PR>(g, a.P, gam, p);
            n_cert += N;
            store_row<T, C>(g, a.vfin + pid * a.P.ld, d, v);
            if (g.lane == 0) {
                const int prior = (a.phase == 2) ? a.iters[pid] : 0;
                const uint8_t fprior = (a.phase == 2) ? (uint8_t)(a.flags[pid] & 2) : (uint8_t)0;
                a.iters[pid] = prior + it;
                a.flags[pid] = (uint8_t)(cap | (bad << 1) | fprior);
                const bool fin = finite_(F) && finite_(r);
                uint8_t pass;
                if (!fin) pass = 0;
                else if (sizeof(T) == 8) pass = ((double)r <= a.tol) ? 1 : 0;
                else if ((double)r < CERT_BAND_LO * a.tol) pass = 1;
                else if ((double)r > CERT_BAND_HI * a.tol) pass = 0;
                else pass = 2;
                a.pF[pid] = (double)F;
                a.pR[pid] = (double)r;
                a.pP[pid] = pass;
                if (pass == 2) {
                    const int pos = atomicAdd(a.amb_count + a.problem, 1);
                    a.amb_wl[begin + pos] = (int32_t)pid;
                }
            }
            active = false;
        }
    }
    if (g.lane == 0 && a.stats) {
        atomicAdd(a.stats + 0, n_it);
        atomicAdd(a.stats + 1, n_f);
        atomicAdd(a.stats + 2, n_g);
        atomicAdd(a.stats + 3, n_rk);
        atomicAdd(a.stats + 4, n_adj);
        atomicAdd(a.stats + 5, n_pairs);
        atomicAdd(a.stats + 6, n_sumN);
        atomicAdd(a.stats + 7, n_cert);
    }
}

}  // namespace hjd
