// hj_r1.cuh -- one thread per (query, start) pair for the smooth non-convex
// family H = c(x) Phi(p), c = 1 + sin(<w,x>)/2, Phi = sum_i e_i s(p_i),
// s(q) = sqrt(q^2 + eps), under the Hopf principle, d <= 32.
//
// Structure of the characteristic field used here (Sec. 4.1's system with
// this H): dp/dtau = Phi(p) c'(u) w is always parallel to w, and gamma enters
// the field only through u = <w, gamma> (c and its derivatives are functions
// of u).  Every RK4 stage adds a multiple of w to p and every stage field is
// a function of (u, p), so the iterates of the discretised system are exactly
//   p_n = v + B_n w,   u_n = <w, gamma_n>,
// with the scalars (u_n, B_n) advanced by the RK4 combination of the stage
// values
//   du/dtau = <w, -c Phi'(p)> = -c D,  D = sum_i w_i e_i p_i / s_i,
//   dB/dtau = Phi c',
// and the Hopf running cost L = Phi (c - c' u) (Sec. 4.1) of the same stages.
// The terminal term g*(p_N) - <x, v> needs p_N = v + B_N w only.  The result
// is the RK4 functional of the general lane-group kernels (hj_device.cuh) up
// to rounding: the same stages, the same weights, the same terminal term; the
// 2d-dimensional state is carried as two scalars.
//
// The discrete adjoint (exact gradient of this functional) follows the
// general adjoint_step stage by stage: with lam = (lam_gamma, lam_p), every
// vector-Jacobian product of this family has its gamma-part along w
// (rg = dE/du w), and the Hopf seed is (0, grad g*(p_N)), so
// lam_gamma = alpha w stays a scalar multiple of w; the weights each stage
// product needs reduce to the scalars a (lam_gamma's coefficient), Bw =
// <weight_p, w> and the quadrature weight, and the p-part of each product is
//   rp_i = e_i r_i (kd p_i - c eps a w_i r_i^2),  r_i = 1/s_i,
// summed into lam_p.  The state checkpoints are the pairs (u_n, B_n): 8 bytes
// per step, every step kept by default.
//
// Per pair the thread holds v and lam_p in registers (2d values); the
// per-problem vectors (w, e, w e, the initial data's coefficients) are kernel
// parameters, read as constant operands.  One thread per pair means no
// shuffles: every dot product is a register sum (two partial sums, over the
// even and the odd components).  A second form runs each pair on two lanes
// (TPP = 2), lane l holding the components i = 2k + l with its own copy of
// their parameters: each lane's sum is then exactly one of the two partial
// sums, and the group sum adds the other lane's, so both forms give the same
// results bit for bit while the two-lane form halves the serial work of a
// pair (for rounds with too few pairs to fill the GPU, where a pair's latency
// sets the time).  The four RK4 stages and the
// four stage products of the adjoint run as loops, not unrolled, so that the
// d-wide stage body exists once per use in the code: with every stage inlined
// the kernel's instruction stream outgrew the instruction cache (the
// dominant stall, measured).  The stage scalars the products need are kept
// per thread in shared memory.
#pragma once

#include "hj_kernels.cuh"

namespace hjd {
namespace r1 {

constexpr unsigned FULL = 0xffffffffu;
constexpr int REC = 8;  // floats per stage record in shared memory

// Resident blocks of BLOCK threads per SM the register allocation aims at.
// A problem with d <= R1_MAXD runs with C = the smallest instantiated size
// >= d; padded components carry w = e = g2 = ga = 0 and drop out of every sum.
template <int C, int TPP>
constexpr int min_blocks()
{
    return TPP == 1 ? (C <= 16 ? 4 : (C <= 20 ? 3 : 2)) : (C <= 20 ? 4 : 3);
}

// The lane's view of the per-component parameters.  One lane per pair: the
// parameter block's values, read as constants (component k is i = k).  Two
// lanes per pair: lane l of the group holds i = 2k + l, with w, e and w e of
// those components copied to registers.
template <int C, int TPP>
struct Lane;
template <int C>
struct Lane<C, 1> {
    static constexpr int CL = C;
    unsigned gm;  // lanes of the group
    int gl;       // lane inside the group
    __device__ void load(const ProbDev<float> &, int lane) { gm = 1u << lane; gl = 0; }
    __device__ __forceinline__ int comp(int k) const { return k; }
    __device__ __forceinline__ float w(const ProbDev<float> &P, int k) const { return P.rw[k]; }
    __device__ __forceinline__ float e(const ProbDev<float> &P, int k) const { return P.re[k]; }
    __device__ __forceinline__ float we(const ProbDev<float> &P, int k) const { return P.rew[k]; }
    __device__ __forceinline__ float g2(const ProbDev<float> &P, int k) const { return P.rg2[k]; }
    __device__ __forceinline__ float ga(const ProbDev<float> &P, int k) const { return P.rga[k]; }
    // the group total of partial sums over even (a0) and odd (a1) components
    __device__ __forceinline__ float total(float a0, float a1) const { return a0 + a1; }
    __device__ __forceinline__ float gmaxf(float a) const { return a; }
};
template <int C>
struct Lane<C, 2> {
    static constexpr int CL = C / 2;
    float w_[CL], e_[CL], we_[CL];
    unsigned gm;
    int gl;
    __device__ void load(const ProbDev<float> &P, int lane)
    {
        gl = lane & 1;
        gm = 3u << (lane & ~1);
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            w_[k] = P.rw[2 * k + gl];
            e_[k] = P.re[2 * k + gl];
            we_[k] = P.rew[2 * k + gl];
        }
    }
    __device__ __forceinline__ int comp(int k) const { return 2 * k + gl; }
    __device__ __forceinline__ float w(const ProbDev<float> &, int k) const { return w_[k]; }
    __device__ __forceinline__ float e(const ProbDev<float> &, int k) const { return e_[k]; }
    __device__ __forceinline__ float we(const ProbDev<float> &, int k) const { return we_[k]; }
    __device__ __forceinline__ float g2(const ProbDev<float> &P, int k) const { return P.rg2[2 * k + gl]; }
    __device__ __forceinline__ float ga(const ProbDev<float> &P, int k) const { return P.rga[2 * k + gl]; }
    // this lane's sum is one parity's partial sum (in a0); the other lane has
    // the other parity's: their sum, the same on both lanes
    __device__ __forceinline__ float total(float a0, float) const { return a0 + __shfl_xor_sync(gm, a0, 1); }
    __device__ __forceinline__ float gmaxf(float a) const { return fmaxf(a, __shfl_xor_sync(gm, a, 1)); }
};

// Partial sums over the lane's components: two (even and odd components)
// with one lane per pair, one (the lane's parity) with two.  Every product
// that feeds a sum in this file is an explicit fmaf or an explicitly rounded
// multiply (__fmul_rn), so the compiler cannot contract the two forms'
// arithmetic differently.
template <int TPP>
struct Acc {
    float a0 = 0.f, a1 = 0.f;
    __device__ __forceinline__ void fma_(int k, float m, float x)
    {
        if (TPP == 2 || !(k & 1)) a0 = fmaf(m, x, a0);
        else a1 = fmaf(m, x, a1);
    }
};

// One lane per pair: components 2j and 2j + 1 side by side, so that the
// even and the odd partial sums advance together in packed FP32x2
// operations (each component rounded exactly as the scalar fmaf, __fmul_rn
// and __fadd_rn it replaces).
__device__ __forceinline__ float2 pair2(const float *a, int j) { return make_float2(a[2 * j], a[2 * j + 1]); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// Scalars of one RK4 stage.
struct St {
    float u, B;       // stage input: u = <w, gamma>, p = v + B w
    float c, c1, c2;  // c(u), c'(u), c''(u)
    float phi, D;     // Phi(p), sum_i w_i e_i p_i / s_i
};

// Per-thread stage records: rec points at the thread's column of a
// [4 * REC][BLOCK] shared array.
__device__ __forceinline__ void put(float *rec, int st, const St &s)
{
    float *r = rec + st * REC * BLOCK;
    r[0] = s.u; r[BLOCK] = s.B; r[2 * BLOCK] = s.c; r[3 * BLOCK] = s.c1;
    r[4 * BLOCK] = s.c2; r[5 * BLOCK] = s.phi; r[6 * BLOCK] = s.D;
}
__device__ __forceinline__ St get(const float *rec, int st)
{
    const float *r = rec + st * REC * BLOCK;
    return St{r[0], r[BLOCK], r[2 * BLOCK], r[3 * BLOCK], r[4 * BLOCK], r[5 * BLOCK], r[6 * BLOCK]};
}

// The sums of a stage at input (u, B): Phi and D, with the reciprocals r
// kept when KEEP.
template <int C, int TPP, bool KEEP>
__device__ __forceinline__ void stage(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *v, float eps,
                                      float u, float B, St &s, float *r)
{
    if constexpr (TPP == 1) {
        float2 ph = splat2(0.f), dd = ph;
        const float2 B2 = splat2(B), eps2 = splat2(eps);
#pragma unroll
        for (int j = 0; j < C / 2; ++j) {
            const float2 p = __ffma2_rn(B2, pair2(P.rw, j), pair2(v, j));
            const float2 q = __ffma2_rn(p, p, eps2);
            const float2 ri = make_float2(rsqrtf(q.x), rsqrtf(q.y));
            if constexpr (KEEP) {
                r[2 * j] = ri.x;
                r[2 * j + 1] = ri.y;
            }
            ph = __ffma2_rn(pair2(P.re, j), __fmul2_rn(q, ri), ph);
            dd = __ffma2_rn(pair2(P.rew, j), __fmul2_rn(ri, p), dd);
        }
        s.phi = L.total(ph.x, ph.y);
        s.D = L.total(dd.x, dd.y);
    } else {
        Acc<TPP> ph, dd;
#pragma unroll
        for (int k = 0; k < Lane<C, TPP>::CL; ++k) {
            const float p = fmaf(B, L.w(P, k), v[k]);
            const float q = fmaf(p, p, eps);
            const float ri = rsqrtf(q);
            if constexpr (KEEP) r[k] = ri;
            ph.fma_(k, L.e(P, k), __fmul_rn(q, ri));
            dd.fma_(k, L.we(P, k), __fmul_rn(ri, p));
        }
        s.phi = L.total(ph.a0, ph.a1);
        s.D = L.total(dd.a0, dd.a1);
    }
    s.u = u;
    s.B = B;
    float su, cu;
    __sincosf(u, &su, &cu);
    s.c = fmaf(0.5f, su, 1.f);
    s.c1 = 0.5f * cu;
    s.c2 = -0.5f * su;
}

// Stage rates: du/dtau, dB/dtau and the Hopf running cost.
__device__ __forceinline__ float rate_u(const St &s) { return __fmul_rn(-s.c, s.D); }
__device__ __forceinline__ float rate_B(const St &s) { return __fmul_rn(s.phi, s.c1); }
__device__ __forceinline__ float cost(const St &s) { return __fmul_rn(s.phi, fmaf(-s.c1, s.u, s.c)); }

// RK4 bookkeeping of stage st (0..3) with rate k: the weighted sum
// a = k1 + 2 k2 + 2 k3 + k4.
__device__ __forceinline__ void rk4_acc(int st, float k, float &a)
{
    if (st == 0) a = k;
    else if (st < 3) a = fmaf(2.f, k, a);
    else a = __fadd_rn(a, k);
}

// One classical RK4 step of (u, B) and the running cost; the four stage
// records go to rec (shared memory) when it is non-null.  With srec
// non-null the step's record for the adjoint goes to the thread's local
// memory: srec[0] = (u_n, B_n), srec[1 + s] = (Phi, D) of stage s (the
// stage inputs follow from these by the step's own arithmetic).
template <int C, int TPP>
__device__ __forceinline__ void step(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *v, float eps,
                                     float h, float &u, float &B, float &dQ, float *rec, float2 *srec = nullptr)
{
    const float h2 = 0.5f * h, h6 = h / 6.f;
    float su = u, sB = B, au = 0.f, aB = 0.f, aL = 0.f;
#pragma unroll 1
    for (int st = 0; st < 4; ++st) {
        St s;
        stage<C, TPP, false>(P, L, v, eps, su, sB, s, nullptr);
        if (rec) put(rec, st, s);
        if (srec) srec[1 + st] = make_float2(s.phi, s.D);
        const float ku = rate_u(s), kB = rate_B(s);
        rk4_acc(st, ku, au);
        rk4_acc(st, kB, aB);
        rk4_acc(st, cost(s), aL);
        const float hs = (st == 2) ? h : h2;
        su = fmaf(hs, ku, u);
        sB = fmaf(hs, kB, B);
    }
    if (srec) srec[0] = make_float2(u, B);
    u = fmaf(h6, au, u);
    B = fmaf(h6, aB, B);
    dQ = __fmul_rn(h6, aL);
}

// <w, x> and <a, b> over the group's components.
template <int C, int TPP>
__device__ __forceinline__ float dot_w(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *x)
{
    if constexpr (TPP == 1) {
        float2 a = splat2(0.f);
#pragma unroll
        for (int j = 0; j < C / 2; ++j) a = __ffma2_rn(pair2(P.rw, j), pair2(x, j), a);
        return L.total(a.x, a.y);
    } else {
        Acc<TPP> a;
#pragma unroll
        for (int k = 0; k < Lane<C, TPP>::CL; ++k) a.fma_(k, L.w(P, k), x[k]);
        return L.total(a.a0, a.a1);
    }
}
// <w e, x> over the group's components (w e = w_i e_i, the products' weights
// of the sign-folded adjoint below).
template <int C, int TPP>
__device__ __forceinline__ float dot_we(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *x)
{
    if constexpr (TPP == 1) {
        float2 a = splat2(0.f);
#pragma unroll
        for (int j = 0; j < C / 2; ++j) a = __ffma2_rn(pair2(P.rew, j), pair2(x, j), a);
        return L.total(a.x, a.y);
    } else {
        Acc<TPP> a;
#pragma unroll
        for (int k = 0; k < Lane<C, TPP>::CL; ++k) a.fma_(k, L.we(P, k), x[k]);
        return L.total(a.a0, a.a1);
    }
}
template <int C, int TPP>
__device__ __forceinline__ float dot(const Lane<C, TPP> &L, const float *x, const float *y)
{
    Acc<TPP> a;
#pragma unroll
    for (int k = 0; k < Lane<C, TPP>::CL; ++k) a.fma_(k, x[k], y[k]);
    return L.total(a.a0, a.a1);
}

// Hopf terminal term g*(p_N) - <x, v> (+ the ellipse data's constant), with
// g*(p) = sum_i p_i (g2_i p_i / 2 + ga_i) and xv = <x, v>; the seed grad g*
// goes to lp when it is non-null.
template <int C, int TPP>
__device__ __forceinline__ float terminal(const ProbDev<float> &P, const Lane<C, TPP> &L, float xv, const float *v,
                                          float B, float *lp)
{
    Acc<TPP> a;
#pragma unroll
    for (int k = 0; k < Lane<C, TPP>::CL; ++k) {
        const float p = fmaf(B, L.w(P, k), v[k]);
        const float g2 = L.g2(P, k), ga = L.ga(P, k);
        a.fma_(k, p, fmaf(0.5f * g2, p, ga));
        if (lp) lp[k] = fmaf(g2, p, ga);
    }
    return (L.total(a.a0, a.a1) - xv) + P.rcst;
}

// Functional G(v) (Hopf) from u0 = <w, x> and xv = <x, v>.  With ck != null
// the step inputs (u_n, B_n) of every K-th step are stored there (the
// adjoint's checkpoints); with sr != null every step's record (sr[5 n ..
// 5 n + 4], see step()).  B_N is returned in Bn.
template <int C, int TPP>
__device__ __forceinline__ float functional(const ProbDev<float> &P, const Lane<C, TPP> &L, int kahan, float u0,
                                            float xv, const float *v, float t, int N, float2 *ck, int K, float &Bn,
                                            float2 *sr = nullptr)
{
    if (N < 1 || N > MAX_N) {
        Bn = NAN;
        return NAN;
    }
    const float eps = P.s_eps, h = t / (float)N;
    float u = u0, B = 0.f, Q = 0.f, Qc = 0.f;
    for (int n = 0, kk = 0; n < N; ++n) {
        if (ck) {
            if (kk == 0) ck[n / K] = make_float2(u, B);
            if (++kk == K) kk = 0;
        }
        float dQ;
        step<C, TPP>(P, L, v, eps, h, u, B, dQ, nullptr, sr ? sr + 5 * n : nullptr);
        add_q(kahan, dQ, Q, Qc);
    }
    Bn = B;
    return terminal<C, TPP>(P, L, xv, v, B, nullptr) + Q;
}

// The functional with gamma carried along as a vector, for the certificate
// (Sec. 4.3): gamma advances by the RK4 combination of the stage rates
// -c Phi'(p); (u, B, Q) advance exactly as in functional().  Returns G; gam
// holds x on entry and gamma(0) on exit (the lane's components), Bn gets B_N.
template <int C, int TPP>
__device__ __forceinline__ float functional_gamma(const ProbDev<float> &P, const Lane<C, TPP> &L, int kahan, float u0,
                                                  float xv, const float *v, float t, int N, float *gam, float &Bn)
{
    if (N < 1 || N > MAX_N) {
        Bn = NAN;
        return NAN;
    }
    constexpr int CL = Lane<C, TPP>::CL;
    const float eps = P.s_eps, h = t / (float)N, h2 = 0.5f * h, h6 = h / 6.f;
    float u = u0, B = 0.f, Q = 0.f, Qc = 0.f;
    for (int n = 0; n < N; ++n) {
        float ag[CL];
        float su = u, sB = B, au = 0.f, aB = 0.f, aL = 0.f;
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
            float r[CL];
            St s;
            stage<C, TPP, true>(P, L, v, eps, su, sB, s, r);
#pragma unroll
            for (int k = 0; k < CL; ++k) {
                const float p = fmaf(sB, L.w(P, k), v[k]);
                const float kg = __fmul_rn(-s.c, __fmul_rn(__fmul_rn(L.e(P, k), r[k]), p));
                if (st == 0) ag[k] = kg;
                else if (st < 3) ag[k] = fmaf(2.f, kg, ag[k]);
                else gam[k] = fmaf(h6, __fadd_rn(ag[k], kg), gam[k]);
            }
            const float ku = rate_u(s), kB = rate_B(s);
            rk4_acc(st, ku, au);
            rk4_acc(st, kB, aB);
            rk4_acc(st, cost(s), aL);
            const float hs = (st == 2) ? h : h2;
            su = fmaf(hs, ku, u);
            sB = fmaf(hs, kB, B);
        }
        u = fmaf(h6, au, u);
        B = fmaf(h6, aB, B);
        add_q(kahan, __fmul_rn(h6, aL), Q, Qc);
    }
    Bn = B;
    return terminal<C, TPP>(P, L, xv, v, B, nullptr) + Q;
}

// Vector-Jacobian product of one stage with scalar weights: gamma weight
// a w, p weight with <weight_p, w> = Bw, quadrature weight bb.  The p-part
// is e_i r_i tt_i; with the signs e_i = +-1 folded into the adjoint state
// (lp holds e_i lam_p,i, exactly, since a product with +-1 is exact and
// rounding is symmetric) it adds r_i tt_i to lp, and its <w, .> is
// <w e, r tt>.  Returns the gamma-part's coefficient (dE/du) in R and
// <w, p-part> in Wr.  The stage's p and reciprocals are recomputed; the stage
// input is made to depend on `after` (the previous product's result, finite
// in any finite solve) so that this happens in order instead of being
// hoisted and kept live across the step.
template <int C, int TPP>
__device__ __forceinline__ void vjp(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *v, float eps,
                                    const St &s, float a, float Bw, float bb, float after, float *lp, float &R,
                                    float &Wr)
{
    const float A = __fmul_rn(a, s.D);
    float dEdu = fmaf(-s.c1, A, __fmul_rn(__fmul_rn(s.phi, s.c2), Bw));
    dEdu = fmaf(-__fmul_rn(__fmul_rn(bb, s.phi), s.c2), s.u, dEdu);
    const float kd = fmaf(s.c1, Bw, __fmul_rn(bb, fmaf(-s.c1, s.u, s.c)));
    const float cea = __fmul_rn(__fmul_rn(s.c, eps), a);
    const float Bs = fmaf(0.f, after, s.B);
    R = dEdu;
    if constexpr (TPP == 1) {
        float2 w = splat2(0.f);
        const float2 Bs2 = splat2(Bs), eps2 = splat2(eps), kd2 = splat2(kd), mcea2 = splat2(-cea);
#pragma unroll
        for (int j = 0; j < C / 2; ++j) {
            const float2 wk = pair2(P.rw, j);
            const float2 p = __ffma2_rn(Bs2, wk, pair2(v, j));
            const float2 q = __ffma2_rn(p, p, eps2);
            const float2 ri = make_float2(rsqrtf(q.x), rsqrtf(q.y));
            const float2 tt = __ffma2_rn(__fmul2_rn(mcea2, wk), __fmul2_rn(ri, ri), __fmul2_rn(kd2, p));
            const float2 rp = __fmul2_rn(ri, tt);
            const float2 l = __fadd2_rn(pair2(lp, j), rp);
            lp[2 * j] = l.x;
            lp[2 * j + 1] = l.y;
            w = __ffma2_rn(pair2(P.rew, j), rp, w);
        }
        Wr = L.total(w.x, w.y);
    } else {
        Acc<TPP> w;
#pragma unroll
        for (int k = 0; k < Lane<C, TPP>::CL; ++k) {
            const float wk = L.w(P, k);
            const float p = fmaf(Bs, wk, v[k]);
            const float ri = rsqrtf(fmaf(p, p, eps));
            const float tt = fmaf(__fmul_rn(-cea, wk), __fmul_rn(ri, ri), __fmul_rn(kd, p));
            const float rp = __fmul_rn(ri, tt);
            lp[k] = __fadd_rn(lp[k], rp);
            w.fma_(k, L.we(P, k), rp);
        }
        Wr = L.total(w.a0, w.a1);
    }
}

// Adjoint of one RK4 step at input (u, B): lam = (alpha w, lp) -> lam_n.
// The rebuild (the forward step from (u, B)) leaves the four stage records
// in rec; the products run from stage 4 down to stage 1 with the weights of
// the RK4 adjoint: (h/6, h/3, h/3, h/6) on lam and the quadrature, and
// (h, h/2, h/2) on the previous stage's product.
template <int C, int TPP>
__device__ __forceinline__ void adjoint_step(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *v, float eps,
                                             float h, float u, float B, float &alpha, float *lp, float *rec)
{
    const float h2 = 0.5f * h, h3 = h / 3.f, h6 = h / 6.f;
    float un = u, Bn = B, dQ;
    step<C, TPP>(P, L, v, eps, h, un, Bn, dQ, rec);
    const float Lw = dot_we<C, TPP>(P, L, lp);
    float R = 0.f, W = 0.f, sumR = 0.f;
#pragma unroll 1
    for (int j = 3; j >= 0; --j) {
        const St s = get(rec, j);
        const float wl = (j == 0 || j == 3) ? h6 : h3;
        const float wp = (j == 2) ? h : h2;
        vjp<C, TPP>(P, L, v, eps, s, fmaf(wl, alpha, __fmul_rn(wp, R)), fmaf(wl, Lw, __fmul_rn(wp, W)), wl, W, lp, R,
                    W);
        sumR = __fadd_rn(sumR, R);
    }
    alpha = __fadd_rn(alpha, sumR);
}

// adjoint_step with the step's record from the forward pass (r[0] = (u_n,
// B_n), r[1 + s] = (Phi, D) of stage s) instead of a rebuild: the stage
// inputs are re-derived from (u_n, B_n) and the stored sums by the forward
// step's own operations (c and its derivatives from sin/cos of u as in
// stage()), so every stage product sees the same values and the result is
// the rebuild's bit for bit, without the rebuild's four d-wide stage sums.
template <int C, int TPP>
__device__ __forceinline__ void adjoint_step_rec(const ProbDev<float> &P, const Lane<C, TPP> &L, const float *v,
                                                 float eps, float h, const float2 *r, float &alpha, float *lp,
                                                 float *rec)
{
    const float h2 = 0.5f * h, h3 = h / 3.f, h6 = h / 6.f;
    const float u = r[0].x, B = r[0].y;
    float su = u, sB = B;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        float sn, cs;
        __sincosf(su, &sn, &cs);
        const St s{su, sB, fmaf(0.5f, sn, 1.f), 0.5f * cs, -0.5f * sn, r[1 + st].x, r[1 + st].y};
        put(rec, st, s);
        const float hs = (st == 2) ? h : h2;
        su = fmaf(hs, rate_u(s), u);
        sB = fmaf(hs, rate_B(s), B);
    }
    const float Lw = dot_we<C, TPP>(P, L, lp);
    float R = 0.f, W = 0.f, sumR = 0.f;
#pragma unroll 1
    for (int j = 3; j >= 0; --j) {
        const St s = get(rec, j);
        const float wl = (j == 0 || j == 3) ? h6 : h3;
        const float wp = (j == 2) ? h : h2;
        vjp<C, TPP>(P, L, v, eps, s, fmaf(wl, alpha, __fmul_rn(wp, R)), fmaf(wl, Lw, __fmul_rn(wp, W)), wl, W, lp, R,
                    W);
        sumR = __fadd_rn(sumR, R);
    }
    alpha = __fadd_rn(alpha, sumR);
}

// Gradient of G with respect to v, less the -x of the Hopf terminal term:
// gr gets lam_p(0) (the caller subtracts x).  Returns G.  K = 1: the forward
// pass keeps every step's record in sr (5 N float2) and the reverse pass
// reads them, the next step's while the current one runs; K > 1: sr holds
// ceil(N/K) checkpoints (u_n, B_n) and each segment's states are recomputed
// into seg (K states), each step's stages rebuilt.  Both give the same
// gradient bit for bit (thread-private scratch).
template <int C, int TPP>
__device__ __forceinline__ float gradient(const ProbDev<float> &P, const Lane<C, TPP> &L, int kahan, int K, float u0,
                                          float xv, const float *v, float t, int N, float *gr, float2 *sr,
                                          float2 *seg, float *rec)
{
    if (N < 1 || N > MAX_N) {
#pragma unroll
        for (int k = 0; k < Lane<C, TPP>::CL; ++k) gr[k] = NAN;
        return NAN;
    }
    const float eps = P.s_eps, h = t / (float)N;
    float Bn;
    float2 *ck = sr;
    const float F = functional<C, TPP>(P, L, kahan, u0, xv, v, t, N, K == 1 ? nullptr : ck, K, Bn,
                                       K == 1 ? sr : nullptr);
    terminal<C, TPP>(P, L, xv, v, Bn, gr);  // seed lam_p = grad g*(p_N), kept in gr
#pragma unroll
    for (int k = 0; k < Lane<C, TPP>::CL; ++k) gr[k] = __fmul_rn(L.e(P, k), gr[k]);  // sign-folded
    float alpha = 0.f;
    if (K == 1) {
        float2 cur[5], nxt[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) cur[i] = sr[5 * (N - 1) + i];
        for (int n = N - 1; n >= 0; --n) {
            const int m = n > 0 ? n - 1 : 0;
#pragma unroll
            for (int i = 0; i < 5; ++i) nxt[i] = sr[5 * m + i];
            adjoint_step_rec<C, TPP>(P, L, v, eps, h, cur, alpha, gr, rec);
#pragma unroll
            for (int i = 0; i < 5; ++i) cur[i] = nxt[i];
        }
    } else {
        const int nseg = (N + K - 1) / K;
        for (int sg = nseg - 1; sg >= 0; --sg) {
            const int n0 = sg * K, n1 = min(N, n0 + K);
            float u = ck[sg].x, B = ck[sg].y;
            for (int n = n0; n < n1; ++n) {
                seg[n - n0] = make_float2(u, B);
                if (n + 1 < n1) {
                    float dQ;
                    step<C, TPP>(P, L, v, eps, h, u, B, dQ, nullptr);
                }
            }
            for (int n = n1 - 1; n >= n0; --n)
                adjoint_step<C, TPP>(P, L, v, eps, h, seg[n - n0].x, seg[n - n0].y, alpha, gr, rec);
        }
    }
#pragma unroll
    for (int k = 0; k < Lane<C, TPP>::CL; ++k) gr[k] = __fmul_rn(L.e(P, k), gr[k]);
    return F;
}

// Checkpoint interval: the caller's, else 1 (a checkpoint is 8 bytes).
__device__ __forceinline__ int ck_interval(int N, int fixed)
{
    int K = fixed > 0 ? fixed : 1;
    K = max(K, (N + MAX_N - 1) / MAX_N);
    return min(K, MAX_SEG);
}

// The lane's components of a row of d values.
template <int C, int TPP>
__device__ __forceinline__ void load_vec(const Lane<C, TPP> &L, const float *row, int d, float *out)
{
#pragma unroll
    for (int k = 0; k < Lane<C, TPP>::CL; ++k) {
        const int i = L.comp(k);
        out[k] = (i < d) ? __ldg(row + i) : 0.f;
    }
}
template <int C, int TPP>
__device__ __forceinline__ void store_vec(const Lane<C, TPP> &L, float *row, int d, const float *val)
{
#pragma unroll
    for (int k = 0; k < Lane<C, TPP>::CL; ++k) {
        const int i = L.comp(k);
        if (i < d) row[i] = val[k];
    }
}

// ---------------------------------------------------------------------------
// Rows: functional values and gradients (one thread per row).
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(BLOCK, (min_blocks<C, 1>())) k_eval(RowArgs<float> a)
{
    Lane<C, 1> L;
    L.load(a.P, threadIdx.x & 31);
    const long long stride = (long long)gridDim.x * BLOCK;
    for (long long r = (long long)blockIdx.x * BLOCK + threadIdx.x; r < a.n; r += stride) {
        if (a.pidx && a.pidx[r] != a.pfilter) continue;
        const int N = a.nsteps ? a.nsteps[r] : a.n_default;
        float x[C], v[C], Bn;
        load_vec<C, 1>(L, a.x + r * a.P.ld, a.P.d, x);
        load_vec<C, 1>(L, a.v + r * a.P.ld, a.P.d, v);
        a.F[r] = functional<C, 1>(a.P, L, a.kahan, dot_w<C, 1>(a.P, L, x), dot<C, 1>(L, x, v), v, a.t[r], N,
                                  nullptr, 1, Bn);
    }
}

template <int C>
__global__ void __launch_bounds__(BLOCK, (min_blocks<C, 1>())) k_grad(RowArgs<float> a)
{
    __shared__ float s_rec[4 * REC][BLOCK];
    float2 sr[5 * MAX_N];
    float2 seg[MAX_SEG];
    float *rec = &s_rec[0][threadIdx.x];
    Lane<C, 1> L;
    L.load(a.P, threadIdx.x & 31);
    const long long stride = (long long)gridDim.x * BLOCK;
    for (long long r = (long long)blockIdx.x * BLOCK + threadIdx.x; r < a.n; r += stride) {
        if (a.pidx && a.pidx[r] != a.pfilter) continue;
        const int N = a.nsteps ? a.nsteps[r] : a.n_default;
        float x[C], v[C], gr[C];
        load_vec<C, 1>(L, a.x + r * a.P.ld, a.P.d, x);
        load_vec<C, 1>(L, a.v + r * a.P.ld, a.P.d, v);
        const int K = ck_interval(N, a.ck_interval);
        const float F = gradient<C, 1>(a.P, L, a.kahan, K, dot_w<C, 1>(a.P, L, x), dot<C, 1>(L, x, v), v, a.t[r], N,
                                       gr, sr, seg, rec);
#pragma unroll
        for (int k = 0; k < C; ++k) gr[k] -= x[k];
        store_vec<C, 1>(L, a.grad + r * a.P.ld, a.P.d, gr);
        if (a.F) a.F[r] = F;
    }
}

// ---------------------------------------------------------------------------
// FP64 value of the functional at each query's chosen start (the solve's
// final phi, Sec. 4.3: phi = -G at the returned optimum), one thread per
// query, in the reduced state: the RK4 iterates are p_n = v + B_n w and
// u_n = <w, gamma_n> exactly as in binary32 above, here with every stage sum
// in double and the problem's parameters read from its FP64 block.  The same
// stages, weights, quadrature (plain sum) and terminal term as the lane-group
// FP64 functional, up to rounding; step counts outside [1, MAX_N] give NaN.
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(BLOCK) k_phi64(CertArgs<float> a)
{
    const ProbDev<double> &P = a.P;
    const int d = P.d;
    const long long stride = (long long)gridDim.x * BLOCK;
    for (long long q = (long long)blockIdx.x * BLOCK + threadIdx.x; q < a.n; q += stride) {
        if (a.pidx && a.pidx[q] != a.pfilter) continue;
        const long long pid = a.best_pid[q];
        if (pid < 0) continue;
        const int N = a.nsteps ? a.nsteps[q] : a.n_default;
        if (N < 1 || N > MAX_N) {
            a.phi[q] = NAN;
            continue;
        }
        double v[C], u = 0.0, xv = 0.0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const double xk = (k < d) ? (double)__ldg(a.x + q * P.ld + k) : 0.0;
            v[k] = (k < d) ? (double)__ldg(a.v + pid * P.ld + k) : 0.0;
            u = fma(__ldg(P.w + k), xk, u);
            xv = fma(xk, v[k], xv);
        }
        const double eps = P.s_eps, h = (double)a.t[q] / (double)N, h2 = 0.5 * h, h6 = h / 6.0;
        double B = 0.0, Q = 0.0;
        for (int n = 0; n < N; ++n) {
            double su = u, sB = B, au = 0.0, aB = 0.0, aL = 0.0;
#pragma unroll 1
            for (int st = 0; st < 4; ++st) {
                double phi = 0.0, D = 0.0;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const double wk = __ldg(P.w + k), ek = __ldg(P.e + k);
                    const double p = fma(sB, wk, v[k]);
                    const double qq = fma(p, p, eps);
                    const double r = rsqrt(qq);
                    phi = fma(ek, qq * r, phi);
                    D = fma(wk * ek, r * p, D);
                }
                double sn, cs;
                sincos(su, &sn, &cs);
                const double c = fma(0.5, sn, 1.0), c1 = 0.5 * cs;
                const double ku = -c * D, kB = phi * c1, kL = phi * fma(-c1, su, c);
                const double wgt = (st == 0 || st == 3) ? 1.0 : 2.0;
                au = fma(wgt, ku, au);
                aB = fma(wgt, kB, aB);
                aL = fma(wgt, kL, aL);
                const double hs = (st == 2) ? h : h2;
                su = fma(hs, ku, u);
                sB = fma(hs, kB, B);
            }
            u = fma(h6, au, u);
            B = fma(h6, aB, B);
            Q += h6 * aL;
        }
        // Hopf terminal term g*(p_N) - <x, v>
        double G = 0.0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const double p = fma(B, __ldg(P.w + k), v[k]);
            if (P.g_kind == HJ_G_QUAD_SHIFT) G += p * fma(0.5, p, __ldg(P.ga + k));
            else G += 0.5 * __ldg(P.gs2 + k) * p * p;
        }
        if (P.g_kind == HJ_G_ELLIPSE) G += 0.5;
        a.phi[q] = -((G - xv) + Q);
    }
}

// ---------------------------------------------------------------------------
// Persistent descent, one pair per group of TPP lanes: Algorithm 1 (MODE
// DESC_CD, cyclic coordinate descent with finite differences; one lane per
// pair) or gradient descent with the adjoint (DESC_GD), the same iteration
// rules, stop tests, coarse-to-fine phases, certificate and outputs as
// k_desc.  Groups without a pair take the next one from the problem's work
// list (one atomic per warp) between iterations.  The launch does nothing
// unless the work list's length lies in [run_lo, run_hi).  v lives in
// registers; the per-coordinate steps and the previous derivatives in shared
// memory ([component][thread], conflict-free); x is read from global memory
// (cached) once per iteration.
// ---------------------------------------------------------------------------
template <int C, int MODE, int TPP>
__global__ void __launch_bounds__(BLOCK, (min_blocks<C, TPP>())) k_desc(DescArgs<float> a)
{
    static_assert(MODE == DESC_GD || TPP == 1, "coordinate descent runs one lane per pair");
    constexpr int CL = C / TPP;
    constexpr unsigned LEAD = TPP == 1 ? FULL : 0x55555555u;  // the first lane of every group
    const long long n = a.wl_count[a.problem];
    if (n < a.run_lo || n >= a.run_hi) return;
    __shared__ float s_al[CL][BLOCK], s_pr[CL][BLOCK];
    __shared__ float s_rec[MODE == DESC_GD ? 4 * REC : 1][BLOCK];
    const int tid = threadIdx.x, lane = tid & 31;
    Lane<C, TPP> L;
    L.load(a.P, lane);
    const int lead = lane - L.gl;
    const int d = a.P.d;
    const long long begin = a.seg_begin[a.problem];
    const float eps_stop = (float)a.S.eps;
    const float fd_h = (float)a.S.fd_h;
    const bool central = (a.S.grad != HJ_GRAD_FD_FORWARD);
    const bool coarse = (MODE != DESC_CD) && a.phase == 1;
    float2 sr[MODE == DESC_GD ? 5 * MAX_N : 1];
    float2 seg[MODE == DESC_GD ? MAX_SEG : 1];
    float *rec = &s_rec[0][tid];
    unsigned long long n_it = 0, n_f = 0, n_g = 0, n_rk = 0, n_adj = 0, n_pairs = 0, n_sumN = 0, n_cert = 0;

    bool active = false, exhausted = false;
    long long pid = 0, q = 0;
    int N = 1, Ncur = 1, it = 0, count = 0, kper = 0, bad = 0;
    float t = 0.f, v[CL];
#pragma unroll
    for (int k = 0; k < CL; ++k) v[k] = 0.f;

    for (;;) {
        // ---- refill: one atomic per warp for all groups that need a pair -----
        const bool need = !active && !exhausted;
        const unsigned nm = __ballot_sync(FULL, need) & LEAD;
        if (nm) {
            const int leader = __ffs(nm) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(a.cursor + a.problem, __popc(nm));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                const long long j = (long long)base + __popc(nm & ((1u << lead) - 1u));
                if (j >= n) {
                    exhausted = true;
                } else {
                    pid = a.wl[begin + j];
                    q = a.pair_q[pid];
                    const int slot = a.pair_slot[pid], round = a.pair_round[pid];
                    N = a.nsteps ? a.nsteps[q] : a.S.n_default;
                    t = a.t[q];
#pragma unroll
                    for (int k = 0; k < CL; ++k) {
                        s_al[k][tid] = (float)a.S.step;
                        s_pr[k][tid] = 0.f;
                    }
                    if (a.phase == 2) {
                        load_vec<C, TPP>(L, a.vfin + pid * a.P.ld, d, v);  // the coarse level's v
                    } else {
#pragma unroll
                        for (int k = 0; k < CL; ++k) {
                            const int i = L.comp(k);
                            v[k] = (i < d) ? start_component<float>(a.S.seed, a.q_begin + q, slot, round, i,
                                                                    a.S.guess_dist)
                                           : 0.f;
                        }
                    }
                    it = count = kper = bad = 0;
                    Ncur = coarse ? max(1, N / a.S.coarse_div) : N;
                    active = true;
                }
            }
        }
        if (!__any_sync(FULL, active)) break;
        if (!active) continue;

        const float *xr = a.x + q * a.P.ld;
        float u0, xv;  // <w, x>, <x, v>
        {
            float x[CL];
            load_vec<C, TPP>(L, xr, d, x);
            u0 = dot_w<C, TPP>(a.P, L, x);
            xv = dot<C, TPP>(L, x, v);
        }
        // ---- one iteration -----------------------------------------------------
        bool stop = (it >= a.S.max_iters), conv = false;
        const float eps_lvl = coarse ? (float)a.S.coarse_eps : eps_stop;
        if (!stop) {
            if constexpr (MODE == DESC_GD) {
                float gr[CL];
                const int K = ck_interval(Ncur, a.S.ck_interval);
                gradient<C, TPP>(a.P, L, a.S.kahan, K, u0, xv, v, t, Ncur, gr, sr, seg, rec);
                if (L.gl == 0) {  // counted once per pair
                    n_g++;
                    n_rk += Ncur;
                    n_adj += Ncur;
                }
                float big = 0.f;
                bool fin = true;
#pragma unroll
                for (int k = 0; k < CL; ++k) {
                    const int i = L.comp(k);
                    const float g = gr[k] - ((i < d) ? __ldg(xr + i) : 0.f);
                    float al = s_al[k][tid];
                    if (a.S.adapt) {
                        const float prod = g * s_pr[k][tid];
                        if (prod < 0.f) al *= (float)a.S.shrink;
                        else if (prod > 0.f) al = fminf(al * (float)a.S.grow, (float)a.S.step_max);
                    }
                    const float st = __fmul_rn(al, g);
                    fin = fin && isfinite(st);
                    v[k] = __fsub_rn(v[k], st);
                    big = fmaxf(big, fabsf(st));
                    s_pr[k][tid] = g;
                    s_al[k][tid] = al;
                }
                big = L.gmaxf(fin ? big : INFINITY);
                ++it;
                if (!(big < INFINITY)) { bad = 1; stop = true; }
                if (a.S.halving_period > 0 && it % a.S.halving_period == 0) {
#pragma unroll
                    for (int k = 0; k < CL; ++k) s_al[k][tid] *= 0.5f;
                }
                if (big < eps_lvl) conv = stop = true;
            } else {
                const int jc = it % d;
                const float xj = __ldg(xr + jc);
                float vp[C], Bn;
#pragma unroll
                for (int k = 0; k < C; ++k) vp[k] = v[k] + ((k == jc) ? fd_h : 0.f);
                const float Fp = functional<C, 1>(a.P, L, a.S.kahan, u0, fmaf(xj, fd_h, xv), vp, t, N, nullptr, 1, Bn);
#pragma unroll
                for (int k = 0; k < C; ++k) vp[k] = v[k] - ((central && k == jc) ? fd_h : 0.f);
                const float Fm = functional<C, 1>(a.P, L, a.S.kahan, u0, central ? fmaf(-xj, fd_h, xv) : xv, vp, t, N,
                                                  nullptr, 1, Bn);
                n_f += 2;
                n_rk += 2 * N;
                const float dj = central ? (Fp - Fm) / (2.f * fd_h) : (Fp - Fm) / fd_h;
                float al = s_al[jc][tid];
                if (a.S.adapt) {
                    const float prod = dj * s_pr[jc][tid];
                    if (prod < 0.f) al *= (float)a.S.shrink;
                    else if (prod > 0.f) al = fminf(al * (float)a.S.grow, (float)a.S.step_max);
                    s_pr[jc][tid] = dj;
                }
                const float st = __fmul_rn(al, dj);
#pragma unroll
                for (int k = 0; k < C; ++k)
                    if (k == jc) v[k] = __fsub_rn(v[k], st);
                ++it;
                if (!isfinite(st)) { bad = 1; stop = true; }
                // steps 3-4 of Algorithm 1: reset on a move > eps, count a move < eps
                if (fabsf(st) > eps_stop) count = 0;
                else if (fabsf(st) < eps_stop) ++count;
                s_al[jc][tid] = al;
                if (a.S.halving_period > 0 && ++kper == a.S.halving_period) {
                    kper = 0;
#pragma unroll
                    for (int k = 0; k < C; ++k) s_al[k][tid] *= 0.5f;
                }
                if (count >= d) conv = stop = true;
            }
            if (it >= a.S.max_iters) stop = true;
        }
        // ---- finished pair: certificate at the final v, then write it out -----
        const bool first = L.gl == 0;  // one writer per pair
        if (stop && a.phase == 1) {
            if (first) n_it += it;
            store_vec<C, TPP>(L, a.vfin + pid * a.P.ld, d, v);
            if (first) {
                a.iters[pid] = it;
                a.flags[pid] = (uint8_t)(bad << 1);
            }
            active = false;
        } else if (stop) {
            const int cap = (!conv && !bad) ? 1 : 0;
            if (first) {
                n_it += it;
                n_pairs++;
                n_sumN += N;
                n_cert += N;
            }
            float gam[CL], Bn;
            load_vec<C, TPP>(L, xr, d, gam);
            const float F = functional_gamma<C, TPP>(a.P, L, a.S.kahan, u0, dot<C, TPP>(L, gam, v), v, t, N, gam, Bn);
            // Hopf residual |gamma(0) - grad g*(p(0))| / (1 + |gamma(0)|)
            Acc<TPP> num, den;
#pragma unroll
            for (int k = 0; k < CL; ++k) {
                const float p = fmaf(Bn, L.w(a.P, k), v[k]);
                const float diff = gam[k] - fmaf(L.g2(a.P, k), p, L.ga(a.P, k));
                num.fma_(k, diff, diff);
                den.fma_(k, gam[k], gam[k]);
            }
            const float r = sqrtf(L.total(num.a0, num.a1)) / (1.f + sqrtf(L.total(den.a0, den.a1)));
            store_vec<C, TPP>(L, a.vfin + pid * a.P.ld, d, v);
            if (first) {
                const int prior = (a.phase == 2) ? a.iters[pid] : 0;
                const uint8_t fprior = (a.phase == 2) ? (uint8_t)(a.flags[pid] & 2) : (uint8_t)0;
                a.iters[pid] = prior + it;
                a.flags[pid] = (uint8_t)(cap | (bad << 1) | fprior);
                const bool fin = isfinite(F) && isfinite(r);
                uint8_t pass;
                if (!fin) pass = 0;
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
    if (a.stats) {
        unsigned long long c[8] = {n_it, n_f, n_g, n_rk, n_adj, n_pairs, n_sumN, n_cert};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(FULL, c[k], o);
            if (lane == 0 && c[k]) atomicAdd(a.stats + k, c[k]);
        }
    }
}

}  // namespace r1
}  // namespace hjd
