// hj_device.cuh -- device arithmetic of the generalized Lax/Hopf solver.
//
// One (query, start) pair is handled by a group of TPP consecutive lanes of
// a warp (TPP in {1,2,4,8,16,32}).  Lane l of a group holds the C vector
// components i = l + k*TPP, k < C, of gamma, p, v and of every per-component
// parameter, all in registers; dot products over the dimension are a local
// sum followed by an xor-shuffle reduction inside the group.  Components
// i >= d are zero and every per-component parameter is zero there (the sign
// vector e included), so they drop out of every sum with no branches.
//
// Time runs backward: tau = t - s goes from 0 to t, the state z = (gamma, p)
// follows dz/dtau = (-dH/dp, +dH/dx) from z(0) = (x, v), and the running
// cost is integrated alongside (Sec. 4.1, final value problem).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hj.h"

namespace hjd {

constexpr int DPAD = 1024;   // parameter vectors are zero padded to this length
constexpr int MAX_N = 256;   // RK4 steps supported by the adjoint buffers
constexpr int MAX_SEG = 16;  // checkpoint segment length cap (ceil(sqrt(MAX_N)))

// ---------------------------------------------------------------------------
// Problem parameters on the device (one problem per launch).
// ---------------------------------------------------------------------------
template <typename T>
struct ProbDev {
    int d, family, principle, g_kind, m, n_neg, n_guesses, ld;
    T s_eps;
    const T *w;     // [DPAD] speed direction
    const T *e;     // [DPAD] signs of the smooth non-convex family (0 past d)
    const T *ga;    // [DPAD] shift a of g = |x-a|^2/2
    const T *gs2;   // [DPAD] sigma^2 of g = sum x^2/(2 sigma^2)
    const T *gis2;  // [DPAD] 1/sigma^2
    const T *A;     // [d*d] row-major (linear-quadratic family)
    const T *B;     // [d*m] row-major
};

// Solver constants on the device.
struct SolverDev {
    int quad, grad, max_iters, halving_period, adapt, max_trials, max_rounds, guess_dist, kahan, n_default;
    double fd_h, step, eps, grow, shrink, step_max, cert_tol;
    unsigned long long seed;
};

// ---------------------------------------------------------------------------
// Lane groups.
// ---------------------------------------------------------------------------
struct Grp {
    int tpp;        // lanes per pair
    int lane;       // lane inside the group
    unsigned mask;  // lanes of this group inside the warp
};

__device__ __forceinline__ Grp make_grp(int tpp)
{
    int l = threadIdx.x & 31;
    int base = l & ~(tpp - 1);
    unsigned m = (tpp == 32) ? 0xffffffffu : (((1u << tpp) - 1u) << base);
    return Grp{tpp, l - base, m};
}

template <typename T>
__device__ __forceinline__ T gsum(const Grp &g, T x)
{
    for (int o = g.tpp >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(g.mask, x, o);
    return x;
}
template <typename T>
__device__ __forceinline__ void gsum2(const Grp &g, T &a, T &b)
{
    for (int o = g.tpp >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(g.mask, a, o);
        b += __shfl_xor_sync(g.mask, b, o);
    }
}
template <typename T>
__device__ __forceinline__ void gsum3(const Grp &g, T &a, T &b, T &c)
{
    for (int o = g.tpp >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(g.mask, a, o);
        b += __shfl_xor_sync(g.mask, b, o);
        c += __shfl_xor_sync(g.mask, c, o);
    }
}
template <typename T>
__device__ __forceinline__ void gsum4(const Grp &g, T &a, T &b, T &c, T &e)
{
    for (int o = g.tpp >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(g.mask, a, o);
        b += __shfl_xor_sync(g.mask, b, o);
        c += __shfl_xor_sync(g.mask, c, o);
        e += __shfl_xor_sync(g.mask, e, o);
    }
}
template <typename T>
__device__ __forceinline__ T gmax(const Grp &g, T x)
{
    for (int o = g.tpp >> 1; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(g.mask, x, o));
    return x;
}

// ---------------------------------------------------------------------------
// Precision-dispatched math.  fp32 uses the hardware reciprocal square root
// and the fast sine/cosine (|<w,gamma>| stays O(1) in these problems); fp64
// uses the correctly rounded library routines.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsq(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsq(double q) { return rsqrt(q); }
__device__ __forceinline__ void sin_cos(float u, float *s, float *c) { __sincosf(u, s, c); }
__device__ __forceinline__ void sin_cos(double u, double *s, double *c) { sincos(u, s, c); }
__device__ __forceinline__ bool finite_(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products with the published multipliers; the key is
// bumped by the published Weyl increments after each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Word j of the start stream of (query id q, slot, round).
__device__ __forceinline__ uint32_t start_word(unsigned long long seed, long long q, int slot, int round, int j)
{
    uint4 c = make_uint4((uint32_t)(j >> 2), (uint32_t)slot | ((uint32_t)round << 16),
                         (uint32_t)((unsigned long long)q & 0xffffffffull), (uint32_t)((unsigned long long)q >> 32));
    uint4 o = philox4x32_10(c, make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32)));
    switch (j & 3) {
    case 0: return o.x;
    case 1: return o.y;
    case 2: return o.z;
    default: return o.w;
    }
}

// Component i of a start: uniform 4u-2 with u = (word>>8) 2^-24 (exact in
// binary32), or Irwin-Hall(12) summed as an integer and shifted by 6.
template <typename T>
__device__ __forceinline__ T start_component(unsigned long long seed, long long q, int slot, int round, int i,
                                             int dist)
{
    if (dist == 0) {
        uint32_t wd = start_word(seed, q, slot, round, i);
        return (T)(4.0 * ((double)(wd >> 8) * 0x1p-24) - 2.0);
    }
    unsigned long long s = 0;
    for (int k = 0; k < 12; ++k) s += start_word(seed, q, slot, round, 12 * i + k) >> 8;
    return (T)((double)s * 0x1p-24 - 6.0);
}

// ---------------------------------------------------------------------------
// Per-thread copies of the per-component parameters.
// ---------------------------------------------------------------------------
template <typename T, int C>
struct TP {
    T w[C], e[C], ga[C], gs2[C], gis2[C];
    __device__ void load(const ProbDev<T> &P, const Grp &g)
    {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            int i = g.lane + k * g.tpp;
            w[k] = P.w[i];
            e[k] = P.e[i];
            ga[k] = P.ga[i];
            gs2[k] = P.gs2[i];
            gis2[k] = P.gis2[i];
        }
    }
};

// ---------------------------------------------------------------------------
// Families.  field(): dz/dtau = (-dH/dp, +dH/dx) and the running cost L
// (Lax: <p, dH/dp> - H;  Hopf: H - <dH/dx, gamma>).  vjp(): for weights
// (ag, ap) on the state rows and b on the cost row, the products
//   rg = ag.d(-H_p)/dgamma + ap.d(H_x)/dgamma + b dL/dgamma, and the same in p.
// Speed c(gamma) = 1 + sin(u)/2, u = <w, gamma>, c' = cos(u)/2, c'' = -sin(u)/2.
// ---------------------------------------------------------------------------
template <typename T, int C, int FAM, int PR>
struct Family;

// H = |p|^2/2: dz/dtau = (-p, 0), L = |p|^2/2 for both principles.
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_QUAD_ISO, PR> {
    __device__ static __forceinline__ void field(const Grp &g, const TP<T, C> &tp, const T *gam, const T *p, T *dg,
                                                 T *dp, T &L)
    {
        T pp = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -p[k];
            dp[k] = 0;
            pp = fma(p[k], p[k], pp);
        }
        L = (T)0.5 * gsum(g, pp);
    }
    __device__ static __forceinline__ void vjp(const Grp &, const TP<T, C> &, const T *, const T *p, const T *ag,
                                               const T *, T b, T *rg, T *rp)
    {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = 0;
            rp[k] = fma(b, p[k], -ag[k]);
        }
    }
    static constexpr int field_flops_per_comp = 3, field_flops_fixed = 2, vjp_flops_per_comp = 2,
                         vjp_flops_fixed = 0;
};

// H = c^2 |p|^2/2: dz/dtau = (-c^2 p, c c' |p|^2 w),
// L_Lax = c^2|p|^2/2, L_Hopf = c^2|p|^2/2 - c c' |p|^2 u.
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_SPEED_QUAD, PR> {
    __device__ static __forceinline__ void field(const Grp &g, const TP<T, C> &tp, const T *gam, const T *p, T *dg,
                                                 T *dp, T &L)
    {
        T u = 0, pp = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            u = fma(tp.w[k], gam[k], u);
            pp = fma(p[k], p[k], pp);
        }
        gsum2(g, u, pp);
        T su, cu;
        sin_cos(u, &su, &cu);
        T c = fma((T)0.5, su, (T)1), c1 = (T)0.5 * cu;
        T c2 = c * c, fx = c * c1 * pp;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -c2 * p[k];
            dp[k] = fx * tp.w[k];
        }
        L = (T)0.5 * c2 * pp;
        if (PR == HJ_HOPF) L -= fx * u;
    }
    __device__ static __forceinline__ void vjp(const Grp &g, const TP<T, C> &tp, const T *gam, const T *p,
                                               const T *ag, const T *ap, T b, T *rg, T *rp)
    {
        T u = 0, pp = 0, A = 0, Bw = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            u = fma(tp.w[k], gam[k], u);
            pp = fma(p[k], p[k], pp);
            A = fma(ag[k], p[k], A);
            Bw = fma(ap[k], tp.w[k], Bw);
        }
        gsum4(g, u, pp, A, Bw);
        T su, cu;
        sin_cos(u, &su, &cu);
        T c = fma((T)0.5, su, (T)1), c1 = (T)0.5 * cu, cc2 = (T)-0.5 * su;
        T q = fma(c1, c1, c * cc2);  // d(c c')/du
        T dEdu = (T)-2 * c * c1 * A + q * pp * Bw;
        T dLp;
        if (PR == HJ_LAX) {
            dEdu += b * c * c1 * pp;
            dLp = c * c;
        } else {
            dEdu -= b * q * pp * u;
            dLp = c * c - (T)2 * c * c1 * u;
        }
        T kp = (T)2 * c * c1 * Bw + b * dLp;
        T mc2 = -c * c;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = dEdu * tp.w[k];
            rp[k] = fma(mc2, ag[k], kp * p[k]);
        }
    }
    static constexpr int field_flops_per_comp = 6, field_flops_fixed = 12, vjp_flops_per_comp = 11,
                         vjp_flops_fixed = 26;
};

// H = c Phi(p), Phi = sum_i e_i s(p_i), s = sqrt(p^2 + eps):
// dz/dtau = (-c Phi', Phi c' w), Phi'_i = e_i p_i / s_i,
// L_Lax = c (<p, Phi'> - Phi) = -c eps sum_i e_i / s_i, L_Hopf = Phi (c - c' u).
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_SMOOTH_NONCONVEX, PR> {
    __device__ static __forceinline__ void field(const Grp &g, const TP<T, C> &tp, const T *gam, const T *p, T *dg,
                                                 T *dp, T &L, T eps)
    {
        T u = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) u = fma(tp.w[k], gam[k], u);
        u = gsum(g, u);
        T su, cu;
        sin_cos(u, &su, &cu);
        T c = fma((T)0.5, su, (T)1), c1 = (T)0.5 * cu;
        T phi = 0, lax = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T q = fma(p[k], p[k], eps);
            T r = rsq(q);
            T er = tp.e[k] * r;
            phi = fma(er, q, phi);   // e s
            if (PR == HJ_LAX) lax += er;
            dg[k] = -c * er * p[k];
        }
        if (PR == HJ_LAX) gsum2(g, phi, lax);
        else phi = gsum(g, phi);
        T fx = phi * c1;
#pragma unroll
        for (int k = 0; k < C; ++k) dp[k] = fx * tp.w[k];
        if (PR == HJ_LAX) L = -c * eps * lax;
        else L = phi * (c - c1 * u);
    }
    __device__ static __forceinline__ void vjp(const Grp &g, const TP<T, C> &tp, const T *gam, const T *p,
                                               const T *ag, const T *ap, T b, T *rg, T *rp, T eps)
    {
        T u = 0, Bw = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            u = fma(tp.w[k], gam[k], u);
            Bw = fma(ap[k], tp.w[k], Bw);
        }
        gsum2(g, u, Bw);
        T su, cu;
        sin_cos(u, &su, &cu);
        T c = fma((T)0.5, su, (T)1), c1 = (T)0.5 * cu, cc2 = (T)-0.5 * su;
        T phi = 0, A = 0, pdphi = 0;
        T r[C];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T q = fma(p[k], p[k], eps);
            r[k] = rsq(q);
            T er = tp.e[k] * r[k];
            phi = fma(er, q, phi);
            T dphi = er * p[k];
            A = fma(ag[k], dphi, A);
            if (PR == HJ_LAX) pdphi = fma(p[k], dphi, pdphi);
        }
        if (PR == HJ_LAX) gsum3(g, phi, A, pdphi);
        else gsum2(g, phi, A);
        T dEdu = -c1 * A + phi * cc2 * Bw;
        T kd;  // coefficient of Phi'_i in rp
        if (PR == HJ_LAX) {
            dEdu += b * c1 * (pdphi - phi);
            kd = c1 * Bw;
        } else {
            dEdu -= b * phi * cc2 * u;
            kd = c1 * Bw + b * (c - c1 * u);
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T er = tp.e[k] * r[k];
            T dphi = er * p[k];
            T ddphi = eps * er * r[k] * r[k];  // e eps / s^3
            rg[k] = dEdu * tp.w[k];
            T v = fma(-c * ag[k], ddphi, kd * dphi);
            if (PR == HJ_LAX) v = fma(b * c * p[k], ddphi, v);
            rp[k] = v;
        }
    }
    static constexpr int field_flops_per_comp = 9, field_flops_fixed = 10, vjp_flops_per_comp = 20,
                         vjp_flops_fixed = 24;
};

// Dispatch helpers so every family shares one call form.
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void field(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p, T *dg,
                                      T *dp, T &L)
{
    if constexpr (FAM == HJ_FAM_SMOOTH_NONCONVEX) Family<T, C, FAM, PR>::field(g, tp, gam, p, dg, dp, L, eps);
    else Family<T, C, FAM, PR>::field(g, tp, gam, p, dg, dp, L);
}
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void vjp(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p, const T *ag,
                                    const T *ap, T b, T *rg, T *rp)
{
    if constexpr (FAM == HJ_FAM_SMOOTH_NONCONVEX) Family<T, C, FAM, PR>::vjp(g, tp, gam, p, ag, ap, b, rg, rp, eps);
    else Family<T, C, FAM, PR>::vjp(g, tp, gam, p, ag, ap, b, rg, rp);
}

// ---------------------------------------------------------------------------
// Initial data: terminal value, its gradient (adjoint seed) and the
// certificate residual.
//   Lax  term g(gamma0), seed (grad g(gamma0), 0)
//   Hopf term g*(p0) - <x, v>, seed (0, grad g*(p0))
// ---------------------------------------------------------------------------
template <typename T, int C, int PR>
__device__ __forceinline__ T terminal(const Grp &g, const TP<T, C> &tp, int g_kind, const T *x, const T *v,
                                      const T *gam, const T *p, T *sg, T *sp)
{
    T acc = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        if (PR == HJ_LAX) {
            T gr = (g_kind == HJ_G_QUAD_SHIFT) ? gam[k] - tp.ga[k] : gam[k] * tp.gis2[k];
            acc = fma((T)0.5 * gr, (g_kind == HJ_G_QUAD_SHIFT) ? gr : gam[k], acc);
            if (sg) { sg[k] = gr; sp[k] = 0; }
        } else {
            T gr = (g_kind == HJ_G_QUAD_SHIFT) ? p[k] + tp.ga[k] : tp.gs2[k] * p[k];
            T val = (g_kind == HJ_G_QUAD_SHIFT) ? p[k] * fma((T)0.5, p[k], tp.ga[k]) : (T)0.5 * gr * p[k];
            acc += val - x[k] * v[k];
            if (sg) { sg[k] = 0; sp[k] = gr; }
        }
    }
    return gsum(g, acc);
}

// Relative certificate residual (Sec. 4.3) from (gamma(0), p(0)).
template <typename T, int C, int PR>
__device__ __forceinline__ T cert_residual(const Grp &g, const TP<T, C> &tp, int g_kind, const T *gam, const T *p)
{
    T num = 0, den = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        T diff, base;
        if (PR == HJ_LAX) {
            T gr = (g_kind == HJ_G_QUAD_SHIFT) ? gam[k] - tp.ga[k] : gam[k] * tp.gis2[k];
            diff = p[k] - gr;
            base = p[k];
        } else {
            T gr = (g_kind == HJ_G_QUAD_SHIFT) ? p[k] + tp.ga[k] : tp.gs2[k] * p[k];
            diff = gam[k] - gr;
            base = gam[k];
        }
        num = fma(diff, diff, num);
        den = fma(base, base, den);
    }
    gsum2(g, num, den);
    return sqrt(num) / ((T)1 + sqrt(den));
}

// ---------------------------------------------------------------------------
// Forward integration.  One classical RK4 step of the augmented system;
// Q accumulates the running cost (RK4 weights, or the rectangle node at the
// new state), with optional Kahan compensation.
// ---------------------------------------------------------------------------
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void rk4_step(const Grp &g, const TP<T, C> &tp, T eps, T h, int quad, int kahan, T *gam,
                                         T *p, T &Q, T &Qc)
{
    T ag[C], ap[C], zg[C], zp[C], kg[C], kp[C], L, aL;
    const T h2 = (T)0.5 * h;
    field<T, C, FAM, PR>(g, tp, eps, gam, p, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = kg[k];
        ap[k] = kp[k];
        zg[k] = fma(h2, kg[k], gam[k]);
        zp[k] = fma(h2, kp[k], p[k]);
    }
    aL = L;
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = fma((T)2, kg[k], ag[k]);
        ap[k] = fma((T)2, kp[k], ap[k]);
        zg[k] = fma(h2, kg[k], gam[k]);
        zp[k] = fma(h2, kp[k], p[k]);
    }
    aL = fma((T)2, L, aL);
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = fma((T)2, kg[k], ag[k]);
        ap[k] = fma((T)2, kp[k], ap[k]);
        zg[k] = fma(h, kg[k], gam[k]);
        zp[k] = fma(h, kp[k], p[k]);
    }
    aL = fma((T)2, L, aL);
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
    const T h6 = h / (T)6;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        gam[k] = fma(h6, ag[k] + kg[k], gam[k]);
        p[k] = fma(h6, ap[k] + kp[k], p[k]);
    }
    aL += L;
    T dQ;
    if (quad == HJ_QUAD_RK4) {
        dQ = h6 * aL;
    } else {
        T Ln, dg_[C], dp_[C];
        field<T, C, FAM, PR>(g, tp, eps, gam, p, dg_, dp_, Ln);
        dQ = h * Ln;
    }
    if (kahan) {
        T y = dQ - Qc;
        T s = Q + y;
        Qc = (s - Q) - y;
        Q = s;
    } else {
        Q += dQ;
    }
}

// Functional value F (Lax) or G (Hopf); gam/p hold (x, v) on entry and
// (gamma(0), p(0)) on exit.
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ T functional(const Grp &g, const TP<T, C> &tp, const ProbDev<T> &P, int quad, int kahan,
                                        const T *x, const T *v, T t, int N, T *gam, T *p)
{
    if (N < 1 || N > MAX_N) return (T)NAN;  // step counts outside [1, MAX_N] are rejected
    const T h = t / (T)N;
    T Q = 0, Qc = 0;
    for (int n = 0; n < N; ++n) rk4_step<T, C, FAM, PR>(g, tp, P.s_eps, h, quad, kahan, gam, p, Q, Qc);
    return terminal<T, C, PR>(g, tp, P.g_kind, x, v, gam, p, (T *)nullptr, (T *)nullptr) + Q;
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the RK4 map (exact gradient of the discretised
// functional).  Forward: checkpoints of z every K = ceil(sqrt(N)) steps.
// Reverse, segment by segment: recompute the segment's steps from its
// checkpoint storing the four stage inputs of every step, then run the
// adjoint of each step backward:
//   a4 = J(Z4)^T(h/6 lam, h/6 b)
//   a3 = J(Z3)^T(h/3 lam + h a4, h/3 b)
//   a2 = J(Z2)^T(h/3 lam + h/2 a3, h/3 b)
//   a1 = J(Z1)^T(h/6 lam + h/2 a2, h/6 b)
//   lam += a1 + a2 + a3 + a4
// with b = 1 for the RK4 quadrature (0 for the rectangle rule, whose nodes
// add h grad L(z_{n+1}) to lam directly).  The seed lam(tau=t) comes from
// the terminal term; dF/dv = lam_p(tau=0) (minus x for Hopf).
// Buffers (per thread, local memory) are sized for N <= MAX_N.
// ---------------------------------------------------------------------------
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void stage_inputs(const Grp &g, const TP<T, C> &tp, T eps, T h, const T *zg, const T *zp,
                                             T *st /* [4][2C] */, T *ng, T *np)
{
    // Computes one RK4 step from (zg, zp), storing its four stage inputs and
    // returning the new state in (ng, np).
    T ag[C], ap[C], kg[C], kp[C], sg[C], sp[C], L;
    const T h2 = (T)0.5 * h, h6 = h / (T)6;
#pragma unroll
    for (int k = 0; k < C; ++k) { st[k] = zg[k]; st[C + k] = zp[k]; }
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = kg[k]; ap[k] = kp[k];
        sg[k] = fma(h2, kg[k], zg[k]); sp[k] = fma(h2, kp[k], zp[k]);
        st[2 * C + k] = sg[k]; st[3 * C + k] = sp[k];
    }
    field<T, C, FAM, PR>(g, tp, eps, sg, sp, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = fma((T)2, kg[k], ag[k]); ap[k] = fma((T)2, kp[k], ap[k]);
        sg[k] = fma(h2, kg[k], zg[k]); sp[k] = fma(h2, kp[k], zp[k]);
        st[4 * C + k] = sg[k]; st[5 * C + k] = sp[k];
    }
    field<T, C, FAM, PR>(g, tp, eps, sg, sp, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = fma((T)2, kg[k], ag[k]); ap[k] = fma((T)2, kp[k], ap[k]);
        sg[k] = fma(h, kg[k], zg[k]); sp[k] = fma(h, kp[k], zp[k]);
        st[6 * C + k] = sg[k]; st[7 * C + k] = sp[k];
    }
    field<T, C, FAM, PR>(g, tp, eps, sg, sp, kg, kp, L);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ng[k] = fma(h6, ag[k] + kg[k], zg[k]);
        np[k] = fma(h6, ap[k] + kp[k], zp[k]);
    }
}

template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void adjoint_step(const Grp &g, const TP<T, C> &tp, T eps, T h, T b, const T *st,
                                             T *lg, T *lp)
{
    T wg[C], wp[C], rg[C], rp[C], sumg[C], sump[C];
    const T h6 = h / (T)6, h3 = h / (T)3, h2 = (T)0.5 * h;
    // stage 4
#pragma unroll
    for (int k = 0; k < C; ++k) { wg[k] = h6 * lg[k]; wp[k] = h6 * lp[k]; }
    vjp<T, C, FAM, PR>(g, tp, eps, st + 6 * C, st + 7 * C, wg, wp, h6 * b, rg, rp);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        sumg[k] = rg[k]; sump[k] = rp[k];
        wg[k] = fma(h3, lg[k], h * rg[k]); wp[k] = fma(h3, lp[k], h * rp[k]);
    }
    // stage 3
    vjp<T, C, FAM, PR>(g, tp, eps, st + 4 * C, st + 5 * C, wg, wp, h3 * b, rg, rp);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        sumg[k] += rg[k]; sump[k] += rp[k];
        wg[k] = fma(h3, lg[k], h2 * rg[k]); wp[k] = fma(h3, lp[k], h2 * rp[k]);
    }
    // stage 2
    vjp<T, C, FAM, PR>(g, tp, eps, st + 2 * C, st + 3 * C, wg, wp, h3 * b, rg, rp);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        sumg[k] += rg[k]; sump[k] += rp[k];
        wg[k] = fma(h6, lg[k], h2 * rg[k]); wp[k] = fma(h6, lp[k], h2 * rp[k]);
    }
    // stage 1
    vjp<T, C, FAM, PR>(g, tp, eps, st, st + C, wg, wp, h6 * b, rg, rp);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        lg[k] += sumg[k] + rg[k];
        lp[k] += sump[k] + rp[k];
    }
}

// Gradient of F with respect to v.  ck: >= ceil(N/K)*2C entries, seg: >= K*8C
// entries of thread-private scratch.  Returns F; grad gets dF/dv.
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ T gradient(const Grp &g, const TP<T, C> &tp, const ProbDev<T> &P, int quad, int kahan,
                                   const T *x, const T *v, T t, int N, T *grad, T *ck, T *seg)
{
    if (N < 1 || N > MAX_N) {
        // the checkpoint buffers hold MAX_N steps: reject other step counts
#pragma unroll
        for (int k = 0; k < C; ++k) grad[k] = (T)NAN;
        return (T)NAN;
    }
    const T h = t / (T)N;
    const T eps = P.s_eps;
    int K = 1;
    while (K * K < N) ++K;
    T gam[C], p[C], Q = 0, Qc = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) { gam[k] = x[k]; p[k] = v[k]; }
    for (int n = 0; n < N; ++n) {
        if (n % K == 0) {
            T *c = ck + (n / K) * 2 * C;
#pragma unroll
            for (int k = 0; k < C; ++k) { c[k] = gam[k]; c[C + k] = p[k]; }
        }
        rk4_step<T, C, FAM, PR>(g, tp, eps, h, quad, kahan, gam, p, Q, Qc);
    }
    T lg[C], lp[C];
    T F = terminal<T, C, PR>(g, tp, P.g_kind, x, v, gam, p, lg, lp) + Q;
    const T b = (quad == HJ_QUAD_RK4) ? (T)1 : (T)0;
    const int nseg = (N + K - 1) / K;
    for (int s = nseg - 1; s >= 0; --s) {
        const int n0 = s * K, n1 = min(N, n0 + K);
        T zg[C], zp[C];
        const T *c = ck + s * 2 * C;
#pragma unroll
        for (int k = 0; k < C; ++k) { zg[k] = c[k]; zp[k] = c[C + k]; }
        for (int n = n0; n < n1; ++n) {
            T ng[C], np[C];
            stage_inputs<T, C, FAM, PR>(g, tp, eps, h, zg, zp, seg + (n - n0) * 8 * C, ng, np);
#pragma unroll
            for (int k = 0; k < C; ++k) { zg[k] = ng[k]; zp[k] = np[k]; }
        }
        // zg, zp now hold z_{n1}
        for (int n = n1 - 1; n >= n0; --n) {
            if (quad == HJ_QUAD_RECT) {
                // rectangle node at z_{n+1}: lam += h grad L(z_{n+1})
                T zeros[C], rg[C], rp[C];
                const T *sn = (n + 1 < n1) ? seg + (n + 1 - n0) * 8 * C : nullptr;
                T ug[C], up[C];
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    zeros[k] = 0;
                    ug[k] = sn ? sn[k] : zg[k];
                    up[k] = sn ? sn[C + k] : zp[k];
                }
                vjp<T, C, FAM, PR>(g, tp, eps, ug, up, zeros, zeros, (T)1, rg, rp);
#pragma unroll
                for (int k = 0; k < C; ++k) { lg[k] = fma(h, rg[k], lg[k]); lp[k] = fma(h, rp[k], lp[k]); }
            }
            adjoint_step<T, C, FAM, PR>(g, tp, eps, h, b, seg + (n - n0) * 8 * C, lg, lp);
        }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) grad[k] = (PR == HJ_HOPF) ? lp[k] - x[k] : lp[k];
    return F;
}

}  // namespace hjd
