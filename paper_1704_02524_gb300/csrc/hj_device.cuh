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
#include "hj_internal.h"

namespace hjd {

constexpr int DPAD = 1024;   // parameter vectors are zero padded to this length
constexpr int MAX_N = 256;   // RK4 steps supported by the adjoint buffers
constexpr int MAX_CK = 128;  // checkpoints per gradient (so N <= MAX_CK * interval)
constexpr int MAX_SEG = 16;  // checkpoint interval cap
constexpr int CK_BUDGET = 3072;  // bytes of checkpoint + segment storage per thread (automatic interval)

// ---------------------------------------------------------------------------
// Problem parameters on the device (one problem per launch).
// ---------------------------------------------------------------------------
template <typename T>
struct ProbDev {
    int d, family, principle, g_kind, m, n_neg, n_guesses, ld;
    int huygens;  // Lax kernels of the split-norm family: minimise F^2 (smallest g over the grid nodes)
    T s_eps;
    // split-norm family (the bump norm is its one-block case): H = c_A |p_A| + c_B |p_B|
    // over the coordinate blocks [0, ksplit) and [ksplit, d), c_b = alpha_b (1 + kappa
    // exp(-mu |x - xc_b|^2)), xc_A in w and xc_B in wb
    int ksplit;
    T kappa, mu, alpha_a, alpha_b;
    // Evans-type family: H = -c(x) p_1 + beta |p_2| - |p| - gamma0, c = alpha_a (1 + kappa
    // exp(-mu |x - xc|^2)), xc in w; harmonic family: H = alpha_a (|p|^2 + |x|^2)/2
    T beta, gamma0;
    // linear game: H(x,p,s) = -<diag(w) x, p> + a(s) |p|, a(s) = r_c - r_d (1 + beta sin(omega s))
    T r_c, r_d, omega;
    const T *w;     // [DPAD] speed direction (split-norm family: the centre xc_A)
    const T *wb;    // [DPAD] split-norm family: the centre xc_B
    const T *e;     // [DPAD] signs of the smooth non-convex family (0 past d)
    const T *ga;    // [DPAD] shift a of g = |x-a|^2/2
    const T *gs2;   // [DPAD] sigma^2 of g = sum x^2/(2 sigma^2)
    const T *gis2;  // [DPAD] 1/sigma^2
    // linear-quadratic family: d rows of ldm (d rounded up to 8, zero padded)
    // values each, all read as M[j*ldm + i]:
    int ldm;
    const T *At;    // At[j*ldm + i] = A[i][j]   (for A gamma)
    const T *A;     // A[j*ldm + i]  = A[j][i]   (for A^T p)
    const T *Cm;    // Cm[j*ldm + i] = (B B^T)[j][i], symmetric
    // The one-thread-per-pair kernels of the smooth non-convex family
    // (hj_r1.cuh) read the per-component vectors as values carried in the
    // kernel's parameters: w, the signs e, w e, and the Hopf data's
    // g*(p) = sum_i p_i (g2_i p_i / 2 + ga_i) + rcst; all zero past d.
    float rw[R1_MAXD], re[R1_MAXD], rew[R1_MAXD], rg2[R1_MAXD], rga[R1_MAXD], rcst;
};

// Solver constants on the device.
struct SolverDev {
    int quad, grad, max_iters, halving_period, adapt, max_trials, max_rounds, guess_dist, kahan, n_default;
    int ck_interval;  // adjoint checkpoint interval K (0: automatic)
    int coarse_div;   // > 1: coarse-to-fine descent (gradient forms)
    double fd_h, step, eps, grow, shrink, step_max, cert_tol, coarse_eps;
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
// and the fast sine/cosine/exponential (|<w,gamma>| stays O(1) in these
// problems, and the bump's exponent is <= 0); fp64 uses the library routines.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsq(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsq(double q) { return rsqrt(q); }
__device__ __forceinline__ void sin_cos(float u, float *s, float *c) { __sincosf(u, s, c); }
__device__ __forceinline__ void sin_cos(double u, double *s, double *c) { sincos(u, s, c); }
__device__ __forceinline__ float exp_(float x) { return __expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
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
// Per-thread copies of the per-component parameters the field needs (the
// initial-data parameters are read from memory at the terminal term).
// ---------------------------------------------------------------------------
// The linear-quadratic family also keeps its matrices' addresses and a
// per-group shared-memory scratch of 2 C tpp values, through which a group
// exchanges the vectors its matrix-vector products need.
template <typename T, int C>
struct TP {
    T w[C], e[C];
    T wb[C], ma[C];  // split-norm family: centre xc_B, and 1 on block A's components
    T m1[C], m2[C];  // 1 on the first / second coordinate (Evans-type family)
    T kap, mu, al_a, al_b, beta, gamma0;
    T r_c, r_d, omega;  // linear game: a(s) = r_c - r_d (1 + beta sin(omega s))
    mutable T st;       // PDE time s = t - tau of the stage being evaluated (set by the integrator)
    bool has_a, has_b;
    const T *At, *A, *Cm;
    T *sh;
    int d, ldm;
    __device__ void load(const ProbDev<T> &P, const Grp &g)
    {
        kap = P.kappa;
        mu = P.mu;
        al_a = P.alpha_a;
        al_b = P.alpha_b;
        beta = P.beta;
        gamma0 = P.gamma0;
        r_c = P.r_c;
        r_d = P.r_d;
        omega = P.omega;
        st = 0;
        has_a = P.ksplit > 0;
        has_b = P.ksplit < P.d;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            int i = g.lane + k * g.tpp;
            w[k] = P.w[i];
            e[k] = P.e[i];
            wb[k] = P.wb ? P.wb[i] : (T)0;
            ma[k] = (i < P.ksplit) ? (T)1 : (T)0;
            m1[k] = (i == 0) ? (T)1 : (T)0;
            m2[k] = (i == 1) ? (T)1 : (T)0;
        }
        At = P.At;
        A = P.A;
        Cm = P.Cm;
        d = P.d;
        ldm = P.ldm;
        sh = nullptr;
    }
};

// Shared scratch of the linear-quadratic family: 5 C values per thread (two
// staged input vectors and three product vectors of the group).
template <typename T, int C, int FAM>
struct LqScratch {
    static constexpr int N = (FAM == HJ_FAM_LINEAR_QUAD) ? 5 * C : 1;
};

// ---------------------------------------------------------------------------
// Families.  Each family splits its work at a stage input Z = (gamma, p):
//   prep()     the quantities that need reductions or special functions
//              (dot products, sin/cos, rsqrt), gathered in an FI record;
//   field_fi() dZ/dtau = (-dH/dp, +dH/dx) and the running cost L
//              (Lax: <p, dH/dp> - H;  Hopf: H - <dH/dx, gamma>) from FI;
//   vjp_fi()   for weights (ag, ap) on the state rows and b on the cost row,
//              rg = ag.d(-H_p)/dgamma + ap.d(H_x)/dgamma + b dL/dgamma and
//              the same in p, from FI (one reduction round).
// The adjoint reuses the FI of a stage for its vector-Jacobian product.
// Speed c(gamma) = 1 + sin(u)/2, u = <w, gamma>, c' = cos(u)/2, c'' = -sin(u)/2.
// ---------------------------------------------------------------------------
// Elementwise vector operations over a lane's C components.  binary32 with
// C even runs them as packed FP32x2 pairs (__ffma2_rn, __fmul2_rn,
// __fadd2_rn: per component the rounding of the scalar fma, multiply and add
// they replace); everything else, and callers that pass PACK = false, in
// scalars.  (The linear-quadratic family's kernels keep scalars: their
// register pressure is already high, and packing added spills that made the
// d=100 descent slower, measured.)
template <typename T, int C, bool PACK = true>
struct Vec {
    static constexpr bool packed = PACK && (sizeof(T) == 4) && (C % 2 == 0);
    // out = a x + y
    __device__ static __forceinline__ void axpy(T a, const T *x, const T *y, T *out)
    {
        if constexpr (packed) {
            const float2 a2 = make_float2(a, a);
#pragma unroll
            for (int j = 0; j < C / 2; ++j) {
                const float2 r = __ffma2_rn(a2, make_float2(x[2 * j], x[2 * j + 1]), make_float2(y[2 * j], y[2 * j + 1]));
                out[2 * j] = r.x;
                out[2 * j + 1] = r.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) out[k] = fma(a, x[k], y[k]);
        }
    }
    // out = a x + b y (b y rounded first)
    __device__ static __forceinline__ void axpby(T a, const T *x, T b, const T *y, T *out)
    {
        if constexpr (packed) {
            const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
            for (int j = 0; j < C / 2; ++j) {
                const float2 by = __fmul2_rn(b2, make_float2(y[2 * j], y[2 * j + 1]));
                const float2 r = __ffma2_rn(a2, make_float2(x[2 * j], x[2 * j + 1]), by);
                out[2 * j] = r.x;
                out[2 * j + 1] = r.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) out[k] = fma(a, x[k], b * y[k]);
        }
    }
    // out = a x
    __device__ static __forceinline__ void scale(T a, const T *x, T *out)
    {
        if constexpr (packed) {
            const float2 a2 = make_float2(a, a);
#pragma unroll
            for (int j = 0; j < C / 2; ++j) {
                const float2 r = __fmul2_rn(a2, make_float2(x[2 * j], x[2 * j + 1]));
                out[2 * j] = r.x;
                out[2 * j + 1] = r.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) out[k] = a * x[k];
        }
    }
    // out = x + y
    __device__ static __forceinline__ void add(const T *x, const T *y, T *out)
    {
        if constexpr (packed) {
#pragma unroll
            for (int j = 0; j < C / 2; ++j) {
                const float2 r = __fadd2_rn(make_float2(x[2 * j], x[2 * j + 1]), make_float2(y[2 * j], y[2 * j + 1]));
                out[2 * j] = r.x;
                out[2 * j + 1] = r.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) out[k] = x[k] + y[k];
        }
    }
};

template <typename T, int C, int FAM, int PR>
struct Family;

// H = |p|^2/2: dZ/dtau = (-p, 0), L = |p|^2/2 for both principles.
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_QUAD_ISO, PR> {
    struct FI {
        T pp;
        T p[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &, T, const T *, const T *p, FI &f)
    {
        T pp = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            f.p[k] = p[k];
            pp = fma(p[k], p[k], pp);
        }
        f.pp = gsum(g, pp);
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &, const FI &f, T, T *dg, T *dp, T &L)
    {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -f.p[k];
            dp[k] = 0;
        }
        L = (T)0.5 * f.pp;
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &, const TP<T, C> &, const FI &f, T, const T *ag,
                                                  const T *, T b, T *rg, T *rp)
    {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = 0;
            rp[k] = fma(b, f.p[k], -ag[k]);
        }
    }
};

// H = c^2 |p|^2/2: dZ/dtau = (-c^2 p, c c' |p|^2 w),
// L_Lax = c^2|p|^2/2, L_Hopf = c^2|p|^2/2 - c c' |p|^2 u.
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_SPEED_QUAD, PR> {
    struct FI {
        T u, pp, c, c1, c2;
        T p[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &tp, T, const T *gam, const T *p, FI &f)
    {
        T u = 0, pp = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            u = fma(tp.w[k], gam[k], u);
            pp = fma(p[k], p[k], pp);
            f.p[k] = p[k];
        }
        gsum2(g, u, pp);
        T su, cu;
        sin_cos(u, &su, &cu);
        f.u = u;
        f.pp = pp;
        f.c = fma((T)0.5, su, (T)1);
        f.c1 = (T)0.5 * cu;
        f.c2 = (T)-0.5 * su;
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &tp, const FI &f, T, T *dg, T *dp, T &L)
    {
        const T cc = f.c * f.c, fx = f.c * f.c1 * f.pp;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -cc * f.p[k];
            dp[k] = fx * tp.w[k];
        }
        L = (T)0.5 * cc * f.pp;
        if (PR == HJ_HOPF) L -= fx * f.u;
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &g, const TP<T, C> &tp, const FI &f, T, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        T A = 0, Bw = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            A = fma(ag[k], f.p[k], A);
            Bw = fma(ap[k], tp.w[k], Bw);
        }
        gsum2(g, A, Bw);
        const T c = f.c, c1 = f.c1;
        const T q = fma(c1, c1, c * f.c2);  // d(c c')/du
        T dEdu = (T)-2 * c * c1 * A + q * f.pp * Bw;
        T dLp;
        if (PR == HJ_LAX) {
            dEdu += b * c * c1 * f.pp;
            dLp = c * c;
        } else {
            dEdu -= b * q * f.pp * f.u;
            dLp = c * c - (T)2 * c * c1 * f.u;
        }
        const T kp = (T)2 * c * c1 * Bw + b * dLp;
        const T mc2 = -c * c;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = dEdu * tp.w[k];
            rp[k] = fma(mc2, ag[k], kp * f.p[k]);
        }
    }
};

// Split norm: H = c_A(gamma) n_A + c_B(gamma) n_B over the coordinate blocks
// A = [0, ksplit), B = [ksplit, d), with n_b = sqrt(|p_b|^2 + eps) (0 for an
// empty block), c_b = alpha_b (1 + kappa exp(-mu |y_b|^2)), y_b = gamma - xc_b,
// grad c_b = k_b y_b, k_b = -2 mu alpha_b kappa exp(-mu |y_b|^2), and m_i the
// block of component i:
// dZ/dtau = (-c_{m_i} p_i / n_{m_i}, sum_b n_b k_b y_b),
// L_Lax = -eps sum_b c_b / n_b,  L_Hopf = sum_b n_b (c_b - k_b <y_b, gamma>).
// With grad k_b = -2 mu k_b y_b and dn_b/dp_i = p_i / n_b on block b the
// vector-Jacobian product is, summed over the blocks,
//   rg = (-k_b <ag,p>_b / n_b - 2 mu n_b k_b <ap,y_b>) y_b + n_b k_b ap
//        + b (Lax: -eps k_b / n_b y_b;  Hopf: n_b k_b (2 mu <y_b,gamma> y_b - gamma)),
// and on block b's components
//   rp = -c_b / n_b ag + (c_b <ag,p>_b / n_b^3 + k_b <ap,y_b> / n_b) p
//        + b (Lax: c_b eps / n_b^3;  Hopf: (c_b - k_b <y_b,gamma>) / n_b) p.
// An empty block has n_b = 1/n_b = 0 and drops out.  The bump norm of Sec. 6,
// Example 3 (H = +-c(x)|p|) is the case ksplit = d, alpha_A = +-1.
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_SPLIT_NORM, PR> {
    struct FI {
        T c[2], k[2], n[2], ni[2], yg[2];
        T ya[C], yb[C], p[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p,
                                                FI &f)
    {
        T ra = 0, rb = 0, pa = 0, pb = 0, ga = 0, gb = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const T ya = gam[k] - tp.w[k], yb = gam[k] - tp.wb[k], pp = p[k] * p[k];
            f.ya[k] = ya;
            f.yb[k] = yb;
            f.p[k] = p[k];
            ra = fma(ya, ya, ra);
            rb = fma(yb, yb, rb);
            pa = fma(tp.ma[k], pp, pa);
            pb = fma((T)1 - tp.ma[k], pp, pb);
            if (PR == HJ_HOPF) {
                ga = fma(ya, gam[k], ga);
                gb = fma(yb, gam[k], gb);
            }
        }
        gsum4(g, ra, rb, pa, pb);
        if (PR == HJ_HOPF) gsum2(g, ga, gb);
        const T ea = exp_(-tp.mu * ra), eb = exp_(-tp.mu * rb);
        f.c[0] = tp.al_a * fma(tp.kap, ea, (T)1);
        f.c[1] = tp.al_b * fma(tp.kap, eb, (T)1);
        f.k[0] = (T)-2 * tp.mu * tp.al_a * tp.kap * ea;
        f.k[1] = (T)-2 * tp.mu * tp.al_b * tp.kap * eb;
        const T qa = pa + eps, qb = pb + eps;
        f.ni[0] = tp.has_a ? rsq(qa) : (T)0;
        f.ni[1] = tp.has_b ? rsq(qb) : (T)0;
        f.n[0] = qa * f.ni[0];
        f.n[1] = qb * f.ni[1];
        f.yg[0] = ga;
        f.yg[1] = gb;
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &tp, const FI &f, T eps, T *dg, T *dp, T &L)
    {
        const T sa = f.c[0] * f.ni[0], sb = f.c[1] * f.ni[1];
        const T fa = f.n[0] * f.k[0], fb = f.n[1] * f.k[1];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -fma(tp.ma[k], sa - sb, sb) * f.p[k];
            dp[k] = fma(fa, f.ya[k], fb * f.yb[k]);
        }
        if (PR == HJ_LAX) L = -eps * (sa + sb);
        else L = f.n[0] * (f.c[0] - f.k[0] * f.yg[0]) + f.n[1] * (f.c[1] - f.k[1] * f.yg[1]);
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &g, const TP<T, C> &tp, const FI &f, T eps, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        T Aa = 0, Ab = 0, Ba = 0, Bb = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const T agp = ag[k] * f.p[k];
            Aa = fma(tp.ma[k], agp, Aa);
            Ab = fma((T)1 - tp.ma[k], agp, Ab);
            Ba = fma(ap[k], f.ya[k], Ba);
            Bb = fma(ap[k], f.yb[k], Bb);
        }
        gsum4(g, Aa, Ab, Ba, Bb);
        const T A_[2] = {Aa, Ab}, B_[2] = {Ba, Bb};
        const T mu = tp.mu;
        T cy[2], nk[2], cag[2], cp[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const T n = f.n[q], ni = f.ni[q], c = f.c[q], kk = f.k[q];
            const T ni3 = ni * ni * ni;
            nk[q] = n * kk;
            cy[q] = -kk * A_[q] * ni - (T)2 * mu * nk[q] * B_[q];
            cag[q] = -c * ni;
            cp[q] = c * A_[q] * ni3 + kk * B_[q] * ni;
            if (PR == HJ_LAX) {
                cy[q] -= b * eps * kk * ni;
                cp[q] += b * c * eps * ni3;
            } else {
                cy[q] += b * (T)2 * mu * nk[q] * f.yg[q];
                cp[q] += b * (c - kk * f.yg[q]) * ni;
            }
        }
        const T nkt = nk[0] + nk[1];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T r = fma(cy[0], f.ya[k], fma(cy[1], f.yb[k], nkt * ap[k]));
            if (PR == HJ_HOPF) r = fma(-b * nkt, f.ya[k] + tp.w[k], r);  // gamma = y_A + xc_A
            rg[k] = r;
            const T m = tp.ma[k];
            rp[k] = fma(fma(m, cag[0] - cag[1], cag[1]), ag[k], fma(m, cp[0] - cp[1], cp[1]) * f.p[k]);
        }
    }
};

// Harmonic oscillator H = S (|p|^2 + |gamma|^2)/2, S = alpha_a (Sec. 6,
// Example 2): dZ/dtau = (-S p, S gamma), L = S (|p|^2 - |gamma|^2)/2 for both
// principles; rg = S ap - b S gamma, rp = -S ag + b S p.
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_HARMONIC, PR> {
    struct FI {
        T pp, gg;
        T g[C], p[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &, T, const T *gam, const T *p, FI &f)
    {
        T pp = 0, gg = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            f.g[k] = gam[k];
            f.p[k] = p[k];
            pp = fma(p[k], p[k], pp);
            gg = fma(gam[k], gam[k], gg);
        }
        gsum2(g, pp, gg);
        f.pp = pp;
        f.gg = gg;
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &tp, const FI &f, T, T *dg, T *dp, T &L)
    {
        const T S = tp.al_a;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -S * f.p[k];
            dp[k] = S * f.g[k];
        }
        L = (T)0.5 * S * (f.pp - f.gg);
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &, const TP<T, C> &tp, const FI &f, T, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        const T S = tp.al_a, bS = b * tp.al_a;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = fma(S, ap[k], -bS * f.g[k]);
            rp[k] = fma(-S, ag[k], bS * f.p[k]);
        }
    }
};

// Evans-type non-convex H = -c(gamma) p_1 + beta s_2 - n - gamma0 (Sec. 6,
// Example 4) with s_2 = sqrt(p_2^2 + eps), n = sqrt(|p|^2 + eps),
// c = alpha (1 + kappa exp(-mu |y|^2)), y = gamma - xc, grad c = k y,
// k = -2 mu alpha kappa exp(-mu |y|^2), grad k = -2 mu k y, e_1, e_2 the
// first two coordinates:
// dZ/dtau = (c e_1 - beta p_2/s_2 e_2 + p/n, -p_1 k y),
// L_Lax = gamma0 - beta eps/s_2 + eps/n,  L_Hopf = H + p_1 k <y, gamma>;
//   rg = (<ag,e_1> k + 2 mu p_1 k <ap,y>) y - p_1 k ap
//        + b (Hopf: p_1 k (gamma - 2 mu <y,gamma> y)),
//   rp = ag/n - <ag,p> p/n^3 - k <ap,y> e_1 - beta eps/s_2^3 <ag,e_2> e_2
//        + b (Lax: -eps p/n^3 + beta eps p_2/s_2^3 e_2;
//             Hopf: -p/n + (-c + k <y,gamma>) e_1 + beta p_2/s_2 e_2).
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_EVANS, PR> {
    struct FI {
        T c, k, n, ni, s2, s2i, p1, p2, yg;
        T y[C], p[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p,
                                                FI &f)
    {
        T rr = 0, pp = 0, p1 = 0, p2 = 0, yg = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const T y = gam[k] - tp.w[k];
            f.y[k] = y;
            f.p[k] = p[k];
            rr = fma(y, y, rr);
            pp = fma(p[k], p[k], pp);
            p1 = fma(tp.m1[k], p[k], p1);
            p2 = fma(tp.m2[k], p[k], p2);
            if (PR == HJ_HOPF) yg = fma(y, gam[k], yg);
        }
        gsum4(g, rr, pp, p1, p2);
        if (PR == HJ_HOPF) yg = gsum(g, yg);
        const T e = exp_(-tp.mu * rr);
        f.c = tp.al_a * fma(tp.kap, e, (T)1);
        f.k = (T)-2 * tp.mu * tp.al_a * tp.kap * e;
        const T q = pp + eps, q2 = fma(p2, p2, eps);
        f.ni = rsq(q);
        f.n = q * f.ni;
        f.s2i = rsq(q2);
        f.s2 = q2 * f.s2i;
        f.p1 = p1;
        f.p2 = p2;
        f.yg = yg;
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &tp, const FI &f, T eps, T *dg, T *dp, T &L)
    {
        const T a2 = -tp.beta * f.p2 * f.s2i, fp = -f.p1 * f.k;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = fma(tp.m1[k], f.c, fma(tp.m2[k], a2, f.p[k] * f.ni));
            dp[k] = fp * f.y[k];
        }
        if (PR == HJ_LAX) {
            L = tp.gamma0 - tp.beta * eps * f.s2i + eps * f.ni;
        } else {
            const T H = -f.c * f.p1 + tp.beta * f.s2 - f.n - tp.gamma0;
            L = fma(f.p1 * f.k, f.yg, H);
        }
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &g, const TP<T, C> &tp, const FI &f, T eps, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        T A = 0, By = 0, ag1 = 0, ag2 = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            A = fma(ag[k], f.p[k], A);
            By = fma(ap[k], f.y[k], By);
            ag1 = fma(tp.m1[k], ag[k], ag1);
            ag2 = fma(tp.m2[k], ag[k], ag2);
        }
        gsum4(g, A, By, ag1, ag2);
        const T kk = f.k, mu = tp.mu, ni = f.ni, ni3 = ni * ni * ni, s2i3 = f.s2i * f.s2i * f.s2i;
        const T p1k = f.p1 * kk;
        T cy = fma(ag1, kk, (T)2 * mu * p1k * By);
        T cgam = 0;
        T cp = -A * ni3;                              // on p
        T c1 = -kk * By;                              // on e_1
        T c2 = -tp.beta * eps * s2i3 * ag2;           // on e_2
        if (PR == HJ_LAX) {
            cp -= b * eps * ni3;
            c2 += b * tp.beta * eps * f.p2 * s2i3;
        } else {
            cy -= b * (T)2 * mu * p1k * f.yg;
            cgam = b * p1k;
            cp -= b * ni;
            c1 += b * (-f.c + kk * f.yg);
            c2 += b * tp.beta * f.p2 * f.s2i;
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T r = fma(cy, f.y[k], -p1k * ap[k]);
            if (PR == HJ_HOPF) r = fma(cgam, f.y[k] + tp.w[k], r);  // gamma = y + xc
            rg[k] = r;
            rp[k] = fma(ag[k], ni, fma(cp, f.p[k], fma(tp.m1[k], c1, tp.m2[k] * c2)));
        }
    }
};

// Linear differential game (Sec. 3.4, Example 3) with a diagonal drift
// M = diag(m) (m in w) and ball-shaped control sets:
// H(gamma, p, s) = -<M gamma, p> + a(s) n, a(s) = r_c - r_d (1 + beta sin(omega s)),
// n = sqrt(|p|^2 + eps), s the PDE time of the stage (tp.st):
// dZ/dtau = (M gamma - a p/n, -M p), L_Lax = -a eps/n, L_Hopf = a n;
//   rg = m ag,  rp = -a (ag/n - <ag,p> p/n^3) - m ap + b (Lax: a eps p/n^3; Hopf: a p/n).
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_LINEAR_GAME, PR> {
    struct FI {
        T a, n, ni;
        T g[C], p[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p,
                                                FI &f)
    {
        T pp = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            f.g[k] = gam[k];
            f.p[k] = p[k];
            pp = fma(p[k], p[k], pp);
        }
        pp = gsum(g, pp);
        T sn, cs;
        sin_cos(tp.omega * tp.st, &sn, &cs);
        f.a = tp.r_c - tp.r_d * fma(tp.beta, sn, (T)1);
        const T q = pp + eps;
        f.ni = rsq(q);
        f.n = q * f.ni;
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &tp, const FI &f, T eps, T *dg, T *dp, T &L)
    {
        const T an = f.a * f.ni;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = fma(tp.w[k], f.g[k], -an * f.p[k]);
            dp[k] = -tp.w[k] * f.p[k];
        }
        L = (PR == HJ_LAX) ? -eps * an : f.a * f.n;
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &g, const TP<T, C> &tp, const FI &f, T eps, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        T A = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) A = fma(ag[k], f.p[k], A);
        A = gsum(g, A);
        const T ni = f.ni, ni3 = ni * ni * ni;
        T cp = f.a * A * ni3 + ((PR == HJ_LAX) ? b * f.a * eps * ni3 : b * f.a * ni);
        const T cag = -f.a * ni;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = tp.w[k] * ag[k];
            rp[k] = fma(cag, ag[k], fma(cp, f.p[k], -tp.w[k] * ap[k]));
        }
    }
};

// H = c Phi(p), Phi = sum_i e_i s(p_i), s = sqrt(p^2 + eps):
// dZ/dtau = (-c Phi', Phi c' w), Phi'_i = e_i p_i / s_i, Phi''_i = e_i eps / s_i^3,
// L_Lax = c (<p, Phi'> - Phi) = -c eps sum_i e_i / s_i, L_Hopf = Phi (c - c' u).
// FI keeps er_i = e_i / s_i and Phi'_i = er_i p_i (e_i^2 = 1 on real
// components, so Phi''_i = eps er_i^3; both are 0 on padding).
template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_SMOOTH_NONCONVEX, PR> {
    struct FI {
        T u, c, c1, c2, phi, lax;
        T er[C], dphi[C];
        T pl[PR == HJ_LAX ? C : 1];  // p_i, kept for the Lax running cost only
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p,
                                                FI &f)
    {
        T u = 0, phi = 0, lax = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            u = fma(tp.w[k], gam[k], u);
            const T q = fma(p[k], p[k], eps);
            const T er = tp.e[k] * rsq(q);
            f.er[k] = er;
            f.dphi[k] = er * p[k];
            if constexpr (PR == HJ_LAX) f.pl[k] = p[k];
            phi = fma(er, q, phi);  // e s
            if (PR == HJ_LAX) lax += er;
        }
        if (PR == HJ_LAX) gsum3(g, u, phi, lax);
        else gsum2(g, u, phi);
        T su, cu;
        sin_cos(u, &su, &cu);
        f.u = u;
        f.phi = phi;
        f.lax = lax;
        f.c = fma((T)0.5, su, (T)1);
        f.c1 = (T)0.5 * cu;
        f.c2 = (T)-0.5 * su;
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &tp, const FI &f, T eps, T *dg, T *dp, T &L)
    {
        const T fx = f.phi * f.c1, mc = -f.c;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = mc * f.dphi[k];
            dp[k] = fx * tp.w[k];
        }
        if (PR == HJ_LAX) L = mc * eps * f.lax;
        else L = f.phi * (f.c - f.c1 * f.u);
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &g, const TP<T, C> &tp, const FI &f, T eps, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        T A = 0, Bw = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            A = fma(ag[k], f.dphi[k], A);
            Bw = fma(ap[k], tp.w[k], Bw);
        }
        gsum2(g, A, Bw);
        const T c = f.c, c1 = f.c1;
        T dEdu = -c1 * A + f.phi * f.c2 * Bw;
        T kd;  // coefficient of Phi'_i in rp
        if (PR == HJ_LAX) {
            // <p, Phi'> - Phi = -eps sum e/s
            dEdu -= b * c1 * eps * f.lax;
            kd = c1 * Bw;
        } else {
            dEdu -= b * f.phi * f.c2 * f.u;
            kd = c1 * Bw + b * (c - c1 * f.u);
        }
        // rp_i = Phi''_i (-c ag_i [+ b c p_i for Lax]) + kd Phi'_i, Phi''_i = eps er_i^3
        const T ce = c * eps;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T a = -ag[k];
            if constexpr (PR == HJ_LAX) a = fma(b, f.pl[k], a);
            const T er = f.er[k];
            rg[k] = dEdu * tp.w[k];
            rp[k] = fma(ce * a * er * er, er, kd * f.dphi[k]);
        }
    }
};

// H = <A gamma, p> + p^T (B B^T) p / 2 (Cm = B B^T):
// dZ/dtau = (-(A gamma + Cm p), A^T p), L = p^T Cm p / 2 for both principles
// (<p, H_p> - H and H - <H_x, gamma> coincide).  The field is linear, so the
// vector-Jacobian product needs only Cm p of the stage (for the cost row):
// rg = -A^T ag,  rp = A ap - Cm ag + b Cm p.
// Each product sum_j M[j][i] u_j runs over j with u staged in the group's
// shared scratch (broadcast reads); for the sums, lane l of the group takes
// the C consecutive rows i = C l .. C l + C - 1, so each matrix row costs one
// vector load per lane, and the sums go back to the owner layout
// (i = l + k tpp) through the scratch.
template <typename T, int C>
__device__ __forceinline__ void lq_stage2(const Grp &g, T *sh, const T *a, const T *b)
{
    const int n = C * g.tpp;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        sh[g.lane + k * g.tpp] = a[k];
        sh[n + g.lane + k * g.tpp] = b[k];
    }
    __syncwarp(g.mask);
}

// C consecutive values at p (aligned to their size, up to 16 bytes per load).
template <typename T, int C>
__device__ __forceinline__ void ld_row(const T *p, T *v)
{
    constexpr int bytes = C * (int)sizeof(T);
    if constexpr (bytes % 16 == 0) {
#pragma unroll
        for (int q = 0; q < bytes / 16; ++q) {
            const float4 f = __ldg((const float4 *)p + q);
            const T *t = (const T *)&f;
#pragma unroll
            for (int k = 0; k < 16 / (int)sizeof(T); ++k) v[q * (16 / (int)sizeof(T)) + k] = t[k];
        }
    } else if constexpr (bytes == 8) {
        const float2 f = __ldg((const float2 *)p);
        const T *t = (const T *)&f;
#pragma unroll
        for (int k = 0; k < C; ++k) v[k] = t[k];
    } else {
#pragma unroll
        for (int k = 0; k < C; ++k) v[k] = __ldg(p + k);
    }
}

// Writes the three row-blocked sums (lane l holds rows C l + k) to the
// scratch and reads them back in the owner layout.
template <typename T, int C>
__device__ __forceinline__ void lq_regather(const Grp &g, T *sh, const T *s0, const T *s1, const T *s2, T *o0, T *o1,
                                            T *o2)
{
    const int n = C * g.tpp, i0 = C * g.lane;
    T *r = sh + 2 * n;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        r[i0 + k] = s0[k];
        r[n + i0 + k] = s1[k];
        r[2 * n + i0 + k] = s2[k];
    }
    __syncwarp(g.mask);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int i = g.lane + k * g.tpp;
        o0[k] = r[i];
        o1[k] = r[n + i];
        o2[k] = r[2 * n + i];
    }
    __syncwarp(g.mask);
}

template <typename T, int C, int PR>
struct Family<T, C, HJ_FAM_LINEAR_QUAD, PR> {
    struct FI {
        T L;
        T ax[C], cp[C], atp[C];
    };
    __device__ static __forceinline__ void prep(const Grp &g, const TP<T, C> &tp, T, const T *gam, const T *p, FI &f)
    {
        T *sh = tp.sh;
        const int n = C * g.tpp, d = tp.d, ldm = tp.ldm, i0 = C * g.lane;
        lq_stage2<T, C>(g, sh, gam, p);
        T ax[C], cp[C], atp[C];
#pragma unroll
        for (int k = 0; k < C; ++k) ax[k] = cp[k] = atp[k] = 0;
        if (i0 < d) {
            for (int j = 0; j < d; ++j) {
                const T gj = sh[j], pj = sh[n + j];
                T m1[C], m2[C], m3[C];
                ld_row<T, C>(tp.At + (size_t)j * ldm + i0, m1);
                ld_row<T, C>(tp.Cm + (size_t)j * ldm + i0, m2);
                ld_row<T, C>(tp.A + (size_t)j * ldm + i0, m3);
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    ax[k] = fma(m1[k], gj, ax[k]);
                    cp[k] = fma(m2[k], pj, cp[k]);
                    atp[k] = fma(m3[k], pj, atp[k]);
                }
            }
        }
        lq_regather<T, C>(g, sh, ax, cp, atp, f.ax, f.cp, f.atp);
        T pcp = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) pcp = fma(p[k], f.cp[k], pcp);
        f.L = (T)0.5 * gsum(g, pcp);
    }
    __device__ static __forceinline__ void field_fi(const TP<T, C> &, const FI &f, T, T *dg, T *dp, T &L)
    {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dg[k] = -(f.ax[k] + f.cp[k]);
            dp[k] = f.atp[k];
        }
        L = f.L;
    }
    __device__ static __forceinline__ void vjp_fi(const Grp &g, const TP<T, C> &tp, const FI &f, T, const T *ag,
                                                  const T *ap, T b, T *rg, T *rp)
    {
        T *sh = tp.sh;
        const int n = C * g.tpp, d = tp.d, ldm = tp.ldm, i0 = C * g.lane;
        lq_stage2<T, C>(g, sh, ag, ap);
        T sg[C], sa[C], sc[C];
#pragma unroll
        for (int k = 0; k < C; ++k) sg[k] = sa[k] = sc[k] = 0;
        if (i0 < d) {
            for (int j = 0; j < d; ++j) {
                const T agj = sh[j], apj = sh[n + j];
                T m1[C], m2[C], m3[C];
                ld_row<T, C>(tp.A + (size_t)j * ldm + i0, m1);
                ld_row<T, C>(tp.At + (size_t)j * ldm + i0, m2);
                ld_row<T, C>(tp.Cm + (size_t)j * ldm + i0, m3);
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    sg[k] = fma(m1[k], agj, sg[k]);  // (A^T ag)_i
                    sa[k] = fma(m2[k], apj, sa[k]);  // (A ap)_i
                    sc[k] = fma(m3[k], agj, sc[k]);  // (Cm ag)_i
                }
            }
        }
        T og[C], oa[C], oc[C];
        lq_regather<T, C>(g, sh, sg, sa, sc, og, oa, oc);
#pragma unroll
        for (int k = 0; k < C; ++k) {
            rg[k] = -og[k];
            rp[k] = fma(b, f.cp[k], oa[k] - oc[k]);
        }
    }
};

// Whole-stage helpers.
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void field(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p, T *dg,
                                      T *dp, T &L)
{
    typename Family<T, C, FAM, PR>::FI f;
    Family<T, C, FAM, PR>::prep(g, tp, eps, gam, p, f);
    Family<T, C, FAM, PR>::field_fi(tp, f, eps, dg, dp, L);
}
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void vjp(const Grp &g, const TP<T, C> &tp, T eps, const T *gam, const T *p, const T *ag,
                                    const T *ap, T b, T *rg, T *rp)
{
    typename Family<T, C, FAM, PR>::FI f;
    Family<T, C, FAM, PR>::prep(g, tp, eps, gam, p, f);
    Family<T, C, FAM, PR>::vjp_fi(g, tp, f, eps, ag, ap, b, rg, rp);
}

// ---------------------------------------------------------------------------
// Initial data: terminal value, its gradient (adjoint seed) and the
// certificate residual.
//   Lax  term g(gamma0), seed (grad g(gamma0), 0)
//   Hopf term g*(p0) - <x, v>, seed (0, grad g*(p0))
// ---------------------------------------------------------------------------
// Rosenbrock data (Sec. 6, Example 2; d = 2, Lax only):
// g = 4e-4 (-100 + (1 - x_1)^2 + 100 (1 + x_2 - x_1^2)^2).  Returns g; gr gets
// grad g on each lane's components (0 past the first two).
template <typename T, int C>
__device__ __forceinline__ T rosenbrock(const Grp &g, const T *gam, T *gr)
{
    T x1 = 0, x2 = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int i = g.lane + k * g.tpp;
        if (i == 0) x1 = gam[k];
        if (i == 1) x2 = gam[k];
    }
    gsum2(g, x1, x2);
    const T a = (T)1 - x1, b = (T)1 + x2 - x1 * x1, s = (T)4e-4;
    const T d1 = s * ((T)-2 * a - (T)400 * b * x1), d2 = s * (T)200 * b;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int i = g.lane + k * g.tpp;
        gr[k] = (i == 0) ? d1 : (i == 1) ? d2 : (T)0;
    }
    return s * ((T)-100 + a * a + (T)100 * b * b);
}

template <typename T, int C, int PR>
__device__ __forceinline__ T terminal(const Grp &g, const ProbDev<T> &P, const T *x, const T *v, const T *gam,
                                      const T *p, T *sg, T *sp)
{
    if (PR == HJ_LAX && P.g_kind == HJ_G_ROSENBROCK) {
        T gr[C];
        const T val = rosenbrock<T, C>(g, gam, gr);
        if (sg) {
#pragma unroll
            for (int k = 0; k < C; ++k) { sg[k] = gr[k]; sp[k] = 0; }
        }
        return val;
    }
    T acc = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int i = g.lane + k * g.tpp;
        if (PR == HJ_LAX) {
            T gr = (P.g_kind == HJ_G_QUAD_SHIFT) ? gam[k] - __ldg(P.ga + i) : gam[k] * __ldg(P.gis2 + i);
            acc = fma((T)0.5 * gr, (P.g_kind == HJ_G_QUAD_SHIFT) ? gr : gam[k], acc);
            if (sg) { sg[k] = gr; sp[k] = 0; }
        } else {
            T gr, val;
            if (P.g_kind == HJ_G_QUAD_SHIFT) {
                const T a = __ldg(P.ga + i);
                gr = p[k] + a;
                val = p[k] * fma((T)0.5, p[k], a);
            } else {
                gr = __ldg(P.gs2 + i) * p[k];
                val = (T)0.5 * gr * p[k];
            }
            acc += val - x[k] * v[k];
            if (sg) { sg[k] = 0; sp[k] = gr; }
        }
    }
    acc = gsum(g, acc);
    // the ellipse data's constant: g - 1/2 (Lax), g* + 1/2 (Hopf)
    if (P.g_kind == HJ_G_ELLIPSE) acc += (PR == HJ_LAX) ? (T)-0.5 : (T)0.5;
    return acc;
}

// Relative certificate residual (Sec. 4.3) from (gamma(0), p(0)).
template <typename T, int C, int PR>
__device__ __forceinline__ T cert_residual(const Grp &g, const ProbDev<T> &P, const T *gam, const T *p)
{
    T num = 0, den = 0;
    T rg[C];
    if (PR == HJ_LAX && P.g_kind == HJ_G_ROSENBROCK) rosenbrock<T, C>(g, gam, rg);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int i = g.lane + k * g.tpp;
        T diff, base;
        if (PR == HJ_LAX) {
            T gr = (P.g_kind == HJ_G_QUAD_SHIFT) ? gam[k] - __ldg(P.ga + i) : gam[k] * __ldg(P.gis2 + i);
            if (P.g_kind == HJ_G_ROSENBROCK) gr = rg[k];
            diff = p[k] - gr;
            base = p[k];
        } else {
            T gr = (P.g_kind == HJ_G_QUAD_SHIFT) ? p[k] + __ldg(P.ga + i) : __ldg(P.gs2 + i) * p[k];
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
// Forward integration.  One step of the augmented system: classical RK4, or
// forward Euler when quad carries HJ_ODE_EULER (Sec. 4.2's example solver).
// Q accumulates the running cost (the integrator's own weights on the
// augmented state, or the rectangle node at the new state), with optional
// Kahan compensation.  quad is uniform across a launch, so the branch is too.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void add_q(int kahan, T dQ, T &Q, T &Qc)
{
    if (kahan) {
        T y = dQ - Qc;
        T s = Q + y;
        Qc = (s - Q) - y;
        Q = s;
    } else {
        Q += dQ;
    }
}

// s0 is the PDE time s = t - tau at the start of the step; each stage sets
// tp.st to its own time (only a time-dependent H reads it).
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void rk4_step(const Grp &g, const TP<T, C> &tp, T eps, T h, T s0, int quad, int kahan,
                                         T *gam, T *p, T &Q, T &Qc)
{
    T ag[C], ap[C], zg[C], zp[C], kg[C], kp[C], L, aL;
    const T h2 = (T)0.5 * h;
    tp.st = s0;
    field<T, C, FAM, PR>(g, tp, eps, gam, p, kg, kp, L);
    if (quad & HJ_ODE_EULER) {
        // z_{n+1} = z_n + h f(z_n); the augmented state gains h L(z_n)
#pragma unroll
        for (int k = 0; k < C; ++k) {
            gam[k] = fma(h, kg[k], gam[k]);
            p[k] = fma(h, kp[k], p[k]);
        }
        T dQ = h * L;
        if (quad & HJ_QUAD_RECT) {
            T dg_[C], dp_[C];
            tp.st = s0 - h;
            field<T, C, FAM, PR>(g, tp, eps, gam, p, dg_, dp_, L);
            dQ = h * L;
        }
        add_q(kahan, dQ, Q, Qc);
        return;
    }
    using V = Vec<T, C, FAM != HJ_FAM_LINEAR_QUAD>;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        ag[k] = kg[k];
        ap[k] = kp[k];
    }
    V::axpy(h2, kg, gam, zg);
    V::axpy(h2, kp, p, zp);
    aL = L;
    tp.st = s0 - h2;
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
    V::axpy((T)2, kg, ag, ag);
    V::axpy((T)2, kp, ap, ap);
    V::axpy(h2, kg, gam, zg);
    V::axpy(h2, kp, p, zp);
    aL = fma((T)2, L, aL);
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
    V::axpy((T)2, kg, ag, ag);
    V::axpy((T)2, kp, ap, ap);
    V::axpy(h, kg, gam, zg);
    V::axpy(h, kp, p, zp);
    aL = fma((T)2, L, aL);
    tp.st = s0 - h;
    field<T, C, FAM, PR>(g, tp, eps, zg, zp, kg, kp, L);
    const T h6 = h / (T)6;
    V::add(ag, kg, ag);
    V::add(ap, kp, ap);
    V::axpy(h6, ag, gam, gam);
    V::axpy(h6, ap, p, p);
    aL += L;
    T dQ;
    if (!(quad & HJ_QUAD_RECT)) {
        dQ = h6 * aL;
    } else {
        T Ln, dg_[C], dp_[C];
        tp.st = s0 - h;
        field<T, C, FAM, PR>(g, tp, eps, gam, p, dg_, dp_, Ln);
        dQ = h * Ln;
    }
    add_q(kahan, dQ, Q, Qc);
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
    if (PR == HJ_LAX && FAM == HJ_FAM_SPLIT_NORM && P.huygens) {
        // F^2: the smallest g over the nodes z_0 .. z_N (first one on ties;
        // group sums are identical on every lane, so the choice is uniform);
        // gam, p return the minimising node for the certificate
        T gb = terminal<T, C, HJ_LAX>(g, P, x, v, gam, p, (T *)nullptr, (T *)nullptr), bg[C], bp[C];
#pragma unroll
        for (int k = 0; k < C; ++k) { bg[k] = gam[k]; bp[k] = p[k]; }
        for (int n = 0; n < N; ++n) {
            rk4_step<T, C, FAM, PR>(g, tp, P.s_eps, h, t - (T)n * h, quad, 0, gam, p, Q, Qc);
            const T gn = terminal<T, C, HJ_LAX>(g, P, x, v, gam, p, (T *)nullptr, (T *)nullptr);
            if (gn < gb) {
                gb = gn;
#pragma unroll
                for (int k = 0; k < C; ++k) { bg[k] = gam[k]; bp[k] = p[k]; }
            }
        }
#pragma unroll
        for (int k = 0; k < C; ++k) { gam[k] = bg[k]; p[k] = bp[k]; }
        return gb;
    }
    for (int n = 0; n < N; ++n) rk4_step<T, C, FAM, PR>(g, tp, P.s_eps, h, t - (T)n * h, quad, kahan, gam, p, Q, Qc);
    return terminal<T, C, PR>(g, P, x, v, gam, p, (T *)nullptr, (T *)nullptr) + Q;
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the RK4 map (exact gradient of the discretised
// functional).  Forward: checkpoints of z every K steps, K from
// ck_interval: the caller's fixed interval, or else the smallest K whose
// ceil(N/K) checkpoints plus a K-state segment fit CK_BUDGET bytes per thread
// (K = 1, every state stored, at d = 20 and N = 64; K = ceil(sqrt(N)) is the
// choice that minimises that storage, at the price of one extra forward
// pass).  Every K gives the same gradient: the recomputed states repeat the
// forward pass's arithmetic.
// Reverse, segment by segment: recompute the segment's states z_n from its
// checkpoint (stored, 2C values per step), then for each step backward
// rebuild its stage inputs Z1 = z_n, Z2 = z_n + h/2 k1, Z3 = z_n + h/2 k2,
// Z4 = z_n + h k3 and run the adjoint of the step:
//   a4 = J(Z4)^T(h/6 lam, h/6 b)
//   a3 = J(Z3)^T(h/3 lam + h a4, h/3 b)
//   a2 = J(Z2)^T(h/3 lam + h/2 a3, h/3 b)
//   a1 = J(Z1)^T(h/6 lam + h/2 a2, h/6 b)
//   lam += a1 + a2 + a3 + a4
// with b = 1 for the RK4 quadrature (0 for the rectangle rule, whose nodes
// add h grad L(z_{n+1}) to lam directly).  The forward Euler map
// z_{n+1} = z_n + h f(z_n) has the one-stage adjoint
//   lam += J(z_n)^T(h lam, h b).
// The seed lam(tau=t) comes from the terminal term; dF/dv = lam_p(tau=0)
// (minus x for Hopf).
// Per-thread scratch (local memory): ck >= ceil(N/K)*2C, seg >= K*2C values,
// both sized for N <= MAX_N.
// ---------------------------------------------------------------------------
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ void adjoint_step(const Grp &g, const TP<T, C> &tp, T eps, T h, T s0, T b, const T *zg,
                                             const T *zp, T *lg, T *lp)
{
    using Fam = Family<T, C, FAM, PR>;
    typename Fam::FI f1, f2, f3, f4;
    T kg[C], kp[C], sg[C], sp[C], L;
    const T h6 = h / (T)6, h3 = h / (T)3, h2 = (T)0.5 * h;
    // rebuild the stage inputs of the step from z_n, keeping each stage's FI
    // (each prepared at its stage's PDE time, s0, s0 - h/2, s0 - h/2, s0 - h)
    using V = Vec<T, C, FAM != HJ_FAM_LINEAR_QUAD>;
    tp.st = s0;
    Fam::prep(g, tp, eps, zg, zp, f1);
    Fam::field_fi(tp, f1, eps, kg, kp, L);
    V::axpy(h2, kg, zg, sg);
    V::axpy(h2, kp, zp, sp);
    tp.st = s0 - h2;
    Fam::prep(g, tp, eps, sg, sp, f2);
    Fam::field_fi(tp, f2, eps, kg, kp, L);
    V::axpy(h2, kg, zg, sg);
    V::axpy(h2, kp, zp, sp);
    Fam::prep(g, tp, eps, sg, sp, f3);
    Fam::field_fi(tp, f3, eps, kg, kp, L);
    V::axpy(h, kg, zg, sg);
    V::axpy(h, kp, zp, sp);
    tp.st = s0 - h;
    Fam::prep(g, tp, eps, sg, sp, f4);

    T wg[C], wp[C], rg[C], rp[C], sumg[C], sump[C];
    // stage 4
    V::scale(h6, lg, wg);
    V::scale(h6, lp, wp);
    Fam::vjp_fi(g, tp, f4, eps, wg, wp, h6 * b, rg, rp);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        sumg[k] = rg[k];
        sump[k] = rp[k];
    }
    V::axpby(h3, lg, h, rg, wg);
    V::axpby(h3, lp, h, rp, wp);
    // stage 3
    Fam::vjp_fi(g, tp, f3, eps, wg, wp, h3 * b, rg, rp);
    V::add(sumg, rg, sumg);
    V::add(sump, rp, sump);
    V::axpby(h3, lg, h2, rg, wg);
    V::axpby(h3, lp, h2, rp, wp);
    // stage 2
    Fam::vjp_fi(g, tp, f2, eps, wg, wp, h3 * b, rg, rp);
    V::add(sumg, rg, sumg);
    V::add(sump, rp, sump);
    V::axpby(h6, lg, h2, rg, wg);
    V::axpby(h6, lp, h2, rp, wp);
    // stage 1
    Fam::vjp_fi(g, tp, f1, eps, wg, wp, h6 * b, rg, rp);
    V::add(sumg, rg, sumg);
    V::add(sump, rp, sump);
    V::add(lg, sumg, lg);
    V::add(lp, sump, lp);
}

// Checkpoint interval: the given K, or the smallest K whose checkpoint and
// segment storage, (ceil(N/K) + K) states of 2C values, fits CK_BUDGET bytes.
template <typename T, int C>
__device__ __forceinline__ int ck_interval(int N, int fixed)
{
    int K = fixed;
    if (K <= 0) {
        K = 1;
        while (K < MAX_SEG && ((N + K - 1) / K + K) * 2 * C * (int)sizeof(T) > CK_BUDGET) ++K;
    }
    K = max(K, (N + MAX_CK - 1) / MAX_CK);
    return min(K, MAX_SEG);
}

// Gradient of F with respect to v.  Returns F; grad gets dF/dv.  ck holds
// MAX_CK states, seg MAX_SEG states (2C values each, thread-private).
template <typename T, int C, int FAM, int PR>
__device__ __forceinline__ T gradient(const Grp &g, const TP<T, C> &tp, const ProbDev<T> &P, int quad, int kahan,
                                      int ck_fixed, const T *x, const T *v, T t, int N, T *grad, T *ck, T *seg)
{
    const int K = ck_interval<T, C>(N, ck_fixed);
    if (N < 1 || N > MAX_N || (N + K - 1) / K > MAX_CK) {
        // the checkpoint buffers hold MAX_N steps: reject other step counts
#pragma unroll
        for (int k = 0; k < C; ++k) grad[k] = (T)NAN;
        return (T)NAN;
    }
    const T h = t / (T)N;
    const T eps = P.s_eps;
    const bool huy = PR == HJ_LAX && FAM == HJ_FAM_SPLIT_NORM && P.huygens;
    T gam[C], p[C], Q = 0, Qc = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) { gam[k] = x[k]; p[k] = v[k]; }
    T *c = ck;
    // F^2: smallest g over the nodes and its node nstar (first on ties)
    T gb = huy ? terminal<T, C, HJ_LAX>(g, P, x, v, gam, p, (T *)nullptr, (T *)nullptr) : (T)0;
    int nstar = 0;
    for (int n = 0, kk = 0; n < N; ++n) {
        if (kk == 0) {
#pragma unroll
            for (int k = 0; k < C; ++k) { c[k] = gam[k]; c[C + k] = p[k]; }
            c += 2 * C;
        }
        if (++kk == K) kk = 0;
        rk4_step<T, C, FAM, PR>(g, tp, eps, h, t - (T)n * h, quad, kahan, gam, p, Q, Qc);
        if (huy) {
            const T gn = terminal<T, C, HJ_LAX>(g, P, x, v, gam, p, (T *)nullptr, (T *)nullptr);
            if (gn < gb) { gb = gn; nstar = n + 1; }
        }
    }
    // gam, p hold z_N
    T lg[C], lp[C];
    T F;
    if (huy) {
        // the seed grad g enters at node nstar during the reverse sweep
        F = gb;
#pragma unroll
        for (int k = 0; k < C; ++k) { lg[k] = 0; lp[k] = 0; }
    } else {
        F = terminal<T, C, PR>(g, P, x, v, gam, p, lg, lp) + Q;
    }
    // F^2 has no running cost: no quadrature weight, no rectangle nodes
    const T b = ((quad & HJ_QUAD_RECT) || huy) ? (T)0 : (T)1;
    const bool rect = (quad & HJ_QUAD_RECT) && !huy;
    const int ode = quad & HJ_ODE_EULER;
    const int nseg = (N + K - 1) / K;
    for (int s = nseg - 1; s >= 0; --s) {
        const int n0 = s * K, n1 = min(N, n0 + K);
        // states z_{n0 .. n1-1}: the checkpoint and K-1 recomputed steps
        T zg[C], zp[C];
        const T *c = ck + s * 2 * C;
#pragma unroll
        for (int k = 0; k < C; ++k) { zg[k] = c[k]; zp[k] = c[C + k]; }
        for (int n = n0; n < n1; ++n) {
            T *st = seg + (n - n0) * 2 * C;
#pragma unroll
            for (int k = 0; k < C; ++k) { st[k] = zg[k]; st[C + k] = zp[k]; }
            if (n + 1 < n1) {
                T Qd = 0, Qcd = 0;
                rk4_step<T, C, FAM, PR>(g, tp, eps, h, t - (T)n * h, ode, 0, zg, zp, Qd, Qcd);
            }
        }
        for (int n = n1 - 1; n >= n0; --n) {
            const T *st = seg + (n - n0) * 2 * C;
            T ug[C], up[C];
#pragma unroll
            for (int k = 0; k < C; ++k) { ug[k] = st[k]; up[k] = st[C + k]; }
            if (rect || (huy && n + 1 == nstar)) {
                // z_{n+1} is the next stored state, the next checkpoint, or z_N
                T zeros[C], rg[C], rp[C], ng[C], np[C];
                const T *sn = (n + 1 < n1) ? seg + (n + 1 - n0) * 2 * C : (s + 1 < nseg ? ck + (s + 1) * 2 * C : nullptr);
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    zeros[k] = 0;
                    ng[k] = sn ? sn[k] : gam[k];
                    np[k] = sn ? sn[C + k] : p[k];
                }
                if (huy) {
                    // F^2 seed at its node: lam_gamma += grad g(gamma_{n+1})
                    terminal<T, C, HJ_LAX>(g, P, x, v, ng, np, rg, rp);
#pragma unroll
                    for (int k = 0; k < C; ++k) lg[k] += rg[k];
                } else {
                    // rectangle node at z_{n+1}: lam += h grad L(z_{n+1})
                    tp.st = t - (T)(n + 1) * h;
                    vjp<T, C, FAM, PR>(g, tp, eps, ng, np, zeros, zeros, (T)1, rg, rp);
#pragma unroll
                    for (int k = 0; k < C; ++k) { lg[k] = fma(h, rg[k], lg[k]); lp[k] = fma(h, rp[k], lp[k]); }
                }
            }
            if (ode) {
                T wg[C], wp[C], rg[C], rp[C];
#pragma unroll
                for (int k = 0; k < C; ++k) { wg[k] = h * lg[k]; wp[k] = h * lp[k]; }
                tp.st = t - (T)n * h;
                vjp<T, C, FAM, PR>(g, tp, eps, ug, up, wg, wp, h * b, rg, rp);
#pragma unroll
                for (int k = 0; k < C; ++k) { lg[k] += rg[k]; lp[k] += rp[k]; }
            } else {
                adjoint_step<T, C, FAM, PR>(g, tp, eps, h, t - (T)n * h, b, ug, up, lg, lp);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) grad[k] = (PR == HJ_HOPF) ? lp[k] - x[k] : lp[k];
    return F;
}

}  // namespace hjd
