// hj_api.cu -- the C ABI of include/hj.h: context, validation, parameter
// upload, kernel choice and the hj_solve pipeline.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hj.h"
#include "hj_device.cuh"
#include "hj_internal.h"
#include "hj_kernels.cuh"
#include "hj_sched.h"
#include "hj_tc.h"

namespace hjd {
void reg_f32_qi_lax(Registry &);
void reg_f32_qi_hopf(Registry &);
void reg_f32_sq_lax(Registry &);
void reg_f32_sq_hopf(Registry &);
void reg_f32_sn_lax(Registry &);
void reg_f32_sn_hopf(Registry &);
void reg_f64_qi_lax(Registry &);
void reg_f64_qi_hopf(Registry &);
void reg_f64_sq_lax(Registry &);
void reg_f64_sq_hopf(Registry &);
void reg_f64_sn_lax(Registry &);
void reg_f64_sn_hopf(Registry &);
void reg_f32_lq_lax(Registry &);
void reg_f32_lq_hopf(Registry &);
void reg_f64_lq_lax(Registry &);
void reg_f64_lq_hopf(Registry &);
void reg_f32_lg_lax(Registry &);
void reg_f32_lg_hopf(Registry &);
void reg_f64_lg_lax(Registry &);
void reg_f64_lg_hopf(Registry &);
void reg_f32_ho_lax(Registry &);
void reg_f32_ho_hopf(Registry &);
void reg_f64_ho_lax(Registry &);
void reg_f64_ho_hopf(Registry &);
void reg_f32_ev_lax(Registry &);
void reg_f32_ev_hopf(Registry &);
void reg_f64_ev_lax(Registry &);
void reg_f64_ev_hopf(Registry &);
void reg_f32_spn_lax(Registry &);
void reg_f32_spn_hopf(Registry &);
void reg_f64_spn_lax(Registry &);
void reg_f64_spn_hopf(Registry &);
void reg_f32_r1_c04(Registry &);
void reg_f32_r1_c08(Registry &);
void reg_f32_r1_c16(Registry &);
void reg_f32_r1_c20(Registry &);
void reg_f32_r1_c32(Registry &);

Registry &registry()
{
    static Registry *r = [] {
        Registry *x = new Registry();
        reg_f32_qi_lax(*x);
        reg_f32_qi_hopf(*x);
        reg_f32_sq_lax(*x);
        reg_f32_sq_hopf(*x);
        reg_f32_sn_lax(*x);
        reg_f32_sn_hopf(*x);
        reg_f64_qi_lax(*x);
        reg_f64_qi_hopf(*x);
        reg_f64_sq_lax(*x);
        reg_f64_sq_hopf(*x);
        reg_f64_sn_lax(*x);
        reg_f64_sn_hopf(*x);
        reg_f32_lq_lax(*x);
        reg_f32_lq_hopf(*x);
        reg_f64_lq_lax(*x);
        reg_f64_lq_hopf(*x);
        reg_f32_lg_lax(*x);
        reg_f32_lg_hopf(*x);
        reg_f64_lg_lax(*x);
        reg_f64_lg_hopf(*x);
        reg_f32_ho_lax(*x);
        reg_f32_ho_hopf(*x);
        reg_f64_ho_lax(*x);
        reg_f64_ho_hopf(*x);
        reg_f32_ev_lax(*x);
        reg_f32_ev_hopf(*x);
        reg_f64_ev_lax(*x);
        reg_f64_ev_hopf(*x);
        reg_f32_spn_lax(*x);
        reg_f32_spn_hopf(*x);
        reg_f64_spn_lax(*x);
        reg_f64_spn_hopf(*x);
        reg_f32_r1_c04(*x);
        reg_f32_r1_c08(*x);
        reg_f32_r1_c16(*x);
        reg_f32_r1_c20(*x);
        reg_f32_r1_c32(*x);
        return x;
    }();
    return *r;
}
}  // namespace hjd

using namespace hjd;

namespace {

thread_local std::string g_create_error;

enum Kind { K_EVAL = 0, K_GRAD = 1, K_CD = 2, K_GD = 3, K_CERT = 4, K_CG = 5 };

// Descent kernel kind of a gradient mode.
int desc_kind(int grad) { return grad == HJ_GRAD_ADJOINT ? K_GD : grad == HJ_GRAD_ADJOINT_CG ? K_CG : K_CD; }

// Arithmetic per integrator step of one pair (FMA = 2, add/mul = 1, sin/cos
// and rsqrt not counted), from the operations written in hj_device.cuh.  The
// reverse step counts only the vector-Jacobian products (the stage
// intermediates they reuse and the recomputation of stage inputs from
// checkpoints are not counted).
struct FlopModel {
    double fwd_step;  // one forward step: 4 field evaluations + stage combinations (Euler: 1 + update)
    double adj_step;  // one reverse step: 4 vector-Jacobian products + combinations (Euler: 1 + update)
};

FlopModel flop_model(int fam, int pr, int d, int quad)
{
    double fld = 0, vjp = 0;
    switch (fam) {
    case HJ_FAM_QUAD_ISO: fld = 3.0 * d + 1; vjp = 2.0 * d; break;
    case HJ_FAM_SPEED_QUAD: fld = 6.0 * d + (pr == HJ_HOPF ? 10 : 8); vjp = 8.0 * d + 25; break;
    case HJ_FAM_SMOOTH_NONCONVEX:
        fld = (pr == HJ_LAX ? 11.0 : 10.0) * d + 7;
        vjp = (pr == HJ_LAX ? 13.0 : 11.0) * d + 20;
        break;
    case HJ_FAM_LINEAR_QUAD:
        // three d x d products (A gamma, Cm p, A^T p) per field and per
        // vector-Jacobian product (A^T ag, A ap, Cm ag)
        fld = 6.0 * d * d + 3.0 * d + 1;
        vjp = 6.0 * d * d + 2.0 * d;
        break;
    case HJ_FAM_BUMP_NORM:  // runs as the split norm with one block
    case HJ_FAM_SPLIT_NORM:
        fld = (pr == HJ_HOPF ? 16.0 : 12.0) * d + 30;
        vjp = (pr == HJ_HOPF ? 16.0 : 14.0) * d + 50;
        break;
    case HJ_FAM_HARMONIC: fld = 6.0 * d + 3; vjp = 4.0 * d + 2; break;
    case HJ_FAM_LINEAR_GAME: fld = 7.0 * d + 12; vjp = 9.0 * d + 10; break;
    case HJ_FAM_EVANS:
        fld = (pr == HJ_HOPF ? 16.0 : 14.0) * d + 30;
        vjp = (pr == HJ_HOPF ? 18.0 : 16.0) * d + 30;
        break;
    default: break;
    }
    if (quad & HJ_ODE_EULER) return FlopModel{fld + 4.0 * d + 2, vjp + 4.0 * d + 1};
    return FlopModel{4 * fld + 26.0 * d + 12, 4 * vjp + 28.0 * d + 6};
}

// Nominal arithmetic of one forward step of one pair in the general RK4
// form (FMA = 2): about 28d for the stage combinations plus four field
// evaluations, the field of H = |p|^2/2 ~2d, c(x)^2|p|^2/2 ~6d,
// c(x) Phi(p) ~9d, <Ax,p> + |B^T p|^2/2 4d^2 + 4md -- 36d, 52d, 64d and
// 4(4d^2 + 4md) + 28d per step.  An adjoint gradient counts as four
// evaluations (one forward, a reverse of about three), the in-kernel
// certificate as one.  These are fixed per-evaluation counts, independent of
// how a kernel arranges the arithmetic; families without one use the
// operation count of the lane-group kernels (flop_model).
double nominal_fwd_step(int fam, int pr, int d, int m, int quad)
{
    switch (fam) {
    case HJ_FAM_QUAD_ISO: return 36.0 * d;
    case HJ_FAM_SPEED_QUAD: return 52.0 * d;
    case HJ_FAM_SMOOTH_NONCONVEX: return 64.0 * d;
    case HJ_FAM_LINEAR_QUAD: return 4.0 * (4.0 * d * d + 4.0 * m * d) + 28.0 * d;
    default: return flop_model(fam, pr, d, quad).fwd_step;
    }
}

struct DevProblem {
    void *block32 = nullptr, *block64 = nullptr;
    ProbDev<float> pf{};
    ProbDev<double> pd{};
    // linear-quadratic problems that fit the tensor-core tile kernel
    bool tc = false;
    LqTcGeom geom{};
    void *wf_hi = nullptr, *wf_lo = nullptr, *wv_hi = nullptr, *wv_lo = nullptr;
};

template <typename T>
void fill_prob(const hj_problem_desc &D, const std::vector<double> &par, int ld, std::vector<T> &host, ProbDev<T> &P)
{
    const int d = D.d, m = (D.family == HJ_FAM_LINEAR_QUAD) ? D.m : 0;
    const int ldm = (d + 7) / 8 * 8;  // matrix rows padded for aligned vector loads
    const size_t nvec = 6 * (size_t)DPAD, nA = (size_t)d * d, nB = (size_t)d * m, nM = (size_t)d * ldm;
    host.assign(nvec + (m ? 3 * nM : 0), (T)0);
    T *w = host.data(), *e = w + DPAD, *ga = e + DPAD, *gs2 = ga + DPAD, *gis2 = gs2 + DPAD, *wb = gis2 + DPAD;
    size_t off = 0;
    if (D.family == HJ_FAM_SPEED_QUAD || D.family == HJ_FAM_SMOOTH_NONCONVEX) {
        for (int i = 0; i < d; ++i) w[i] = (T)par[i];
        off = d;
    }
    P.kappa = P.mu = P.alpha_a = P.alpha_b = P.beta = P.gamma0 = P.r_c = P.r_d = P.omega = (T)0;
    if (D.family == HJ_FAM_LINEAR_GAME) {
        for (int i = 0; i < d; ++i) w[i] = (T)par[i];  // the diagonal drift m
        P.r_c = (T)par[d];
        P.r_d = (T)par[d + 1];
        P.beta = (T)par[d + 2];
        P.omega = (T)par[d + 3];
        off = d + 4;
    }
    P.ksplit = d;
    if (D.family == HJ_FAM_HARMONIC) {
        P.alpha_a = (T)par[0];  // the sign
        off = 1;
    }
    if (D.family == HJ_FAM_EVANS) {
        for (int i = 0; i < d; ++i) w[i] = (T)par[i];
        P.kappa = (T)par[d];
        P.mu = (T)par[d + 1];
        P.alpha_a = (T)par[d + 2];
        P.beta = (T)par[d + 3];
        P.gamma0 = (T)par[d + 4];
        off = d + 5;
    }
    if (D.family == HJ_FAM_BUMP_NORM) {
        // the split norm with block A = all coordinates: xc_A = xc, alpha_A = sign
        for (int i = 0; i < d; ++i) w[i] = (T)par[i];
        P.kappa = (T)par[d];
        P.mu = (T)par[d + 1];
        P.alpha_a = (T)par[d + 2];
        off = d + 3;
    }
    if (D.family == HJ_FAM_SPLIT_NORM) {
        for (int i = 0; i < d; ++i) {
            w[i] = (T)par[i];
            wb[i] = (T)par[d + i];
        }
        P.ksplit = (int)par[2 * d];
        P.kappa = (T)par[2 * d + 1];
        P.mu = (T)par[2 * d + 2];
        P.alpha_a = (T)par[2 * d + 3];
        P.alpha_b = (T)par[2 * d + 4];
        off = 2 * d + 5;
    }
    if (D.family == HJ_FAM_LINEAR_QUAD) {
        // At[j][i] = A[i][j], A[j][i], Cm = B B^T (double sums, then rounded),
        // rows of ldm values
        T *At = host.data() + nvec, *A = At + nM, *Cm = A + nM;
        const double *pA = par.data(), *pB = par.data() + nA;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                At[(size_t)j * ldm + i] = (T)pA[(size_t)i * d + j];
                A[(size_t)j * ldm + i] = (T)pA[(size_t)j * d + i];
                double c = 0;
                for (int k = 0; k < m; ++k) c += pB[(size_t)i * m + k] * pB[(size_t)j * m + k];
                Cm[(size_t)j * ldm + i] = (T)c;
            }
        off = nA + nB;
    }
    for (int i = 0; i < d; ++i) {
        e[i] = (T)((i < D.n_neg) ? -1 : 1);
        if (D.g_kind == HJ_G_ROSENBROCK) continue;  // no g parameters
        if (D.g_kind == HJ_G_QUAD_SHIFT) {
            ga[i] = (T)par[off + i];
        } else {
            const T s = (T)par[off + i];
            gs2[i] = s * s;
            gis2[i] = (T)1 / (s * s);
        }
    }
    for (int i = 0; i < R1_MAXD; ++i) P.rw[i] = P.re[i] = P.rew[i] = P.rg2[i] = P.rga[i] = 0.f;
    P.rcst = 0.f;
    if (D.family == HJ_FAM_SMOOTH_NONCONVEX && d <= R1_MAXD) {
        for (int i = 0; i < d; ++i) {
            const float wi = (float)par[i], ei = (i < D.n_neg) ? -1.f : 1.f;
            P.rw[i] = wi;
            P.re[i] = ei;
            P.rew[i] = wi * ei;
            if (D.g_kind == HJ_G_QUAD_SHIFT) {
                P.rg2[i] = 1.f;
                P.rga[i] = (float)par[off + i];
            } else {
                const float s = (float)par[off + i];
                P.rg2[i] = s * s;
            }
        }
        if (D.g_kind == HJ_G_ELLIPSE) P.rcst = 0.5f;
    }
    P.d = d;
    P.family = D.family;
    P.principle = D.principle;
    P.huygens = D.principle == HJ_HUYGENS;
    P.g_kind = D.g_kind;
    P.m = m;
    P.n_neg = D.n_neg;
    P.ld = ld;
    P.ldm = ldm;
    P.s_eps = (T)D.s_eps;
}

template <typename T>
void bind_prob(void *block, int m, ProbDev<T> &P)
{
    T *b = (T *)block;
    P.w = b;
    P.e = b + DPAD;
    P.ga = b + 2 * DPAD;
    P.gs2 = b + 3 * DPAD;
    P.gis2 = b + 4 * DPAD;
    P.wb = b + 5 * DPAD;
    const size_t nM = (size_t)P.d * P.ldm;
    P.At = m ? b + 6 * DPAD : nullptr;
    P.A = m ? b + 6 * DPAD + nM : nullptr;
    P.Cm = m ? b + 6 * DPAD + 2 * nM : nullptr;
}

}  // namespace

struct hj_ctx {
    int device = 0, nsm = 0, np = 0, ld = 0, prec = 0, gmax = 1, tmax = 1;  // most starts, most trials of a problem
    hj_solver_opts opts{};
    std::vector<hj_problem_desc> desc;
    std::vector<hj_solver_opts> popts;  // per-problem descent constants (context-wide fields overridden)
    std::vector<std::vector<double>> params;
    std::vector<DevProblem> dev;
    std::vector<int> tpp_override, ck_interval;
    int32_t *d_pg = nullptr, *d_pd = nullptr, *d_pprin = nullptr, *d_pt = nullptr;
    // scratch
    long long cap_q = 0, cap_p = 0;
    int32_t *starts = nullptr, *pair_base = nullptr, *block_sums = nullptr, *trials = nullptr, *qflags = nullptr,
            *best_pid = nullptr;
    int32_t *pair_q = nullptr, *pair_slot = nullptr, *pair_round = nullptr, *iters = nullptr, *wl = nullptr,
            *amb_wl = nullptr;
    uint8_t *flags = nullptr, *pP = nullptr;
    double *pF = nullptr, *pR = nullptr;
    void *vfin = nullptr;
    int32_t *pcount = nullptr, *seg_begin = nullptr, *wl_count = nullptr, *cursor = nullptr, *amb_count = nullptr;
    int32_t *wl_lpt = nullptr, *lpt_bins = nullptr;  // fine-level work lists in longest-first order
    unsigned long long *stats = nullptr;
    // tensor-core tile kernel scratch (per CTA slot) and its error word
    float *tc_vec = nullptr, *tc_ybuf = nullptr;
    size_t tc_vec_cap = 0, tc_ybuf_cap = 0;
    int *tc_err = nullptr;
    // last solve
    cudaStream_t last_stream = nullptr;
    long long last_nq = 0;
    int last_tpp = 0, last_c = 0;
    std::vector<char> last_tc;  // problem ran on the tensor-core tile kernel in the last solve
    bool timing = true;
    std::vector<cudaEvent_t> ev_desc, ev_cert;
    // concurrent per-problem descent launches (several problems): auxiliary
    // streams forked from and joined back into the caller's stream
    bool concurrent = true;
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    // per-problem descent timing of round 0 (autotuner)
    bool pp_timing = false;
    std::vector<cudaEvent_t> pp_ev;
    // CUDA graph of the last solve's launch sequence (hj_set_graph)
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    struct GraphKey {
        long long q_begin = -1, nq = -1;
        const void *pidx = nullptr, *x = nullptr, *t = nullptr, *ns = nullptr, *phi = nullptr, *v = nullptr,
                   *st = nullptr;
        cudaStream_t s = nullptr;
        bool operator==(const GraphKey &o) const
        {
            return q_begin == o.q_begin && nq == o.nq && pidx == o.pidx && x == o.x && t == o.t && ns == o.ns &&
                   phi == o.phi && v == o.v && st == o.st && s == o.s;
        }
    } gkey;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    int n_desc_ev = 0, n_cert_ev = 0;
    long long launches = 0;
    std::string err;
};

namespace {

hj_status fail(hj_ctx *ctx, hj_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_error = buf;
    return s;
}

#define CU(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HJ_ENOMEM : HJ_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

size_t expected_params(const hj_problem_desc &D)
{
    size_t n = 0;
    if (D.family == HJ_FAM_SPEED_QUAD || D.family == HJ_FAM_SMOOTH_NONCONVEX) n += D.d;
    if (D.family == HJ_FAM_LINEAR_QUAD) n += (size_t)D.d * D.d + (size_t)D.d * D.m;
    if (D.family == HJ_FAM_BUMP_NORM) n += D.d + 3;
    if (D.family == HJ_FAM_SPLIT_NORM) n += 2 * (size_t)D.d + 5;
    if (D.family == HJ_FAM_HARMONIC) n += 1;
    if (D.family == HJ_FAM_EVANS) n += D.d + 5;
    if (D.family == HJ_FAM_LINEAR_GAME) n += D.d + 4;
    if (D.g_kind != HJ_G_ROSENBROCK) n += D.d;
    return n;
}

hj_status validate_problem(hj_ctx *ctx, const hj_problem_desc &D, int idx)
{
    if (D.d < 1 || D.d > DPAD) return fail(ctx, HJ_EINVAL, "problem %d: d=%d outside [1, %d]", idx, D.d, DPAD);
    if (D.family < HJ_FAM_QUAD_ISO || D.family > HJ_FAM_LINEAR_GAME)
        return fail(ctx, HJ_EINVAL, "problem %d: unknown family %d", idx, (int)D.family);
    if (D.principle != HJ_LAX && D.principle != HJ_HOPF && D.principle != HJ_HUYGENS)
        return fail(ctx, HJ_EINVAL, "problem %d: unknown principle %d", idx, (int)D.principle);
    if (D.g_kind == HJ_G_ROSENBROCK && (D.d != 2 || D.principle == HJ_HOPF))
        return fail(ctx, HJ_EINVAL, "problem %d: the Rosenbrock data needs d = 2 and no Hopf principle", idx);
    if (D.principle == HJ_HUYGENS && D.family != HJ_FAM_BUMP_NORM && D.family != HJ_FAM_SPLIT_NORM)
        return fail(ctx, HJ_EINVAL, "problem %d: the Huygens functional needs a degree-one H (BUMP_NORM, SPLIT_NORM)",
                    idx);
    if (D.g_kind < HJ_G_QUAD_SHIFT || D.g_kind > HJ_G_ROSENBROCK)
        return fail(ctx, HJ_EINVAL, "problem %d: unknown initial data %d", idx, (int)D.g_kind);
    if (D.family == HJ_FAM_LINEAR_QUAD) {
        if (D.m < 1 || D.m > 64 || D.d > 128)
            return fail(ctx, HJ_EINVAL, "problem %d: linear-quadratic needs m in [1,64], d <= 128", idx);
    }
    if (D.family == HJ_FAM_SMOOTH_NONCONVEX && !(D.s_eps > 0))
        return fail(ctx, HJ_EINVAL, "problem %d: s_eps must be > 0", idx);
    if (D.n_guesses < 0 || D.n_guesses > 65535)
        return fail(ctx, HJ_EINVAL, "problem %d: n_guesses=%d outside [0, 65535]", idx, D.n_guesses);
    if (!D.params && expected_params(D) > 0) return fail(ctx, HJ_EINVAL, "problem %d: params is NULL", idx);
    if (D.n_params != expected_params(D))
        return fail(ctx, HJ_EINVAL, "problem %d: n_params=%zu, expected %zu", idx, D.n_params, expected_params(D));
    size_t off = expected_params(D) - (D.g_kind == HJ_G_ROSENBROCK ? 0 : D.d);
    for (size_t i = 0; i < D.n_params; ++i)
        if (!std::isfinite(D.params[i])) return fail(ctx, HJ_EINVAL, "problem %d: params[%zu] not finite", idx, i);
    if (D.family == HJ_FAM_HARMONIC && D.params[0] != 1.0 && D.params[0] != -1.0)
        return fail(ctx, HJ_EINVAL, "problem %d: harmonic sign must be +1 or -1", idx);
    if (D.family == HJ_FAM_EVANS) {
        if (D.d < 2) return fail(ctx, HJ_EINVAL, "problem %d: the Evans-type family needs d >= 2", idx);
        if (!(D.params[D.d + 1] >= 0)) return fail(ctx, HJ_EINVAL, "problem %d: Evans mu must be >= 0", idx);
    }
    if (D.family == HJ_FAM_BUMP_NORM || D.family == HJ_FAM_SPLIT_NORM || D.family == HJ_FAM_EVANS ||
        D.family == HJ_FAM_LINEAR_GAME) {
        if (!(D.s_eps >= 0) || !std::isfinite(D.s_eps))
            return fail(ctx, HJ_EINVAL, "problem %d: s_eps must be >= 0", idx);
    }
    if (D.family == HJ_FAM_BUMP_NORM) {
        const double *sc = D.params + D.d;
        if (!(sc[1] >= 0)) return fail(ctx, HJ_EINVAL, "problem %d: bump mu must be >= 0", idx);
        if (sc[2] != 1.0 && sc[2] != -1.0) return fail(ctx, HJ_EINVAL, "problem %d: bump sign must be +1 or -1", idx);
    }
    if (D.family == HJ_FAM_SPLIT_NORM) {
        const double *sc = D.params + 2 * D.d;
        if (!(sc[0] >= 0 && sc[0] <= D.d && sc[0] == std::floor(sc[0])))
            return fail(ctx, HJ_EINVAL, "problem %d: split k must be an integer in [0, d]", idx);
        if (!(sc[2] >= 0)) return fail(ctx, HJ_EINVAL, "problem %d: split mu must be >= 0", idx);
    }
    if (D.g_kind == HJ_G_DIAG_QUAD || D.g_kind == HJ_G_ELLIPSE)
        for (int i = 0; i < D.d; ++i)
            if (!(D.params[off + i] > 0)) return fail(ctx, HJ_EINVAL, "problem %d: sigma[%d] must be > 0", idx, i);
    return HJ_OK;
}

hj_status validate_opts(hj_ctx *ctx, const hj_solver_opts &o)
{
    if (o.n_steps_default < 1 || o.n_steps_default > MAX_N)
        return fail(ctx, HJ_EINVAL, "n_steps_default=%d outside [1, %d]", o.n_steps_default, MAX_N);
    if ((int)o.quad < 0 || (int)o.quad > (HJ_QUAD_RECT | HJ_ODE_EULER))
        return fail(ctx, HJ_EINVAL, "unknown quad %d", (int)o.quad);
    if (o.grad < HJ_GRAD_FD_CENTRAL || o.grad > HJ_GRAD_ADJOINT_CG)
        return fail(ctx, HJ_EINVAL, "unknown grad mode %d", (int)o.grad);
    if ((o.grad == HJ_GRAD_FD_CENTRAL || o.grad == HJ_GRAD_FD_FORWARD) && !(o.fd_h > 0))
        return fail(ctx, HJ_EINVAL, "fd_h must be > 0");
    if (o.grad == HJ_GRAD_ADJOINT_CG && !(o.step_max > 0))
        return fail(ctx, HJ_EINVAL, "conjugate gradients need step_max > 0");
    if (o.coarse_div < 1 || o.coarse_div > 64) return fail(ctx, HJ_EINVAL, "coarse_div=%d outside [1, 64]", o.coarse_div);
    if (o.coarse_div > 1 && o.grad != HJ_GRAD_ADJOINT && o.grad != HJ_GRAD_ADJOINT_CG)
        return fail(ctx, HJ_EINVAL, "coarse_div > 1 needs a gradient descent (adjoint or adjoint CG)");
    if (o.coarse_div > 1 && !(o.coarse_eps >= 0)) return fail(ctx, HJ_EINVAL, "coarse_eps must be >= 0");
    if (!(o.step > 0) || !std::isfinite(o.step)) return fail(ctx, HJ_EINVAL, "step must be finite and > 0");
    if (o.max_iters < 0) return fail(ctx, HJ_EINVAL, "max_iters must be >= 0");
    if (o.halving_period < 0) return fail(ctx, HJ_EINVAL, "halving_period must be >= 0");
    if (!(o.eps >= 0)) return fail(ctx, HJ_EINVAL, "eps must be >= 0");
    if (o.adapt && (!(o.grow >= 1) || !(o.shrink > 0 && o.shrink <= 1) || !(o.step_max > 0)))
        return fail(ctx, HJ_EINVAL, "adapt needs grow >= 1, 0 < shrink <= 1, step_max > 0");
    if (o.n_guesses < 1 || o.n_guesses > 65535) return fail(ctx, HJ_EINVAL, "n_guesses=%d outside [1, 65535]", o.n_guesses);
    if (o.max_rounds < 0 || o.max_rounds > 64) return fail(ctx, HJ_EINVAL, "max_rounds=%d outside [0, 64]", o.max_rounds);
    if (o.max_trials < 0) return fail(ctx, HJ_EINVAL, "max_trials must be >= 0");
    if (o.guess_dist != 0 && o.guess_dist != 1) return fail(ctx, HJ_EINVAL, "guess_dist must be 0 or 1");
    if (!(o.cert_tol >= 0)) return fail(ctx, HJ_EINVAL, "cert_tol must be >= 0");
    if (o.precision != HJ_PREC_FP32 && o.precision != HJ_PREC_FP64)
        return fail(ctx, HJ_EINVAL, "unknown precision %d", (int)o.precision);
    return HJ_OK;
}

// Kernel set of a principle: F^2 runs in the Lax kernels (a runtime switch
// on the problem).
int kprin(int principle) { return principle == HJ_HOPF ? HJ_HOPF : HJ_LAX; }

// Kernel set of a family: the bump norm runs as the one-block split norm.
int kfam(int family) { return family == HJ_FAM_BUMP_NORM ? HJ_FAM_SPLIT_NORM : family; }

// Smallest instantiated C >= need for this (precision, family, principle, kind).
int pick_c(int prec, int fam, int pr, int kind, int need)
{
    const Registry &R = registry();
    for (int c = need; c <= MAXC; ++c) {
        const KSet &k = R.k[prec][fam][pr][c];
        const void *f = kind == K_EVAL ? (const void *)k.eval : kind == K_GRAD ? (const void *)k.grad
                      : kind == K_CD ? (const void *)k.cd : kind == K_GD ? (const void *)k.gd
                      : kind == K_CG ? (const void *)k.cg : (const void *)k.cert_pairs;
        if (f) return c;
    }
    return -1;
}

// Padded dimension of the one-thread-per-pair kernel for problem p and
// kernel kind, or 0 when those kernels do not apply: fp32 context, smooth
// non-convex family, Hopf principle, d <= R1_MAXD, RK4 with its own
// quadrature, no lane-count override, and a functional, gradient, coordinate
// or gradient descent kernel (conjugate gradients and the FP64 certificate
// use the lane groups).
int r1_c(const hj_ctx *ctx, int p, int kind)
{
    const hj_problem_desc &D = ctx->desc[p];
    if (ctx->prec != 0 || D.family != HJ_FAM_SMOOTH_NONCONVEX || D.principle != HJ_HOPF || D.d > R1_MAXD) return 0;
    if (ctx->tpp_override[p] > 0 || ctx->opts.quad != HJ_QUAD_RK4) return 0;
    if (kind != K_EVAL && kind != K_GRAD && kind != K_CD && kind != K_GD) return 0;
    const Registry &R = registry();
    for (int c = D.d; c <= R1_MAXD; ++c)
        if (R.r1[c].eval) return c;
    return 0;
}

// Threads per pair and components per thread for one launch.  The
// one-thread-per-pair kernels where they apply (reported as tpp 1 and a
// negative C, the padded dimension); otherwise lane groups with at most
// `pref` components per thread (fewer registers for the adjoint and for
// FP64), then the fewest lanes.
bool choose(const hj_ctx *ctx, int p, int kind, int *tpp_out, int *c_out)
{
    const hj_problem_desc &D = ctx->desc[p];
    if (const int c1 = r1_c(ctx, p, kind)) {
        *tpp_out = 1;
        *c_out = -c1;
        return true;
    }
    const int prec = (kind == K_CERT) ? ctx->prec : ctx->prec;
    int pref;
    if (kind == K_CERT) pref = 2;
    else if (ctx->prec == 1) pref = 4;
    else if (kind == K_GRAD || kind == K_GD || kind == K_CG) pref = 5;
    else pref = 10;
    // the -1 / -2 pins concern the one-pair-per-thread kernels only
    const int ov = std::max(0, ctx->tpp_override[p]);
    for (int tpp = 1; tpp <= 32; tpp <<= 1) {
        if (ov && kind != K_CERT && tpp != ov) continue;
        const int need = (D.d + tpp - 1) / tpp;
        if (!ov && need > pref && tpp < 32) continue;
        const int c = pick_c(prec, kfam(D.family), kprin(D.principle), kind, need);
        if (c > 0) {
            *tpp_out = tpp;
            *c_out = c;
            return true;
        }
    }
    return false;
}

const KSet &kset(const hj_ctx *ctx, int p, int c)
{
    const hj_problem_desc &D = ctx->desc[p];
    if (c < 0) return registry().r1[-c];
    return registry().k[ctx->prec][kfam(D.family)][kprin(D.principle)][c];
}

int persistent_grid(hj_ctx *ctx, const void *fn)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, BLOCK, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb * ctx->nsm;
}

// Descent launches of one fp32 problem and round: the coarse level first
// when coarse-to-fine is on (phase 1, then the cursor reset, then phase 2).
// One-thread-per-pair sets enqueue both their variants with complementary
// ranges of the round's pair count (read on the device): one lane per pair
// from twice the launch's resident threads up, two lanes per pair below,
// where a round is too small to fill the GPU and a pair's latency sets its
// time.  *launched gets the number of kernels launched.
// One round's fp32 descent launches of a problem (two levels: coarse, then
// fine).  With lpt_out non-null the fine level takes the round's pairs in
// longest-first order (written there; lpt_bins is the problem's bin scratch).
cudaError_t launch_desc_f32(hj_ctx *ctx, const KSet &k, int kind, bool r1, bool two, DescArgs<float> &a,
                            int32_t *cursor, cudaStream_t sp, int *launched, int32_t *lpt_out, int32_t *lpt_bins)
{
    const Launch L = kind == K_GD ? k.gd : kind == K_CG ? k.cg : k.cd;
    const void *fn = kind == K_GD ? k.f_gd : kind == K_CG ? k.f_cg : k.f_cd;
    const bool dual = r1 && kind == K_GD && k.gd_lat;
    const long long big = persistent_grid(ctx, fn);
    // a lane-count override of -1 / -2 pins one / two lanes per pair for every round
    const int ov = ctx->tpp_override[a.problem];
    const long long split = !dual ? 0 : ov == -1 ? 0 : ov == -2 ? LLONG_MAX : 2 * big * BLOCK;
    *launched = 0;
    for (int ph = two ? 1 : 0; ph <= (two ? 2 : 0); ++ph) {
        a.phase = ph;
        cudaError_t e;
        if (ph == 2 && (e = cudaMemsetAsync(cursor, 0, sizeof(int32_t), sp)) != cudaSuccess) return e;
        if (ph == 2 && lpt_out) {
            if ((e = launch_lpt_order(a.wl, a.seg_begin, a.wl_count, a.problem, a.iters, a.S.max_iters, lpt_bins,
                                      lpt_out, 4 * ctx->nsm, sp)) != cudaSuccess)
                return e;
            a.wl = lpt_out;
            *launched += 3;
        }
        a.run_lo = split;
        a.run_hi = LLONG_MAX;
        if ((e = L(&a, (int)big, sp)) != cudaSuccess) return e;
        ++*launched;
        if (dual) {
            a.run_lo = 0;
            a.run_hi = split;
            if ((e = k.gd_lat(&a, persistent_grid(ctx, k.f_gd_lat), sp)) != cudaSuccess) return e;
            ++*launched;
        }
    }
    return cudaSuccess;
}

int rows_grid(hj_ctx *ctx, const void *fn, long long n, int tpp)
{
    long long need = (n * tpp + BLOCK - 1) / BLOCK;
    long long cap = (long long)persistent_grid(ctx, fn) * 8;
    if (need < 1) need = 1;
    return (int)std::min(need, cap);
}

template <typename T>
void *as_ptr(T *p) { return (void *)p; }

// The tensor-core tile kernel runs problem p: fp32 context, linear-quadratic
// problem that fits it, RK4 quadrature, no lane-group tuning override.
bool tc_eligible(const hj_ctx *ctx, int p)
{
    return ctx->prec == 0 && ctx->dev[p].tc && ctx->tpp_override[p] == 0 && ctx->opts.quad == HJ_QUAD_RK4 &&
           (ctx->desc[p].g_kind == HJ_G_QUAD_SHIFT || ctx->desc[p].g_kind == HJ_G_DIAG_QUAD) &&
           ctx->desc[p].principle != HJ_HUYGENS &&
           ctx->popts[p].coarse_div <= 1;
}

hj_status ensure_tc_scratch(hj_ctx *ctx, int p)
{
    const LqTcGeom &g = ctx->dev[p].geom;
    const size_t nv = (size_t)ctx->nsm * lq_tc_vec_slot(g), ny = (size_t)ctx->nsm * lq_tc_ybuf_slot(g);
    if (nv > ctx->tc_vec_cap) {
        cudaFree(ctx->tc_vec);
        ctx->tc_vec = nullptr;
        ctx->tc_vec_cap = 0;
        CU(cudaMalloc(&ctx->tc_vec, nv * sizeof(float)));
        ctx->tc_vec_cap = nv;
    }
    if (ny > ctx->tc_ybuf_cap) {
        cudaFree(ctx->tc_ybuf);
        ctx->tc_ybuf = nullptr;
        ctx->tc_ybuf_cap = 0;
        CU(cudaMalloc(&ctx->tc_ybuf, ny * sizeof(float)));
        ctx->tc_ybuf_cap = ny;
    }
    return HJ_OK;
}

LqTcArgs tc_args(const hj_ctx *ctx, int p)
{
    const DevProblem &D = ctx->dev[p];
    const LqTcGeom &g = D.geom;
    LqTcArgs a{};
    a.d = g.d; a.dp = g.dp; a.m = g.m; a.mp = g.mp; a.ld = ctx->ld;
    a.KV = g.KV; a.KZ = g.KZ;
    a.fwd[0] = g.fwd[0]; a.fwd[1] = g.fwd[1]; a.rev[0] = g.rev[0]; a.rev[1] = g.rev[1];
    a.w_bytes = g.w_bytes; a.z_bytes = g.z_bytes;
    a.wf_hi = (const uint4 *)D.wf_hi; a.wf_lo = (const uint4 *)D.wf_lo;
    a.wv_hi = (const uint4 *)D.wv_hi; a.wv_lo = (const uint4 *)D.wv_lo;
    a.principle = D.pf.principle; a.g_kind = D.pf.g_kind;
    a.ga = D.pf.ga; a.gs2 = D.pf.gs2; a.gis2 = D.pf.gis2;
    a.n_default = ctx->opts.n_steps_default;
    a.vec = ctx->tc_vec; a.vec_slot = lq_tc_vec_slot(g);
    a.ybuf = ctx->tc_ybuf; a.ybuf_slot = lq_tc_ybuf_slot(g);
    a.err = ctx->tc_err;
    return a;
}

size_t tc_smem(const hj_ctx *ctx, int p) { return std::max(ctx->dev[p].geom.smem, LQ_TC_SMEM_MIN); }

hj_status ensure_scratch(hj_ctx *ctx, long long nq, long long npairs)
{
    if (nq > ctx->cap_q) {
        cudaFree(ctx->starts); cudaFree(ctx->pair_base); cudaFree(ctx->block_sums);
        cudaFree(ctx->trials); cudaFree(ctx->qflags); cudaFree(ctx->best_pid);
        ctx->starts = ctx->pair_base = ctx->block_sums = ctx->trials = ctx->qflags = ctx->best_pid = nullptr;
        ctx->cap_q = 0;
        long long nb = (nq + 1023) / 1024 + 1;
        CU(cudaMalloc(&ctx->starts, sizeof(int32_t) * nq));
        CU(cudaMalloc(&ctx->pair_base, sizeof(int32_t) * nq));
        CU(cudaMalloc(&ctx->block_sums, sizeof(int32_t) * nb));
        CU(cudaMalloc(&ctx->trials, sizeof(int32_t) * nq));
        CU(cudaMalloc(&ctx->qflags, sizeof(int32_t) * nq));
        CU(cudaMalloc(&ctx->best_pid, sizeof(int32_t) * nq));
        ctx->cap_q = nq;
    }
    if (npairs > ctx->cap_p) {
        cudaFree(ctx->pair_q); cudaFree(ctx->pair_slot); cudaFree(ctx->pair_round); cudaFree(ctx->iters);
        cudaFree(ctx->wl); cudaFree(ctx->flags); cudaFree(ctx->pP); cudaFree(ctx->pF); cudaFree(ctx->pR);
        cudaFree(ctx->vfin); cudaFree(ctx->amb_wl); cudaFree(ctx->wl_lpt);
        ctx->pair_q = ctx->pair_slot = ctx->pair_round = ctx->iters = ctx->wl = ctx->amb_wl = ctx->wl_lpt = nullptr;
        ctx->flags = ctx->pP = nullptr;
        ctx->pF = ctx->pR = nullptr;
        ctx->vfin = nullptr;
        ctx->cap_p = 0;
        const size_t es = ctx->prec ? sizeof(double) : sizeof(float);
        CU(cudaMalloc(&ctx->pair_q, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->pair_slot, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->pair_round, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->iters, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->wl, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->amb_wl, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->wl_lpt, sizeof(int32_t) * npairs));
        CU(cudaMalloc(&ctx->flags, npairs));
        CU(cudaMalloc(&ctx->pP, npairs));
        CU(cudaMalloc(&ctx->pF, sizeof(double) * npairs));
        CU(cudaMalloc(&ctx->pR, sizeof(double) * npairs));
        CU(cudaMalloc(&ctx->vfin, es * npairs * ctx->ld));
        ctx->cap_p = npairs;
    }
    return HJ_OK;
}

SolverDev solver_dev(const hj_solver_opts &o)
{
    SolverDev S;
    S.quad = o.quad;
    S.grad = o.grad;
    S.max_iters = o.max_iters;
    S.halving_period = o.halving_period;
    S.adapt = o.adapt;
    S.max_trials = o.max_trials;
    S.max_rounds = o.max_rounds;
    S.guess_dist = o.guess_dist;
    S.kahan = o.kahan;
    S.n_default = o.n_steps_default;
    S.fd_h = o.fd_h;
    S.step = o.step;
    S.eps = o.eps;
    S.grow = o.grow;
    S.shrink = o.shrink;
    S.step_max = o.step_max;
    S.cert_tol = o.cert_tol;
    S.seed = o.seed;
    S.coarse_div = o.coarse_div;
    S.coarse_eps = o.coarse_eps;
    return S;
}

hj_status check_rows(hj_ctx *ctx, int64_t n, const void *x, const void *t, const void *v)
{
    if (!ctx) return HJ_EINVAL;
    if (n < 0) return fail(ctx, HJ_EINVAL, "n must be >= 0");
    if (n > (int64_t)1 << 30) return fail(ctx, HJ_EINVAL, "n=%lld too large (max 2^30)", (long long)n);
    if (n > 0 && (!x || !t || !v)) return fail(ctx, HJ_EINVAL, "x, t and v must be non-NULL");
    return HJ_OK;
}

template <typename T>
RowArgs<T> row_args(hj_ctx *ctx, int p, int tpp, int64_t n, const int32_t *pidx, const void *x, const void *t,
                    const int32_t *ns, const void *v, void *F, void *grad)
{
    RowArgs<T> a{};
    a.P = *(ProbDev<T> *)(sizeof(T) == 8 ? (void *)&ctx->dev[p].pd : (void *)&ctx->dev[p].pf);
    a.tpp = tpp;
    a.n = n;
    a.x = (const T *)x;
    a.t = (const T *)t;
    a.nsteps = ns;
    a.n_default = ctx->opts.n_steps_default;
    a.v = (const T *)v;
    a.F = (T *)F;
    a.grad = (T *)grad;
    a.pidx = (ctx->np > 1) ? pidx : nullptr;
    a.pfilter = p;
    a.quad = ctx->opts.quad;
    a.kahan = ctx->opts.kahan;
    a.ck_interval = ctx->ck_interval[p];
    return a;
}

}  // namespace

extern "C" {

hj_status hj_create(const hj_problem_desc *problems, int n_problems, const hj_solver_opts *opts, int cuda_device,
                    hj_ctx **out)
{
    hj_ctx *ctx = nullptr;
    if (!problems || n_problems < 1 || !opts || !out)
        return fail(nullptr, HJ_EINVAL, "hj_create: problems, opts and out must be non-NULL, n_problems >= 1");
    if (n_problems > 4096) return fail(nullptr, HJ_EINVAL, "hj_create: at most 4096 problems");
    {
        hj_status s = validate_opts(nullptr, *opts);
        if (s != HJ_OK) return s;
    }
    for (int i = 0; i < n_problems; ++i) {
        hj_status s = validate_problem(nullptr, problems[i], i);
        if (s != HJ_OK) return s;
        if (problems[i].solver) {
            hj_solver_opts o = *problems[i].solver;
            o.precision = opts->precision;
            o.n_steps_default = opts->n_steps_default;
            o.quad = opts->quad;
            s = validate_opts(nullptr, o);
            if (s != HJ_OK) {
                g_create_error = "problem " + std::to_string(i) + " solver: " + g_create_error;
                return s;
            }
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
        return fail(nullptr, HJ_ECUDA, "hj_create: no CUDA device available");
    if (cuda_device < 0 || cuda_device >= ndev)
        return fail(nullptr, HJ_EINVAL, "hj_create: device %d outside [0, %d)", cuda_device, ndev);
    ctx = new (std::nothrow) hj_ctx();
    if (!ctx) return fail(nullptr, HJ_ENOMEM, "hj_create: out of host memory");
    ctx->device = cuda_device;
    ctx->np = n_problems;
    ctx->opts = *opts;
    ctx->prec = opts->precision == HJ_PREC_FP64 ? 1 : 0;
    ctx->desc.assign(problems, problems + n_problems);
    ctx->popts.resize(n_problems);
    ctx->params.resize(n_problems);
    ctx->dev.resize(n_problems);
    ctx->tpp_override.assign(n_problems, 0);
    ctx->ck_interval.assign(n_problems, 0);
    for (int i = 0; i < n_problems; ++i) {
        ctx->params[i].assign(problems[i].params, problems[i].params + problems[i].n_params);
        ctx->desc[i].params = ctx->params[i].data();
        hj_solver_opts &po = ctx->popts[i];
        po = problems[i].solver ? *problems[i].solver : *opts;
        po.precision = opts->precision;
        po.quad = opts->quad;
        po.kahan = opts->kahan;
        po.seed = opts->seed;
        po.guess_dist = opts->guess_dist;
        po.n_steps_default = opts->n_steps_default;
        po.max_rounds = opts->max_rounds;
        ctx->desc[i].solver = nullptr;
        if (ctx->desc[i].n_guesses == 0) ctx->desc[i].n_guesses = po.n_guesses;
        ctx->ld = std::max(ctx->ld, problems[i].d);
        ctx->gmax = std::max(ctx->gmax, ctx->desc[i].n_guesses);
    }
    auto bail = [&](hj_status s) {
        g_create_error = ctx->err;
        hj_destroy(ctx);
        return s;
    };
#define CUC(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            fail(ctx, e_ == cudaErrorMemoryAllocation ? HJ_ENOMEM : HJ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
            return bail(e_ == cudaErrorMemoryAllocation ? HJ_ENOMEM : HJ_ECUDA);                  \
        }                                                                                          \
    } while (0)
    CUC(cudaSetDevice(cuda_device));
    CUC(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, cuda_device));
    std::vector<int32_t> pg(n_problems), pd(n_problems), pprin(n_problems), ptr(n_problems);
    for (int i = 0; i < n_problems; ++i) {
        const hj_problem_desc &D = ctx->desc[i];
        std::vector<float> hf;
        std::vector<double> hd;
        fill_prob<float>(D, ctx->params[i], ctx->ld, hf, ctx->dev[i].pf);
        fill_prob<double>(D, ctx->params[i], ctx->ld, hd, ctx->dev[i].pd);
        CUC(cudaMalloc(&ctx->dev[i].block32, hf.size() * sizeof(float)));
        CUC(cudaMalloc(&ctx->dev[i].block64, hd.size() * sizeof(double)));
        CUC(cudaMemcpy(ctx->dev[i].block32, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice));
        CUC(cudaMemcpy(ctx->dev[i].block64, hd.data(), hd.size() * sizeof(double), cudaMemcpyHostToDevice));
        bind_prob<float>(ctx->dev[i].block32, ctx->dev[i].pf.m, ctx->dev[i].pf);
        bind_prob<double>(ctx->dev[i].block64, ctx->dev[i].pd.m, ctx->dev[i].pd);
        ctx->dev[i].pf.n_guesses = ctx->dev[i].pd.n_guesses = D.n_guesses;
        if (D.family == HJ_FAM_LINEAR_QUAD && ctx->prec == 0 && lq_tc_geometry(D.d, D.m, &ctx->dev[i].geom)) {
            std::vector<uint8_t> fh, fl, vh, vl;
            const double *pA = ctx->params[i].data(), *pB = pA + (size_t)D.d * D.d;
            lq_tc_matrices(ctx->dev[i].geom, pA, pB, fh, fl, vh, vl);
            CUC(cudaMalloc(&ctx->dev[i].wf_hi, fh.size()));
            CUC(cudaMalloc(&ctx->dev[i].wf_lo, fl.size()));
            CUC(cudaMalloc(&ctx->dev[i].wv_hi, vh.size()));
            CUC(cudaMalloc(&ctx->dev[i].wv_lo, vl.size()));
            CUC(cudaMemcpy(ctx->dev[i].wf_hi, fh.data(), fh.size(), cudaMemcpyHostToDevice));
            CUC(cudaMemcpy(ctx->dev[i].wf_lo, fl.data(), fl.size(), cudaMemcpyHostToDevice));
            CUC(cudaMemcpy(ctx->dev[i].wv_hi, vh.data(), vh.size(), cudaMemcpyHostToDevice));
            CUC(cudaMemcpy(ctx->dev[i].wv_lo, vl.data(), vl.size(), cudaMemcpyHostToDevice));
            ctx->dev[i].tc = true;
        }
        pg[i] = D.n_guesses;
        pd[i] = D.d;
        pprin[i] = D.principle;
        // pair entries of a query: its starts, then (when reseeding is on)
        // the rest of its trial budget, run together in one reseed round
        const int budget = ctx->popts[i].max_trials;
        ptr[i] = D.n_guesses + ((opts->max_rounds >= 1 && budget > D.n_guesses) ? budget - D.n_guesses : 0);
        ctx->tmax = std::max(ctx->tmax, ptr[i]);
        int tpp, c;
        if (!choose(ctx, i, K_EVAL, &tpp, &c) || !choose(ctx, i, K_CERT, &tpp, &c) ||
            !choose(ctx, i, desc_kind(ctx->popts[i].grad), &tpp, &c)) {
            fail(ctx, HJ_EUNSUPPORTED, "problem %d: no kernel built for d=%d in this precision", i, D.d);
            return bail(HJ_EUNSUPPORTED);
        }
    }
    CUC(cudaMalloc(&ctx->d_pg, sizeof(int32_t) * n_problems));
    CUC(cudaMalloc(&ctx->d_pd, sizeof(int32_t) * n_problems));
    CUC(cudaMalloc(&ctx->d_pprin, sizeof(int32_t) * n_problems));
    CUC(cudaMemcpy(ctx->d_pg, pg.data(), sizeof(int32_t) * n_problems, cudaMemcpyHostToDevice));
    CUC(cudaMemcpy(ctx->d_pd, pd.data(), sizeof(int32_t) * n_problems, cudaMemcpyHostToDevice));
    CUC(cudaMemcpy(ctx->d_pprin, pprin.data(), sizeof(int32_t) * n_problems, cudaMemcpyHostToDevice));
    CUC(cudaMalloc(&ctx->d_pt, sizeof(int32_t) * n_problems));
    CUC(cudaMemcpy(ctx->d_pt, ptr.data(), sizeof(int32_t) * n_problems, cudaMemcpyHostToDevice));
    CUC(cudaMalloc(&ctx->pcount, sizeof(int32_t) * n_problems));
    CUC(cudaMalloc(&ctx->seg_begin, sizeof(int32_t) * (n_problems + 1)));
    CUC(cudaMalloc(&ctx->wl_count, sizeof(int32_t) * n_problems));
    CUC(cudaMalloc(&ctx->cursor, sizeof(int32_t) * n_problems));
    CUC(cudaMalloc(&ctx->amb_count, sizeof(int32_t) * n_problems));
    CUC(cudaMalloc(&ctx->lpt_bins, sizeof(int32_t) * LPT_BINS_HOST * n_problems));
    CUC(cudaMalloc(&ctx->stats, sizeof(unsigned long long) * 8 * n_problems));
    CUC(cudaMemset(ctx->stats, 0, sizeof(unsigned long long) * 8 * n_problems));
    CUC(cudaMalloc(&ctx->tc_err, sizeof(int)));
    CUC(cudaMemset(ctx->tc_err, 0, sizeof(int)));
    CUC(cudaEventCreate(&ctx->ev_begin));
    CUC(cudaEventCreate(&ctx->ev_end));
#undef CUC
    *out = ctx;
    return HJ_OK;
}

hj_status hj_destroy(hj_ctx *ctx)
{
    if (!ctx) return HJ_EINVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &d : ctx->dev) {
        cudaFree(d.block32);
        cudaFree(d.block64);
        cudaFree(d.wf_hi);
        cudaFree(d.wf_lo);
        cudaFree(d.wv_hi);
        cudaFree(d.wv_lo);
    }
    cudaFree(ctx->tc_vec);
    cudaFree(ctx->tc_ybuf);
    cudaFree(ctx->tc_err);
    void *ptrs[] = {ctx->d_pg, ctx->d_pd, ctx->d_pprin, ctx->d_pt, ctx->starts, ctx->pair_base, ctx->block_sums, ctx->trials,
                    ctx->qflags, ctx->pair_q, ctx->pair_slot, ctx->pair_round, ctx->iters, ctx->wl, ctx->flags,
                    ctx->pP, ctx->pF, ctx->pR, ctx->vfin, ctx->pcount, ctx->seg_begin, ctx->wl_count, ctx->cursor,
                    ctx->stats, ctx->amb_wl, ctx->amb_count, ctx->best_pid, ctx->wl_lpt, ctx->lpt_bins};
    for (void *p : ptrs) cudaFree(p);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    for (auto a : ctx->aux) cudaStreamDestroy(a);
    for (auto e : ctx->ev_join) cudaEventDestroy(e);
    for (auto e : ctx->pp_ev) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (auto e : ctx->ev_desc) cudaEventDestroy(e);
    for (auto e : ctx->ev_cert) cudaEventDestroy(e);
    if (ctx->ev_begin) cudaEventDestroy(ctx->ev_begin);
    if (ctx->ev_end) cudaEventDestroy(ctx->ev_end);
    delete ctx;
    return HJ_OK;
}

const char *hj_last_error(const hj_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

hj_status hj_set_tuning(hj_ctx *ctx, int problem, int tpp, int ck_interval)
{
    if (!ctx) return HJ_EINVAL;
    if (problem < 0 || problem >= ctx->np) return fail(ctx, HJ_EINVAL, "problem %d outside [0, %d)", problem, ctx->np);
    if (tpp != 0 && tpp != -1 && tpp != -2 && tpp != 1 && tpp != 2 && tpp != 4 && tpp != 8 && tpp != 16 && tpp != 32)
        return fail(ctx, HJ_EINVAL, "tpp must be 0, -1, -2 or a power of two <= 32");

    if (ck_interval < 0 || ck_interval > MAX_SEG)
        return fail(ctx, HJ_EINVAL, "ck_interval must be in [0, %d]", MAX_SEG);
    int old = ctx->tpp_override[problem];
    ctx->tpp_override[problem] = tpp;
    if (tpp < 0 && (desc_kind(ctx->popts[problem].grad) != K_GD || !r1_c(ctx, problem, K_GD))) {
        ctx->tpp_override[problem] = old;
        return fail(ctx, HJ_EUNSUPPORTED, "tpp %d needs a problem that runs one pair per thread (the fp32 smooth "
                    "non-convex Hopf family, d <= %d, RK4, adjoint gradient descent)", tpp, R1_MAXD);
    }
    int t, c;
    const int kind = desc_kind(ctx->popts[problem].grad);
    if (!choose(ctx, problem, kind, &t, &c) || !choose(ctx, problem, K_EVAL, &t, &c) ||
        !choose(ctx, problem, K_GRAD, &t, &c)) {
        ctx->tpp_override[problem] = old;
        return fail(ctx, HJ_EUNSUPPORTED, "no kernel for d=%d with %d threads per pair", ctx->desc[problem].d, tpp);
    }
    ctx->ck_interval[problem] = ck_interval;
    ctx->gkey = hj_ctx::GraphKey();  // launch parameters changed: record a new graph
    return HJ_OK;
}

hj_status hj_set_graph(hj_ctx *ctx, int enable)
{
    if (!ctx) return HJ_EINVAL;
    ctx->use_graph = enable != 0;
    if (!ctx->use_graph && ctx->gexec) {
        CU(cudaSetDevice(ctx->device));
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->gkey = hj_ctx::GraphKey();
    return HJ_OK;
}

static hj_status rows_launch(hj_ctx *ctx, int kind, int64_t n, const int32_t *pidx, const void *x, const void *t,
                             const int32_t *ns, const void *v, void *F, void *grad, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    for (int p = 0; p < ctx->np; ++p) {
        if (tc_eligible(ctx, p)) {
            hj_status st = ensure_tc_scratch(ctx, p);
            if (st != HJ_OK) return st;
            LqTcArgs a = tc_args(ctx, p);
            a.n = n;
            a.x = (const float *)x;
            a.t = (const float *)t;
            a.nsteps = ns;
            a.v = (const float *)v;
            a.F = (float *)F;
            a.grad = (float *)grad;
            a.pidx = (ctx->np > 1) ? pidx : nullptr;
            a.pfilter = p;
            const int grid = (int)std::min<long long>(ctx->nsm, (n + 127) / 128);
            CU(lq_tc_launch(kind == K_EVAL ? LQ_ROWS_EVAL : LQ_ROWS_GRAD, a, std::max(grid, 1), tc_smem(ctx, p), s));
            continue;
        }
        int tpp, c;
        if (!choose(ctx, p, kind, &tpp, &c)) return fail(ctx, HJ_EUNSUPPORTED, "no kernel for problem %d", p);
        const KSet &k = kset(ctx, p, c);
        if (ctx->prec) {
            RowArgs<double> a = row_args<double>(ctx, p, tpp, n, pidx, x, t, ns, v, F, grad);
            const void *fn = kind == K_EVAL ? k.f_eval : k.f_grad;
            CU((kind == K_EVAL ? k.eval : k.grad)(&a, rows_grid(ctx, fn, n, tpp), s));
        } else {
            RowArgs<float> a = row_args<float>(ctx, p, tpp, n, pidx, x, t, ns, v, F, grad);
            const void *fn = kind == K_EVAL ? k.f_eval : k.f_grad;
            CU((kind == K_EVAL ? k.eval : k.grad)(&a, rows_grid(ctx, fn, n, tpp), s));
        }
    }
    return HJ_OK;
}

hj_status hj_eval_functional(hj_ctx *ctx, int64_t n, const int32_t *problem_idx, const void *x, const void *t,
                             const int32_t *n_steps, const void *v, void *F_out, void *stream)
{
    hj_status s = check_rows(ctx, n, x, t, v);
    if (s != HJ_OK) return s;
    if (n > 0 && !F_out) return fail(ctx, HJ_EINVAL, "F_out must be non-NULL");
    if (n == 0) return HJ_OK;
    return rows_launch(ctx, K_EVAL, n, problem_idx, x, t, n_steps, v, F_out, nullptr, stream);
}

hj_status hj_grad(hj_ctx *ctx, int64_t n, const int32_t *problem_idx, const void *x, const void *t,
                  const int32_t *n_steps, const void *v, void *F_out, void *grad_out, void *stream)
{
    hj_status s = check_rows(ctx, n, x, t, v);
    if (s != HJ_OK) return s;
    if (n > 0 && !grad_out) return fail(ctx, HJ_EINVAL, "grad_out must be non-NULL");
    if (n == 0) return HJ_OK;
    return rows_launch(ctx, K_GRAD, n, problem_idx, x, t, n_steps, v, F_out, grad_out, stream);
}

hj_status hj_certify(hj_ctx *ctx, int64_t n, const int32_t *problem_idx, const void *x, const void *t,
                     const int32_t *n_steps, const void *v, double *residual_out, uint8_t *pass_out, double *F_out,
                     void *stream)
{
    hj_status st = check_rows(ctx, n, x, t, v);
    if (st != HJ_OK) return st;
    if (n > 0 && (!residual_out || !pass_out)) return fail(ctx, HJ_EINVAL, "residual_out and pass_out must be non-NULL");
    if (n == 0) return HJ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    double *F = F_out;
    double *tmp = nullptr;
    if (!F) {
        CU(cudaMallocAsync(&tmp, sizeof(double) * n, s));
        F = tmp;
    }
    for (int p = 0; p < ctx->np; ++p) {
        int tpp, c;
        if (!choose(ctx, p, K_CERT, &tpp, &c)) return fail(ctx, HJ_EUNSUPPORTED, "no certificate kernel for problem %d", p);
        const KSet &k = kset(ctx, p, c);
        auto fill = [&](auto &a) {
            a.P = ctx->dev[p].pd;
            a.tpp = tpp;
            a.n = n;
            a.nsteps = n_steps;
            a.n_default = ctx->opts.n_steps_default;
            a.F = F;
            a.resid = residual_out;
            a.pass = pass_out;
            a.tol = ctx->popts[p].cert_tol;
            a.pidx = ctx->np > 1 ? problem_idx : nullptr;
            a.pfilter = p;
            a.quad = ctx->opts.quad;
        };
        if (ctx->prec) {
            CertArgs<double> a{};
            fill(a);
            a.x = (const double *)x; a.t = (const double *)t; a.v = (const double *)v;
            CU(k.cert_rows(&a, rows_grid(ctx, k.f_cert_rows, n, tpp), s));
        } else {
            CertArgs<float> a{};
            fill(a);
            a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)v;
            CU(k.cert_rows(&a, rows_grid(ctx, k.f_cert_rows, n, tpp), s));
        }
    }
    if (tmp) CU(cudaFreeAsync(tmp, s));
    return HJ_OK;
}

hj_status hj_guesses(hj_ctx *ctx, int64_t n, const int64_t *query_id, const int32_t *slot, const int32_t *round,
                     const int32_t *problem_idx, void *v_out, void *stream)
{
    if (!ctx) return HJ_EINVAL;
    if (n < 0) return fail(ctx, HJ_EINVAL, "n must be >= 0");
    if (n == 0) return HJ_OK;
    if (!query_id || !slot || !round || !v_out) return fail(ctx, HJ_EINVAL, "query_id, slot, round, v_out must be non-NULL");
    CU(cudaSetDevice(ctx->device));
    CU(launch_guess(n, (const long long *)query_id, slot, round, ctx->np > 1 ? problem_idx : nullptr, ctx->np, ctx->d_pd,
                    ctx->ld, ctx->opts.seed, ctx->opts.guess_dist, ctx->prec, v_out, (cudaStream_t)stream));
    return HJ_OK;
}

// Auxiliary streams of the concurrent descent launches (created once).
static hj_status ensure_aux(hj_ctx *ctx)
{
    // the tensor-core problems share the first stream; every other problem
    // gets one of its own (up to 16), so that no problem's launches wait
    // behind another's on a shared stream
    const int want = std::min(ctx->np + 1, 17);
    if ((int)ctx->aux.size() >= want) return HJ_OK;
    if (!ctx->ev_fork) CU(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    while ((int)ctx->aux.size() < want) {
        cudaStream_t st;
        cudaEvent_t ev;
        CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ctx->aux.push_back(st);
        ctx->ev_join.push_back(ev);
    }
    return HJ_OK;
}

static hj_status record(hj_ctx *ctx, std::vector<cudaEvent_t> &pool, int idx, cudaStream_t s)
{
    while ((int)pool.size() <= idx) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        pool.push_back(e);
    }
    CU(cudaEventRecord(pool[idx], s));
    return HJ_OK;
}

hj_status hj_solve(hj_ctx *ctx, int64_t q_begin, int64_t n_queries, const int32_t *problem_idx, const void *x,
                   const void *t, const int32_t *n_steps, double *phi_out, void *v_out, int32_t *status_out,
                   void *stream)
{
    if (!ctx) return HJ_EINVAL;
    if (n_queries < 0) return fail(ctx, HJ_EINVAL, "n_queries must be >= 0");
    if (q_begin < 0) return fail(ctx, HJ_EINVAL, "q_begin must be >= 0");
    if (n_queries == 0) return HJ_OK;
    if (!x || !t || !phi_out || !v_out || !status_out)
        return fail(ctx, HJ_EINVAL, "x, t, phi_out, v_out and status_out must be non-NULL");
    if (ctx->np > 1 && !problem_idx) return fail(ctx, HJ_EINVAL, "problem_idx is required with several problems");
    if (n_queries > (((long long)1 << 31) - 1) / ctx->tmax) return fail(ctx, HJ_EINVAL, "too many (query, trial) pairs");
    const long long npairs = (long long)n_queries * ctx->tmax;
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    hj_status st = ensure_scratch(ctx, n_queries, npairs);
    if (st != HJ_OK) return st;
    const int32_t *pidx = ctx->np > 1 ? problem_idx : nullptr;
    std::vector<int> kinds(ctx->np);
    for (int p = 0; p < ctx->np; ++p) kinds[p] = desc_kind(ctx->popts[p].grad);
    for (int p = 0; p < ctx->np; ++p)
        if (tc_eligible(ctx, p) && kinds[p] != K_CD) {
            st = ensure_tc_scratch(ctx, p);
            if (st != HJ_OK) return st;
        }
    // choose kernels up front so nothing is enqueued on failure
    std::vector<int> tpp_d(ctx->np), c_d(ctx->np), tpp_c(ctx->np), c_c(ctx->np);
    for (int p = 0; p < ctx->np; ++p)
        if (!choose(ctx, p, kinds[p], &tpp_d[p], &c_d[p]) || !choose(ctx, p, K_CERT, &tpp_c[p], &c_c[p]))
            return fail(ctx, HJ_EUNSUPPORTED, "no kernel for problem %d", p);
    ctx->last_stream = s;
    ctx->last_nq = n_queries;
    ctx->last_tpp = tpp_d[0];
    ctx->last_c = std::abs(c_d[0]);
    if (tc_eligible(ctx, 0) && kinds[0] != K_CD) {
        ctx->last_tpp = 1;  // one thread (and TMEM lane) per pair
        ctx->last_c = ctx->dev[0].geom.dp;
    }
    ctx->last_tc.assign(ctx->np, 0);
    for (int p = 0; p < ctx->np; ++p) ctx->last_tc[p] = (tc_eligible(ctx, p) && kinds[p] != K_CD) ? 1 : 0;
    // everything the solve enqueues on `s` (recorded into a CUDA graph when
    // hj_set_graph is on)
    // (events recorded inside a graph cannot be timed: a captured solve keeps
    // only the begin/end events, recorded around the graph launch)
    bool capturing = false;
    auto enqueue = [&]() -> hj_status {
        ctx->n_desc_ev = ctx->n_cert_ev = 0;
        const bool timing_saved = ctx->timing;
        if (capturing) ctx->timing = false;
        else CU(cudaEventRecord(ctx->ev_begin, s));
        CU(cudaMemsetAsync(ctx->stats, 0, sizeof(unsigned long long) * 8 * ctx->np, s));
        ctx->launches = 6;  // count, offsets, three scan phases, pair build
        CU(launch_count(n_queries, pidx, ctx->d_pt, ctx->starts, ctx->pcount, ctx->np, ctx->seg_begin, ctx->wl_count, s));
        CU(launch_scan(n_queries, ctx->starts, ctx->pair_base, ctx->block_sums, s));
        CU(launch_build_pairs(n_queries, pidx, ctx->np, ctx->d_pg, ctx->d_pt, ctx->pair_base, ctx->pair_q, ctx->pair_slot,
                              ctx->pair_round, ctx->trials, ctx->qflags, ctx->seg_begin, ctx->wl_count, ctx->wl,
                              ctx->pF, ctx->pP, ctx->flags, s));
        // Several problems: each round's descent launches go to auxiliary streams
        // (tensor-core problems share the first, the lane-group ones take the
        // others in turn) so that their tails overlap and the tensor-core tile
        // kernel runs beside the FP32 kernels; the caller's stream joins them.
        const bool conc = ctx->concurrent && ctx->np > 1 && !ctx->pp_timing;
        if (conc) {
            st = ensure_aux(ctx);
            if (st != HJ_OK) return st;
        }
        auto stream_of = [&](int p) -> cudaStream_t {
            if (!conc) return s;
            const int na = (int)ctx->aux.size();
            if (ctx->last_tc[p] || na == 1) return ctx->aux[0];
            return ctx->aux[1 + p % (na - 1)];
        };
        if (ctx->pp_timing)
            while ((int)ctx->pp_ev.size() < 2 * ctx->np) {
                cudaEvent_t e;
                CU(cudaEventCreate(&e));
                ctx->pp_ev.push_back(e);
            }
        const int nrounds = std::min(ctx->opts.max_rounds, 1);  // round 0, then one reseed round
        // phi in FP64 at each query's chosen start
        auto phi_pass = [&](cudaStream_t ps) -> hj_status {
            for (int p = 0; p < ctx->np; ++p) {
                const KSet &k = kset(ctx, p, c_c[p]);
                auto fill = [&](auto &a) {
                    a.P = ctx->dev[p].pd;
                    a.tpp = tpp_c[p];
                    a.n = n_queries;
                    a.nsteps = n_steps;
                    a.n_default = ctx->opts.n_steps_default;
                    a.quad = ctx->opts.quad;
                    a.pidx = pidx;
                    a.pfilter = p;
                    a.best_pid = ctx->best_pid;
                    a.phi = phi_out;
                };
                if (ctx->prec) {
                    CertArgs<double> a{};
                    fill(a);
                    a.x = (const double *)x; a.t = (const double *)t; a.v = (const double *)ctx->vfin;
                    CU(k.cert_final(&a, rows_grid(ctx, k.f_cert_final, n_queries, tpp_c[p]), ps));
                } else if (c_d[p] < 0) {
                    // one-thread-per-pair family: FP64 phi in its reduced state
                    const KSet &kr = kset(ctx, p, c_d[p]);
                    CertArgs<float> a{};
                    fill(a);
                    a.tpp = 1;
                    a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)ctx->vfin;
                    CU(kr.cert_final(&a, rows_grid(ctx, kr.f_cert_final, n_queries, 1), ps));
                } else {
                    CertArgs<float> a{};
                    fill(a);
                    a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)ctx->vfin;
                    CU(k.cert_final(&a, rows_grid(ctx, k.f_cert_final, n_queries, tpp_c[p]), ps));
                }
                ctx->launches++;
            }
            return HJ_OK;
        };
        for (int round = 0; round <= nrounds; ++round) {
            CU(cudaMemsetAsync(ctx->cursor, 0, sizeof(int32_t) * ctx->np, s));
            CU(cudaMemsetAsync(ctx->amb_count, 0, sizeof(int32_t) * ctx->np, s));
            if (ctx->timing) { st = record(ctx, ctx->ev_desc, ctx->n_desc_ev++, s); if (st != HJ_OK) return st; }
            if (conc) {
                CU(cudaEventRecord(ctx->ev_fork, s));
                for (cudaStream_t a : ctx->aux) CU(cudaStreamWaitEvent(a, ctx->ev_fork, 0));
            }
            for (int p = 0; p < ctx->np; ++p) {
                const KSet &k = kset(ctx, p, c_d[p]);
                const int kind = kinds[p];
                const cudaStream_t sp = stream_of(p);
                if (ctx->pp_timing && round == 0) CU(cudaEventRecord(ctx->pp_ev[2 * p], s));
                Launch L = kind == K_GD ? k.gd : kind == K_CG ? k.cg : k.cd;
                const void *fn = kind == K_GD ? k.f_gd : kind == K_CG ? k.f_cg : k.f_cd;
                auto fill = [&](auto &a) {
                    a.tpp = tpp_d[p];
                    a.problem = p;
                    a.nsteps = n_steps;
                    a.q_begin = q_begin;
                    a.S = solver_dev(ctx->popts[p]);
                    a.S.ck_interval = ctx->ck_interval[p];
                    a.wl = ctx->wl;
                    a.seg_begin = ctx->seg_begin;
                    a.wl_count = ctx->wl_count;
                    a.cursor = ctx->cursor;
                    a.pair_q = ctx->pair_q;
                    a.pair_slot = ctx->pair_slot;
                    a.pair_round = ctx->pair_round;
                    a.iters = ctx->iters;
                    a.flags = ctx->flags;
                    a.stats = ctx->stats + 8 * p;
                    a.pF = ctx->pF;
                    a.pR = ctx->pR;
                    a.pP = ctx->pP;
                    a.amb_wl = ctx->amb_wl;
                    a.amb_count = ctx->amb_count;
                    a.tol = ctx->popts[p].cert_tol;
                };
                if (ctx->prec) {
                    DescArgs<double> a{};
                    fill(a);
                    a.P = ctx->dev[p].pd;
                    a.x = (const double *)x; a.t = (const double *)t; a.vfin = (double *)ctx->vfin;
                    if (kind != K_CD && ctx->popts[p].coarse_div > 1) {
                        a.phase = 1;
                        CU(L(&a, persistent_grid(ctx, fn), sp));
                        CU(cudaMemsetAsync(ctx->cursor + p, 0, sizeof(int32_t), sp));
                        a.phase = 2;
                        ctx->launches++;
                    }
                    CU(L(&a, persistent_grid(ctx, fn), sp));
                } else if (tc_eligible(ctx, p) && kind != K_CD) {
                    // tensor-core tile kernel: 128 pairs per CTA, one CTA per SM
                    LqTcArgs a = tc_args(ctx, p);
                    fill(a.D);
                    a.D.P = ctx->dev[p].pf;
                    a.D.x = (const float *)x; a.D.t = (const float *)t; a.D.vfin = (float *)ctx->vfin;
                    a.x = (const float *)x; a.t = (const float *)t; a.nsteps = n_steps;
                    a.mode_desc = (kind == K_CG) ? DESC_CG : DESC_GD;
                    CU(lq_tc_launch(LQ_DESC, a, ctx->nsm, tc_smem(ctx, p), sp));
                } else {
                    DescArgs<float> a{};
                    fill(a);
                    a.P = ctx->dev[p].pf;
                    a.x = (const float *)x; a.t = (const float *)t; a.vfin = (float *)ctx->vfin;
                    // coarse-to-fine as two launches, so that every warp runs one step count
                    int nl = 0;
                    CU(launch_desc_f32(ctx, k, kind, c_d[p] < 0, kind != K_CD && ctx->popts[p].coarse_div > 1, a,
                                       ctx->cursor + p, sp, &nl, ctx->wl_lpt, ctx->lpt_bins + LPT_BINS_HOST * p));
                    ctx->launches += nl - 1;
                }
                if (ctx->pp_timing && round == 0) CU(cudaEventRecord(ctx->pp_ev[2 * p + 1], s));
                ctx->launches++;
            }
            if (conc)
                for (size_t i = 0; i < ctx->aux.size(); ++i) {
                    CU(cudaEventRecord(ctx->ev_join[i], ctx->aux[i]));
                    CU(cudaStreamWaitEvent(s, ctx->ev_join[i], 0));
                }
            if (ctx->timing) { st = record(ctx, ctx->ev_desc, ctx->n_desc_ev++, s); if (st != HJ_OK) return st; }
            for (int p = 0; p < ctx->np; ++p) {
                const KSet &k = kset(ctx, p, c_c[p]);
                auto fill = [&](auto &a) {
                    a.P = ctx->dev[p].pd;
                    a.tpp = tpp_c[p];
                    a.nsteps = n_steps;
                    a.n_default = ctx->opts.n_steps_default;
                    a.F = ctx->pF;
                    a.resid = ctx->pR;
                    a.pass = ctx->pP;
                    a.tol = ctx->popts[p].cert_tol;
                    a.quad = ctx->opts.quad;
                    a.wl = ctx->amb_wl;
                    a.seg_begin = ctx->seg_begin;
                    a.wl_count = ctx->amb_count;
                    a.problem = p;
                    a.pair_q = ctx->pair_q;
                };
                // FP64 certificate of the starts whose binary32 residual fell in
                // the band around the tolerance (few): a small grid suffices
                const long long cap = std::min<long long>(npairs, 1 << 16);
                if (ctx->prec) {
                    CertArgs<double> a{};
                    fill(a);
                    a.x = (const double *)x; a.t = (const double *)t; a.v = (const double *)ctx->vfin;
                    CU(k.cert_pairs(&a, rows_grid(ctx, k.f_cert_pairs, cap, tpp_c[p]), s));
                } else {
                    CertArgs<float> a{};
                    fill(a);
                    a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)ctx->vfin;
                    CU(k.cert_pairs(&a, rows_grid(ctx, k.f_cert_pairs, cap, tpp_c[p]), s));
                }
                ctx->launches++;
            }
            if (ctx->timing) { st = record(ctx, ctx->ev_cert, ctx->n_cert_ev++, s); if (st != HJ_OK) return st; }
            const int schedule = round < nrounds;
            if (schedule) CU(cudaMemsetAsync(ctx->wl_count, 0, sizeof(int32_t) * ctx->np, s));
            SelectArgs a{};
            a.nq = n_queries;
            a.pidx = pidx;
            a.np = ctx->np;
            a.pg = ctx->d_pg;
            a.pt = ctx->d_pt;
            a.pd = ctx->d_pd;
            a.pprin = ctx->d_pprin;
            a.ld = ctx->ld;
            a.pair_base = ctx->pair_base;
            a.pF = ctx->pF;
            a.pP = ctx->pP;
            a.flags = ctx->flags;
            a.vfin = ctx->vfin;
            a.pair_slot = ctx->pair_slot;
            a.pair_round = ctx->pair_round;
            a.trials = ctx->trials;
            a.qflags = ctx->qflags;
            a.round = round;
            a.schedule = schedule;
            a.seg_begin = ctx->seg_begin;
            a.wl_count = ctx->wl_count;
            a.wl = ctx->wl;
            a.phi = phi_out;
            a.v_out = v_out;
            a.status = status_out;
            a.best_pid = ctx->best_pid;
            CU(launch_select(a, ctx->prec, s));
            ctx->launches++;
        }
        st = phi_pass(s);
        if (st != HJ_OK) return st;
        if (ctx->timing) { st = record(ctx, ctx->ev_cert, ctx->n_cert_ev++, s); if (st != HJ_OK) return st; }
        ctx->timing = timing_saved;
        if (!capturing) CU(cudaEventRecord(ctx->ev_end, s));
        return HJ_OK;
    };
    if (ctx->use_graph && s != nullptr && !ctx->pp_timing) {
        hj_ctx::GraphKey key;
        key.q_begin = q_begin; key.nq = n_queries; key.pidx = pidx; key.x = x; key.t = t; key.ns = n_steps;
        key.phi = phi_out; key.v = v_out; key.st = status_out; key.s = s;
        if (ctx->gexec && key == ctx->gkey) {
            CU(cudaEventRecord(ctx->ev_begin, s));
            CU(cudaGraphLaunch(ctx->gexec, s));
            CU(cudaEventRecord(ctx->ev_end, s));
            return HJ_OK;
        }
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
        if (ctx->np > 1 && ctx->concurrent) {
            st = ensure_aux(ctx);
            if (st != HJ_OK) return st;
        }
        CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        capturing = true;
        st = enqueue();
        capturing = false;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != HJ_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(ctx, HJ_ECUDA, "graph capture of hj_solve: %s", cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            ctx->gexec = nullptr;
            return fail(ctx, HJ_ECUDA, "graph instantiation of hj_solve: %s", cudaGetErrorString(e2));
        }
        ctx->gkey = key;
        CU(cudaEventRecord(ctx->ev_begin, s));
        CU(cudaGraphLaunch(ctx->gexec, s));
        CU(cudaEventRecord(ctx->ev_end, s));
        return HJ_OK;
    }
    return enqueue();
}

hj_status hj_last_solve_info(hj_ctx *ctx, hj_solve_info *out)
{
    if (!ctx || !out) return HJ_EINVAL;
    std::memset(out, 0, sizeof *out);
    if (!ctx->last_nq) return HJ_OK;
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->last_stream));
    int tc_err = 0;
    CU(cudaMemcpy(&tc_err, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (tc_err)
        return fail(ctx, HJ_ETIMEOUT, "tensor-core tile kernel: a bounded wait for the tensor cores ran out");
    std::vector<unsigned long long> st(8 * ctx->np);
    CU(cudaMemcpy(st.data(), ctx->stats, sizeof(unsigned long long) * st.size(), cudaMemcpyDeviceToHost));
    out->n_queries = ctx->last_nq;
    for (int p = 0; p < ctx->np; ++p) {
        const unsigned long long *c = st.data() + 8 * p;
        const hj_problem_desc &D = ctx->desc[p];
        FlopModel fm = flop_model(D.family, D.principle, D.d, (int)ctx->opts.quad);
        out->iterations += (int64_t)c[0];
        out->functional_evals += (int64_t)c[1];
        out->gradient_evals += (int64_t)c[2];
        out->rk4_steps += (int64_t)c[3];
        out->n_pairs += (int64_t)c[5];
        out->algorithmic_flops += (double)c[3] * fm.fwd_step + (double)c[4] * fm.adj_step;
        const double nf = nominal_fwd_step(D.family, D.principle, D.d, D.m, (int)ctx->opts.quad);
        out->adjoint_steps += (int64_t)c[4];
        out->nominal_flops += nf * (double)(c[3] + c[7]) + 3.0 * nf * (double)c[4];
        out->certify_flops += (double)c[7] * fm.fwd_step;
        if (p < (int)ctx->last_tc.size() && ctx->last_tc[p]) {
            const double d = D.d, m = D.m;
            out->tensor_flops += (double)(c[3] + c[4] + c[7]) * 4.0 * 3.0 * 2.0 * (3.0 * d * d + d * m);
        }
    }
    out->threads_per_pair = ctx->last_tpp;
    out->comps_per_thread = ctx->last_c;
    float ms = 0;
    double desc_ms = 0, cert_ms = 0;
    double round0_ms = 0;
    for (int i = 0; i + 1 < ctx->n_desc_ev; i += 2) {
        CU(cudaEventElapsedTime(&ms, ctx->ev_desc[i], ctx->ev_desc[i + 1]));
        desc_ms += ms;
        if (i == 0) round0_ms = ms;
        if (i / 2 < ctx->n_cert_ev) {
            CU(cudaEventElapsedTime(&ms, ctx->ev_desc[i + 1], ctx->ev_cert[i / 2]));
            cert_ms += ms;
        }
    }
    if (ctx->n_cert_ev > ctx->n_desc_ev / 2 && ctx->n_cert_ev >= 2) {
        // final FP64 evaluation of phi: from the last select to the last event
        CU(cudaEventElapsedTime(&ms, ctx->ev_cert[ctx->n_cert_ev - 2], ctx->ev_cert[ctx->n_cert_ev - 1]));
        cert_ms += ms;
    }
    out->descent_ms_round0 = round0_ms;
    CU(cudaEventElapsedTime(&ms, ctx->ev_begin, ctx->ev_end));
    out->total_ms = ms;
    out->descent_ms = desc_ms;
    out->certify_ms = cert_ms;
    out->descent_launches = ctx->n_desc_ev / 2;
    out->kernel_launches = ctx->launches;
    return HJ_OK;
}

hj_status hj_autotune(hj_ctx *ctx, int64_t n_queries, const int32_t *problem_idx, const void *x, const void *t,
                      const int32_t *n_steps, int iters, int32_t *tpp_out, void *stream)
{
    if (!ctx) return HJ_EINVAL;
    if (n_queries < 1) return fail(ctx, HJ_EINVAL, "hj_autotune needs at least one query");
    if (iters < 1) return fail(ctx, HJ_EINVAL, "iters must be >= 1");
    if (!x || !t) return fail(ctx, HJ_EINVAL, "x and t must be non-NULL");
    if (ctx->np > 1 && !problem_idx) return fail(ctx, HJ_EINVAL, "problem_idx is required with several problems");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    // candidates: the automatic choice first, then every lane count with a kernel
    std::vector<std::vector<int>> cand(ctx->np);
    size_t maxc = 0;
    const std::vector<int> saved_tpp = ctx->tpp_override;
    for (int p = 0; p < ctx->np; ++p) {
        const int kind = desc_kind(ctx->popts[p].grad);
        cand[p].push_back(0);
        for (int tp = 1; tp <= 32; tp <<= 1) {
            ctx->tpp_override[p] = tp;
            int a_, c_;
            if (choose(ctx, p, kind, &a_, &c_)) cand[p].push_back(tp);
        }
        ctx->tpp_override[p] = saved_tpp[p];
        maxc = std::max(maxc, cand[p].size());
    }
    double *phi = nullptr;
    void *v = nullptr;
    int32_t *status = nullptr;
    const size_t es = ctx->prec ? sizeof(double) : sizeof(float);
    CU(cudaMalloc(&phi, sizeof(double) * n_queries));
    CU(cudaMalloc(&v, es * n_queries * ctx->ld));
    CU(cudaMalloc(&status, sizeof(int32_t) * n_queries));
    const std::vector<hj_solver_opts> saved_popts = ctx->popts;
    const int saved_rounds = ctx->opts.max_rounds;
    for (int p = 0; p < ctx->np; ++p)
        ctx->popts[p].max_iters =
            (desc_kind(ctx->popts[p].grad) == K_CD) ? iters * ctx->desc[p].d : iters;  // CD counts coordinate moves
    ctx->opts.max_rounds = 0;
    ctx->pp_timing = true;
    std::vector<double> best_ms(ctx->np, 1e300);
    std::vector<int> best(ctx->np, 0);
    hj_status st = HJ_OK;
    for (size_t c = 0; c <= maxc && st == HJ_OK; ++c) {
        // pass 0 warms up (module load, attributes) with the automatic choice
        const size_t ci = c == 0 ? 0 : c - 1;
        for (int p = 0; p < ctx->np; ++p) ctx->tpp_override[p] = cand[p][std::min(ci, cand[p].size() - 1)];
        st = hj_solve(ctx, 0, n_queries, problem_idx, x, t, n_steps, phi, v, status, stream);
        if (st != HJ_OK) break;
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = fail(ctx, HJ_ECUDA, "hj_autotune: solve failed");
            break;
        }
        if (c == 0) continue;
        for (int p = 0; p < ctx->np; ++p) {
            if (ci >= cand[p].size()) continue;
            float ms = 0;
            cudaEventElapsedTime(&ms, ctx->pp_ev[2 * p], ctx->pp_ev[2 * p + 1]);
            // a later candidate must beat the earlier ones by 3% (ties keep the automatic choice)
            if (ms < best_ms[p] * 0.97) {
                best_ms[p] = ms;
                best[p] = cand[p][ci];
            }
        }
    }
    ctx->pp_timing = false;
    ctx->opts.max_rounds = saved_rounds;
    ctx->popts = saved_popts;
    ctx->last_nq = 0;
    cudaFree(phi);
    cudaFree(v);
    cudaFree(status);
    if (st != HJ_OK) {
        ctx->tpp_override = saved_tpp;
        return st;
    }
    for (int p = 0; p < ctx->np; ++p) {
        ctx->tpp_override[p] = best[p];
        if (tpp_out) tpp_out[p] = best[p];
    }
    ctx->gkey = hj_ctx::GraphKey();
    return HJ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// hj_solve_noalloc: hj_solve with every piece of per-call scratch taken from
// one fixed, statically allocated device array instead of cudaMalloc.
//
// Who needs it: programs that cannot make driver allocations at call time,
// for example ones whose device memory is entirely owned by another
// allocator (a framework's caching pool or a pre-reserved arena, where an
// extra cudaMalloc fails or fragments memory), or latency-critical loops that
// must not pay for, or risk failing, an allocation.  They create the context
// once at start-up and then solve without allocating anything.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// this library reserves it for the life of the process.  Host code must not
// pass its name to a kernel (on the host the name is only a stand-in for the
// symbol); the device address comes from cudaGetSymbolAddress, fetched once
// per device with that device current, on the first hj_solve_noalloc call
// made on that device.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char hj_noalloc_scratch[HJ_SOLVE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
unsigned char *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

struct NoallocLayout {
    int32_t *pcount, *seg_begin, *wl_count, *cursor, *amb_count;
    int32_t *starts, *pair_base, *block_sums, *trials, *qflags, *best_pid;
    int32_t *pair_q, *pair_slot, *pair_round, *iters, *wl, *amb_wl;
    uint8_t *flags, *pP;
    double *pF, *pR;
    void *vfin;
};

// Carves the scratch into the solve's arrays (each 256-byte aligned) and
// returns the bytes needed; base == nullptr only measures.
size_t noalloc_layout(unsigned char *base, int np, long long nq, long long npairs, int ld, size_t es, NoallocLayout *L)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> unsigned char * {
        off = (off + 255) & ~(size_t)255;
        unsigned char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    L->pcount = (int32_t *)take(sizeof(int32_t) * np);
    L->seg_begin = (int32_t *)take(sizeof(int32_t) * (np + 1));
    L->wl_count = (int32_t *)take(sizeof(int32_t) * np);
    L->cursor = (int32_t *)take(sizeof(int32_t) * np);
    L->amb_count = (int32_t *)take(sizeof(int32_t) * np);
    L->starts = (int32_t *)take(sizeof(int32_t) * nq);
    L->pair_base = (int32_t *)take(sizeof(int32_t) * nq);
    L->block_sums = (int32_t *)take(sizeof(int32_t) * ((nq + 1023) / 1024 + 1));
    L->trials = (int32_t *)take(sizeof(int32_t) * nq);
    L->qflags = (int32_t *)take(sizeof(int32_t) * nq);
    L->best_pid = (int32_t *)take(sizeof(int32_t) * nq);
    L->pair_q = (int32_t *)take(sizeof(int32_t) * npairs);
    L->pair_slot = (int32_t *)take(sizeof(int32_t) * npairs);
    L->pair_round = (int32_t *)take(sizeof(int32_t) * npairs);
    L->iters = (int32_t *)take(sizeof(int32_t) * npairs);
    L->wl = (int32_t *)take(sizeof(int32_t) * npairs);
    L->amb_wl = (int32_t *)take(sizeof(int32_t) * npairs);
    L->flags = (uint8_t *)take(npairs);
    L->pP = (uint8_t *)take(npairs);
    L->pF = (double *)take(sizeof(double) * npairs);
    L->pR = (double *)take(sizeof(double) * npairs);
    L->vfin = (void *)take(es * npairs * ld);
    return off;
}

}  // namespace

extern "C" hj_status hj_solve_noalloc(hj_ctx *ctx, int64_t q_begin, int64_t n_queries, const int32_t *problem_idx,
                                      const void *x, const void *t, const int32_t *n_steps, double *phi_out,
                                      void *v_out, int32_t *status_out, void *stream)
{
    if (!ctx) return HJ_EINVAL;
    if (n_queries < 0) return fail(ctx, HJ_EINVAL, "n_queries must be >= 0");
    if (q_begin < 0) return fail(ctx, HJ_EINVAL, "q_begin must be >= 0");
    if (n_queries == 0) return HJ_OK;
    if (!x || !t || !phi_out || !v_out || !status_out)
        return fail(ctx, HJ_EINVAL, "x, t, phi_out, v_out and status_out must be non-NULL");
    if (ctx->np > 1 && !problem_idx) return fail(ctx, HJ_EINVAL, "problem_idx is required with several problems");
    if (ctx->device < 0 || ctx->device >= NOALLOC_MAX_DEVICES)
        return fail(ctx, HJ_EUNSUPPORTED, "hj_solve_noalloc supports devices 0..%d", NOALLOC_MAX_DEVICES - 1);
    // bound the batch before any size arithmetic: (query, start) pairs are
    // indexed in int32, and n_queries * starts must not wrap
    if (n_queries > (((long long)1 << 31) - 1) / ctx->tmax) return fail(ctx, HJ_EINVAL, "too many (query, trial) pairs");
    const long long npairs = (long long)n_queries * ctx->tmax;
    const size_t es = ctx->prec ? sizeof(double) : sizeof(float);
    NoallocLayout L{};
    const size_t need = noalloc_layout(nullptr, ctx->np, n_queries, npairs, ctx->ld, es, &L);
    if (need > (size_t)HJ_SOLVE_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, HJ_EINVAL,
                    "hj_solve_noalloc: %lld queries x %d trials need %zu bytes of scratch, the static array holds %zu "
                    "(split the batch or use hj_solve)",
                    (long long)n_queries, ctx->tmax, need, (size_t)HJ_SOLVE_NOALLOC_SCRATCH_BYTES);
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    if (!g_noalloc_ptr[ctx->device]) {
        // once per device, with that device current
        void *p = nullptr;
        CU(cudaGetSymbolAddress(&p, hj_noalloc_scratch));
        g_noalloc_ptr[ctx->device] = (unsigned char *)p;
    }
    noalloc_layout(g_noalloc_ptr[ctx->device], ctx->np, n_queries, npairs, ctx->ld, es, &L);
    const int32_t *pidx = ctx->np > 1 ? problem_idx : nullptr;
    std::vector<int> kinds(ctx->np);
    for (int p = 0; p < ctx->np; ++p) kinds[p] = desc_kind(ctx->popts[p].grad);
    std::vector<int> tpp_d(ctx->np), c_d(ctx->np), tpp_c(ctx->np), c_c(ctx->np);
    for (int p = 0; p < ctx->np; ++p)
        if (!choose(ctx, p, kinds[p], &tpp_d[p], &c_d[p]) || !choose(ctx, p, K_CERT, &tpp_c[p], &c_c[p]))
            return fail(ctx, HJ_EUNSUPPORTED, "no kernel for problem %d", p);
    // Every array read below is written earlier in this call; only the
    // per-problem counters must start at zero, and they are cleared here.
    CU(launch_count(n_queries, pidx, ctx->d_pt, L.starts, L.pcount, ctx->np, L.seg_begin, L.wl_count, s));
    CU(launch_scan(n_queries, L.starts, L.pair_base, L.block_sums, s));
    CU(launch_build_pairs(n_queries, pidx, ctx->np, ctx->d_pg, ctx->d_pt, L.pair_base, L.pair_q, L.pair_slot,
                          L.pair_round, L.trials, L.qflags, L.seg_begin, L.wl_count, L.wl, L.pF, L.pP, L.flags, s));
    const int nrounds = std::min(ctx->opts.max_rounds, 1);  // round 0, then one reseed round
    for (int round = 0; round <= nrounds; ++round) {
        CU(cudaMemsetAsync(L.cursor, 0, sizeof(int32_t) * ctx->np, s));
        CU(cudaMemsetAsync(L.amb_count, 0, sizeof(int32_t) * ctx->np, s));
        for (int p = 0; p < ctx->np; ++p) {
            const KSet &k = kset(ctx, p, c_d[p]);
            const int kind = kinds[p];
            Launch Lk = kind == K_GD ? k.gd : kind == K_CG ? k.cg : k.cd;
            const void *fn = kind == K_GD ? k.f_gd : kind == K_CG ? k.f_cg : k.f_cd;
            auto fill = [&](auto &a) {
                a.tpp = tpp_d[p];
                a.problem = p;
                a.nsteps = n_steps;
                a.q_begin = q_begin;
                a.S = solver_dev(ctx->popts[p]);
                a.S.ck_interval = ctx->ck_interval[p];
                a.wl = L.wl;
                a.seg_begin = L.seg_begin;
                a.wl_count = L.wl_count;
                a.cursor = L.cursor;
                a.pair_q = L.pair_q;
                a.pair_slot = L.pair_slot;
                a.pair_round = L.pair_round;
                a.iters = L.iters;
                a.flags = L.flags;
                a.stats = nullptr;
                a.pF = L.pF;
                a.pR = L.pR;
                a.pP = L.pP;
                a.amb_wl = L.amb_wl;
                a.amb_count = L.amb_count;
                a.tol = ctx->popts[p].cert_tol;
            };
            const bool two = kind != K_CD && ctx->popts[p].coarse_div > 1;
            if (ctx->prec) {
                DescArgs<double> a{};
                fill(a);
                a.P = ctx->dev[p].pd;
                a.x = (const double *)x; a.t = (const double *)t; a.vfin = (double *)L.vfin;
                if (two) {
                    a.phase = 1;
                    CU(Lk(&a, persistent_grid(ctx, fn), s));
                    CU(cudaMemsetAsync(L.cursor + p, 0, sizeof(int32_t), s));
                    a.phase = 2;
                }
                CU(Lk(&a, persistent_grid(ctx, fn), s));
            } else {
                DescArgs<float> a{};
                fill(a);
                a.P = ctx->dev[p].pf;
                a.x = (const float *)x; a.t = (const float *)t; a.vfin = (float *)L.vfin;
                int nl = 0;
                CU(launch_desc_f32(ctx, k, kind, c_d[p] < 0, two, a, L.cursor + p, s, &nl, nullptr, nullptr));
            }
        }
        for (int p = 0; p < ctx->np; ++p) {
            const KSet &k = kset(ctx, p, c_c[p]);
            auto fill = [&](auto &a) {
                a.P = ctx->dev[p].pd;
                a.tpp = tpp_c[p];
                a.nsteps = n_steps;
                a.n_default = ctx->opts.n_steps_default;
                a.F = L.pF;
                a.resid = L.pR;
                a.pass = L.pP;
                a.tol = ctx->popts[p].cert_tol;
                a.quad = ctx->opts.quad;
                a.wl = L.amb_wl;
                a.seg_begin = L.seg_begin;
                a.wl_count = L.amb_count;
                a.problem = p;
                a.pair_q = L.pair_q;
            };
            const long long cap = std::min<long long>(npairs, 1 << 16);
            if (ctx->prec) {
                CertArgs<double> a{};
                fill(a);
                a.x = (const double *)x; a.t = (const double *)t; a.v = (const double *)L.vfin;
                CU(k.cert_pairs(&a, rows_grid(ctx, k.f_cert_pairs, cap, tpp_c[p]), s));
            } else {
                CertArgs<float> a{};
                fill(a);
                a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)L.vfin;
                CU(k.cert_pairs(&a, rows_grid(ctx, k.f_cert_pairs, cap, tpp_c[p]), s));
            }
        }
        const int schedule = round < nrounds;
        if (schedule) CU(cudaMemsetAsync(L.wl_count, 0, sizeof(int32_t) * ctx->np, s));
        SelectArgs a{};
        a.nq = n_queries;
        a.pidx = pidx;
        a.np = ctx->np;
        a.pg = ctx->d_pg;
        a.pt = ctx->d_pt;
        a.pd = ctx->d_pd;
        a.pprin = ctx->d_pprin;
        a.ld = ctx->ld;
        a.pair_base = L.pair_base;
        a.pF = L.pF;
        a.pP = L.pP;
        a.flags = L.flags;
        a.vfin = L.vfin;
        a.pair_slot = L.pair_slot;
        a.pair_round = L.pair_round;
        a.trials = L.trials;
        a.qflags = L.qflags;
        a.round = round;
        a.schedule = schedule;
        a.seg_begin = L.seg_begin;
        a.wl_count = L.wl_count;
        a.wl = L.wl;
        a.phi = phi_out;
        a.v_out = v_out;
        a.status = status_out;
        a.best_pid = L.best_pid;
        CU(launch_select(a, ctx->prec, s));
    }
    for (int p = 0; p < ctx->np; ++p) {
        const KSet &k = kset(ctx, p, c_c[p]);
        auto fill = [&](auto &a) {
            a.P = ctx->dev[p].pd;
            a.tpp = tpp_c[p];
            a.n = n_queries;
            a.nsteps = n_steps;
            a.n_default = ctx->opts.n_steps_default;
            a.quad = ctx->opts.quad;
            a.pidx = pidx;
            a.pfilter = p;
            a.best_pid = L.best_pid;
            a.phi = phi_out;
        };
        if (ctx->prec) {
            CertArgs<double> a{};
            fill(a);
            a.x = (const double *)x; a.t = (const double *)t; a.v = (const double *)L.vfin;
            CU(k.cert_final(&a, rows_grid(ctx, k.f_cert_final, n_queries, tpp_c[p]), s));
        } else if (c_d[p] < 0) {
            const KSet &kr = kset(ctx, p, c_d[p]);
            CertArgs<float> a{};
            fill(a);
            a.tpp = 1;
            a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)L.vfin;
            CU(kr.cert_final(&a, rows_grid(ctx, kr.f_cert_final, n_queries, 1), s));
        } else {
            CertArgs<float> a{};
            fill(a);
            a.x = (const float *)x; a.t = (const float *)t; a.v = (const float *)L.vfin;
            CU(k.cert_final(&a, rows_grid(ctx, k.f_cert_final, n_queries, tpp_c[p]), s));
        }
    }
    return HJ_OK;
}
