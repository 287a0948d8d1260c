/*
 * hj_oracle.c -- plain, slow, FP64 CPU oracle for the generalized Lax/Hopf
 * method of Chow, Darbon, Osher and Yin (arXiv 1704.02524).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file's library.
 * The CUDA path shares no code, header, table or helper with it.
 *
 * Everything is double precision and written as directly as possible:
 * straight loops over coordinates, full storage of every RK4 stage for the
 * adjoint, one pair at a time.  Each function names the passage it follows.
 *
 * Families: H = |p|^2/2; H = c(x)^2|p|^2/2 with c = 1 + sin<w,x>/2; the
 * smooth non-convex H = c(x) sum_i e_i sqrt(p_i^2 + eps); the linear-
 * quadratic H = <Ax,p> + |B^T p|^2/2; and H = +-c(x)|p| with the Gaussian
 * bump speed c = 1 + kappa exp(-mu|x - xc|^2) of Sec. 6, Example 3; and the
 * split norm H = c_A(x)|p_A| + c_B(x)|p_B| over two coordinate blocks, each
 * speed a signed multiple of such a bump (Sec. 6, Example 5); the harmonic
 * oscillator H = +-(|p|^2 + |x|^2)/2 (Sec. 6, Example 2); and the non-convex
 * H = -c(x) p_1 + beta|p_2| - |p| - gamma0 with c a bump (Sec. 6, Example 4);
 * and the time-dependent linear differential game of Sec. 3.4, Example 3,
 * H(x,p,s) = -<Mx,p> + a(s)|p| with M diagonal and the support functions of
 * balls, a(s) = r_C - r_D (1 + beta sin(omega s)).
 * Initial data: |x - a|^2/2, sum x_i^2/(2 s_i^2), and the ellipse data
 * (<x, Ax> - 1)/2, A diagonal, of Sec. 6.
 *
 * What it computes, per (query x, time t, initial guess v):
 *   - the bi-characteristics (Sec. 4.1, final value problem):
 *         d gamma/ds = dH/dp,  dp/ds = -dH/dx,  gamma(t) = x,  p(t) = v,
 *     integrated backward from s = t to s = 0 with N classical RK4 steps,
 *     or with N forward Euler steps, the solver Sec. 4.2 uses as its
 *     example while leaving higher-order schemes open;
 *   - the functional F^1 (Lax, eq. lax_formula / Sec. 4.1) or G (Hopf,
 *     eq. hopf_formula / Sec. 4.1) with the running-cost integral taken
 *     either by RK4 on an augmented quadrature state (default) or by the
 *     rectangular rule of eq. num_int;
 *   - derivatives by the finite differences of eq. num_diff (forward) or
 *     the central form, and the exact gradient of the discretised
 *     functional by the discrete adjoint of the RK4 (or Euler) map;
 *   - cyclic coordinate descent (Algorithm 1), gradient descent, and a
 *     conjugate-gradient (momentum) descent for ill-conditioned functionals
 *     (Sec. 5 points to momentum methods when plain descent drags);
 *   - the certificate p(0) in dg(gamma(0)) (Sec. 4.3), reseeding of failed
 *     starts and best-of-guesses (Sec. 5: multiple random initial guesses).
 *
 * Random initial guesses come from Philox4x32-10 (Salmon, Moraes, Dror,
 * Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11), written here
 * from that paper's definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Largest dimension and control width the oracle accepts (stack buffers). */
#define ORC_DMAX 128
#define ORC_MMAX 64

/* ------------------------------------------------------------------------ */
/* Problem description                                                       */
/* ------------------------------------------------------------------------ */

enum { FAM_QUAD_ISO = 0, FAM_SPEED_QUAD = 1, FAM_SMOOTH_NONCONVEX = 2, FAM_LINEAR_QUAD = 3, FAM_BUMP_NORM = 4,
       FAM_SPLIT_NORM = 5, FAM_HARMONIC = 6, FAM_EVANS = 7, FAM_LINEAR_GAME = 8 };
/* HUYGENS: the Lax principle through F^2 (Sec. 4.1), the smallest g over the
 * endpoints gamma(x, v, r, 0), 0 <= r <= t, taken on the solver grid r = n dt
 * (eq. num_min) -- for Hamiltonians of degree one in p, with no running cost. */
enum { LAX = 0, HOPF = 1, HUYGENS = 2 };
/* G_ROSENBROCK (Sec. 6, Example 2, d = 2): g = 4e-4 (-100 + (1 - x_1)^2 + 100 (1 + x_2 - x_1^2)^2),
 * non-convex, so it has no Legendre transform here: Lax and Huygens only. */
enum { G_QUAD_SHIFT = 0, G_DIAG_QUAD = 1, G_ELLIPSE = 2, G_ROSENBROCK = 3 };
enum { QUAD_RK4 = 0, QUAD_RECT = 1 };
/* Flag or-ed into a `quad` argument: integrate with forward Euler (the
 * solver Sec. 4.2 suggests) instead of RK4.  With QUAD_RK4 the running cost
 * is then integrated by the same Euler steps on the augmented state. */
enum { ODE_EULER = 2 };
enum { GRAD_FD_CENTRAL = 0, GRAD_FD_FORWARD = 1, GRAD_ADJOINT = 2 };
enum { DESC_CD = 0, DESC_GD = 1, DESC_CG = 2 };

/* Per-query status bits (same meaning as the library's, defined separately). */
#define ST_CERTIFIED 1
#define ST_MAX_ITERS 2
#define ST_NONFINITE 4
#define ST_RESEEDED 8

typedef struct {
    int d;            /* dimension of x, p, v                                   */
    int family;       /* FAM_*                                                  */
    int principle;    /* LAX, HOPF or HUYGENS                                   */
    int g_kind;       /* G_*                                                    */
    int m;            /* columns of B (linear-quadratic family)                 */
    int n_neg;        /* smooth non-convex family: first n_neg signs negative   */
    double s_eps;     /* smooth non-convex family: s(q) = sqrt(q^2 + s_eps)     */
    const double *w;  /* [d]   speed c(x) = 1 + sin(<w,x>)/2                    */
    const double *A;  /* [d*d] row-major drift matrix                           */
    const double *B;  /* [d*m] row-major control matrix                         */
    const double *ga; /* [d]   shift a of g = |x-a|^2/2                         */
    const double *gs; /* [d]   sigma of g = sum x_i^2/(2 sigma_i^2) (- 1/2 for  */
                      /*       the ellipse data of Sec. 6)                      */
    /* bump-norm family (Sec. 6, Example 3): H = sign c(x) |p|_eps with
     * c(x) = 1 + kappa exp(-mu |x - xc|^2), |p|_eps = sqrt(|p|^2 + s_eps) */
    const double *xc; /* [d] */
    double kappa, mu, hsign;
    /* split-norm family (Sec. 6, Example 5): H = c_A(x)|p_A|_eps + c_B(x)|p_B|_eps
     * over the blocks A = coordinates 0..k-1 and B = k..d-1, with
     * c_A = alpha_a (1 + kappa exp(-mu |x - xc|^2)),
     * c_B = alpha_b (1 + kappa exp(-mu |x - xcb|^2)); signs in the alphas */
    const double *xcb; /* [d] */
    int ksplit;
    double alpha_a, alpha_b;
    /* harmonic family (Example 2): H = hsign (|p|^2 + |x|^2)/2.
     * Evans-type family (Example 4): H = -c(x) p_1 + beta |p_2|_eps - |p|_eps - gamma0
     * with c = alpha_a (1 + kappa exp(-mu |x - xc|^2)) and |q|_eps = sqrt(q^2 + s_eps) */
    double beta, gamma0;
    /* linear game (Sec. 3.4, Example 3): H(x,p,s) = -<Mx,p> + a(s)|p|_eps with
     * M = diag(m), a(s) = r_C - r_D (1 + beta sin(omega s)); m in w */
    double r_c, r_d, omega;
} orc_problem;

typedef struct {
    int quad;            /* QUAD_RK4 / QUAD_RECT, optionally | ODE_EULER          */
    int descent;         /* DESC_CD / DESC_GD / DESC_CG                          */
    int grad;            /* GRAD_FD_CENTRAL / GRAD_FD_FORWARD / GRAD_ADJOINT     */
    double fd_h;         /* finite-difference step sigma of eq. num_diff         */
    double step;         /* alpha = 1/L of Algorithm 1                           */
    int max_iters;       /* iteration cap (CD: coordinate iterations; GD: steps) */
    int halving_period;  /* M of Algorithm 1 (0: never halve)                    */
    double eps;          /* stopping tolerance epsilon of Algorithm 1            */
    int adapt;           /* GD only: per-coordinate sign-change step control     */
    double grow;         /* GD adapt: factor applied when the sign is kept       */
    double shrink;       /* GD adapt: factor applied when the sign flips         */
    double step_max;     /* GD adapt: upper bound on a coordinate's step         */
    int n_guesses;       /* initial guesses per query                            */
    int max_trials;      /* total trials per query (guesses + reseeds)           */
    int max_rounds;      /* >= 1: one reseed round spends the trial budget       */
    uint64_t seed;       /* Philox key                                           */
    int guess_dist;      /* 0: U[-2,2]^d, 1: Irwin-Hall(12) approximate N(0,1)   */
    double cert_tol;     /* certificate tolerance tau                            */
    int coarse_div;      /* > 1: descend first on the functional with N/coarse_div */
                         /* RK4 steps until moves < coarse_eps, then on the full  */
                         /* functional from there (gradient forms only)           */
    double coarse_eps;
} orc_opts;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 4): ten rounds of two 32x32->64 multiplies with */
/* the published multipliers, key bumped by the published Weyl constants.   */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Word number `j` of the stream for (query q, guess slot g, round r).
 * Counter = (j / 4, g | r << 16, q low word, q high word); key = seed. */
static uint32_t guess_word(uint64_t seed, int64_t q, int g, int r, int j)
{
    uint32_t ctr[4] = { (uint32_t)(j / 4), (uint32_t)g | ((uint32_t)r << 16),
                        (uint32_t)((uint64_t)q & 0xffffffffu), (uint32_t)((uint64_t)q >> 32) };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[j % 4];
}

/* Initial guess (Sec. 5: random starting points uniform in [-2,2]^d).
 * dist 0: v_j = 4 u - 2 with u = (word >> 8) 2^-24, exact in binary32.
 * dist 1: Irwin-Hall(12): sum of twelve 24-bit uniforms minus 6, summed as an
 *         integer so the value is exact in binary64. */
void orc_guess(uint64_t seed, int64_t q, int g, int r, int d, int dist, double *v)
{
    for (int j = 0; j < d; ++j) {
        if (dist == 0) {
            uint32_t wd = guess_word(seed, q, g, r, j);
            v[j] = 4.0 * ((double)(wd >> 8) * 0x1p-24) - 2.0;
        } else {
            uint64_t s = 0;
            for (int k = 0; k < 12; ++k) s += guess_word(seed, q, g, r, 12 * j + k) >> 8;
            v[j] = (double)s * 0x1p-24 - 6.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Hamiltonian families: right-hand side of the characteristic system and the */
/* running cost of the functional (Sec. 4.1; per family in the comments).    */
/* ------------------------------------------------------------------------ */

static double dot(const double *a, const double *b, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

static double sgn_of(const orc_problem *P, int i) { return i < P->n_neg ? -1.0 : 1.0; }

/* Speed c(x) = 1 + sin(u)/2, u = <w,x>, with c' = cos(u)/2, c'' = -sin(u)/2
 * along w (so grad c = c' w). */
static void speed(const orc_problem *P, const double *gam, double *u, double *c, double *c1, double *c2)
{
    *u = dot(P->w, gam, P->d);
    *c = 1.0 + 0.5 * sin(*u);
    *c1 = 0.5 * cos(*u);
    *c2 = -0.5 * sin(*u);
}

/* Bump speed c(x) = 1 + kappa exp(-mu |x - xc|^2) with grad c = k (x - xc),
 * k = -2 mu kappa exp(-mu |x - xc|^2); y receives x - xc. */
static void bump(const orc_problem *P, const double *gam, double *y, double *c, double *k)
{
    double rr = 0.0;
    for (int i = 0; i < P->d; ++i) {
        y[i] = gam[i] - P->xc[i];
        rr += y[i] * y[i];
    }
    double e = exp(-P->mu * rr);
    *c = 1.0 + P->kappa * e;
    *k = -2.0 * P->mu * P->kappa * e;
}

/* Split-norm family: per block b in {A, B}, the speed c_b, its gradient
 * factor k_b (grad c_b = k_b (x - xc_b)), y_b = x - xc_b, and the block norm
 * n_b = sqrt(|p_b|^2 + s_eps) (0 for an empty block). */
typedef struct {
    double c[2], k[2], n[2];
    double y[2][ORC_DMAX];
} split_t;
static int block_of(const orc_problem *P, int i) { return i < P->ksplit ? 0 : 1; }
static void split_eval(const orc_problem *P, const double *gam, const double *p, split_t *S)
{
    const double *ctr[2] = { P->xc, P->xcb };
    const double alpha[2] = { P->alpha_a, P->alpha_b };
    for (int b = 0; b < 2; ++b) {
        double rr = 0.0;
        for (int i = 0; i < P->d; ++i) {
            S->y[b][i] = gam[i] - ctr[b][i];
            rr += S->y[b][i] * S->y[b][i];
        }
        double e = exp(-P->mu * rr);
        S->c[b] = alpha[b] * (1.0 + P->kappa * e);
        S->k[b] = -2.0 * P->mu * alpha[b] * P->kappa * e;
        double pp = 0.0;
        int cnt = 0;
        for (int i = 0; i < P->d; ++i)
            if (block_of(P, i) == b) { pp += p[i] * p[i]; ++cnt; }
        S->n[b] = cnt ? sqrt(pp + P->s_eps) : 0.0;
    }
}

/* Speed of the linear game at PDE time s. */
static double game_speed(const orc_problem *P, double s)
{
    return P->r_c - P->r_d * (1.0 + P->beta * sin(P->omega * s));
}

/* Hamiltonian value H(gamma, p) at PDE time s (only the linear game uses s). */
static double ham(const orc_problem *P, const double *gam, const double *p, double s)
{
    int d = P->d;
    double u, c, c1, c2;
    switch (P->family) {
    case FAM_QUAD_ISO:
        return 0.5 * dot(p, p, d);
    case FAM_SPEED_QUAD:
        speed(P, gam, &u, &c, &c1, &c2);
        return 0.5 * c * c * dot(p, p, d);
    case FAM_SMOOTH_NONCONVEX: {
        speed(P, gam, &u, &c, &c1, &c2);
        double phi = 0.0;
        for (int i = 0; i < d; ++i) phi += sgn_of(P, i) * sqrt(p[i] * p[i] + P->s_eps);
        return c * phi;
    }
    case FAM_LINEAR_QUAD: {
        double h = 0.0;
        for (int i = 0; i < d; ++i) {
            double ax = 0.0;
            for (int j = 0; j < d; ++j) ax += P->A[i * d + j] * gam[j];
            h += ax * p[i];
        }
        for (int k = 0; k < P->m; ++k) {
            double btp = 0.0;
            for (int i = 0; i < d; ++i) btp += P->B[i * P->m + k] * p[i];
            h += 0.5 * btp * btp;
        }
        return h;
    }
    case FAM_BUMP_NORM: {
        double y[ORC_DMAX], c, k;
        bump(P, gam, y, &c, &k);
        return P->hsign * c * sqrt(dot(p, p, d) + P->s_eps);
    }
    case FAM_SPLIT_NORM: {
        split_t S;
        split_eval(P, gam, p, &S);
        return S.c[0] * S.n[0] + S.c[1] * S.n[1];
    }
    case FAM_HARMONIC:
        return P->hsign * 0.5 * (dot(p, p, d) + dot(gam, gam, d));
    case FAM_LINEAR_GAME: {
        double mxp = 0.0;
        for (int i = 0; i < d; ++i) mxp += P->w[i] * gam[i] * p[i];
        return -mxp + game_speed(P, s) * sqrt(dot(p, p, d) + P->s_eps);
    }
    case FAM_EVANS: {
        double y[ORC_DMAX], c, k;
        bump(P, gam, y, &c, &k);
        c *= P->alpha_a;
        return -c * p[0] + P->beta * sqrt(p[1] * p[1] + P->s_eps) - sqrt(dot(p, p, d) + P->s_eps) - P->gamma0;
    }
    }
    return NAN;
}

/* dH/dp and dH/dx at (gamma, p). */
static void ham_grads(const orc_problem *P, const double *gam, const double *p, double s, double *Hp, double *Hx)
{
    int d = P->d;
    double u, c, c1, c2;
    switch (P->family) {
    case FAM_QUAD_ISO:
        for (int i = 0; i < d; ++i) { Hp[i] = p[i]; Hx[i] = 0.0; }
        return;
    case FAM_SPEED_QUAD: {
        speed(P, gam, &u, &c, &c1, &c2);
        double pp = dot(p, p, d);
        for (int i = 0; i < d; ++i) {
            Hp[i] = c * c * p[i];
            Hx[i] = c * c1 * pp * P->w[i];
        }
        return;
    }
    case FAM_SMOOTH_NONCONVEX: {
        speed(P, gam, &u, &c, &c1, &c2);
        double phi = 0.0;
        for (int i = 0; i < d; ++i) {
            double s = sqrt(p[i] * p[i] + P->s_eps);
            phi += sgn_of(P, i) * s;
            Hp[i] = c * sgn_of(P, i) * p[i] / s;
        }
        for (int i = 0; i < d; ++i) Hx[i] = phi * c1 * P->w[i];
        return;
    }
    case FAM_LINEAR_QUAD: {
        double btp[ORC_MMAX];
        for (int k = 0; k < P->m; ++k) {
            btp[k] = 0.0;
            for (int i = 0; i < d; ++i) btp[k] += P->B[i * P->m + k] * p[i];
        }
        for (int i = 0; i < d; ++i) {
            double ax = 0.0, atp = 0.0, bbtp = 0.0;
            for (int j = 0; j < d; ++j) {
                ax += P->A[i * d + j] * gam[j];
                atp += P->A[j * d + i] * p[j];
            }
            for (int k = 0; k < P->m; ++k) bbtp += P->B[i * P->m + k] * btp[k];
            Hp[i] = ax + bbtp;
            Hx[i] = atp;
        }
        return;
    }
    case FAM_BUMP_NORM: {
        /* H_p = sign c p / |p|_eps,  H_x = sign |p|_eps grad c */
        double y[ORC_DMAX], c, k;
        bump(P, gam, y, &c, &k);
        double n = sqrt(dot(p, p, d) + P->s_eps);
        for (int i = 0; i < d; ++i) {
            Hp[i] = P->hsign * c * p[i] / n;
            Hx[i] = P->hsign * n * k * y[i];
        }
        return;
    }
    case FAM_HARMONIC:
        for (int i = 0; i < d; ++i) {
            Hp[i] = P->hsign * p[i];
            Hx[i] = P->hsign * gam[i];
        }
        return;
    case FAM_LINEAR_GAME: {
        /* H_p = -M gamma + a(s) p/n,  H_x = -M p */
        double a = game_speed(P, s), n = sqrt(dot(p, p, d) + P->s_eps);
        for (int i = 0; i < d; ++i) {
            Hp[i] = -P->w[i] * gam[i] + a * p[i] / n;
            Hx[i] = -P->w[i] * p[i];
        }
        return;
    }
    case FAM_EVANS: {
        /* H_p = -c e_1 + beta p_2/s_2 e_2 - p/n,  H_x = -p_1 grad c = -p_1 alpha k y */
        double y[ORC_DMAX], c, k;
        bump(P, gam, y, &c, &k);
        c *= P->alpha_a;
        k *= P->alpha_a;
        double n = sqrt(dot(p, p, d) + P->s_eps), s2 = sqrt(p[1] * p[1] + P->s_eps);
        for (int i = 0; i < d; ++i) {
            Hp[i] = -p[i] / n;
            Hx[i] = -p[0] * k * y[i];
        }
        Hp[0] -= c;
        Hp[1] += P->beta * p[1] / s2;
        return;
    }
    case FAM_SPLIT_NORM: {
        /* H_p on block b = c_b p_b / n_b;  H_x = sum_b n_b k_b y_b */
        split_t S;
        split_eval(P, gam, p, &S);
        for (int i = 0; i < d; ++i) {
            int b = block_of(P, i);
            Hp[i] = S.c[b] * p[i] / S.n[b];
            Hx[i] = S.n[0] * S.k[0] * S.y[0][i] + S.n[1] * S.k[1] * S.y[1][i];
        }
        return;
    }
    }
}

/* Running cost inside the integral: Lax <p, dH/dp> - H (eq. lax_formula),
 * Hopf H - <dH/dx, gamma> (eq. hopf_formula). */
static double running_cost(const orc_problem *P, const double *gam, const double *p, double s)
{
    int d = P->d;
    double Hp[ORC_DMAX], Hx[ORC_DMAX];
    ham_grads(P, gam, p, s, Hp, Hx);
    double H = ham(P, gam, p, s);
    return (P->principle == LAX) ? dot(p, Hp, d) - H : H - dot(Hx, gam, d);
}

/* Right-hand side in reversed time tau = t - s: the state z = (gamma, p)
 * moves by dz/dtau = (-dH/dp, +dH/dx) and the quadrature state by the
 * running cost.  out has 2d + 1 entries. */
static void field(const orc_problem *P, const double *z, double s, double *out)
{
    int d = P->d;
    const double *gam = z, *p = z + d;
    double Hp[ORC_DMAX], Hx[ORC_DMAX];
    ham_grads(P, gam, p, s, Hp, Hx);
    for (int i = 0; i < d; ++i) {
        out[i] = -Hp[i];
        out[d + i] = Hx[i];
    }
    out[2 * d] = running_cost(P, gam, p, s);
}

/* Vector-Jacobian product of `field`: given weights a (2d entries, on the
 * state rows) and b (on the quadrature row), return
 *     r = a^T d(field_z)/dz + b d(field_Q)/dz     (2d entries).
 * The Jacobians are written out per family from the formulas above. */
static void field_vjp(const orc_problem *P, const double *z, double s, const double *a, double b, double *r)
{
    int d = P->d;
    const double *gam = z, *p = z + d;
    const double *ag = a, *ap = a + d;
    double *rg = r, *rp = r + d;
    switch (P->family) {
    case FAM_QUAD_ISO:
        /* field = (-p, 0, |p|^2/2) for both principles */
        for (int i = 0; i < d; ++i) { rg[i] = 0.0; rp[i] = -ag[i] + b * p[i]; }
        return;
    case FAM_SPEED_QUAD: {
        double u, c, c1, c2;
        speed(P, gam, &u, &c, &c1, &c2);
        double A = dot(ag, p, d), Bw = dot(ap, P->w, d), pp = dot(p, p, d);
        /* field_gamma = -c^2 p, field_p = c c' |p|^2 w
         * Lax L = c^2 |p|^2 / 2 ; Hopf L = c^2|p|^2/2 - c c' |p|^2 u */
        double dE_du = -2.0 * c * c1 * A + (c1 * c1 + c * c2) * pp * Bw;
        if (P->principle == LAX) dE_du += b * c * c1 * pp;
        else dE_du += b * (-(c1 * c1 + c * c2) * pp * u);
        for (int i = 0; i < d; ++i) {
            rg[i] = dE_du * P->w[i];
            double dLdp = (P->principle == LAX) ? c * c * p[i] : (c * c - 2.0 * c * c1 * u) * p[i];
            rp[i] = -c * c * ag[i] + 2.0 * c * c1 * Bw * p[i] + b * dLdp;
        }
        return;
    }
    case FAM_SMOOTH_NONCONVEX: {
        double u, c, c1, c2;
        speed(P, gam, &u, &c, &c1, &c2);
        double phi = 0.0, A = 0.0, pdphi = 0.0;
        for (int i = 0; i < d; ++i) {
            double s = sqrt(p[i] * p[i] + P->s_eps);
            double dphi = sgn_of(P, i) * p[i] / s;
            phi += sgn_of(P, i) * s;
            A += ag[i] * dphi;
            pdphi += p[i] * dphi;
        }
        double Bw = dot(ap, P->w, d);
        /* field_gamma = -c Phi'(p), field_p = Phi c' w
         * Lax L = c (<p,Phi'> - Phi) ; Hopf L = Phi (c - c' u) */
        double dE_du = -c1 * A + phi * c2 * Bw;
        if (P->principle == LAX) dE_du += b * c1 * (pdphi - phi);
        else dE_du += b * (-phi * c2 * u);
        for (int i = 0; i < d; ++i) {
            double s = sqrt(p[i] * p[i] + P->s_eps);
            double dphi = sgn_of(P, i) * p[i] / s;
            double ddphi = sgn_of(P, i) * P->s_eps / (s * s * s);
            double dLdp = (P->principle == LAX) ? c * p[i] * ddphi : dphi * (c - c1 * u);
            rg[i] = dE_du * P->w[i];
            rp[i] = -c * ag[i] * ddphi + dphi * c1 * Bw + b * dLdp;
        }
        return;
    }
    case FAM_LINEAR_QUAD: {
        /* field_gamma = -(A gamma + B B^T p), field_p = A^T p, L = |B^T p|^2/2 */
        int m = P->m;
        double btag[ORC_MMAX], btp[ORC_MMAX];
        for (int k = 0; k < m; ++k) {
            btag[k] = 0.0; btp[k] = 0.0;
            for (int i = 0; i < d; ++i) {
                btag[k] += P->B[i * m + k] * ag[i];
                btp[k] += P->B[i * m + k] * p[i];
            }
        }
        for (int i = 0; i < d; ++i) {
            double atag = 0.0, aap = 0.0, bb = 0.0;
            for (int j = 0; j < d; ++j) {
                atag += P->A[j * d + i] * ag[j];
                aap += P->A[i * d + j] * ap[j];
            }
            for (int k = 0; k < m; ++k) bb += P->B[i * m + k] * (-btag[k] + b * btp[k]);
            rg[i] = -atag;
            rp[i] = aap + bb;
        }
        return;
    }
    case FAM_BUMP_NORM: {
        /* field_gamma = -S c p/n, field_p = S n k y with y = gamma - xc,
         * n = |p|_eps, grad c = k y, grad k = -2 mu k y;
         * Lax L = S c (|p|^2/n - n) = -S c eps/n;
         * Hopf L = H - <H_x, gamma> = S n (c - k <y, gamma>) */
        double y[ORC_DMAX], c, k;
        bump(P, gam, y, &c, &k);
        const double S = P->hsign, eps = P->s_eps, mu = P->mu;
        double n = sqrt(dot(p, p, d) + eps);
        double Agp = dot(ag, p, d), Apy = dot(ap, y, d), yg = dot(y, gam, d);
        for (int i = 0; i < d; ++i) {
            /* d/dgamma of <ag, field_gamma> and <ap, field_p> */
            double g_i = -S * (Agp / n) * k * y[i] + S * n * (-2.0 * mu * k * Apy * y[i] + k * ap[i]);
            /* d/dp of the same */
            double p_i = -S * c * (ag[i] / n - Agp * p[i] / (n * n * n)) + S * k * Apy * p[i] / n;
            if (P->principle == LAX) {
                g_i += b * (-S * eps / n) * k * y[i];
                p_i += b * S * c * eps * p[i] / (n * n * n);
            } else {
                /* d<y,gamma>/dgamma = y + gamma */
                g_i += b * S * n * (k * y[i] + 2.0 * mu * k * yg * y[i] - k * (y[i] + gam[i]));
                p_i += b * S * (c - k * yg) * p[i] / n;
            }
            rg[i] = g_i;
            rp[i] = p_i;
        }
        return;
    }
    case FAM_LINEAR_GAME: {
        /* field = (M gamma - a p/n, -M p); Lax L = a (|p|^2/n - n) = -a eps/n,
         * Hopf L = H - <H_x, gamma> = a n (M diagonal) */
        const double a_s = game_speed(P, s), eps = P->s_eps;
        const double n = sqrt(dot(p, p, d) + eps), Agp = dot(ag, p, d);
        for (int i = 0; i < d; ++i) {
            rg[i] = ag[i] * P->w[i];
            rp[i] = -a_s * (ag[i] / n - Agp * p[i] / (n * n * n)) - ap[i] * P->w[i];
            if (P->principle == LAX) rp[i] += b * a_s * eps * p[i] / (n * n * n);
            else rp[i] += b * a_s * p[i] / n;
        }
        return;
    }
    case FAM_HARMONIC: {
        /* field = (-S p, S gamma), Lax and Hopf L = S (|p|^2 - |gamma|^2)/2 */
        const double S = P->hsign;
        for (int i = 0; i < d; ++i) {
            rg[i] = S * ap[i] - b * S * gam[i];
            rp[i] = -S * ag[i] + b * S * p[i];
        }
        return;
    }
    case FAM_EVANS: {
        /* field_gamma = c e_1 - beta p_2/s_2 e_2 + p/n, field_p = -p_1 k y
         * (c, k including alpha); grad c = k y, grad k = -2 mu k y;
         * Lax L = <p,H_p> - H = gamma0 - beta eps/s_2 + eps/n;
         * Hopf L = H - <H_x, gamma> = H + p_1 k <y, gamma> */
        double y[ORC_DMAX], c, k;
        bump(P, gam, y, &c, &k);
        c *= P->alpha_a;
        k *= P->alpha_a;
        const double eps = P->s_eps, mu = P->mu, beta = P->beta;
        const double n = sqrt(dot(p, p, d) + eps), s2 = sqrt(p[1] * p[1] + eps);
        const double Agp = dot(ag, p, d), Apy = dot(ap, y, d), yg = dot(y, gam, d);
        for (int i = 0; i < d; ++i) {
            /* d/dgamma: ag_1 grad c, and -p_1 (grad k <ap,y> + k ap) */
            double g_i = ag[0] * k * y[i] + 2.0 * mu * p[0] * k * Apy * y[i] - p[0] * k * ap[i];
            /* d/dp: ag/n - <ag,p> p/n^3 (- beta eps/s_2^3 ag_2 on p_2), -k <ap,y> on p_1 */
            double p_i = ag[i] / n - Agp * p[i] / (n * n * n);
            if (P->principle == LAX) {
                p_i += b * (-eps * p[i] / (n * n * n));
            } else {
                g_i += b * p[0] * k * (gam[i] - 2.0 * mu * yg * y[i]);
                p_i += b * (-p[i] / n);
            }
            rg[i] = g_i;
            rp[i] = p_i;
        }
        rp[0] += -k * Apy;
        rp[1] += -beta * eps / (s2 * s2 * s2) * ag[1];
        if (P->principle == LAX) {
            rp[1] += b * beta * eps * p[1] / (s2 * s2 * s2);
        } else {
            rp[0] += b * (-c + k * yg);
            rp[1] += b * beta * p[1] / s2;
        }
        return;
    }
    case FAM_SPLIT_NORM: {
        /* each block contributes the bump-norm terms with S c -> c_blk:
         * field_gamma on the block = -c_blk p_blk/n_blk, field_p = sum_blk n_blk k_blk y_blk,
         * Lax L = -eps sum_blk c_blk/n_blk, Hopf L = sum_blk n_blk (c_blk - k_blk <y_blk, gamma>) */
        split_t S;
        split_eval(P, gam, p, &S);
        const double eps = P->s_eps, mu = P->mu;
        double Agp[2] = { 0.0, 0.0 }, Apy[2], yg[2];
        for (int i = 0; i < d; ++i) Agp[block_of(P, i)] += ag[i] * p[i];
        for (int bl = 0; bl < 2; ++bl) {
            Apy[bl] = dot(ap, S.y[bl], d);
            yg[bl] = dot(S.y[bl], gam, d);
        }
        for (int i = 0; i < d; ++i) {
            double g_i = 0.0;
            for (int bl = 0; bl < 2; ++bl) {
                if (S.n[bl] == 0.0) continue; /* empty block */
                const double n = S.n[bl], k = S.k[bl], y = S.y[bl][i];
                g_i += -(Agp[bl] / n) * k * y + n * (-2.0 * mu * k * Apy[bl] * y + k * ap[i]);
                if (P->principle == LAX) g_i += b * (-eps / n) * k * y;
                else g_i += b * n * (2.0 * mu * k * yg[bl] * y - k * gam[i]);
            }
            const int bi = block_of(P, i);
            const double n = S.n[bi], c = S.c[bi], k = S.k[bi];
            double p_i = -c * (ag[i] / n - Agp[bi] * p[i] / (n * n * n)) + k * Apy[bi] * p[i] / n;
            if (P->principle == LAX) p_i += b * c * eps * p[i] / (n * n * n);
            else p_i += b * (c - k * yg[bi]) * p[i] / n;
            rg[i] = g_i;
            rp[i] = p_i;
        }
        return;
    }
    }
}

/* Initial data g, its gradient, its Legendre transform g* and grad g*. */
static double g_val(const orc_problem *P, const double *x)
{
    if (P->g_kind == G_ROSENBROCK) {
        double a = 1.0 - x[0], b = 1.0 + x[1] - x[0] * x[0];
        return 4e-4 * (-100.0 + a * a + 100.0 * b * b);
    }
    double s = (P->g_kind == G_ELLIPSE) ? -0.5 : 0.0;
    for (int i = 0; i < P->d; ++i) {
        if (P->g_kind == G_QUAD_SHIFT) {
            double a = P->ga ? P->ga[i] : 0.0;
            s += 0.5 * (x[i] - a) * (x[i] - a);
        } else {
            s += 0.5 * x[i] * x[i] / (P->gs[i] * P->gs[i]);
        }
    }
    return s;
}
static void g_grad(const orc_problem *P, const double *x, double *out)
{
    if (P->g_kind == G_ROSENBROCK) {
        double a = 1.0 - x[0], b = 1.0 + x[1] - x[0] * x[0];
        out[0] = 4e-4 * (-2.0 * a - 400.0 * b * x[0]);
        out[1] = 4e-4 * 200.0 * b;
        return;
    }
    for (int i = 0; i < P->d; ++i)
        out[i] = (P->g_kind == G_QUAD_SHIFT) ? x[i] - (P->ga ? P->ga[i] : 0.0) : x[i] / (P->gs[i] * P->gs[i]);
}
static double gstar_val(const orc_problem *P, const double *p)
{
    if (P->g_kind == G_ROSENBROCK) return NAN; /* not convex: no transform */
    /* the ellipse data's constant -1/2 becomes +1/2 in the transform */
    double s = (P->g_kind == G_ELLIPSE) ? 0.5 : 0.0;
    for (int i = 0; i < P->d; ++i) {
        if (P->g_kind == G_QUAD_SHIFT) s += 0.5 * p[i] * p[i] + (P->ga ? P->ga[i] : 0.0) * p[i];
        else s += 0.5 * P->gs[i] * P->gs[i] * p[i] * p[i];
    }
    return s;
}
static void gstar_grad(const orc_problem *P, const double *p, double *out)
{
    for (int i = 0; i < P->d; ++i)
        out[i] = (P->g_kind == G_QUAD_SHIFT) ? p[i] + (P->ga ? P->ga[i] : 0.0) : P->gs[i] * P->gs[i] * p[i];
}

/* ------------------------------------------------------------------------ */
/* Functional evaluation (Sec. 4.1 functionals F^1 and G; Sec. 4.2 solver and */
/* quadrature).                                                              */
/* ------------------------------------------------------------------------ */

/* Integrate from s = t (tau = 0) to s = 0 (tau = t) in N RK4 steps.  The
 * trajectory z_n (n = 0..N, tau_n = n t/N) and, for the adjoint, the four
 * stage inputs of every step are written when the buffers are non-NULL.
 * Returns the quadrature of the running cost over [0, t]. */
static double integrate(const orc_problem *P, int quad, const double *x, double t, int N, const double *v,
                        double *traj /* [(N+1)*2d] */, double *stages /* [N*4*2d] */)
{
    int d = P->d, n2 = 2 * d;
    double h = t / N;
    double z[2 * ORC_DMAX + 1], zs[2 * ORC_DMAX + 1];
    double k1[2 * ORC_DMAX + 1], k2[2 * ORC_DMAX + 1], k3[2 * ORC_DMAX + 1], k4[2 * ORC_DMAX + 1];
    const int euler = quad & ODE_EULER;
    quad &= ~ODE_EULER;
    for (int i = 0; i < d; ++i) { z[i] = x[i]; z[d + i] = v[i]; }
    double Q = 0.0;
    if (traj) memcpy(traj, z, sizeof(double) * n2);
    if (euler) {
        /* forward Euler, z_{n+1} = z_n + h f(z_n); the Euler step of the
         * augmented state adds h L(z_n), the rectangle rule h L(z_{n+1}) */
        for (int n = 0; n < N; ++n) {
            if (stages) memcpy(stages + (size_t)(4 * n) * n2, z, sizeof(double) * n2);
            field(P, z, t - n * h, k1);
            for (int i = 0; i < n2; ++i) z[i] += h * k1[i];
            if (quad == QUAD_RK4) Q += h * k1[n2];
            else Q += h * running_cost(P, z, z + d, t - (n + 1) * h);
            if (traj) memcpy(traj + (size_t)(n + 1) * n2, z, sizeof(double) * n2);
        }
        return Q;
    }
    for (int n = 0; n < N; ++n) {
        if (stages) memcpy(stages + (size_t)(4 * n + 0) * n2, z, sizeof(double) * n2);
        /* stage times in the PDE's own time s = t - tau */
        const double s0 = t - n * h, sm = t - (n + 0.5) * h, s1 = t - (n + 1) * h;
        field(P, z, s0, k1);
        for (int i = 0; i < n2; ++i) zs[i] = z[i] + 0.5 * h * k1[i];
        if (stages) memcpy(stages + (size_t)(4 * n + 1) * n2, zs, sizeof(double) * n2);
        field(P, zs, sm, k2);
        for (int i = 0; i < n2; ++i) zs[i] = z[i] + 0.5 * h * k2[i];
        if (stages) memcpy(stages + (size_t)(4 * n + 2) * n2, zs, sizeof(double) * n2);
        field(P, zs, sm, k3);
        for (int i = 0; i < n2; ++i) zs[i] = z[i] + h * k3[i];
        if (stages) memcpy(stages + (size_t)(4 * n + 3) * n2, zs, sizeof(double) * n2);
        field(P, zs, s1, k4);
        for (int i = 0; i < n2; ++i) z[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        if (quad == QUAD_RK4) {
            /* RK4 on the augmented quadrature state */
            Q += h / 6.0 * (k1[n2] + 2.0 * k2[n2] + 2.0 * k3[n2] + k4[n2]);
        } else {
            /* eq. num_int: rectangle rule on the solver's mesh.  The node
             * s_i = i ds (i = 0..N-1) is the state after N - i steps of
             * reversed time, i.e. the states z_1..z_N reached here. */
            Q += h * running_cost(P, z, z + d, s1);
        }
        if (traj) memcpy(traj + (size_t)(n + 1) * n2, z, sizeof(double) * n2);
    }
    return Q;
}

/* F^1 (Lax) = g(gamma(0)) + int_0^t (<p, H_p> - H) ds;
 * G (Hopf)  = g*(p(0)) + int_0^t (H - <H_x, gamma>) ds - <x, v>.
 * gamma0, p0 may be NULL. */
/* Node of the smallest g(gamma_n), n = 0..N (first one on ties). */
static int huygens_node(const orc_problem *P, const double *traj, int N)
{
    int best = 0;
    double gb = g_val(P, traj);
    for (int n = 1; n <= N; ++n) {
        double gn = g_val(P, traj + (size_t)n * 2 * P->d);
        if (gn < gb) { gb = gn; best = n; }
    }
    return best;
}

double orc_functional(const orc_problem *P, int quad, const double *x, double t, int N, const double *v,
                      double *gamma0, double *p0)
{
    int d = P->d, n2 = 2 * d;
    double *traj = (double *)malloc(sizeof(double) * (size_t)(N + 1) * n2);
    double Q = integrate(P, quad, x, t, N, v, traj, NULL);
    const double *zN = traj + (size_t)N * n2; /* (gamma(0), p(0)) */
    double F;
    if (P->principle == HUYGENS) {
        /* eq. num_min: the grid node n = r/dt after n steps holds
         * (gamma(x,v,r,0), p(x,v,r,0)); the first smallest g wins, and its
         * node is the one reported (and certified) */
        int ns = huygens_node(P, traj, N);
        zN = traj + (size_t)ns * n2;
        F = g_val(P, zN);
    } else {
        F = (P->principle == LAX) ? g_val(P, zN) + Q : gstar_val(P, zN + d) + Q - dot(x, v, d);
    }
    if (gamma0) memcpy(gamma0, zN, sizeof(double) * d);
    if (p0) memcpy(p0, zN + d, sizeof(double) * d);
    free(traj);
    return F;
}

/* Exact gradient of the discretised functional with respect to v: the
 * discrete adjoint of the RK4 map (reverse accumulation through the four
 * stages of every step; all stage inputs are stored).  Returns F. */
double orc_gradient(const orc_problem *P, int quad, const double *x, double t, int N, const double *v,
                    double *grad)
{
    int d = P->d, n2 = 2 * d;
    double h = t / N;
    double *traj = (double *)malloc(sizeof(double) * (size_t)(N + 1) * n2);
    double *stages = (double *)malloc(sizeof(double) * (size_t)N * 4 * n2);
    double lam[2 * ORC_DMAX], a1[2 * ORC_DMAX], a2[2 * ORC_DMAX], a3[2 * ORC_DMAX], a4[2 * ORC_DMAX];
    double w[2 * ORC_DMAX];
    double Q = integrate(P, quad, x, t, N, v, traj, stages);
    const double *zN = traj + (size_t)N * n2;
    double F;
    /* adjoint of the terminal term; for F^2 the seed grad g enters at the
     * minimising node ns instead (no running cost) */
    int ns = N;
    for (int i = 0; i < n2; ++i) lam[i] = 0.0;
    if (P->principle == HUYGENS) {
        ns = huygens_node(P, traj, N);
        F = g_val(P, traj + (size_t)ns * n2);
    } else if (P->principle == LAX) {
        F = g_val(P, zN) + Q;
        g_grad(P, zN, lam);
    } else {
        F = gstar_val(P, zN + d) + Q - dot(x, v, d);
        gstar_grad(P, zN + d, lam + d);
    }
    const int euler = quad & ODE_EULER;
    quad &= ~ODE_EULER;
    double beta_q = (quad == QUAD_RK4) ? 1.0 : 0.0; /* dF/dQ flows through the stages only for RK4 quadrature */
    if (P->principle == HUYGENS) {
        beta_q = 0.0;
        quad = QUAD_RK4; /* no rectangle nodes either */
    }
    for (int n = N - 1; n >= 0; --n) {
        const double *Z1 = stages + (size_t)(4 * n + 0) * n2, *Z2 = Z1 + n2, *Z3 = Z2 + n2, *Z4 = Z3 + n2;
        if (P->principle == HUYGENS && n + 1 == ns) {
            double gs[2 * ORC_DMAX];
            g_grad(P, traj + (size_t)ns * n2, gs);
            for (int i = 0; i < d; ++i) lam[i] += gs[i];
        }
        if (euler) {
            /* z_{n+1} = z_n + h f(z_n) (and Q += h L(z_n)); reverse:
             * lam_n = lam_{n+1} + h J(z_n)^T lam_{n+1} + h beta dL/dz(z_n),
             * after the rectangle node at z_{n+1} when that rule is used */
            if (quad == QUAD_RECT) {
                double gl[2 * ORC_DMAX], zero[2 * ORC_DMAX];
                for (int i = 0; i < n2; ++i) zero[i] = 0.0;
                field_vjp(P, traj + (size_t)(n + 1) * n2, t - (n + 1) * h, zero, 1.0, gl);
                for (int i = 0; i < n2; ++i) lam[i] += h * gl[i];
            }
            for (int i = 0; i < n2; ++i) w[i] = h * lam[i];
            field_vjp(P, Z1, t - n * h, w, beta_q * h, a1);
            for (int i = 0; i < n2; ++i) lam[i] += a1[i];
            continue;
        }
        if (quad == QUAD_RECT) {
            /* rectangle node at the state after step n, weight h: add h grad L */
            double gl[2 * ORC_DMAX], zero[2 * ORC_DMAX];
            for (int i = 0; i < n2; ++i) zero[i] = 0.0;
            field_vjp(P, traj + (size_t)(n + 1) * n2, t - (n + 1) * h, zero, 1.0, gl);
            for (int i = 0; i < n2; ++i) lam[i] += h * gl[i];
        }
        /* z_{n+1} = z_n + h/6 (k1 + 2k2 + 2k3 + k4), Q likewise; reverse
         * (each stage at its own time, as in the forward step): */
        const double s0 = t - n * h, sm = t - (n + 0.5) * h, s1 = t - (n + 1) * h;
        for (int i = 0; i < n2; ++i) w[i] = h / 6.0 * lam[i];
        field_vjp(P, Z4, s1, w, beta_q * h / 6.0, a4);
        for (int i = 0; i < n2; ++i) w[i] = h / 3.0 * lam[i] + h * a4[i];
        field_vjp(P, Z3, sm, w, beta_q * h / 3.0, a3);
        for (int i = 0; i < n2; ++i) w[i] = h / 3.0 * lam[i] + 0.5 * h * a3[i];
        field_vjp(P, Z2, sm, w, beta_q * h / 3.0, a2);
        for (int i = 0; i < n2; ++i) w[i] = h / 6.0 * lam[i] + 0.5 * h * a2[i];
        field_vjp(P, Z1, s0, w, beta_q * h / 6.0, a1);
        for (int i = 0; i < n2; ++i) lam[i] += a1[i] + a2[i] + a3[i] + a4[i];
    }
    for (int i = 0; i < d; ++i) grad[i] = lam[d + i] - (P->principle == HOPF ? x[i] : 0.0);
    free(traj);
    free(stages);
    return F;
}

/* Finite-difference partial derivative along e_j (eq. num_diff; central form
 * when central != 0).  F0 is F(v), used by the forward form. */
static double fd_partial(const orc_problem *P, int quad, const double *x, double t, int N, double *v, int j,
                         double h, int central, double F0)
{
    double vj = v[j];
    v[j] = vj + h;
    double Fp = orc_functional(P, quad, x, t, N, v, NULL, NULL);
    double deriv;
    if (central) {
        v[j] = vj - h;
        double Fm = orc_functional(P, quad, x, t, N, v, NULL, NULL);
        deriv = (Fp - Fm) / (2.0 * h);
    } else {
        deriv = (Fp - F0) / h;
    }
    v[j] = vj;
    return deriv;
}

/* Central-difference full gradient (the plain definition of the derivative,
 * used to check the adjoint). */
void orc_gradient_fd(const orc_problem *P, int quad, const double *x, double t, int N, const double *v, double h,
                     double *grad)
{
    double *vv = (double *)malloc(sizeof(double) * (size_t)P->d);
    memcpy(vv, v, sizeof(double) * P->d);
    for (int j = 0; j < P->d; ++j) grad[j] = fd_partial(P, quad, x, t, N, vv, j, h, 1, 0.0);
    free(vv);
}

/* ------------------------------------------------------------------------ */
/* Descent (Sec. 4.1, Algorithm 1, and its gradient form).                  */
/* ------------------------------------------------------------------------ */

/* Algorithm 1, cyclic coordinate descent, read as follows.  alpha = step;
 * at iteration k the coordinate j_k = k mod d moves by alpha * dF/dv_j; a
 * move |dv_j| > eps resets the counter, a move |dv_j| < eps increments it
 * (both strict, as in steps 3-4; eps = 0 therefore never stops early), and
 * the descent stops when it reaches d (a full sweep of small moves);
 * every `halving_period` iterations alpha is halved; max_iters caps k.
 * Gradient form: every iteration moves all coordinates by alpha_i dF/dv_i
 * with the adjoint gradient; it stops after one iteration whose largest
 * move is < eps.
 * Per-coordinate step control (`adapt`, both forms): each coordinate keeps
 * its own alpha_i.  When its derivative changes sign between two
 * consecutive visits (an overshoot) alpha_i is multiplied by `shrink`; when
 * the sign is kept, by `grow` (capped at step_max).  This is a per-
 * coordinate trigger for Algorithm 1's "alpha := alpha/2"; the global
 * halving every `halving_period` iterations still applies on top.
 * Returns the number of iterations; *hit_cap is set when the cap stopped it. */
static int descend_cg(const orc_problem *P, const orc_opts *O, const double *x, double t, int N, double *v,
                      int *hit_cap, int *nonfinite);

int orc_descend(const orc_problem *P, const orc_opts *O, const double *x, double t, int N, double *v, int *hit_cap,
                int *nonfinite)
{
    int d = P->d;
    *hit_cap = 0;
    *nonfinite = 0;
    if (O->coarse_div > 1 && O->descent != DESC_CD) {
        /* continuation in the step size: the same descent, first on the
         * functional discretised with N / coarse_div steps (stopping at moves
         * < coarse_eps), then, with its step control started afresh, on the
         * functional with N steps from the point reached */
        orc_opts C = *O, F = *O;
        C.coarse_div = F.coarse_div = 1;
        C.eps = O->coarse_eps;
        int Nc = N / O->coarse_div;
        if (Nc < 1) Nc = 1;
        int cap1 = 0, nf1 = 0;
        int it1 = orc_descend(P, &C, x, t, Nc, v, &cap1, &nf1);
        if (nf1) { *nonfinite = 1; return it1; }
        int it2 = orc_descend(P, &F, x, t, N, v, hit_cap, nonfinite);
        return it1 + it2;
    }
    if (O->descent == DESC_CG) return descend_cg(P, O, x, t, N, v, hit_cap, nonfinite);
    if (O->descent == DESC_CD) {
        double alpha[ORC_DMAX], dprev[ORC_DMAX];
        for (int i = 0; i < d; ++i) { alpha[i] = O->step; dprev[i] = 0.0; }
        int count = 0, k_in_period = 0, it;
        for (it = 0; it < O->max_iters; ++it) {
            int j = it % d;
            double F0 = 0.0;
            if (O->grad == GRAD_FD_FORWARD) F0 = orc_functional(P, O->quad, x, t, N, v, NULL, NULL);
            double dj = fd_partial(P, O->quad, x, t, N, v, j, O->fd_h, O->grad != GRAD_FD_FORWARD, F0);
            if (O->adapt) {
                double prod = dj * dprev[j];
                if (prod < 0.0) alpha[j] *= O->shrink;
                else if (prod > 0.0) alpha[j] = fmin(alpha[j] * O->grow, O->step_max);
                dprev[j] = dj;
            }
            double step = alpha[j] * dj;
            if (!isfinite(step)) { *nonfinite = 1; return it + 1; }
            v[j] -= step;
            /* steps 3-4: reset on a move > eps, count a move < eps (strict) */
            if (fabs(step) > O->eps) count = 0;
            else if (fabs(step) < O->eps) count += 1;
            if (O->halving_period > 0 && ++k_in_period == O->halving_period) {
                k_in_period = 0;
                for (int i = 0; i < d; ++i) alpha[i] *= 0.5;
            }
            if (count >= d) return it + 1;
        }
        *hit_cap = 1;
        return it;
    } else {
        double *g = (double *)malloc(sizeof(double) * 3 * (size_t)d), *gprev = g + d, *alpha = gprev + d;
        for (int i = 0; i < d; ++i) { alpha[i] = O->step; gprev[i] = 0.0; }
        int it;
        for (it = 0; it < O->max_iters; ++it) {
            if (O->grad == GRAD_ADJOINT) orc_gradient(P, O->quad, x, t, N, v, g);
            else orc_gradient_fd(P, O->quad, x, t, N, v, O->fd_h, g);
            double big = 0.0;
            for (int i = 0; i < d; ++i) {
                if (O->adapt) {
                    double prod = g[i] * gprev[i];
                    if (prod < 0.0) alpha[i] *= O->shrink;
                    else if (prod > 0.0) alpha[i] = fmin(alpha[i] * O->grow, O->step_max);
                }
                double step = alpha[i] * g[i];
                if (!isfinite(step)) { *nonfinite = 1; free(g); return it + 1; }
                v[i] -= step;
                if (fabs(step) > big) big = fabs(step);
                gprev[i] = g[i];
            }
            if (O->halving_period > 0 && (it + 1) % O->halving_period == 0)
                for (int i = 0; i < d; ++i) alpha[i] *= 0.5;
            if (big < O->eps) { free(g); return it + 1; }
        }
        free(g);
        *hit_cap = 1;
        return it;
    }
}

/* Conjugate-gradient descent with the adjoint gradient (Sec. 5 remarks that
 * descent along long, flat trenches needs momentum; conjugate directions are
 * the momentum that is exact for quadratic functionals, such as the
 * linear-quadratic family's, where plain descent needs ~condition-number
 * iterations).  Polak-Ribiere+ directions with one secant line search per
 * iteration:
 *   g = grad F(v); dir = -g
 *   repeat (one iteration):
 *     n = max_i |dir_i|;  sigma = step / n           (probe: largest move = step)
 *     gp = grad F(v + sigma dir)
 *     s0 = <g, dir>, s1 = <gp, dir>, curv = (s1 - s0) / sigma
 *     alpha = -s0 / curv if curv > 0, else sigma;  alpha <= step_max / n
 *     v += alpha dir;  stop if alpha n < eps, or at max_iters
 *     gn = grad F(v);  beta = max(0, <gn, gn - g> / <g, g>)
 *     dir = -gn + beta dir;  dir = -gn if <gn, dir> >= 0;  g = gn
 * On a quadratic the secant slope is its exact curvature along dir, so this
 * is linear CG with exact line searches.  Returns the iteration count. */
static int descend_cg(const orc_problem *P, const orc_opts *O, const double *x, double t, int N, double *v,
                      int *hit_cap, int *nonfinite)
{
    int d = P->d;
    double *g = (double *)malloc(sizeof(double) * 4 * (size_t)d), *dir = g + d, *gp = dir + d, *u = gp + d;
    orc_gradient(P, O->quad, x, t, N, v, g);
    for (int i = 0; i < d; ++i) dir[i] = -g[i];
    int it = 0;
    while (it < O->max_iters) {
        double n = 0.0;
        for (int i = 0; i < d; ++i) n = fmax(n, fabs(dir[i]));
        if (!isfinite(n)) { *nonfinite = 1; free(g); return it; }
        if (n == 0.0) { free(g); return it; }
        double sigma = O->step / n;
        for (int i = 0; i < d; ++i) u[i] = v[i] + sigma * dir[i];
        orc_gradient(P, O->quad, x, t, N, u, gp);
        double s0 = dot(g, dir, d), s1 = dot(gp, dir, d);
        double curv = (s1 - s0) / sigma;
        double alpha = (curv > 0.0) ? -s0 / curv : sigma;
        if (alpha > O->step_max / n) alpha = O->step_max / n;
        if (!isfinite(alpha)) { *nonfinite = 1; free(g); return it + 1; }
        for (int i = 0; i < d; ++i) v[i] += alpha * dir[i];
        ++it;
        if (alpha * n < O->eps) { free(g); return it; }
        if (it >= O->max_iters) break;
        orc_gradient(P, O->quad, x, t, N, v, gp);
        double gg = dot(g, g, d), gy = 0.0;
        for (int i = 0; i < d; ++i) gy += gp[i] * (gp[i] - g[i]);
        double beta = (gg > 0.0) ? fmax(0.0, gy / gg) : 0.0;
        for (int i = 0; i < d; ++i) dir[i] = -gp[i] + beta * dir[i];
        if (dot(gp, dir, d) >= 0.0)
            for (int i = 0; i < d; ++i) dir[i] = -gp[i];
        memcpy(g, gp, sizeof(double) * d);
    }
    free(g);
    *hit_cap = 1;
    return it;
}

/* ------------------------------------------------------------------------ */
/* Certificate (Sec. 4.3): p(0) in dg(gamma(0)).  Lax: residual             */
/* |p(0) - grad g(gamma(0))| / (1 + |p(0)|); Hopf (g convex, so the inclusion */
/* is gamma(0) = grad g*(p(0))): |gamma(0) - grad g*(p(0))| / (1 + |gamma(0)|). */
/* Also returns the FP64 functional value at v.                              */
/* ------------------------------------------------------------------------ */
double orc_certify(const orc_problem *P, int quad, const double *x, double t, int N, const double *v,
                   double *residual)
{
    int d = P->d;
    double *g0 = (double *)malloc(sizeof(double) * 3 * (size_t)d), *p0 = g0 + d, *gr = p0 + d;
    double F = orc_functional(P, quad, x, t, N, v, g0, p0);
    double num = 0.0, den = 0.0;
    if (P->principle != HOPF) { /* F^2: the Lax test at the minimising node */
        g_grad(P, g0, gr);
        for (int i = 0; i < d; ++i) { num += (p0[i] - gr[i]) * (p0[i] - gr[i]); den += p0[i] * p0[i]; }
    } else {
        gstar_grad(P, p0, gr);
        for (int i = 0; i < d; ++i) { num += (g0[i] - gr[i]) * (g0[i] - gr[i]); den += g0[i] * g0[i]; }
    }
    *residual = sqrt(num) / (1.0 + sqrt(den));
    free(g0);
    return F;
}

/* ------------------------------------------------------------------------ */
/* One query: guesses, descent, certificate, reseeding of failed starts and  */
/* best-of-guesses (Sec. 4.3 and Sec. 5).                                    */
/*                                                                          */
/* Trial g < n_guesses is slot g from Philox draw (q, g, 0).  When           */
/* max_rounds >= 1 and some of them fail the certificate, the rest of the    */
/* query's budget of max_trials independent trials (Sec. 5) is spent at      */
/* once: restart j in [0, max_trials - n_guesses) draws (q, S[j mod |S|],    */
/* 1 + j / |S|), S the failed slots in slot order.  The answer is the        */
/* certified trial with the smallest FP64 functional value (ties: the lowest */
/* trial), with no certified trial the smallest over all trials.  Lax:       */
/* phi = F^1; Hopf: phi = -G.                                                */
/*                                                                          */
/* Per-trial diagnostics (may be NULL), each [orc_trials(O)] (trials that   */
/* did not run are left untouched): functional, residual, pass flag,         */
/* iterations, round and slot of the draw, and the final v ([trials * d]).   */
/* ------------------------------------------------------------------------ */
int orc_trials(const orc_opts *O)
{
    const int G = O->n_guesses;
    return G + ((O->max_rounds >= 1 && O->max_trials > G) ? O->max_trials - G : 0);
}

int orc_solve_query(const orc_problem *P, const orc_opts *O, int64_t q, const double *x, double t, int N,
                    double *phi, double *vstar, double *slot_F, double *slot_res, int *slot_pass, int *slot_iters,
                    int *slot_round, double *slot_v, int *slot_slot)
{
    const int d = P->d, G = O->n_guesses, T = orc_trials(O);
    double *V = (double *)malloc(sizeof(double) * (size_t)T * d);
    double *F = (double *)malloc(sizeof(double) * (size_t)T * 2), *R = F + T;
    int *pass = (int *)malloc(sizeof(int) * (size_t)T * 6), *iters = pass + T, *round = iters + T, *cap = round + T,
        *slot = cap + T, *failed = slot + T;
    int any_nonfinite = 0, reseeded = 0, nt = 0;
    /* trial nt: slot s, round r */
#define RUN_TRIAL(s, r)                                                                \
    do {                                                                               \
        double *v_ = V + (size_t)nt * d;                                               \
        int nf_;                                                                       \
        orc_guess(O->seed, q, (s), (r), d, O->guess_dist, v_);                        \
        iters[nt] = orc_descend(P, O, x, t, N, v_, &cap[nt], &nf_);                   \
        any_nonfinite |= nf_;                                                          \
        F[nt] = orc_certify(P, O->quad, x, t, N, v_, &R[nt]);                         \
        pass[nt] = (R[nt] <= O->cert_tol) && isfinite(F[nt]);                         \
        round[nt] = (r);                                                               \
        slot[nt] = (s);                                                                \
        ++nt;                                                                          \
    } while (0)
    for (int g = 0; g < G; ++g) RUN_TRIAL(g, 0);
    int nfail = 0;
    for (int g = 0; g < G; ++g)
        if (!pass[g]) failed[nfail++] = g;
    if (nfail > 0)
        for (int j = 0; G + j < T; ++j) {
            RUN_TRIAL(failed[j % nfail], 1 + j / nfail);
            reseeded = 1;
        }
#undef RUN_TRIAL
    int best = -1, best_cert = 0;
    for (int g = 0; g < nt; ++g) {
        if (!isfinite(F[g])) continue;
        if (pass[g] && !best_cert) { best = g; best_cert = 1; continue; }
        if (pass[g] != best_cert) continue;
        if (best < 0 || F[g] < F[best]) best = g;
    }
    int status = 0;
    if (best >= 0) {
        *phi = (P->principle == HOPF) ? -F[best] : F[best];
        memcpy(vstar, V + (size_t)best * d, sizeof(double) * d);
        if (best_cert) status |= ST_CERTIFIED;
        if (cap[best]) status |= ST_MAX_ITERS;
    } else {
        *phi = NAN;
        for (int i = 0; i < d; ++i) vstar[i] = NAN;
        status |= ST_NONFINITE;
    }
    if (any_nonfinite) status |= ST_NONFINITE;
    if (reseeded) status |= ST_RESEEDED;
    for (int g = 0; g < nt; ++g) {
        if (slot_F) slot_F[g] = F[g];
        if (slot_res) slot_res[g] = R[g];
        if (slot_pass) slot_pass[g] = pass[g];
        if (slot_iters) slot_iters[g] = iters[g];
        if (slot_round) slot_round[g] = round[g];
        if (slot_slot) slot_slot[g] = slot[g];
        if (slot_v) memcpy(slot_v + (size_t)g * d, V + (size_t)g * d, sizeof(double) * d);
    }
    free(V);
    free(F);
    free(pass);
    return status;
}
