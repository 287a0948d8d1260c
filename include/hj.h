/*
 * hj.h -- C ABI of the GB300 (sm_103a) solver for state-dependent
 * Hamilton-Jacobi equations by the generalized Lax minimisation and Hopf
 * maximisation principles of Chow, Darbon, Osher and Yin (arXiv 1704.02524).
 *
 * The equation is phi_t + H(x, grad phi, t) = 0, phi(x, 0) = g(x) (Sec. 2.1).
 * For a query (x, t) and a vector v the library integrates the
 * bi-characteristics (Sec. 4.1)
 *      d gamma/ds = dH/dp(gamma, p, s),  dp/ds = -dH/dx(gamma, p, s),
 *      gamma(t) = x,  p(t) = v,
 * backward from s = t to s = 0 with N classical RK4 steps (or N forward
 * Euler steps, HJ_ODE_EULER), and evaluates
 *   Lax  (convex H, eq. lax_formula):
 *      F(v) = g(gamma(0)) + int_0^t ( <p, dH/dp> - H ) ds,       phi = min_v F
 *   Hopf (g convex, eq. hopf_formula):
 *      G(v) = g*(p(0)) + int_0^t ( H - <dH/dx, gamma> ) ds - <x, v>,
 *                                                                phi = -min_v G
 *   Huygens (H of degree one in p, eq. num_min): the smallest g(gamma) over
 *      the solver's grid nodes, phi = min_v of it (see hj_principle).
 * It minimises over v by the paper's cyclic coordinate descent with
 * finite differences (Algorithm 1, eq. num_diff), by gradient descent with
 * the exact gradient of the discretised functional (discrete adjoint of
 * the integrator), or by conjugate gradients with that gradient, checks the
 * certificate p(0) in dg(gamma(0)) (Sec. 4.3), reseeds failed starts and
 * keeps the best of several random guesses (Sec. 5).
 *
 * Conventions for every entry point below
 *  - Array arguments are DEVICE pointers owned by the caller, contiguous,
 *    row-major, on the context's device, unless a comment says "host".
 *  - Element type of x, t, v, F, grad: float when opts.precision is
 *    HJ_PREC_FP32, double when HJ_PREC_FP64.  phi, residuals: double.
 *  - Vectors of a query are rows of length ld = the largest d over the
 *    context's problems; a row of a problem with smaller d uses its first d
 *    entries (the rest is ignored on input and left untouched on output).
 *  - problem_idx (int32 [n], nullable = all 0) selects the problem of each
 *    row (a row whose index is outside [0, n problems) is skipped: its
 *    outputs are left untouched, or for hj_solve phi = NaN and status
 *    HJ_ST_NONFINITE); n_steps (int32 [n], nullable = opts.n_steps_default)
 *    its integrator step count N.  t must be > 0, N in [1, 256] (other step counts
 *    give NaN results).
 *  - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  Argument errors are detected on the host and
 *    returned before anything is enqueued; the message is available from
 *    hj_last_error().  Non-convergence is reported per query in the status
 *    bits, never by trapping.
 *  - A context is not thread safe: serialise calls that share one.
 */
#ifndef HJ_H
#define HJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hj_ctx hj_ctx;

typedef enum {
    HJ_OK = 0,
    HJ_EINVAL = 1,        /* invalid argument (message in hj_last_error)        */
    HJ_ENOMEM = 2,        /* device or host allocation failed                   */
    HJ_ECUDA = 3,         /* a CUDA call failed                                 */
    HJ_ETIMEOUT = 4,      /* reserved: a bounded device wait ran out            */
    HJ_EUNSUPPORTED = 5   /* combination not built into this library            */
} hj_status;

/* Hamiltonian families (per-family parameters in hj_problem_desc.params). */
typedef enum {
    HJ_FAM_QUAD_ISO = 0,         /* H = |p|^2/2                                              */
    HJ_FAM_SPEED_QUAD = 1,       /* H = c(x)^2 |p|^2/2,  c = 1 + sin(<w,x>)/2                 */
    HJ_FAM_SMOOTH_NONCONVEX = 2, /* H = c(x) sum_i e_i s(p_i), s(q) = sqrt(q^2 + s_eps),
                                    e_i = -1 for i < n_neg, +1 otherwise                       */
    HJ_FAM_LINEAR_QUAD = 3,      /* H = <A x, p> + |B^T p|^2/2                               */
    HJ_FAM_BUMP_NORM = 4,        /* H = sign c(x) |p|_eps,  c = 1 + kappa exp(-mu |x - xc|^2),
                                    |p|_eps = sqrt(|p|^2 + s_eps) (Sec. 6, Example 3)        */
    HJ_FAM_SPLIT_NORM = 5,       /* H = c_A(x) |p_A|_eps + c_B(x) |p_B|_eps over the blocks
                                    A = coordinates [0, k), B = [k, d), with
                                    c_b = alpha_b (1 + kappa exp(-mu |x - xc_b|^2))
                                    (Sec. 6, Example 5; signs in the alphas)                */
    HJ_FAM_HARMONIC = 6,         /* H = sign (|p|^2 + |x|^2)/2 (Sec. 6, Example 2)          */
    HJ_FAM_EVANS = 7,            /* H = -c(x) p_1 + beta |p_2|_eps - |p|_eps - gamma0, d >= 2,
                                    c = alpha (1 + kappa exp(-mu |x - xc|^2))
                                    (Sec. 6, Example 4)                                      */
    HJ_FAM_LINEAR_GAME = 8       /* time dependent: H(x, p, s) = -<diag(m) x, p> + a(s) |p|_eps,
                                    a(s) = r_C - r_D (1 + beta sin(omega s)), s the PDE time
                                    (the linear differential game of Sec. 3.4, Example 3,
                                    with ball-shaped control sets)                           */
} hj_family;

/* Which functional is minimised over v (Sec. 4.1):
 *   HJ_LAX      F^1 = g(gamma(0)) + int_0^t (<p, H_p> - H) ds,  phi = min F^1;
 *   HJ_HOPF     G = g*(p(0)) + int_0^t (H - <H_x, gamma>) ds - <x, v>,  phi = -min G;
 *   HJ_HUYGENS  F^2 = min over 0 <= r <= t of g(gamma(x, v, r, 0)), taken on the
 *               solver grid r = n t/N, n = 0..N (eq. num_min; the first smallest
 *               node on ties), phi = min F^2 -- for Hamiltonians of degree one
 *               in p (the BUMP_NORM and SPLIT_NORM families, the only ones
 *               accepted with it);
 *               no running cost, the certificate is the Lax test at the
 *               minimising node, and the gradient is the adjoint seeded there. */
typedef enum { HJ_LAX = 0, HJ_HOPF = 1, HJ_HUYGENS = 2 } hj_principle;

/* Initial data g. */
typedef enum {
    HJ_G_QUAD_SHIFT = 0,  /* g = |x - a|^2/2,          g* = |p|^2/2 + <a,p>       */
    HJ_G_DIAG_QUAD = 1,   /* g = sum x_i^2/(2 s_i^2),  g* = sum s_i^2 p_i^2/2     */
    HJ_G_ELLIPSE = 2,     /* g = (sum x_i^2/s_i^2 - 1)/2, g* = (sum s_i^2 p_i^2 + 1)/2:
                             zero level set the ellipse <x, Ax> = 1 with
                             A = diag(1/s_i^2) (the initial data of Sec. 6)  */
    HJ_G_ROSENBROCK = 3   /* d = 2: g = 4e-4 (-100 + (1 - x_1)^2 + 100 (1 + x_2 - x_1^2)^2)
                             (Sec. 6, Example 2); not convex, so Lax and Huygens
                             only                                             */
} hj_initial;

typedef enum {
    HJ_GRAD_FD_CENTRAL = 0, /* cyclic coordinate descent, (F(v+he)-F(v-he))/2h            */
    HJ_GRAD_FD_FORWARD = 1, /* cyclic coordinate descent, (F(v+he)-F(v))/h  (eq. num_diff) */
    HJ_GRAD_ADJOINT = 2,    /* gradient descent with the discrete-adjoint gradient         */
    HJ_GRAD_ADJOINT_CG = 3  /* conjugate-gradient descent with the discrete-adjoint
                               gradient (the momentum Sec. 5 recommends when descent drags
                               along flat trenches; see hj_solver_opts)                     */
} hj_grad_mode;

/* Integrator and quadrature of the characteristic system (Sec. 4.2).  The
 * characteristics are integrated by N classical RK4 steps, or by N forward
 * Euler steps (Sec. 4.2's example solver) when HJ_ODE_EULER is or-ed into
 * the value (HJ_QUAD_RK4 | HJ_ODE_EULER: Euler on the augmented state, which
 * sums h L(z_n) at the left nodes; HJ_QUAD_RECT | HJ_ODE_EULER: Euler with
 * the rectangle rule).  The discrete adjoint follows the chosen integrator,
 * so gradients stay exact for the discretised functional. */
typedef enum {
    HJ_QUAD_RK4 = 0,  /* running cost integrated by the integrator on an augmented state */
    HJ_QUAD_RECT = 1, /* rectangle rule on the solver mesh, nodes s_i = i t/N, i<N       */
    HJ_ODE_EULER = 2  /* flag: forward Euler instead of RK4                              */
} hj_quad_mode;

typedef enum { HJ_PREC_FP32 = 0, HJ_PREC_FP64 = 1 } hj_precision;

/* Per-query status bits written by hj_solve. */
#define HJ_ST_CERTIFIED 1  /* the returned start passed the certificate           */
#define HJ_ST_MAX_ITERS 2  /* the returned start stopped at the iteration cap     */
#define HJ_ST_NONFINITE 4  /* some start produced a non-finite value              */
#define HJ_ST_RESEEDED 8   /* at least one failed start was restarted             */

/*
 * Solver constants.  Names follow Algorithm 1: step = alpha = 1/L; every
 * `halving_period` iterations alpha is halved (0: never); the descent stops
 * when every move of a full sweep is smaller than `eps` (coordinate descent:
 * d consecutive coordinate moves, a move larger than eps restarting the
 * count; gradient descent: one iteration; eps = 0 never stops early), or at
 * `max_iters` (coordinate descent counts coordinate moves, gradient descent
 * counts gradient steps).  With `adapt`, each coordinate keeps its own
 * alpha_i, multiplied by `shrink` when its derivative changes sign between
 * consecutive visits and by `grow` (capped at step_max) when it keeps it.
 * HJ_GRAD_ADJOINT_CG: Polak-Ribiere+ conjugate directions with one secant
 * line search per iteration: from the gradient g at v and dir (first
 * dir = -g), probe the gradient gp at v + sigma dir with sigma = step /
 * max|dir|, move v by alpha dir with alpha = -<g,dir> / ((<gp,dir> -
 * <g,dir>) / sigma) when that curvature is positive (else sigma), capped at
 * step_max / max|dir|; stop when alpha max|dir| < eps or at max_iters
 * (iterations, each two gradients); then dir = -gn + beta dir with
 * beta = max(0, <gn, gn - g> / <g, g>), restarted at -gn when it is not a
 * descent direction.  Exact line searches on quadratic functionals (the
 * linear-quadratic family), whose conditioning defeats plain gradient steps.
 * Round 0 of hj_solve runs n_guesses starts per query (Philox4x32-10 draws
 * keyed by `seed`, counter (component/4, slot | round<<16, query id)).
 * Reseeding (Sec. 4.3, Sec. 5: at most max_trials independent trials per
 * query): with max_rounds >= 1, a query some of whose starts failed the
 * certificate runs the rest of its budget, max_trials - n_guesses trials,
 * in one more round; restart j uses the draw (slot S[j mod |S|], round
 * 1 + j / |S|), S the failed slots in slot order.  max_rounds = 0 turns
 * reseeding off (values above 1 act as 1).  The answer is the best trial:
 * certified first, then the smallest functional, ties to the lowest trial
 * (starts in slot order, then restarts in order).
 * guess_dist: 0 = uniform on [-2,2]^d (Sec. 5), 1 = Irwin-Hall(12) N(0,1)
 * approximation.  cert_tol: certificate tolerance on the relative residual
 *   Lax  |p(0) - grad g(gamma(0))| / (1 + |p(0)|),
 *   Hopf |gamma(0) - grad g*(p(0))| / (1 + |gamma(0)|).
 * kahan: compensated summation of the running-cost quadrature.
 */
typedef struct {
    int n_steps_default;
    hj_quad_mode quad;
    hj_grad_mode grad;
    double fd_h;
    double step;
    int max_iters;
    int halving_period;
    double eps;
    int adapt;
    double grow;
    double shrink;
    double step_max;
    int n_guesses;
    int max_trials;
    int max_rounds;
    uint64_t seed;
    int guess_dist;
    double cert_tol;
    hj_precision precision;
    int kahan;
    int coarse_div;     /* gradient and CG descents: > 1 descends first on the
                           functional with N / coarse_div steps until every
                           move is < coarse_eps (or max_iters), then, with the
                           step control started afresh, on the N-step functional
                           from there (continuation in the step size; iterations
                           of both levels are counted); 1 = off                   */
    double coarse_eps;
} hj_solver_opts;

/*
 * One problem: a Hamiltonian family instance and its initial data.
 * params (HOST, double, copied by hj_create) holds, in order:
 *   family block:  SPEED_QUAD, SMOOTH_NONCONVEX: w[d]
 *                  LINEAR_QUAD: A[d*d] (row-major), then B[d*m] (row-major)
 *                  BUMP_NORM: xc[d], then kappa, mu (>= 0), sign (+1 or -1)
 *                  SPLIT_NORM: xc_A[d], xc_B[d], then k (integer in [0, d]), kappa,
 *                              mu (>= 0), alpha_A, alpha_B
 *                  HARMONIC: sign (+1 or -1)
 *                  EVANS: xc[d], then kappa, mu (>= 0), alpha, beta, gamma0
 *                  LINEAR_GAME: m[d] (the diagonal drift), then r_C, r_D, beta, omega
 *                  QUAD_ISO: nothing
 *   g block:       HJ_G_QUAD_SHIFT: a[d];  HJ_G_DIAG_QUAD, HJ_G_ELLIPSE: s[d] (all > 0);
 *                  HJ_G_ROSENBROCK: nothing
 * n_params must equal the total.  d in [1, 1024]; m in [1, 64] for
 * LINEAR_QUAD (d in [1, 128] there), else ignored.  LINEAR_QUAD computes
 * B B^T once in double precision at hj_create and integrates
 * d gamma/ds = A gamma + (B B^T) p, dp/ds = -A^T p with running cost
 * p^T (B B^T) p / 2 (the same for both principles).
 */
typedef struct {
    int d;
    hj_family family;
    hj_principle principle;
    hj_initial g_kind;
    int m;             /* LINEAR_QUAD: columns of B                             */
    int n_neg;         /* SMOOTH_NONCONVEX: number of leading negative signs     */
    double s_eps;      /* SMOOTH_NONCONVEX: smoothing of |q|, > 0;
                          BUMP_NORM, SPLIT_NORM, EVANS, LINEAR_GAME: smoothing of the norms,
                          >= 0 (0: the plain norms)                                */
    int n_guesses;     /* random starts per query for hj_solve (0: the solver value) */
    const double *params;
    size_t n_params;
    /* HOST, nullable, copied by hj_create: this problem's descent constants
     * (grad, fd_h, step, max_iters, halving_period, eps, adapt, grow, shrink,
     * step_max, n_guesses, max_trials, cert_tol); NULL takes the context's.
     * precision, quad, kahan, seed, guess_dist, n_steps_default and
     * max_rounds always come from the context's options. */
    const hj_solver_opts *solver;
} hj_problem_desc;


/* Counters and device timings of the last hj_solve on a context
 * (hj_last_solve_info); times come from CUDA events on the solve's stream. */
typedef struct {
    int64_t n_queries;
    int64_t n_pairs;            /* (query, trial) pairs run, restarts included     */
    int64_t iterations;         /* descent iterations summed over pairs             */
    int64_t functional_evals;   /* forward functional evaluations                   */
    int64_t gradient_evals;     /* adjoint gradients                                */
    int64_t rk4_steps;          /* integrator (RK4 or Euler) steps of all evaluations
                                   (forward sweeps)                                 */
    double algorithmic_flops;   /* fp32/fp64 arithmetic of the descent, FMA = 2     */
    double certify_flops;       /* arithmetic of the in-kernel certificate passes   */
    int threads_per_pair;       /* of the first problem's descent launch            */
    int comps_per_thread;
    int descent_launches;       /* rounds run (round 0 and, with reseeding, one
                                   reseed round; each one descent launch per problem) */
    double descent_ms;          /* device time of the descent launches (CUDA events) */
    double certify_ms;          /* device time of the certificate launches           */
    double total_ms;            /* device time of the whole hj_solve                 */
    int64_t kernel_launches;    /* kernels the library launched in the last hj_solve */
    double descent_ms_round0;   /* device time of the first round's descent launches */
    double tensor_flops;        /* tensor-core tile kernel: BF16 flops of its stage products,
                                   3 x 2 (3 d^2 + d m) per pair and RK4 stage (the fp32
                                   product, unpadded, times the three BF16x3 terms)       */
    int64_t adjoint_steps;      /* reverse integrator steps of all adjoint gradients       */
    double nominal_flops;       /* the descent launches' work at fixed per-evaluation counts
                                   of the general RK4 form: per forward step and pair 36d
                                   (H = |p|^2/2), 52d (c^2|p|^2/2), 64d (c Phi(p)),
                                   4(4d^2 + 4md) + 28d (linear-quadratic), the lane-group
                                   operation count for the other families; an adjoint
                                   gradient counts as four functional evaluations and the
                                   in-kernel certificate as one.  Independent of how the
                                   kernels arrange the arithmetic (the one-thread-per-pair
                                   kernels execute fewer operations than these counts)   */
} hj_solve_info;

/*
 * hj_create -- copy the problems and options to `cuda_device`, validate them
 * and return a context in *out.  The context owns its parameter copies and
 * its scratch memory; the caller owns every I/O buffer.
 * Errors: HJ_EINVAL (bad description; *out untouched), HJ_ENOMEM, HJ_ECUDA.
 */
hj_status hj_create(const hj_problem_desc *problems, int n_problems, const hj_solver_opts *opts,
                    int cuda_device, hj_ctx **out);

/* hj_destroy -- synchronise the device and free the context. */
hj_status hj_destroy(hj_ctx *ctx);

/*
 * hj_eval_functional -- F (Lax) or G (Hopf) of Sec. 4.1 at n (x, t, v):
 * x, v [n, ld], t [n], F_out [n].
 */
hj_status hj_eval_functional(hj_ctx *ctx, int64_t n, const int32_t *problem_idx, const void *x, const void *t,
                             const int32_t *n_steps, const void *v, void *F_out, void *stream);

/*
 * hj_grad -- F and its exact gradient dF/dv of the discretised functional
 * (discrete adjoint of the RK4 or Euler map with sqrt(N)-step checkpointing):
 * F_out [n] (nullable), grad_out [n, ld].
 */
hj_status hj_grad(hj_ctx *ctx, int64_t n, const int32_t *problem_idx, const void *x, const void *t,
                  const int32_t *n_steps, const void *v, void *F_out, void *grad_out, void *stream);

/*
 * hj_certify -- the certificate of Sec. 4.3 at n (x, t, v), always in FP64
 * (v is read in the context precision): residual_out [n] (relative
 * residual above), pass_out [n] (1 iff residual <= opts.cert_tol and the
 * value is finite), F_out [n] (double, nullable): the FP64 functional.
 */
hj_status hj_certify(hj_ctx *ctx, int64_t n, const int32_t *problem_idx, const void *x, const void *t,
                     const int32_t *n_steps, const void *v, double *residual_out, uint8_t *pass_out,
                     double *F_out, void *stream);

/*
 * hj_solve -- phi(x, t) for n_queries queries: random starts, descent,
 * certificate, reseeding, best of the starts (certified first; ties go to
 * the lowest slot), phi from the FP64 value at the chosen v.  The
 * certificate of each start is evaluated in the context precision at the
 * end of its descent; in FP32 a residual inside [0.95, 1.05] x cert_tol is
 * re-evaluated in FP64 before the pass/fail decision.
 * q_begin: global index of the first query (the Philox counter uses
 * q_begin + row), so a batch split across devices draws the same starts.
 * phi_out [nq] double, v_out [nq, ld] (the chosen v, an estimate of
 * grad phi), status_out [nq] int32 (HJ_ST_* bits).
 */
hj_status hj_solve(hj_ctx *ctx, int64_t q_begin, int64_t n_queries, const int32_t *problem_idx, const void *x,
                   const void *t, const int32_t *n_steps, double *phi_out, void *v_out, int32_t *status_out,
                   void *stream);

/*
 * hj_guesses -- the initial guesses hj_solve draws, for testing the
 * counter-based generator: for each of n entries, the start of query id
 * query_id[i] (int64), slot slot[i], round round[i] (int32) for problem
 * problem_idx[i] (nullable): v_out [n, ld].
 */
hj_status hj_guesses(hj_ctx *ctx, int64_t n, const int64_t *query_id, const int32_t *slot, const int32_t *round,
                     const int32_t *problem_idx, void *v_out, void *stream);

/* hj_last_solve_info -- counters of the last hj_solve (synchronises its stream). */
hj_status hj_last_solve_info(hj_ctx *ctx, hj_solve_info *out);

/*
 * hj_set_tuning -- launch parameters of problem `problem` (used by the
 * autotuner and for experiments): tpp = threads per (query, start) pair of
 * the descent and gradient kernels, in {1,2,4,8,16,32} (0: automatic;
 * for a LINEAR_QUAD problem with quadratic data (HJ_G_QUAD_SHIFT or
 * HJ_G_DIAG_QUAD) in an fp32 context with RK4 and its quadrature, no
 * coarse-to-fine descent, d <= 64 and 2 d + m <= 256 after padding to
 * multiples of 16, automatic means the
 * tensor-core tile kernel for hj_eval_functional, hj_grad and the gradient
 * and conjugate-gradient descents of hj_solve: 128 pairs per CTA, the stage
 * products on the tensor cores in split-precision BF16x3 (relative error
 * ~2^-16); any non-zero tpp selects the lane-group kernels instead;
 * for a SMOOTH_NONCONVEX problem under the Hopf principle in an fp32 context
 * with RK4 and its quadrature and d <= 32, automatic means the
 * one-pair-per-thread kernels, which carry the RK4 iterate as the two scalars
 * (u, B) with p = v + B w: one lane per pair in rounds of at least twice the
 * GPU's resident threads of pairs, two lanes per pair in smaller rounds,
 * with bit-identical results; tpp = -1 / -2 pins one / two lanes per pair in
 * every round for such a problem with gradient descent, HJ_EUNSUPPORTED for
 * any other); ck_interval = integrator steps between checkpoints of the
 * adjoint, in [1, 16] (0: automatic, the smallest interval whose checkpoint
 * storage fits a fixed per-thread budget; 1 for the one-pair-per-thread
 * kernels, where interval 1 means the forward pass keeps every step's stage
 * record (40 bytes) and the reverse pass reads it instead of rebuilding the
 * step, and intervals > 1 keep (u, B) checkpoints and rebuild, with the same
 * gradient bit for bit).  Returns HJ_EUNSUPPORTED when no kernel is built for
 * the resulting components per thread.
 */
hj_status hj_set_tuning(hj_ctx *ctx, int problem, int tpp, int ck_interval);

/*
 * hj_set_graph -- enable (1) or disable (0) CUDA graphs for hj_solve: with
 * graphs on, the first hj_solve on a non-NULL stream records its whole
 * launch sequence (kernels, memsets, events, the forks and joins of the
 * concurrent per-problem launches) into a CUDA graph and launches it;
 * later calls with the same q_begin, n_queries, pointers and stream replay
 * that graph instead of enqueuing ~30-70 operations again (the buffers'
 * contents may change between calls, their addresses not).  Calls with other
 * arguments record a new graph; hj_set_tuning and hj_autotune discard it.
 * The NULL (legacy default) stream cannot be captured: calls on it enqueue
 * directly.  A graph-launched solve reports its total device time in
 * hj_last_solve_info (descent_ms, certify_ms and descent_ms_round0 are 0:
 * events recorded inside a graph cannot be timed).  Off by default.
 */
hj_status hj_set_graph(hj_ctx *ctx, int enable);

/*
 * hj_autotune -- choose each problem's launch parameters by measurement (the
 * batching scheme of the solver, not a step of the paper): for every
 * candidate -- the automatic choice (for a linear-quadratic problem that fits
 * it, the tensor-core tile kernel) and every threads-per-pair count with a
 * built kernel -- run hj_solve on the given sample of queries with each
 * problem's descent capped at `iters` iterations (coordinate descent: iters
 * sweeps) and no reseeding, time each problem's descent launch with CUDA
 * events, and keep the fastest (a later candidate must be 3% faster).  The
 * choice is applied as by hj_set_tuning and, when tpp_out (HOST, int32 [n
 * problems]) is non-NULL, returned there (0 = automatic).  Synchronous;
 * allocates and frees temporary outputs; hj_last_solve_info is cleared.
 */
hj_status hj_autotune(hj_ctx *ctx, int64_t n_queries, const int32_t *problem_idx, const void *x, const void *t,
                      const int32_t *n_steps, int iters, int32_t *tpp_out, void *stream);

/*
 * hj_solve_noalloc -- hj_solve that allocates nothing.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * while they solve, e.g. programs whose GPU memory is owned by another
 * allocator (a framework's caching pool, a pre-reserved arena) or
 * latency-critical loops that must not risk an allocation.  Create the
 * context once beforehand (hj_create allocates); this call then makes no
 * cudaMalloc/cudaFree and uses no allocating library routine.
 *
 * Arguments, results and status codes are those of hj_solve, and so are the
 * kernels, with one exception: a linear-quadratic problem that hj_solve
 * would run on the tensor-core tile kernel (see hj_solve) runs here on the
 * lane-group kernels, whose results agree with it within the tile kernel's
 * BF16x3 rounding but not bit for bit; every other problem gets hj_solve's
 * results bit for bit.  A batch of more than 2^31 - 1 (query, trial) pairs
 * (a query's trials: its starts plus, with reseeding on, the rest of its
 * trial budget) returns HJ_EINVAL before any size arithmetic.  All of the
 * call's scratch lives in one static device array of
 * HJ_SOLVE_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps
 * for the life of the process; a call that needs more (about
 * n_queries * max_trials * (42 + ld * element size) bytes plus ~20 bytes per
 * query, max_trials the largest per-query trial count of the context's
 * problems) returns HJ_EINVAL with the sizes in hj_last_error and enqueues
 * nothing.  The first call on each device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture starts.  Every call on a device shares the one array: calls that
 * overlap on the GPU (other streams, other threads, other contexts) race
 * and corrupt each other's results, so serialise them.  hj_last_solve_info
 * keeps describing the last hj_solve call.
 */
#define HJ_SOLVE_NOALLOC_SCRATCH_BYTES (16u << 20)
hj_status hj_solve_noalloc(hj_ctx *ctx, int64_t q_begin, int64_t n_queries, const int32_t *problem_idx,
                           const void *x, const void *t, const int32_t *n_steps, double *phi_out, void *v_out,
                           int32_t *status_out, void *stream);

/* Message of the last error on ctx (or of the last failed hj_create when ctx is NULL). */
const char *hj_last_error(const hj_ctx *ctx);

/*
 * hj_fp32_fma_rate -- measured FP32 FMA rate of CUDA device `device` in
 * TFLOP/s (FMA = 2 flops), written to *tflops (HOST): every thread of
 * 8 x 256-thread blocks per SM runs 8 independent chains of 65,536 FMAs;
 * the best of five timed launches (after one warm-up) is reported.  It is the
 * measured counterpart of the ALU roofline peak (SMs x 128 lanes x 2 x
 * clock), with no context needed.  Allocates and frees its own 2048 floats
 * per SM.  HJ_EINVAL for a NULL tflops, HJ_ECUDA / HJ_ENOMEM on CUDA errors.
 */
hj_status hj_fp32_fma_rate(int device, double *tflops);

#ifdef __cplusplus
}
#endif
#endif /* HJ_H */
