"""Seeded synthetic workloads for the generalized Lax/Hopf solver.

This module only draws inputs: query points, times, step counts and the
parameters of each Hamiltonian family, rounded to binary32 and returned as
float64 arrays, so the GPU (which computes in fp32) and the FP64 oracle
solve exactly the same problem.  It holds none of the method's arithmetic
and imports neither the CUDA library nor the oracle; tests and bench.py
feed its arrays to both sides.

The paper (arXiv 1704.02524, Sec. 5) evaluates analytic examples only, on
2-D cross-sections of [-3,3]^d with random initial guesses in [-2,2]^d; it
uses no dataset.  The five workloads below are synthetic in the same
spirit, with the sizes listed in each docstring.  Every draw comes from
numpy's Philox bit generator keyed by 0x170402524 + workload number, in a
fixed order (family parameters first, then queries), so the first n rows
of a workload do not depend on how many rows are drawn.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

(FAM_QUAD_ISO, FAM_SPEED_QUAD, FAM_SMOOTH_NONCONVEX, FAM_LINEAR_QUAD, FAM_BUMP_NORM, FAM_SPLIT_NORM, FAM_HARMONIC,
 FAM_EVANS, FAM_LINEAR_GAME) = range(9)
LAX, HOPF, HUYGENS = 0, 1, 2
G_QUAD_SHIFT, G_DIAG_QUAD, G_ELLIPSE, G_ROSENBROCK = 0, 1, 2, 3

HARNESS_SEED = 0x170402524


def f32(a) -> np.ndarray:
    """Round to binary32, return as float64 (the values both sides receive)."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def rng_for(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=HARNESS_SEED + index))


@dataclass
class ProblemSpec:
    """A Hamiltonian family instance and its initial data g."""
    d: int
    family: int
    principle: int
    g_kind: int
    w: Optional[np.ndarray] = None       # [d]   speed c(x) = 1 + sin(<w,x>)/2
    A: Optional[np.ndarray] = None       # [d,d] drift
    B: Optional[np.ndarray] = None       # [d,m] control
    a: Optional[np.ndarray] = None       # [d]   g = |x-a|^2/2
    sigma: Optional[np.ndarray] = None   # [d]   g = sum x_i^2/(2 sigma_i^2) (ellipse data: minus 1/2)
    n_neg: int = 1
    s_eps: float = 1e-6
    n_guesses: int = 1
    solver: Optional[Dict] = None        # this problem's descent constants (None: the workload's)
    xc: Optional[np.ndarray] = None      # [d]   bump-norm family: H = hsign c(x)|p|,
    kappa: float = 0.0                   #       c = 1 + kappa exp(-mu |x - xc|^2)
    mu: float = 0.0
    hsign: float = 1.0
    xcb: Optional[np.ndarray] = None     # [d]   split-norm family: H = c_A|p_A| + c_B|p_B| over the
    ksplit: int = 0                      #       blocks [0,k), [k,d); c_A = alpha_a (1 + kappa
    alpha_a: float = 0.0                 #       exp(-mu|x - xc|^2)), c_B likewise around xcb
    alpha_b: float = 0.0
    beta: float = 0.0                    # Evans-type family: H = -c(x) p_1 + beta|p_2| - |p| - gamma0,
    gamma0: float = 0.0                  #       c = alpha_a (1 + kappa exp(-mu|x - xc|^2))
                                         # harmonic family: H = hsign (|p|^2 + |x|^2)/2
    r_c: float = 0.0                     # linear game: H(x,p,s) = -<diag(w) x, p> + a(s)|p|,
    r_d: float = 0.0                     #       a(s) = r_c - r_d (1 + beta sin(omega s))
    omega: float = 0.0

    def params(self) -> np.ndarray:
        """Flat parameter vector in the library's documented order:
        family block (w | A row-major then B row-major | xc, kappa, mu, sign |
        xc_A, xc_B, k, kappa, mu, alpha_A, alpha_B | sign | xc, kappa, mu, alpha,
        beta, gamma0 | m, r_C, r_D, beta, omega),
        then g block (a | sigma)."""
        parts: List[np.ndarray] = []
        if self.family in (FAM_SPEED_QUAD, FAM_SMOOTH_NONCONVEX):
            parts.append(self.w)
        if self.family == FAM_LINEAR_QUAD:
            parts += [self.A.reshape(-1), self.B.reshape(-1)]
        if self.family == FAM_BUMP_NORM:
            parts += [self.xc, np.array([self.kappa, self.mu, self.hsign])]
        if self.family == FAM_SPLIT_NORM:
            parts += [self.xc, self.xcb, np.array([self.ksplit, self.kappa, self.mu, self.alpha_a, self.alpha_b])]
        if self.family == FAM_HARMONIC:
            parts.append(np.array([self.hsign]))
        if self.family == FAM_EVANS:
            parts += [self.xc, np.array([self.kappa, self.mu, self.alpha_a, self.beta, self.gamma0])]
        if self.family == FAM_LINEAR_GAME:
            parts += [self.w, np.array([self.r_c, self.r_d, self.beta, self.omega])]
        if self.g_kind != G_ROSENBROCK:  # the Rosenbrock data has no parameters
            parts.append(self.a if self.g_kind == G_QUAD_SHIFT else self.sigma)
        return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])

    @property
    def m(self) -> int:
        return 0 if self.B is None else int(self.B.shape[1])


@dataclass
class Workload:
    name: str
    problems: List[ProblemSpec]
    x: np.ndarray            # [nq, ld] float64 (binary32 values), zero padded past each row's d
    t: np.ndarray            # [nq]
    n_steps: np.ndarray      # [nq] int32
    problem_idx: np.ndarray  # [nq] int32
    solver: Dict             # solver constants (see solver_constants)
    precision: str           # "fp32" or "fp64"
    note: str = ""

    @property
    def nq(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(sum(self.problems[int(i)].n_guesses for i in self.problem_idx))

    def head(self, n: int) -> "Workload":
        """The first n queries (same problems and constants)."""
        return Workload(self.name, self.problems, self.x[:n].copy(), self.t[:n].copy(), self.n_steps[:n].copy(),
                        self.problem_idx[:n].copy(), dict(self.solver), self.precision, self.note)

    def take(self, idx) -> "Workload":
        idx = np.asarray(idx)
        return Workload(self.name, self.problems, self.x[idx].copy(), self.t[idx].copy(),
                        self.n_steps[idx].copy(), self.problem_idx[idx].copy(), dict(self.solver),
                        self.precision, self.note)


def solver_constants(**over) -> Dict:
    """Default solver constants (names follow Algorithm 1 of the paper).
    eps = 1e-5 on the largest move of a gradient step: on 128 queries of the
    d=20 Hopf workload (16 starts each) it takes 75.6 iterations per start
    against 89.4 at 1e-6, every query still certifies, and phi stays within
    2.2e-8 (relative) of the eps = 1e-8 solution; 3e-5 lets one query stop in
    a worse minimum (9e-2).  The step-control constants (alpha_0 = 0.05,
    grow 1.2, shrink 0.5) were the only robust ones of a grid over grow in
    {1.2, 1.5, 2}, shrink in {0.3, 0.5}, alpha_0 in {0.05, 0.2}.
    Coarse-to-fine (coarse_div = 4, coarse_eps = 1e-4: the descent first on
    the N/4-step functional, then on the N-step one) took 0.61x the oracle's
    time on 128 queries of the d=20 workload and 0.23x on the d=10 one, with
    phi within 2e-8 and every query still certified."""
    c = dict(grad="adjoint", quad="rk4", fd_h=2.0 ** -10, step=0.05, max_iters=200, halving_period=0,
             eps=1e-5, adapt=1, grow=1.2, shrink=0.5, step_max=1.0, n_guesses=1, max_trials=20,
             max_rounds=4, seed=0x5EED1704, guess_dist=0, cert_tol=1e-3, coarse_div=4, coarse_eps=1e-4)
    c.update(over)
    if c["grad"] not in ("adjoint", "adjoint_cg") and "coarse_div" not in over:
        c["coarse_div"] = 1  # coarse-to-fine is a gradient-descent option
    return c


def _speed_w(rng, d):
    return f32(rng.normal(size=d) / math.sqrt(d))


def c1_quad_iso(nq: Optional[int] = None) -> Workload:
    """d=2 Lax, H=|p|^2/2, g=|x|^2/2, t=1: 64 queries on the 8x8 grid over
    [-2,2]^2 (endpoints included), RK4 N=20, coordinate descent with central
    differences (h=1e-4, alpha=0.1, exactly 200 sweeps), 4 Irwin-Hall
    guesses, all in FP64.  Closed form phi = |x|^2 / (2 (1 + t))."""
    g = -2.0 + 4.0 * np.arange(8) / 7.0
    X = np.array([[a, b] for a in g for b in g])
    P = ProblemSpec(d=2, family=FAM_QUAD_ISO, principle=LAX, g_kind=G_QUAD_SHIFT, a=np.zeros(2), n_guesses=4)
    nq = 64 if nq is None else nq
    X = X[:nq]
    solver = solver_constants(grad="fd_central", fd_h=1e-4, step=0.1, max_iters=200 * 2, eps=0.0, adapt=0,
                              n_guesses=4, max_trials=4, max_rounds=0, guess_dist=1, cert_tol=1e-6)
    return Workload("quad_iso_d2_lax", [P], X, np.ones(nq), np.full(nq, 20, np.int32), np.zeros(nq, np.int32),
                    solver, "fp64")


def c2_speed_quad(nq_x: int = 16384) -> Workload:
    """d=10 Lax, H = c(x)^2 |p|^2 / 2 with c = 1 + sin(<w,x>)/2, w ~ N(0, I/d);
    g = |x-a|^2/2, a ~ U[-1,1]^d; x ~ U[-2,2]^d, each at t in {0.25, 0.5, 1}
    (query 3i+k is point i at time k); RK4 N=50; 8 uniform guesses."""
    rng = rng_for(2)
    d = 10
    w = _speed_w(rng, d)
    a = f32(rng.uniform(-1, 1, d))
    X = f32(rng.uniform(-2, 2, (nq_x, d)))
    T = np.array([0.25, 0.5, 1.0])
    P = ProblemSpec(d=d, family=FAM_SPEED_QUAD, principle=LAX, g_kind=G_QUAD_SHIFT, w=w, a=a, n_guesses=8)
    x = np.repeat(X, 3, axis=0)
    t = np.tile(T, nq_x)
    nq = x.shape[0]
    return Workload("speed_quad_d10_lax", [P], x, t, np.full(nq, 50, np.int32), np.zeros(nq, np.int32),
                    solver_constants(n_guesses=8), "fp32")


def c3_smooth_nonconvex(nq: int = 65536) -> Workload:
    """d=20 Hopf, H = c(x) (-s(p_1) + sum_{i>=2} s(p_i)), s(q) = sqrt(q^2+1e-6),
    c as in the d=10 workload (its own w); g = sum x_i^2/(2 sigma_i^2),
    sigma ~ U[0.5,2]; x ~ U[-1,1]^d; t = 0.5; RK4 N=64; 16 uniform guesses,
    certificate and reseeding (at most 20 trials per query)."""
    rng = rng_for(3)
    d = 20
    w = _speed_w(rng, d)
    sigma = f32(rng.uniform(0.5, 2.0, d))
    X = f32(rng.uniform(-1, 1, (nq, d)))
    P = ProblemSpec(d=d, family=FAM_SMOOTH_NONCONVEX, principle=HOPF, g_kind=G_DIAG_QUAD, w=w, sigma=sigma,
                    n_neg=1, s_eps=1e-6, n_guesses=16)
    return Workload("smooth_nonconvex_d20_hopf", [P], X, np.full(nq, 0.5), np.full(nq, 64, np.int32),
                    np.zeros(nq, np.int32), solver_constants(n_guesses=16), "fp32")


def _lq_matrices(rng, d, m=32):
    G0 = rng.normal(size=(d, d))
    A = f32(G0 / (2.0 * np.linalg.norm(G0, 2)))
    B = f32(rng.normal(size=(d, m)) / math.sqrt(d))
    return A, B


def c4_linear_quad(nq: int = 32768) -> Workload:
    """d=64 Lax, H = <Ax,p> + |B^T p|^2/2 with A = G/(2||G||_2), G a standard
    Gaussian d x d, B a d x 32 Gaussian scaled by 1/sqrt(d); g = |x|^2/2;
    x ~ N(0, I); t = 1; RK4 N=100; one guess, conjugate-gradient descent
    (lq_solver).  The exact solution is x^T P(t) x / 2 with the Riccati
    matrix P."""
    rng = rng_for(4)
    d = 64
    A, B = _lq_matrices(rng, d)
    X = f32(rng.normal(size=(nq, d)))
    P = ProblemSpec(d=d, family=FAM_LINEAR_QUAD, principle=LAX, g_kind=G_QUAD_SHIFT, A=A, B=B, a=np.zeros(d),
                    n_guesses=1)
    return Workload("linear_quad_d64_lax", [P], X, np.ones(nq), np.full(nq, 100, np.int32), np.zeros(nq, np.int32),
                    lq_solver(), "fp32")


def lq_solver(**over) -> Dict:
    """Constants of the linear-quadratic workloads.  The functional is a
    convex quadratic in v whose Hessian has eigenvalues down to ~1e-6 in the
    directions B does not reach (B has rank 32 of 64; condition ~3e6 at
    d=64), so gradient steps stall and conjugate directions are used: 100
    Polak-Ribiere+ iterations with secant line searches (probe length 1),
    one start (convex H, Sec. 5), no reseeding.  The certificate residual
    stays far above any useful tolerance there (the flat directions of F are
    not flat for p(0) - grad g(gamma(0))), on the oracle as on the GPU."""
    c = solver_constants(grad="adjoint_cg", step=1.0, step_max=100.0, eps=0.0, max_iters=100, n_guesses=1,
                         max_trials=1, max_rounds=0, coarse_div=1)
    c.update(over)
    return c


def c5_mixed(n_pairs: int = 1 << 20) -> Workload:
    """Uneven batch of (query, guess) pairs: a third of the pairs each from
    the d=10-style speed-quadratic Lax family (8 guesses), the d=20-style
    non-convex Hopf family (16 guesses) and the linear-quadratic Lax family
    (1 guess).  Each query draws d from {8, 16, 32, 100}, t ~ U[0.1, 2] and
    N = ceil(64 t).  Family parameters are drawn per (family, d).  Each
    family keeps the descent constants of its own workload: gradient descent
    with reseeding (at most 20 trials) for the first two, conjugate
    gradients with one start for the linear-quadratic one."""
    rng = rng_for(5)
    dims = [8, 16, 32, 100]
    probs: List[ProblemSpec] = []
    for d in dims:
        probs.append(ProblemSpec(d=d, family=FAM_SPEED_QUAD, principle=LAX, g_kind=G_QUAD_SHIFT,
                                 w=_speed_w(rng, d), a=f32(rng.uniform(-1, 1, d)), n_guesses=8,
                                 solver=solver_constants(n_guesses=8)))
    for d in dims:
        probs.append(ProblemSpec(d=d, family=FAM_SMOOTH_NONCONVEX, principle=HOPF, g_kind=G_DIAG_QUAD,
                                 w=_speed_w(rng, d), sigma=f32(rng.uniform(0.5, 2.0, d)), n_guesses=16,
                                 solver=solver_constants(n_guesses=16)))
    for d in dims:
        A, B = _lq_matrices(rng, d)
        probs.append(ProblemSpec(d=d, family=FAM_LINEAR_QUAD, principle=LAX, g_kind=G_QUAD_SHIFT, A=A, B=B,
                                 a=np.zeros(d), n_guesses=1, solver=lq_solver()))
    per_fam = n_pairs // 3
    n_q = [per_fam // 8, per_fam // 16]
    n_q.append(n_pairs - 8 * n_q[0] - 16 * n_q[1])
    ld = max(dims)
    xs, ts, idx = [], [], []
    for f, nqf in enumerate(n_q):
        dsel = rng.integers(0, len(dims), nqf)
        tt = f32(rng.uniform(0.1, 2.0, nqf))
        X = np.zeros((nqf, ld))
        raw = rng.uniform(-1, 1, (nqf, ld)) if f != 2 else rng.normal(size=(nqf, ld))
        for k, d in enumerate(dims):
            rows = dsel == k
            X[rows, :d] = f32(raw[rows, :d])
        xs.append(X)
        ts.append(tt)
        idx.append(4 * f + dsel)
    x = np.concatenate(xs)
    t = np.concatenate(ts)
    pidx = np.concatenate(idx).astype(np.int32)
    N = np.ceil(64.0 * t).astype(np.int32)
    return Workload("mixed_persistent", probs, x, t, N, pidx, solver_constants(), "fp32")


def paper_solver(**over) -> Dict:
    """The paper's own numerics (Sec. 5, Sec. 6): forward Euler with the
    rectangle rule, forward differences (eq. num_diff), and Algorithm 1 with
    alpha = 1/L, halving every M = 500 iterations and eps = 0.5e-7; random
    starts uniform in [-2,2]^d and no reseeding (Sec. 6 makes one start per
    convex problem and up to 20 independent ones otherwise).  The paper sets
    no iteration cap; 20000 coordinate moves is twice what the d=2 runs
    below need after the halvings have shrunk alpha."""
    c = solver_constants(quad="euler_rect", grad="fd_forward", fd_h=1e-3, step=1.0 / 0.02, max_iters=20000,
                         halving_period=500, eps=0.5e-7, adapt=0, n_guesses=5, max_trials=5, max_rounds=0,
                         coarse_div=1)
    c.update(over)
    return c


def ellipse_sigma(d: int) -> np.ndarray:
    """sigma of the ellipse data of Sec. 6: A^-1 = diag(1, 25/4, 1/4, ...)."""
    s = np.full(d, 0.5)
    s[0] = 1.0
    if d > 1:
        s[1] = 2.5
    return s


def _paper_precision(precision: Optional[str], fp32_every_row: bool) -> str:
    """Default precision of a paper-numerics workload: binary32 where its
    solve meets the 1e-4 gate against the FP64 oracle on every row, else
    FP64 (the paper's own precision).  The paper's forward differences with
    sigma = 1e-3 carry ~eps |F| / sigma ~ 1e-4 of binary32 rounding in every
    derivative; on the flat or kinked functionals of Sec. 6's Examples 2, 4
    and 5 and of the Huygens form that noise moves where Algorithm 1 stops
    (or which basin a start ends in) by more than the gate."""
    if precision is not None:
        return precision
    return "fp32" if fp32_every_row else "fp64"


def bump_ex3(n_side: int = 128, d: int = 2, sign: float = 1.0, t: float = 0.3, ds: float = 0.02,
             fd_h: float = 1e-3, n_guesses: int = 5, precision: Optional[str] = None,
             principle: int = LAX) -> Workload:
    """Sec. 6 Example 3 in the paper's numerics: H = sign c(x)|p| with
    c = 1 + 3 exp(-4 |x - (1,1,0,...)|^2), the ellipse data g, the Lax
    functional, on the n_side x n_side grid over the cross-section
    [-3,3]^2 x {0}^(d-2) at time t (0.3 for H+, as in the paper's d=2 run),
    forward Euler with step ds (N = t/ds), forward differences with step
    fd_h and L = 0.02, five starts per point (the paper's time format
    counts five).  principle = HUYGENS minimises F^2 (eq. num_min) instead
    of F^1.  Nothing is random but the starts."""
    g = np.linspace(-3.0, 3.0, n_side)
    X = np.zeros((n_side * n_side, d))
    X[:, 0] = np.repeat(g, n_side)
    X[:, 1] = np.tile(g, n_side)
    X = f32(X)
    xc = np.zeros(d)
    xc[:2] = 1.0
    P = ProblemSpec(d=d, family=FAM_BUMP_NORM, principle=principle, g_kind=G_ELLIPSE, sigma=ellipse_sigma(d),
                    xc=xc, kappa=3.0, mu=4.0, hsign=sign, s_eps=0.0, n_guesses=n_guesses)
    nq = X.shape[0]
    N = int(round(t / ds))
    pname = {LAX: "lax", HUYGENS: "huygens", HOPF: "hopf"}[principle]
    name = f"bump_norm_d{d}_{'plus' if sign > 0 else 'minus'}_{pname}_paper"
    return Workload(name, [P], X, np.full(nq, t), np.full(nq, N, np.int32), np.zeros(nq, np.int32),
                    paper_solver(fd_h=fd_h, n_guesses=n_guesses, max_trials=n_guesses),
                    _paper_precision(precision, principle != HUYGENS))


def split_ex5(n_side: int = 128, d: int = 2, k: int = 1, t: float = 0.3, ds: float = 0.02, fd_h: float = 1e-3,
              n_guesses: int = 20, precision: Optional[str] = None, descent: str = "paper") -> Workload:
    """Sec. 6 Example 5: H = c(x)|p_1..k| - c(-x)|p_k+1..d| with
    c(x) = 2 (1 + 3 exp(-4 |x - (1,1,0,...)|^2)), the ellipse data, the Hopf
    functional, on the n_side x n_side grid over [-3,3]^2 x {0}^(d-2) at
    t = 0.3, twenty starts per point.  descent "paper": the paper's numerics
    with its constants (forward Euler ds = 0.02, forward differences
    sigma = 1e-3, Algorithm 1 with L = 50); "cg": the momentum the paper
    proposes against this example's trench -- conjugate gradients on the
    same Euler functional with its exact adjoint gradient."""
    g = np.linspace(-3.0, 3.0, n_side)
    X = np.zeros((n_side * n_side, d))
    X[:, 0] = np.repeat(g, n_side)
    X[:, 1] = np.tile(g, n_side)
    X = f32(X)
    xc = np.zeros(d)
    xc[:2] = 1.0
    P = ProblemSpec(d=d, family=FAM_SPLIT_NORM, principle=HOPF, g_kind=G_ELLIPSE, sigma=ellipse_sigma(d), xc=xc,
                    xcb=-xc, ksplit=k, kappa=3.0, mu=4.0, alpha_a=2.0, alpha_b=-2.0, s_eps=0.0, n_guesses=n_guesses)
    nq = X.shape[0]
    N = int(round(t / ds))
    if descent == "paper":
        solver = paper_solver(fd_h=fd_h, step=1.0 / 50.0, n_guesses=n_guesses, max_trials=n_guesses)
    else:
        solver = solver_constants(quad="euler_rect", grad="adjoint_cg", step=0.05, step_max=1.0, max_iters=500,
                                  eps=1e-7, n_guesses=n_guesses, max_trials=n_guesses, max_rounds=0, coarse_div=1)
    return Workload(f"split_norm_d{d}_hopf_{descent}", [P], X, np.full(nq, t), np.full(nq, N, np.int32),
                    np.zeros(nq, np.int32), solver, _paper_precision(precision, False))


def _grid(n_side: int, d: int) -> np.ndarray:
    g = np.linspace(-3.0, 3.0, n_side)
    X = np.zeros((n_side * n_side, d))
    X[:, 0] = np.repeat(g, n_side)
    X[:, 1] = np.tile(g, n_side)
    return f32(X)


def harmonic_ex2(n_side: int = 128, d: int = 2, sign: float = -1.0, t: float = 0.5, ds: float = 0.02,
                 n_guesses: int = 5, precision: Optional[str] = None, rosenbrock: bool = False) -> Workload:
    """Sec. 6 Example 2: H = sign (|p|^2 + |x|^2)/2 with the ellipse data, the
    Hopf functional for both signs, on the n_side x n_side grid over
    [-3,3]^2 x {0}^(d-2) (t = 0.5 at d = 2; the paper's d = 7 run uses
    t = 0.2), in the paper's numerics with ds = 0.02, sigma = 1e-3, L = 3.
    rosenbrock: the non-convex Rosenbrock data instead, with H+ and the Lax
    functional (d = 2), as in the paper's last run of this example."""
    X = _grid(n_side, d)
    if rosenbrock:
        P = ProblemSpec(d=2, family=FAM_HARMONIC, principle=LAX, g_kind=G_ROSENBROCK, hsign=1.0,
                        n_guesses=n_guesses)
        sign = 1.0
    else:
        P = ProblemSpec(d=d, family=FAM_HARMONIC, principle=HOPF, g_kind=G_ELLIPSE, sigma=ellipse_sigma(d),
                        hsign=sign, n_guesses=n_guesses)
    nq = X.shape[0]
    N = int(round(t / ds))
    pname = "lax_rosenbrock" if rosenbrock else "hopf"
    return Workload(f"harmonic_d{d}_{'plus' if sign > 0 else 'minus'}_{pname}_paper", [P], X, np.full(nq, t),
                    np.full(nq, N, np.int32), np.zeros(nq, np.int32),
                    paper_solver(step=1.0 / 3.0, n_guesses=n_guesses, max_trials=n_guesses),
                    _paper_precision(precision, False))


def evans_ex4(n_side: int = 128, t: float = 0.1, ds: float = 0.005, n_guesses: int = 5,
              precision: Optional[str] = None) -> Workload:
    """Sec. 6 Example 4: H = -c(x) p_1 + 2|p_2| - |p| - 1 with
    c = 2 (1 + 3 exp(-4 |x - (1,1)|^2)), d = 2, the ellipse data, the Hopf
    functional, on the n_side x n_side grid over [-3,3]^2 at t = 0.1, in the
    paper's numerics with ds = 0.005, sigma = 1e-3, L = 4."""
    X = _grid(n_side, 2)
    P = ProblemSpec(d=2, family=FAM_EVANS, principle=HOPF, g_kind=G_ELLIPSE, sigma=ellipse_sigma(2),
                    xc=np.array([1.0, 1.0]), kappa=3.0, mu=4.0, alpha_a=2.0, beta=2.0, gamma0=1.0, s_eps=0.0,
                    n_guesses=n_guesses)
    nq = X.shape[0]
    N = int(round(t / ds))
    return Workload("evans_d2_hopf_paper", [P], X, np.full(nq, t), np.full(nq, N, np.int32), np.zeros(nq, np.int32),
                    paper_solver(step=1.0 / 4.0, n_guesses=n_guesses, max_trials=n_guesses),
                    _paper_precision(precision, False))


def linear_game(nq: int = 65536, d: int = 16, t: float = 0.8, n_steps: int = 64, r_d: float = 0.4,
                n_guesses: int = 2) -> Workload:
    """The time-dependent linear differential game of Sec. 3.4, Example 3:
    dynamics dx/ds = M x + a + b with controls a, b in balls of radii r_C = 1
    and r_D (1 + beta sin(omega s)), beta = 0.5, omega = 3, M = diag(m) with
    m ~ U[-0.5, 0.5]^d, giving H(x,p,s) = -<Mx,p> + (r_C - r_D (1 + beta
    sin(omega s)))|p|; the ellipse data, the Hopf functional (the formula
    that section derives), x ~ U[-2,2]^d, t = 0.8, RK4 with 64 steps, the
    default gradient descent with two starts.  With r_d = 0.4 the speed
    stays positive and the functional convex in v; r_d > 1/1.5 lets it
    change sign (a non-convex game)."""
    rng = rng_for(6)
    m = f32(rng.uniform(-0.5, 0.5, d))
    X = f32(rng.uniform(-2, 2, (nq, d)))
    P = ProblemSpec(d=d, family=FAM_LINEAR_GAME, principle=HOPF, g_kind=G_ELLIPSE, sigma=ellipse_sigma(d), w=m,
                    r_c=1.0, r_d=r_d, beta=0.5, omega=3.0, s_eps=0.0, n_guesses=n_guesses)
    name = f"linear_game_d{d}_hopf" if r_d == 0.4 else f"linear_game_d{d}_rd{r_d:g}_hopf"
    return Workload(name, [P], X, np.full(nq, t), np.full(nq, n_steps, np.int32),
                    np.zeros(nq, np.int32), solver_constants(n_guesses=n_guesses), "fp32")


WORKLOADS = {
    "quad_iso_d2_lax": c1_quad_iso,
    "speed_quad_d10_lax": c2_speed_quad,
    "smooth_nonconvex_d20_hopf": c3_smooth_nonconvex,
    "linear_quad_d64_lax": c4_linear_quad,
    "mixed_persistent": c5_mixed,
    "bump_norm_d2_plus_lax_paper": bump_ex3,
    "split_norm_d2_hopf_paper": split_ex5,
    "harmonic_d2_minus_hopf_paper": harmonic_ex2,
    "evans_d2_hopf_paper": evans_ex4,
    "linear_game_d16_hopf": linear_game,
}


def plain_cd_solver(solver: Dict, d: int, sweeps: int = 100) -> Dict:
    """Constants of the plain path for a workload whose own descent is the
    adjoint gradient descent: Algorithm 1 (cyclic coordinate descent) with
    central differences, h = 2^-10 (the binary32 functional carries ~1e-6
    absolute rounding, so smaller steps drown the difference in noise), at
    most `sweeps` sweeps, the same per-coordinate step control, starts,
    reseeding and certificate."""
    c = dict(solver, grad="fd_central", fd_h=2.0 ** -10, max_iters=sweeps * d, coarse_div=1)
    return c


def c3_cd_solver() -> Dict:
    """The plain path's constants on the d=20 Hopf workload (plain_cd_solver)."""
    return plain_cd_solver(solver_constants(n_guesses=16), 20)
