"""Test-side glue: workload specs -> oracle objects, and tolerances."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1704_02524_gb300 import workloads as W

GRAD_CODES = {"fd_central": O.GRAD_FD_CENTRAL, "fd_forward": O.GRAD_FD_FORWARD, "adjoint": O.GRAD_ADJOINT,
              "adjoint_cg": O.GRAD_ADJOINT}
DESCENT_CODES = {"fd_central": O.DESC_CD, "fd_forward": O.DESC_CD, "adjoint": O.DESC_GD, "adjoint_cg": O.DESC_CG}
QUAD_CODES = {"rk4": O.QUAD_RK4, "rect": O.QUAD_RECT, "euler": O.QUAD_RK4 | O.ODE_EULER,
              "euler_rect": O.QUAD_RECT | O.ODE_EULER}


def oracle_problem(spec: W.ProblemSpec) -> O.Problem:
    return O.Problem(d=spec.d, family=spec.family, principle=spec.principle, g_kind=spec.g_kind, w=spec.w,
                     A=spec.A, B=spec.B, a=spec.a, sigma=spec.sigma, n_neg=spec.n_neg, s_eps=spec.s_eps,
                     xc=spec.xc, kappa=spec.kappa, mu=spec.mu, hsign=spec.hsign, xcb=spec.xcb,
                     ksplit=spec.ksplit, alpha_a=spec.alpha_a, alpha_b=spec.alpha_b, beta=spec.beta,
                     gamma0=spec.gamma0, r_c=spec.r_c, r_d=spec.r_d, omega=spec.omega)


def oracle_opts(solver: dict, n_guesses: int) -> O.Opts:
    g = GRAD_CODES[solver["grad"]]
    return O.Opts(quad=QUAD_CODES[solver["quad"]], descent=DESCENT_CODES[solver["grad"]],
                  grad=g, fd_h=solver["fd_h"] if g != O.GRAD_ADJOINT else 1e-6, step=solver["step"],
                  max_iters=solver["max_iters"], halving_period=solver["halving_period"], eps=solver["eps"],
                  adapt=solver["adapt"], grow=solver["grow"], shrink=solver["shrink"],
                  step_max=solver["step_max"], n_guesses=n_guesses, max_trials=solver["max_trials"],
                  max_rounds=solver["max_rounds"], seed=solver["seed"], guess_dist=solver["guess_dist"],
                  cert_tol=solver["cert_tol"], coarse_div=solver.get("coarse_div", 1),
                  coarse_eps=solver.get("coarse_eps", 1e-4))


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / (1.0 + np.abs(b))


def oracle_opts_list(wl) -> list:
    """One oracle Opts per problem of a workload: the problem's own descent
    constants where it has them, the workload's otherwise; the context-wide
    fields (quadrature, seed, start distribution, reseed rounds) are the
    workload's, as in the library."""
    out = []
    for p in wl.problems:
        s = dict(p.solver) if p.solver is not None else dict(wl.solver)
        for k in ("quad", "seed", "guess_dist", "max_rounds"):
            s[k] = wl.solver[k]
        out.append(oracle_opts(s, p.n_guesses))
    return out
