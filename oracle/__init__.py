"""FP64 CPU oracle for the generalized Lax/Hopf method (arXiv 1704.02524).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product library never does, and the two share no code.

The arithmetic lives in ``hj_oracle.c`` (plain double-precision C, one pair
at a time).  This module compiles it with gcc on first use, wraps it with
ctypes and runs independent queries on a thread pool (ctypes releases the
GIL during each foreign call, so the threads run in parallel).

Paper passages followed (all in arXiv 1704.02524):
  * Sec. 4.1 -- the functionals F^1 (Lax) and G (Hopf) and the backward
    final-value characteristic system; Algorithm 1 (cyclic coordinate
    descent with step 1/L halved every M iterations).
  * Sec. 4.2 -- ODE solver (RK4 here; forward Euler is the paper's
    illustration), eq. num_int (rectangle rule), eq. num_diff (finite
    differences).
  * Sec. 4.3 -- the certificate p(0) in dg(gamma(0)) and restart on failure.
  * Sec. 5 -- random initial guesses in [-2,2]^d, at most 20 trials; the
    remark that momentum helps descents that drag along flat trenches
    (conjugate-gradient descent, DESC_CG).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hj_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libhj_oracle.so")
_lock = threading.Lock()
_lib = None

(FAM_QUAD_ISO, FAM_SPEED_QUAD, FAM_SMOOTH_NONCONVEX, FAM_LINEAR_QUAD, FAM_BUMP_NORM, FAM_SPLIT_NORM, FAM_HARMONIC,
 FAM_EVANS, FAM_LINEAR_GAME) = range(9)
LAX, HOPF, HUYGENS = 0, 1, 2  # HUYGENS: the Lax principle through F^2 (eq. num_min)
G_QUAD_SHIFT, G_DIAG_QUAD, G_ELLIPSE, G_ROSENBROCK = 0, 1, 2, 3
QUAD_RK4, QUAD_RECT = 0, 1
ODE_EULER = 2  # or-ed into a quad argument: forward Euler instead of RK4
GRAD_FD_CENTRAL, GRAD_FD_FORWARD, GRAD_ADJOINT = 0, 1, 2
DESC_CD, DESC_GD, DESC_CG = 0, 1, 2
ST_CERTIFIED, ST_MAX_ITERS, ST_NONFINITE, ST_RESEEDED = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile hj_oracle.c into libhj_oracle.so next to it (gcc, -O2)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                            "-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("d", C.c_int), ("family", C.c_int), ("principle", C.c_int), ("g_kind", C.c_int),
                ("m", C.c_int), ("n_neg", C.c_int), ("s_eps", C.c_double),
                ("w", C.POINTER(C.c_double)), ("A", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)),
                ("ga", C.POINTER(C.c_double)), ("gs", C.POINTER(C.c_double)),
                ("xc", C.POINTER(C.c_double)), ("kappa", C.c_double), ("mu", C.c_double), ("hsign", C.c_double),
                ("xcb", C.POINTER(C.c_double)), ("ksplit", C.c_int), ("alpha_a", C.c_double),
                ("alpha_b", C.c_double), ("beta", C.c_double), ("gamma0", C.c_double),
                ("r_c", C.c_double), ("r_d", C.c_double), ("omega", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("quad", C.c_int), ("descent", C.c_int), ("grad", C.c_int), ("fd_h", C.c_double),
                ("step", C.c_double), ("max_iters", C.c_int), ("halving_period", C.c_int),
                ("eps", C.c_double), ("adapt", C.c_int), ("grow", C.c_double), ("shrink", C.c_double),
                ("step_max", C.c_double), ("n_guesses", C.c_int), ("max_trials", C.c_int),
                ("max_rounds", C.c_int), ("seed", C.c_uint64), ("guess_dist", C.c_int),
                ("cert_tol", C.c_double), ("coarse_div", C.c_int), ("coarse_eps", C.c_double)]


_DP = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.orc_guess.argtypes = [C.c_uint64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, _DP]
    lib.orc_functional.argtypes = [C.POINTER(_Problem), C.c_int, _DP, C.c_double, C.c_int, _DP, _DP, _DP]
    lib.orc_functional.restype = C.c_double
    lib.orc_gradient.argtypes = [C.POINTER(_Problem), C.c_int, _DP, C.c_double, C.c_int, _DP, _DP]
    lib.orc_gradient.restype = C.c_double
    lib.orc_gradient_fd.argtypes = [C.POINTER(_Problem), C.c_int, _DP, C.c_double, C.c_int, _DP, C.c_double, _DP]
    lib.orc_descend.argtypes = [C.POINTER(_Problem), C.POINTER(_Opts), _DP, C.c_double, C.c_int, _DP,
                                C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.orc_descend.restype = C.c_int
    lib.orc_certify.argtypes = [C.POINTER(_Problem), C.c_int, _DP, C.c_double, C.c_int, _DP, _DP]
    lib.orc_certify.restype = C.c_double
    _IP = C.POINTER(C.c_int)
    lib.orc_solve_query.argtypes = [C.POINTER(_Problem), C.POINTER(_Opts), C.c_int64, _DP, C.c_double, C.c_int,
                                    _DP, _DP, _DP, _DP, _IP, _IP, _IP, _DP, _IP]
    lib.orc_solve_query.restype = C.c_int
    lib.orc_trials.argtypes = [C.POINTER(_Opts)]
    lib.orc_trials.restype = C.c_int
    _lib = lib
    return lib


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_DP)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Problem:
    """One Hamiltonian/initial-data pair.  Arrays are float64 (the values the
    GPU receives, already rounded to float32 where the GPU computes in fp32)."""
    d: int
    family: int
    principle: int
    g_kind: int
    w: Optional[np.ndarray] = None
    A: Optional[np.ndarray] = None
    B: Optional[np.ndarray] = None
    a: Optional[np.ndarray] = None
    sigma: Optional[np.ndarray] = None
    n_neg: int = 1
    s_eps: float = 1e-6
    xc: Optional[np.ndarray] = None  # bump-norm family: centre of c(x)
    kappa: float = 0.0               # bump-norm family: c(x) = 1 + kappa exp(-mu |x - xc|^2)
    mu: float = 0.0
    hsign: float = 1.0               # bump-norm family: H = hsign c(x) |p|
    xcb: Optional[np.ndarray] = None  # split-norm family: H = c_A|p_A| + c_B|p_B| over blocks [0,k), [k,d),
    ksplit: int = 0                   #   c_A = alpha_a (1 + kappa exp(-mu|x - xc|^2)),
    alpha_a: float = 0.0              #   c_B = alpha_b (1 + kappa exp(-mu|x - xcb|^2))
    alpha_b: float = 0.0
    beta: float = 0.0                 # Evans-type family: H = -c(x) p_1 + beta|p_2| - |p| - gamma0,
    gamma0: float = 0.0               #   c = alpha_a (1 + kappa exp(-mu|x - xc|^2)); harmonic: H = hsign(|p|^2+|x|^2)/2
    r_c: float = 0.0                  # linear game: H(x,p,s) = -<diag(w) x, p> + a(s)|p|,
    r_d: float = 0.0                  #   a(s) = r_c - r_d (1 + beta sin(omega s))
    omega: float = 0.0
    _c: Optional[_Problem] = field(default=None, repr=False)

    def c(self) -> _Problem:
        if self._c is None:
            for name in ("w", "A", "B", "a", "sigma", "xc", "xcb"):
                v = getattr(self, name)
                if v is not None:
                    setattr(self, name, _f64(v))
            m = 0 if self.B is None else int(self.B.shape[1])
            self._c = _Problem(self.d, self.family, self.principle, self.g_kind, m, self.n_neg, self.s_eps,
                               _dp(self.w), _dp(self.A), _dp(self.B), _dp(self.a), _dp(self.sigma),
                               _dp(self.xc), float(self.kappa), float(self.mu), float(self.hsign),
                               _dp(self.xcb), int(self.ksplit), float(self.alpha_a), float(self.alpha_b),
                               float(self.beta), float(self.gamma0), float(self.r_c), float(self.r_d),
                               float(self.omega))
        return self._c


@dataclass
class Opts:
    """Solver constants (names follow Algorithm 1 and Sec. 4.2/5)."""
    quad: int = QUAD_RK4
    descent: int = DESC_CD
    grad: int = GRAD_FD_CENTRAL
    fd_h: float = 1e-4
    step: float = 0.1
    max_iters: int = 400
    halving_period: int = 0
    eps: float = 0.0
    adapt: int = 0
    grow: float = 1.2
    shrink: float = 0.5
    step_max: float = 1.0
    n_guesses: int = 1
    max_trials: int = 1
    max_rounds: int = 0
    seed: int = 0
    guess_dist: int = 0
    cert_tol: float = 1e-3
    coarse_div: int = 1
    coarse_eps: float = 1e-4

    def c(self) -> _Opts:
        return _Opts(self.quad, self.descent, self.grad, self.fd_h, self.step, self.max_iters,
                     self.halving_period, self.eps, self.adapt, self.grow, self.shrink, self.step_max,
                     self.n_guesses, self.max_trials, self.max_rounds, self.seed & (2**64 - 1),
                     self.guess_dist, self.cert_tol, self.coarse_div, self.coarse_eps)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def guess(seed: int, q: int, g: int, r: int, d: int, dist: int = 0) -> np.ndarray:
    lib = _load()
    v = np.zeros(d)
    lib.orc_guess(seed & (2**64 - 1), q, g, r, d, dist, _dp(v))
    return v


def functional(P: Problem, x, t: float, N: int, v, quad: int = QUAD_RK4, with_ends: bool = False):
    """F^1 (Lax) or G (Hopf) at one (x, t, v); optionally (F, gamma(0), p(0))."""
    lib = _load()
    x, v = _f64(x), _f64(v)
    g0, p0 = np.zeros(P.d), np.zeros(P.d)
    F = lib.orc_functional(C.byref(P.c()), quad, _dp(x), float(t), int(N), _dp(v), _dp(g0), _dp(p0))
    return (F, g0, p0) if with_ends else F


def gradient(P: Problem, x, t: float, N: int, v, quad: int = QUAD_RK4):
    """(F, dF/dv) by the discrete adjoint of the RK4 map."""
    lib = _load()
    x, v = _f64(x), _f64(v)
    g = np.zeros(P.d)
    F = lib.orc_gradient(C.byref(P.c()), quad, _dp(x), float(t), int(N), _dp(v), _dp(g))
    return F, g


def gradient_fd(P: Problem, x, t: float, N: int, v, h: float = 1e-6, quad: int = QUAD_RK4) -> np.ndarray:
    """Central finite-difference gradient of the discretised functional."""
    lib = _load()
    x, v = _f64(x), _f64(v)
    g = np.zeros(P.d)
    lib.orc_gradient_fd(C.byref(P.c()), quad, _dp(x), float(t), int(N), _dp(v), float(h), _dp(g))
    return g


def descend(P: Problem, O: Opts, x, t: float, N: int, v0):
    """Run the descent from v0; returns (v_final, iterations, hit_cap, nonfinite)."""
    lib = _load()
    x, v = _f64(x), _f64(v0).copy()
    cap, nf = C.c_int(0), C.c_int(0)
    it = lib.orc_descend(C.byref(P.c()), C.byref(O.c()), _dp(x), float(t), int(N), _dp(v),
                         C.byref(cap), C.byref(nf))
    return v, it, bool(cap.value), bool(nf.value)


def certify(P: Problem, x, t: float, N: int, v, tol: float, quad: int = QUAD_RK4):
    """(F, residual, pass) of the Sec. 4.3 certificate at v."""
    lib = _load()
    x, v = _f64(x), _f64(v)
    r = C.c_double(0.0)
    F = lib.orc_certify(C.byref(P.c()), quad, _dp(x), float(t), int(N), _dp(v), C.byref(r))
    return F, r.value, bool(r.value <= tol and np.isfinite(F))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))


def solve(problems, O: Opts, x, t, N, problem_idx=None, query_ids=None, threads: Optional[int] = None,
          guesses=None):
    """Solve every query: guesses, descent, certificate, reseed, best-of-guesses.

    problems    : one Problem or a list of them
    x           : [nq, ld] float64 (row q uses its problem's first d entries)
    t, N        : [nq] times and RK4 step counts
    problem_idx : [nq] index into problems (None: all 0)
    query_ids   : [nq] global query index used in the Philox counter (None: 0..nq-1)
    guesses     : per-problem number of initial guesses (None: O.n_guesses for all)
    O may also be a list with one Opts per problem (each with its own guesses).
    Returns a dict of arrays: phi, v [nq, ld], status, and per-trial
    diagnostics ([nq, T] with T the largest trial count, guesses plus the
    reseed budget; trials that did not run stay NaN / -1): slot_F, slot_res,
    slot_pass, slot_iters, slot_round, slot_slot (the slot of the draw),
    slot_v [nq, T, ld].  Trial g < guesses is slot g.
    """
    lib = _load()
    probs = problems if isinstance(problems, (list, tuple)) else [problems]
    cprobs = [p.c() for p in probs]
    olist = list(O) if isinstance(O, (list, tuple)) else [O] * len(probs)
    if guesses is None:
        gper = [o.n_guesses for o in olist]
    else:
        gper = [int(g) for g in guesses]
    copts = []
    for o_, g in zip(olist, gper):
        o = o_.c()
        o.n_guesses = g
        copts.append(o)
    x = _f64(x)
    nq = x.shape[0]
    ld = x.shape[1]
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), (nq,)).copy()
    N = np.broadcast_to(np.asarray(N, dtype=np.int64), (nq,)).copy()
    pidx = np.zeros(nq, dtype=np.int64) if problem_idx is None else np.asarray(problem_idx, dtype=np.int64)
    qids = np.arange(nq, dtype=np.int64) if query_ids is None else np.asarray(query_ids, dtype=np.int64)
    tper = [lib.orc_trials(C.byref(o)) for o in copts]
    T = max(tper)
    phi = np.full(nq, np.nan)
    vout = np.full((nq, ld), np.nan)
    status = np.zeros(nq, dtype=np.int32)
    sF = np.full((nq, T), np.nan)
    sR = np.full((nq, T), np.nan)
    sP = np.zeros((nq, T), dtype=np.int32)
    sI = np.zeros((nq, T), dtype=np.int32)
    sRd = np.full((nq, T), -1, dtype=np.int32)
    sS = np.full((nq, T), -1, dtype=np.int32)
    sV = np.full((nq, T, ld), np.nan)
    _IP = C.POINTER(C.c_int)

    def one(q):
        P = probs[pidx[q]]
        d = P.d
        g = tper[pidx[q]]
        xq = np.ascontiguousarray(x[q, :d])
        ph = C.c_double(0.0)
        vs = np.zeros(d)
        f, r_ = np.full(g, np.nan), np.full(g, np.nan)
        pa, it = np.zeros(g, dtype=np.int32), np.zeros(g, dtype=np.int32)
        rd, sl = np.full(g, -1, dtype=np.int32), np.full(g, -1, dtype=np.int32)
        sv = np.full(g * d, np.nan)
        st = lib.orc_solve_query(C.byref(cprobs[pidx[q]]), C.byref(copts[pidx[q]]), int(qids[q]), _dp(xq),
                                 float(t[q]), int(N[q]), C.byref(ph), _dp(vs), _dp(f), _dp(r_),
                                 pa.ctypes.data_as(_IP), it.ctypes.data_as(_IP), rd.ctypes.data_as(_IP), _dp(sv),
                                 sl.ctypes.data_as(_IP))
        phi[q] = ph.value
        vout[q, :d] = vs
        status[q] = st
        sF[q, :g], sR[q, :g], sP[q, :g], sI[q, :g], sRd[q, :g], sS[q, :g] = f, r_, pa, it, rd, sl
        sV[q, :g, :d] = sv.reshape(g, d)

    nthreads = threads or default_threads()
    if nthreads <= 1 or nq == 1:
        for q in range(nq):
            one(q)
    else:
        with ThreadPoolExecutor(max_workers=nthreads) as ex:
            list(ex.map(one, range(nq)))
    return dict(phi=phi, v=vout, status=status, slot_F=sF, slot_res=sR, slot_pass=sP, slot_iters=sI,
                slot_round=sRd, slot_slot=sS, slot_v=sV, threads=nthreads)
