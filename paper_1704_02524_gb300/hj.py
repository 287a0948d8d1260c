"""Thin Python binding of libhj.so (include/hj.h), argument marshalling only.

Every entry point keeps the C name and takes torch CUDA tensors (or None
for nullable arguments); the work runs in the library's CUDA kernels on the
current torch stream.  There is no CPU path: if libhj.so is missing or no
GPU is present, the calls raise.

    ctx = hj_create(problems, opts, device=0)
    hj_solve(ctx, q_begin, x, t, n_steps, problem_idx) -> (phi, v, status)
    hj_eval_functional / hj_grad / hj_certify / hj_guesses
    Functional.apply(ctx, x, t, v, n_steps, problem_idx)  # autograd on v
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhj.so")

HJ_OK, HJ_EINVAL, HJ_ENOMEM, HJ_ECUDA, HJ_ETIMEOUT, HJ_EUNSUPPORTED = range(6)
(HJ_FAM_QUAD_ISO, HJ_FAM_SPEED_QUAD, HJ_FAM_SMOOTH_NONCONVEX, HJ_FAM_LINEAR_QUAD, HJ_FAM_BUMP_NORM,
 HJ_FAM_SPLIT_NORM, HJ_FAM_HARMONIC, HJ_FAM_EVANS, HJ_FAM_LINEAR_GAME) = range(9)
HJ_LAX, HJ_HOPF, HJ_HUYGENS = 0, 1, 2
HJ_G_QUAD_SHIFT, HJ_G_DIAG_QUAD, HJ_G_ELLIPSE = 0, 1, 2
HJ_GRAD_FD_CENTRAL, HJ_GRAD_FD_FORWARD, HJ_GRAD_ADJOINT, HJ_GRAD_ADJOINT_CG = 0, 1, 2, 3
HJ_QUAD_RK4, HJ_QUAD_RECT, HJ_ODE_EULER = 0, 1, 2
HJ_PREC_FP32, HJ_PREC_FP64 = 0, 1
HJ_ST_CERTIFIED, HJ_ST_MAX_ITERS, HJ_ST_NONFINITE, HJ_ST_RESEEDED = 1, 2, 4, 8

EXPORTED = ("hj_create", "hj_destroy", "hj_eval_functional", "hj_grad", "hj_certify", "hj_solve", "hj_guesses",
            "hj_last_solve_info", "hj_set_tuning", "hj_last_error", "hj_solve_noalloc", "hj_autotune",
            "hj_set_graph", "hj_fp32_fma_rate")


class hj_solver_opts(C.Structure):
    _fields_ = [("n_steps_default", C.c_int), ("quad", C.c_int), ("grad", C.c_int), ("fd_h", C.c_double),
                ("step", C.c_double), ("max_iters", C.c_int), ("halving_period", C.c_int), ("eps", C.c_double),
                ("adapt", C.c_int), ("grow", C.c_double), ("shrink", C.c_double), ("step_max", C.c_double),
                ("n_guesses", C.c_int), ("max_trials", C.c_int), ("max_rounds", C.c_int), ("seed", C.c_uint64),
                ("guess_dist", C.c_int), ("cert_tol", C.c_double), ("precision", C.c_int), ("kahan", C.c_int),
                ("coarse_div", C.c_int), ("coarse_eps", C.c_double)]


class hj_problem_desc(C.Structure):
    _fields_ = [("d", C.c_int), ("family", C.c_int), ("principle", C.c_int), ("g_kind", C.c_int), ("m", C.c_int),
                ("n_neg", C.c_int), ("s_eps", C.c_double), ("n_guesses", C.c_int),
                ("params", C.POINTER(C.c_double)), ("n_params", C.c_size_t),
                ("solver", C.POINTER(hj_solver_opts))]


class hj_solve_info(C.Structure):
    _fields_ = [("n_queries", C.c_int64), ("n_pairs", C.c_int64), ("iterations", C.c_int64),
                ("functional_evals", C.c_int64), ("gradient_evals", C.c_int64), ("rk4_steps", C.c_int64),
                ("algorithmic_flops", C.c_double), ("certify_flops", C.c_double), ("threads_per_pair", C.c_int),
                ("comps_per_thread", C.c_int), ("descent_launches", C.c_int), ("descent_ms", C.c_double),
                ("certify_ms", C.c_double), ("total_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("descent_ms_round0", C.c_double), ("tensor_flops", C.c_double), ("adjoint_steps", C.c_int64),
                ("nominal_flops", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libhj.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhj.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i64, i32p = C.c_void_p, C.c_int64, C.POINTER(C.c_int32)
    lib.hj_create.argtypes = [C.POINTER(hj_problem_desc), C.c_int, C.POINTER(hj_solver_opts), C.c_int,
                              C.POINTER(C.c_void_p)]
    lib.hj_destroy.argtypes = [vp]
    lib.hj_eval_functional.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
    lib.hj_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.hj_certify.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.hj_solve.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.hj_solve_noalloc.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.hj_guesses.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    lib.hj_last_solve_info.argtypes = [vp, C.POINTER(hj_solve_info)]
    lib.hj_set_tuning.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    lib.hj_autotune.argtypes = [vp, i64, vp, vp, vp, vp, C.c_int, i32p, vp]
    lib.hj_set_graph.argtypes = [vp, C.c_int]
    lib.hj_fp32_fma_rate.argtypes = [C.c_int, C.POINTER(C.c_double)]
    lib.hj_last_error.argtypes = [vp]
    lib.hj_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name != "hj_last_error":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class HJError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hj status {status}: {msg}")
        self.status = status


class Context:
    """Owns an hj_ctx; keeps the problem descriptions alive."""

    def __init__(self, handle: int, problems, opts: hj_solver_opts, device: int):
        self.handle = handle
        self.problems = problems
        self.opts = opts
        self.device = device
        self.ld = max(p.d for p in problems)
        self.dtype = torch.float64 if opts.precision == HJ_PREC_FP64 else torch.float32

    def close(self):
        if self.handle:
            load_library().hj_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(ctx: Optional[Context], st: int):
    if st != HJ_OK:
        lib = load_library()
        msg = lib.hj_last_error(ctx.handle if ctx else None)
        raise HJError(st, msg.decode() if msg else "")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev(ctx: Context, t: Optional[torch.Tensor], name: str, dtype=None, shape=None):
    if t is None:
        return None
    if not t.is_cuda or t.device.index != ctx.device:
        raise ValueError(f"{name} must be on cuda:{ctx.device}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _solve_out(ctx: Context, out, n: int):
    """Caller-supplied (phi, v, status) of a solve: checked for device, dtype,
    shape and contiguity, since the kernels write every row of each."""
    if len(out) != 3:
        raise ValueError("out must be (phi, v, status)")
    phi, v, status = out
    _dev(ctx, phi, "phi", torch.float64, (n,))
    _dev(ctx, v, "v", ctx.dtype, (n, ctx.ld))
    _dev(ctx, status, "status", torch.int32, (n,))
    for name, o in (("phi", phi), ("v", v), ("status", status)):
        if o is None:
            raise ValueError(f"out {name} must be a tensor")
    return phi, v, status


def opts_from_dict(solver: Dict, precision: int = HJ_PREC_FP32, n_steps_default: int = 64,
                   kahan: int = 1) -> hj_solver_opts:
    grad = {"fd_central": HJ_GRAD_FD_CENTRAL, "fd_forward": HJ_GRAD_FD_FORWARD, "adjoint": HJ_GRAD_ADJOINT,
            "adjoint_cg": HJ_GRAD_ADJOINT_CG}
    quad = {"rk4": HJ_QUAD_RK4, "rect": HJ_QUAD_RECT, "euler": HJ_QUAD_RK4 | HJ_ODE_EULER,
            "euler_rect": HJ_QUAD_RECT | HJ_ODE_EULER}
    return hj_solver_opts(n_steps_default, quad[solver["quad"]], grad[solver["grad"]], solver["fd_h"],
                          solver["step"], solver["max_iters"], solver["halving_period"], solver["eps"],
                          solver["adapt"], solver["grow"], solver["shrink"], solver["step_max"],
                          solver["n_guesses"], solver["max_trials"], solver["max_rounds"],
                          solver["seed"] & (2 ** 64 - 1), solver["guess_dist"], solver["cert_tol"], precision, kahan,
                          solver.get("coarse_div", 1), solver.get("coarse_eps", 1e-4))


def hj_create(problems: Sequence, opts: hj_solver_opts, device: int = 0) -> Context:
    """problems: objects with d, family, principle, g_kind, m, n_neg, s_eps,
    n_guesses and params() (the flat parameter vector of include/hj.h), and
    optionally `solver` (a dict as for opts_from_dict: that problem's own
    descent constants)."""
    lib = load_library()
    arr = (hj_problem_desc * len(problems))()
    keep: List = []
    for i, p in enumerate(problems):
        par = np.ascontiguousarray(np.asarray(p.params(), dtype=np.float64))
        keep.append(par)
        sol = getattr(p, "solver", None)
        sp = None
        if sol is not None:
            so = opts_from_dict(sol, opts.precision, opts.n_steps_default, opts.kahan)
            keep.append(so)
            sp = C.pointer(so)
        arr[i] = hj_problem_desc(p.d, p.family, p.principle, p.g_kind, getattr(p, "m", 0), getattr(p, "n_neg", 0),
                                 getattr(p, "s_eps", 1e-6), getattr(p, "n_guesses", 0),
                                 par.ctypes.data_as(C.POINTER(C.c_double)), par.size, sp)
    h = C.c_void_p()
    st = lib.hj_create(arr, len(problems), C.byref(opts), device, C.byref(h))
    _check(None, st)
    return Context(h.value, list(problems), opts, device)


def hj_destroy(ctx: Context):
    ctx.close()


def hj_eval_functional(ctx: Context, x: torch.Tensor, t: torch.Tensor, v: torch.Tensor,
                       n_steps: Optional[torch.Tensor] = None, problem_idx: Optional[torch.Tensor] = None,
                       F: Optional[torch.Tensor] = None) -> torch.Tensor:
    n = x.shape[0]
    _dev(ctx, x, "x", ctx.dtype, (n, ctx.ld)); _dev(ctx, t, "t", ctx.dtype, (n,))
    _dev(ctx, v, "v", ctx.dtype, (n, ctx.ld))
    _dev(ctx, n_steps, "n_steps", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    F = torch.empty(n, dtype=ctx.dtype, device=x.device) if F is None else _dev(ctx, F, "F", ctx.dtype, (n,))
    _check(ctx, load_library().hj_eval_functional(ctx.handle, n, _ptr(problem_idx), _ptr(x), _ptr(t),
                                                  _ptr(n_steps), _ptr(v), _ptr(F), _stream(x.device)))
    return F


def hj_grad(ctx: Context, x: torch.Tensor, t: torch.Tensor, v: torch.Tensor,
            n_steps: Optional[torch.Tensor] = None, problem_idx: Optional[torch.Tensor] = None):
    n = x.shape[0]
    _dev(ctx, x, "x", ctx.dtype, (n, ctx.ld)); _dev(ctx, t, "t", ctx.dtype, (n,))
    _dev(ctx, v, "v", ctx.dtype, (n, ctx.ld))
    _dev(ctx, n_steps, "n_steps", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    F = torch.empty(n, dtype=ctx.dtype, device=x.device)
    G = torch.zeros(n, ctx.ld, dtype=ctx.dtype, device=x.device)
    _check(ctx, load_library().hj_grad(ctx.handle, n, _ptr(problem_idx), _ptr(x), _ptr(t), _ptr(n_steps), _ptr(v),
                                       _ptr(F), _ptr(G), _stream(x.device)))
    return F, G


def hj_certify(ctx: Context, x: torch.Tensor, t: torch.Tensor, v: torch.Tensor,
               n_steps: Optional[torch.Tensor] = None, problem_idx: Optional[torch.Tensor] = None):
    n = x.shape[0]
    _dev(ctx, x, "x", ctx.dtype, (n, ctx.ld)); _dev(ctx, t, "t", ctx.dtype, (n,))
    _dev(ctx, v, "v", ctx.dtype, (n, ctx.ld))
    _dev(ctx, n_steps, "n_steps", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    R = torch.empty(n, dtype=torch.float64, device=x.device)
    P = torch.empty(n, dtype=torch.uint8, device=x.device)
    F = torch.empty(n, dtype=torch.float64, device=x.device)
    _check(ctx, load_library().hj_certify(ctx.handle, n, _ptr(problem_idx), _ptr(x), _ptr(t), _ptr(n_steps),
                                          _ptr(v), _ptr(R), _ptr(P), _ptr(F), _stream(x.device)))
    return F, R, P


def hj_solve(ctx: Context, x: torch.Tensor, t: torch.Tensor, n_steps: Optional[torch.Tensor] = None,
             problem_idx: Optional[torch.Tensor] = None, q_begin: int = 0, out=None):
    """Returns (phi [nq] float64, v [nq, ld], status [nq] int32)."""
    n = x.shape[0]
    _dev(ctx, x, "x", ctx.dtype, (n, ctx.ld)); _dev(ctx, t, "t", ctx.dtype, (n,))
    _dev(ctx, n_steps, "n_steps", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    if out is None:
        phi = torch.empty(n, dtype=torch.float64, device=x.device)
        v = torch.zeros(n, ctx.ld, dtype=ctx.dtype, device=x.device)
        status = torch.empty(n, dtype=torch.int32, device=x.device)
    else:
        phi, v, status = _solve_out(ctx, out, n)
    _check(ctx, load_library().hj_solve(ctx.handle, q_begin, n, _ptr(problem_idx), _ptr(x), _ptr(t), _ptr(n_steps),
                                        _ptr(phi), _ptr(v), _ptr(status), _stream(x.device)))
    return phi, v, status


def hj_solve_noalloc(ctx: Context, x: torch.Tensor, t: torch.Tensor, n_steps: Optional[torch.Tensor] = None,
                     problem_idx: Optional[torch.Tensor] = None, q_begin: int = 0, out=None):
    """hj_solve without any device allocation inside the library (its scratch
    is a fixed static array); for callers that cannot allocate while solving.
    The output tensors are the caller's: pass them in `out` to keep the call
    free of allocations on the Python side too."""
    n = x.shape[0]
    _dev(ctx, x, "x", ctx.dtype, (n, ctx.ld)); _dev(ctx, t, "t", ctx.dtype, (n,))
    _dev(ctx, n_steps, "n_steps", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    if out is None:
        phi = torch.empty(n, dtype=torch.float64, device=x.device)
        v = torch.zeros(n, ctx.ld, dtype=ctx.dtype, device=x.device)
        status = torch.empty(n, dtype=torch.int32, device=x.device)
    else:
        phi, v, status = _solve_out(ctx, out, n)
    _check(ctx, load_library().hj_solve_noalloc(ctx.handle, q_begin, n, _ptr(problem_idx), _ptr(x), _ptr(t),
                                                _ptr(n_steps), _ptr(phi), _ptr(v), _ptr(status), _stream(x.device)))
    return phi, v, status


def hj_guesses(ctx: Context, query_id: torch.Tensor, slot: torch.Tensor, rnd: torch.Tensor,
               problem_idx: Optional[torch.Tensor] = None) -> torch.Tensor:
    n = query_id.shape[0]
    _dev(ctx, query_id, "query_id", torch.int64, (n,)); _dev(ctx, slot, "slot", torch.int32, (n,))
    _dev(ctx, rnd, "round", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    v = torch.zeros(n, ctx.ld, dtype=ctx.dtype, device=query_id.device)
    _check(ctx, load_library().hj_guesses(ctx.handle, n, _ptr(query_id), _ptr(slot), _ptr(rnd), _ptr(problem_idx),
                                          _ptr(v), _stream(query_id.device)))
    return v


def hj_last_solve_info(ctx: Context) -> Dict:
    info = hj_solve_info()
    _check(ctx, load_library().hj_last_solve_info(ctx.handle, C.byref(info)))
    return {name: getattr(info, name) for name, _ in hj_solve_info._fields_}


def hj_set_tuning(ctx: Context, problem: int, tpp: int = 0, ck_interval: int = 0):
    _check(ctx, load_library().hj_set_tuning(ctx.handle, problem, tpp, ck_interval))


def hj_fp32_fma_rate(device: int = 0) -> float:
    """Measured FP32 FMA rate of the device in TFLOP/s (FMA-chain microbenchmark)."""
    out = C.c_double(0.0)
    st = load_library().hj_fp32_fma_rate(int(device), C.byref(out))
    if st != HJ_OK:
        raise HJError(st, f"hj_fp32_fma_rate failed with status {st}")
    return out.value


def hj_set_graph(ctx: Context, enable: bool = True):
    _check(ctx, load_library().hj_set_graph(ctx.handle, 1 if enable else 0))


def hj_autotune(ctx: Context, x: torch.Tensor, t: torch.Tensor, n_steps: Optional[torch.Tensor] = None,
                problem_idx: Optional[torch.Tensor] = None, iters: int = 4) -> List[int]:
    """Times the launch candidates of every problem on the sample (x, t, ...)
    and applies the fastest; returns the chosen threads per pair (0 = automatic)."""
    n = x.shape[0]
    _dev(ctx, x, "x", ctx.dtype, (n, ctx.ld)); _dev(ctx, t, "t", ctx.dtype, (n,))
    _dev(ctx, n_steps, "n_steps", torch.int32, (n,)); _dev(ctx, problem_idx, "problem_idx", torch.int32, (n,))
    out = (C.c_int32 * len(ctx.problems))()
    _check(ctx, load_library().hj_autotune(ctx.handle, n, _ptr(problem_idx), _ptr(x), _ptr(t), _ptr(n_steps), iters,
                                           out, _stream(x.device)))
    return list(out)


class Functional(torch.autograd.Function):
    """F(v) (Lax) or G(v) (Hopf) with the adjoint gradient as backward:
    forward calls hj_eval_functional, backward calls hj_grad."""

    @staticmethod
    def forward(fctx, ctx: Context, x, t, v, n_steps=None, problem_idx=None):
        v = v.contiguous()
        fctx.hj = ctx
        fctx.save_for_backward(x, t, v, n_steps, problem_idx)
        return hj_eval_functional(ctx, x, t, v, n_steps, problem_idx)

    @staticmethod
    def backward(fctx, gout):
        x, t, v, n_steps, problem_idx = fctx.saved_tensors
        _, G = hj_grad(fctx.hj, x, t, v, n_steps, problem_idx)
        return None, None, None, G * gout[:, None], None, None


def hj_last_error(ctx: Optional[Context] = None) -> str:
    msg = load_library().hj_last_error(ctx.handle if ctx else None)
    return msg.decode() if msg else ""
