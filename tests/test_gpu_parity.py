"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: fp32 functional values 2e-5 relative (RK4 state and Kahan
quadrature in binary32 over <= 256 steps); fp64 paths 1e-11; solved phi
within 1e-4 (1 + |phi|) as the accuracy target of the solver states;
integer/bit outputs (starts, certificate decisions) exactly.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1704_02524_gb300 import workloads as W
from tests.helpers import QUAD_CODES, oracle_opts, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def hj():
    from paper_1704_02524_gb300 import hj as H
    H.load_library()
    return H


def _spec(family, principle, d, seed=0, n_neg=1, s_eps=1e-6, g_kind=None, m=None):
    rng = np.random.default_rng(seed)
    if g_kind is None:
        g_kind = {W.FAM_SMOOTH_NONCONVEX: W.G_DIAG_QUAD, W.FAM_BUMP_NORM: W.G_ELLIPSE, W.FAM_SPLIT_NORM: W.G_ELLIPSE,
                  W.FAM_HARMONIC: W.G_ELLIPSE, W.FAM_EVANS: W.G_ELLIPSE,
                  W.FAM_LINEAR_GAME: W.G_ELLIPSE}.get(family, W.G_QUAD_SHIFT)
    A = B = None
    if family == W.FAM_LINEAR_QUAD:
        G0 = rng.normal(size=(d, d))
        A = W.f32(G0 / (2 * np.linalg.norm(G0, 2)))
        B = W.f32(rng.normal(size=(d, m or max(1, d // 2))) / np.sqrt(d))
    return W.ProblemSpec(d=d, family=family, principle=principle, g_kind=g_kind,
                         w=W.f32(rng.normal(size=d) / np.sqrt(d)), a=W.f32(rng.uniform(-1, 1, d)),
                         sigma=W.f32(rng.uniform(0.5, 2, d)), A=A, B=B, n_neg=n_neg, s_eps=s_eps, n_guesses=4,
                         xc=W.f32(rng.uniform(-0.5, 0.5, d)), kappa=3.0, mu=1.5,
                         hsign=-1.0 if principle == W.HOPF else 1.0, xcb=W.f32(rng.uniform(-0.5, 0.5, d)),
                         ksplit=d // 2, alpha_a=1.5, alpha_b=-1.25, beta=2.0, gamma0=1.0, r_c=1.0, r_d=0.6,
                         omega=3.0)


def _rows(n, d, seed, prec):
    rng = np.random.default_rng(seed)
    x = W.f32(rng.uniform(-1, 1, (n, d)))
    v = W.f32(rng.uniform(-1.5, 1.5, (n, d)))
    t = W.f32(rng.uniform(0.2, 1.0, n))
    N = rng.integers(1, 70, n).astype(np.int32)
    return x, v, t, N


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


FAMS = [(W.FAM_QUAD_ISO, W.LAX), (W.FAM_QUAD_ISO, W.HOPF), (W.FAM_SPEED_QUAD, W.LAX), (W.FAM_SPEED_QUAD, W.HOPF),
        (W.FAM_SMOOTH_NONCONVEX, W.HOPF), (W.FAM_SMOOTH_NONCONVEX, W.LAX), (W.FAM_LINEAR_QUAD, W.LAX),
        (W.FAM_LINEAR_QUAD, W.HOPF), (W.FAM_BUMP_NORM, W.LAX), (W.FAM_BUMP_NORM, W.HOPF),
        (W.FAM_SPLIT_NORM, W.LAX), (W.FAM_SPLIT_NORM, W.HOPF), (W.FAM_HARMONIC, W.LAX), (W.FAM_HARMONIC, W.HOPF),
        (W.FAM_EVANS, W.LAX), (W.FAM_EVANS, W.HOPF), (W.FAM_LINEAR_GAME, W.LAX), (W.FAM_LINEAR_GAME, W.HOPF)]


@pytest.mark.parametrize("family,principle", FAMS)
@pytest.mark.parametrize("d", [1, 3, 10, 20, 37])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_functional_and_gradient_match_oracle(hj, family, principle, d, prec):
    if family == W.FAM_EVANS and d < 2:
        pytest.skip("the Evans-type family needs d >= 2")
    spec = _spec(family, principle, d, seed=d, s_eps=1e-2)
    dt = torch.float32 if prec == "fp32" else torch.float64
    opts = hj.opts_from_dict(W.solver_constants(), hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64, 32)
    ctx = hj.hj_create([spec], opts, 0)
    n = 67  # several groups and a ragged tail
    x, v, t, N = _rows(n, d, 100 + d, prec)
    F = hj.hj_eval_functional(ctx, _t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32)).cpu().numpy()
    Fg, G = hj.hj_grad(ctx, _t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32))
    Fg, G = Fg.cpu().numpy(), G.cpu().numpy()
    P = oracle_problem(spec)
    tolF = 2e-5 if prec == "fp32" else 1e-11
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i])
        assert rel_err(F[i], Fo) <= tolF, (i, F[i], Fo)
        assert rel_err(Fg[i], Fo) <= tolF
        scale = 1 + np.abs(Go).max()
        assert np.abs(G[i] - Go).max() <= (5e-4 if prec == "fp32" else 1e-9) * scale, (i, G[i], Go)
    ctx.close()


@pytest.mark.parametrize("family,principle", FAMS)
@pytest.mark.parametrize("quad", ["euler", "euler_rect"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_forward_euler_functional_gradient_and_certificate_match_oracle(hj, family, principle, quad, prec):
    # forward Euler (Sec. 4.2's example solver) on every family: values,
    # discrete-adjoint gradients and the FP64 certificate against the oracle
    d = 13
    spec = _spec(family, principle, d, seed=40 + d, s_eps=1e-2)
    dt = torch.float32 if prec == "fp32" else torch.float64
    solver = W.solver_constants(quad=quad, cert_tol=0.3)
    ctx = hj.hj_create([spec], hj.opts_from_dict(solver, hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64, 32),
                       0)
    n = 67
    x, v, t, N = _rows(n, d, 200 + family, prec)
    args = (_t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32))
    F = hj.hj_eval_functional(ctx, *args).cpu().numpy()
    Fg, G = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
    Fc, R, Pa = (a.cpu().numpy() for a in hj.hj_certify(ctx, *args))
    P = oracle_problem(spec)
    q = QUAD_CODES[quad]
    tolF = 2e-5 if prec == "fp32" else 1e-11
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i], quad=q)
        assert rel_err(F[i], Fo) <= tolF and rel_err(Fg[i], Fo) <= tolF, (i, F[i], Fo)
        assert np.abs(G[i] - Go).max() <= (5e-4 if prec == "fp32" else 1e-9) * (1 + np.abs(Go).max()), i
        Fco, Ro, ok = O.certify(P, x[i], t[i], int(N[i]), v[i], 0.3, quad=q)
        assert rel_err(Fc[i], Fco) < 1e-11 and abs(R[i] - Ro) < 1e-11 and bool(Pa[i]) == ok, i
    ctx.close()


def test_solve_speed_quad_d10_with_forward_euler_matches_oracle(hj):
    # the whole solve (descent on the Euler-discretised functional, reseeds,
    # certificate) against the oracle run with the same integrator
    wl = W.c2_speed_quad(nq_x=16)
    wl.solver = dict(wl.solver, quad="euler")
    phi, v, st, ref, info = _solve_both(hj, wl, 48)
    assert np.all(rel_err(phi, ref["phi"]) <= 1e-4), rel_err(phi, ref["phi"]).max()
    assert np.array_equal(st & 1, ref["status"] & 1)
    assert info["rk4_steps"] > 0


def _huygens_node_gaps(spec, x, v, t, N):
    # gap between the two smallest g over the grid nodes of each row (the
    # Lax functional of the same path with s_eps = 0 has no running cost,
    # so its value after n steps of length t/N is g at node n)
    lax = oracle_problem(W.ProblemSpec(**{**spec.__dict__, "principle": W.LAX}))
    gaps = []
    for i in range(len(x)):
        h = t[i] / N[i]
        g = np.sort([O.functional(lax, x[i], n * h, n, v[i]) if n else 0.5 * (np.sum(x[i][:spec.d] ** 2 /
                     spec.sigma ** 2) - 1) for n in range(int(N[i]) + 1)])
        gaps.append((g[1] - g[0]) / (1 + abs(g[0])))
    return np.array(gaps)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("quad", ["rk4", "euler"])
@pytest.mark.parametrize("d", [2, 13])
def test_huygens_functional_gradient_and_certificate_match_oracle(hj, prec, quad, d):
    # F^2 (eq. num_min) on H = c(x)|p| with the ellipse data: values, the
    # adjoint seeded at the minimising node, and the Lax certificate there.
    # The gradient is compared on rows whose two smallest node values differ
    # by more than the functional's rounding (else either node may win).
    spec = _spec(W.FAM_BUMP_NORM, W.HUYGENS, d, seed=50 + d, s_eps=0.0)
    dt = torch.float32 if prec == "fp32" else torch.float64
    solver = W.solver_constants(quad=quad, cert_tol=0.3)
    ctx = hj.hj_create([spec], hj.opts_from_dict(solver, hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64, 32),
                       0)
    n = 67
    x, v, t, N = _rows(n, d, 300 + d, prec)
    args = (_t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32))
    F = hj.hj_eval_functional(ctx, *args).cpu().numpy()
    Fg, G = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
    Fc, R, Pa = (a.cpu().numpy() for a in hj.hj_certify(ctx, *args))
    P = oracle_problem(spec)
    q = QUAD_CODES[quad]
    gaps = _huygens_node_gaps(spec, x, v, t, N)
    tie = 3e-5 if prec == "fp32" else 1e-10
    assert np.mean(gaps > tie) > 0.8
    tolF = 2e-5 if prec == "fp32" else 1e-11
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i], quad=q)
        assert rel_err(F[i], Fo) <= tolF and rel_err(Fg[i], Fo) <= tolF, (i, F[i], Fo)
        if gaps[i] > tie:
            assert np.abs(G[i] - Go).max() <= (5e-4 if prec == "fp32" else 1e-9) * (1 + np.abs(Go).max()), i
            Fco, Ro, ok = O.certify(P, x[i], t[i], int(N[i]), v[i], 0.3, quad=q)
            assert rel_err(Fc[i], Fco) < 1e-11 and abs(R[i] - Ro) < 1e-11 and bool(Pa[i]) == ok, i
    ctx.close()


# The solves below run in FP64, these workloads' default precision (the
# paper's own): their forward differences with sigma = 1e-3 carry ~1e-4 of
# binary32 rounding in every derivative, and on these flat or kinked
# functionals that moves where a start stops (or which basin it ends in) by
# more than the 1e-4 gate, so binary32 solves of them are a stated gap (their
# measured errors are in the design notes); the binary32 functionals,
# gradients and certificates of these families are checked row by row above.
def test_paper_mode_example3_huygens_solve_matches_oracle(hj):
    # F^2 in the paper's numerics on the Example 3 grid: the whole solve
    # against the oracle on every row, and min g = -1/2 wherever the
    # reachable set holds the ellipse's centre (|x| < t suffices, since c >= 1)
    wl = W.bump_ex3(n_side=128, principle=W.HUYGENS, ds=0.005)
    assert wl.precision == "fp64"
    near = np.flatnonzero(np.hypot(wl.x[:, 0], wl.x[:, 1]) < 0.25)
    w = wl.take(np.concatenate([np.arange(0, wl.nq, wl.nq // 64)[:64], near]))
    phi, v, st, ref, info = _solve_both(hj, w, w.nq)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), (err.max(), int(np.argmax(err)))
    assert np.array_equal(st & 1, ref["status"] & 1)
    # truth where the reachable set holds the centre: never below min g, and
    # min g itself on nearly every row (a row whose five starts all stall
    # short of the ray through the centre stays above it, on both sides)
    assert len(near) > 0 and np.all(phi[64:] >= -0.5 - 1e-5)
    assert np.mean(np.abs(phi[64:] + 0.5) < 1e-4) >= 0.9


@pytest.mark.parametrize("descent", ["paper", "cg"])
def test_example5_split_norm_hopf_solve_matches_oracle(hj, descent):
    # Sec. 6 Example 5 (H = c(x)|p_1| - c(-x)|p_2|, Hopf, twenty starts) on 64
    # points spread over the [-3,3]^2 grid, in the paper's numerics and with
    # the conjugate-gradient momentum on the same Euler functional, every row
    wl = W.split_ex5(n_side=128, descent=descent)
    assert wl.precision == "fp64"
    w = wl.take(np.arange(0, wl.nq, wl.nq // 64)[:64])
    phi, v, st, ref, info = _solve_both(hj, w, w.nq)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), (err.max(), int(np.argmax(err)))
    assert np.array_equal(st & 1, ref["status"] & 1)


@pytest.mark.parametrize("example", ["ex2_minus", "ex2_plus", "ex2_rosenbrock", "ex4"])
def test_examples_2_and_4_solve_matches_oracle(hj, example):
    # Sec. 6 Examples 2 (harmonic oscillator, both signs, Hopf; the
    # Rosenbrock data with the Lax functional) and 4 (Evans-type non-convex,
    # Hopf) in the paper's numerics on 64 points spread over the [-3,3]^2
    # grid, every row
    if example == "ex4":
        wl = W.evans_ex4(n_side=128)
    elif example == "ex2_rosenbrock":
        wl = W.harmonic_ex2(n_side=128, rosenbrock=True)
    else:
        wl = W.harmonic_ex2(n_side=128, sign=-1.0 if example == "ex2_minus" else 1.0)
    assert wl.precision == "fp64"
    w = wl.take(np.arange(0, wl.nq, wl.nq // 64)[:64])
    phi, v, st, ref, info = _solve_both(hj, w, w.nq)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), (err.max(), int(np.argmax(err)))
    assert np.array_equal(st & 1, ref["status"] & 1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("r_d", [0.4, 1.0])
def test_linear_game_solve_matches_oracle(hj, prec, r_d):
    # the time-dependent game (Sec. 3.4, Example 3) at d = 16: convex
    # (r_d = 0.4, speed > 0) and sign-changing speed (r_d = 1.0), Hopf
    wl = W.linear_game(nq=96, r_d=r_d)
    prec_code = hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64
    phi, v, st, ref, info = _solve_both(hj, wl, 96, prec_code=prec_code)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), (err.max(), int(np.argmax(err)))
    assert np.array_equal(st & 1, ref["status"] & 1)


@pytest.mark.parametrize("name,sample", [("smooth_nonconvex_d20_hopf", 64), ("speed_quad_d10_lax", 64),
                                         ("linear_quad_d64_lax", 16)])
def test_full_size_workloads_match_oracle_on_sampled_queries(hj, name, sample):
    # the benchmark's full batches (65,536 d=20 Hopf queries x 16 starts;
    # 49,152 d=10 Lax queries x 8; 32,768 d=64 linear-quadratic queries on the
    # tensor-core tile kernel) in one solve each, with the library's automatic
    # launch choice; sampled queries against the oracle run one by one with the
    # same query ids (the Philox counters)
    builders = {"smooth_nonconvex_d20_hopf": W.c3_smooth_nonconvex, "speed_quad_d10_lax": W.c2_speed_quad,
                "linear_quad_d64_lax": W.c4_linear_quad}
    wl = builders[name]()
    spec = wl.problems[0]
    ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, int(wl.n_steps[0])), 0)
    phi, v, st = hj.hj_solve(ctx, _t(wl.x, torch.float32), _t(wl.t, torch.float32), _t(wl.n_steps, torch.int32))
    phi, st = phi.cpu().numpy(), st.cpu().numpy()
    ctx.close()
    ids = np.sort(np.random.default_rng(11).choice(wl.nq, sample, replace=False))
    ref = O.solve(oracle_problem(spec), oracle_opts(wl.solver, spec.n_guesses), wl.x[ids], wl.t[ids],
                  wl.n_steps[ids], query_ids=ids)
    err = rel_err(phi[ids], ref["phi"])
    assert np.all(err <= 1e-4), (err.max(), int(ids[np.argmax(err)]))
    assert np.array_equal(st[ids] & 1, ref["status"] & 1)


def test_fp32_fma_rate_microbenchmark_is_below_the_formula_peak(hj):
    # the measured FMA rate cannot exceed SMs x 128 lanes x 2 flop x the
    # highest clock this part runs (2.07 GHz; 2.2 as a margin) and, with 16
    # chains' worth of independent FMAs per scheduler slot, reaches most of it
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rate = hj.hj_fp32_fma_rate(0)
    bound = nsm * 128 * 2 * 2.2e9 / 1e12
    assert 0.5 * bound < rate < bound, (rate, bound)


def test_rosenbrock_data_rows_match_oracle(hj):
    # the non-convex data's value, gradient and certificate through the
    # harmonic family's Lax kernels (fp32 and fp64 rows)
    spec = W.harmonic_ex2(n_side=2, rosenbrock=True).problems[0]
    P = oracle_problem(spec)
    for prec, dt, tolF, tolG in (("fp32", torch.float32, 2e-5, 5e-4), ("fp64", torch.float64, 1e-11, 1e-9)):
        solver = W.solver_constants(quad="euler_rect", cert_tol=0.3)
        ctx = hj.hj_create([spec], hj.opts_from_dict(solver, hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64,
                                                     25), 0)
        x, v, t, N = _rows(67, 2, 400, prec)
        args = (_t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32))
        F = hj.hj_eval_functional(ctx, *args).cpu().numpy()
        Fg, G = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
        Fc, R, Pa = (a.cpu().numpy() for a in hj.hj_certify(ctx, *args))
        for i in range(67):
            Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i], quad=QUAD_CODES["euler_rect"])
            assert rel_err(F[i], Fo) <= tolF and rel_err(Fg[i], Fo) <= tolF, (prec, i)
            assert np.abs(G[i] - Go).max() <= tolG * (1 + np.abs(Go).max()), (prec, i)
            Fco, Ro, ok = O.certify(P, x[i], t[i], int(N[i]), v[i], 0.3, quad=QUAD_CODES["euler_rect"])
            assert abs(R[i] - Ro) < 1e-11 and bool(Pa[i]) == ok, (prec, i)
        ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_paper_mode_example3_solve_matches_oracle(hj, prec):
    # Sec. 6 Example 3 (H+ = c(x)|p|, ellipse data, t = 0.3) in the paper's
    # numerics -- forward Euler, rectangle rule, forward differences,
    # Algorithm 1 with halving, five starts -- on 96 points spread over the
    # [-3,3]^2 grid, against the oracle run with the same constants
    wl = W.bump_ex3(n_side=128, precision=prec)
    w = wl.take(np.arange(0, wl.nq, wl.nq // 96)[:96])
    phi, v, st, ref, info = _solve_both(hj, w, w.nq)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), (err.max(), int(np.argmax(err)))
    assert np.array_equal(st & 1, ref["status"] & 1)
    assert info["iterations"] > 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("dist", [0, 1])
def test_starts_are_bit_exact(hj, prec, dist):
    spec = _spec(W.FAM_SMOOTH_NONCONVEX, W.HOPF, 20)
    dt = torch.float32 if prec == "fp32" else torch.float64
    solver = W.solver_constants(guess_dist=dist, seed=0x1234ABCD5678)
    ctx = hj.hj_create([spec], hj.opts_from_dict(solver, hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64), 0)
    rng = np.random.default_rng(5)
    n = 300
    q = rng.integers(0, 2 ** 40, n).astype(np.int64)
    s = rng.integers(0, 20, n).astype(np.int32)
    r = rng.integers(0, 5, n).astype(np.int32)
    v = hj.hj_guesses(ctx, _t(q, torch.int64), _t(s, torch.int32), _t(r, torch.int32)).cpu().numpy()
    for i in range(n):
        ref = O.guess(solver["seed"], int(q[i]), int(s[i]), int(r[i]), 20, dist)
        if prec == "fp32":
            ref = ref.astype(np.float32).astype(np.float64)
        assert np.array_equal(v[i].astype(np.float64), ref), i
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_certificate_matches_oracle(hj, prec):
    spec = _spec(W.FAM_SMOOTH_NONCONVEX, W.HOPF, 20, seed=3)
    dt = torch.float32 if prec == "fp32" else torch.float64
    solver = W.solver_constants(cert_tol=0.3)
    ctx = hj.hj_create([spec], hj.opts_from_dict(solver, hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64, 64), 0)
    n = 50
    x, v, t, N = _rows(n, 20, 9, prec)
    F, R, Pa = hj.hj_certify(ctx, _t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32))
    F, R, Pa = F.cpu().numpy(), R.cpu().numpy(), Pa.cpu().numpy()
    P = oracle_problem(spec)
    for i in range(n):
        Fo, Ro, ok = O.certify(P, x[i], t[i], int(N[i]), v[i], 0.3)
        assert rel_err(F[i], Fo) < 1e-11 and abs(R[i] - Ro) < 1e-11
        assert bool(Pa[i]) == ok
    ctx.close()


def _solve_both(hj, wl, nq, prec_code=None, tpp=0):
    w = wl.head(nq)
    spec = w.problems[0]
    prec = prec_code if prec_code is not None else (hj.HJ_PREC_FP64 if w.precision == "fp64" else hj.HJ_PREC_FP32)
    dt = torch.float64 if prec == hj.HJ_PREC_FP64 else torch.float32
    ctx = hj.hj_create(w.problems, hj.opts_from_dict(w.solver, prec, int(w.n_steps[0])), 0)
    if tpp:
        hj.hj_set_tuning(ctx, 0, tpp, 0)
    phi, v, st = hj.hj_solve(ctx, _t(w.x, dt), _t(w.t, dt), _t(w.n_steps, torch.int32))
    info = hj.hj_last_solve_info(ctx)
    ctx.close()
    key = (w.name, nq, repr(sorted(w.solver.items())), repr([p.params().tolist() for p in w.problems]),
           hash(w.x.tobytes()), hash(w.t.tobytes()), hash(w.n_steps.tobytes()))
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = O.solve(oracle_problem(spec), oracle_opts(w.solver, spec.n_guesses), w.x, w.t, w.n_steps)
    return phi.cpu().numpy(), v.cpu().numpy(), st.cpu().numpy(), _ORACLE_CACHE[key], info


_ORACLE_CACHE = {}


def test_solve_quad_iso_d2_fp64_matches_closed_form_and_oracle(hj):
    wl = W.c1_quad_iso()
    phi, v, st, ref, info = _solve_both(hj, wl, 64)
    exact = np.sum(wl.x ** 2, axis=1) / 4
    assert np.abs(phi - exact).max() < 1e-12
    assert np.abs(phi - ref["phi"]).max() < 1e-12
    assert np.array_equal(st, ref["status"])
    assert info["iterations"] == 64 * 4 * 400


def test_solve_speed_quad_d10_matches_oracle(hj):
    phi, v, st, ref, info = _solve_both(hj, W.c2_speed_quad(nq_x=16), 48)
    assert np.all(rel_err(phi, ref["phi"]) <= 1e-4)
    assert np.array_equal(st & 1, ref["status"] & 1)


def test_solve_smooth_nonconvex_d20_matches_oracle(hj):
    phi, v, st, ref, info = _solve_both(hj, W.c3_smooth_nonconvex(nq=40), 40)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), err.max()
    assert np.array_equal(st & 1, ref["status"] & 1)


@pytest.mark.parametrize("nq,split", [(40, False), (300, True)])
def test_solve_phi_is_the_fp64_functional_at_the_returned_start(hj, nq, split):
    # phi comes from an FP64 evaluation at each query's returned v (for this
    # family the one-thread-per-query reduced-state kernel): the oracle's FP64
    # functional at the same v agrees to rounding, in hj_solve and in the
    # no-alloc entry point
    wl = W.c3_smooth_nonconvex(nq=nq).head(nq)
    ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, int(wl.n_steps[0])), 0)
    args = (_t(wl.x, torch.float32), _t(wl.t, torch.float32), _t(wl.n_steps, torch.int32))
    phi, v, st = (hj.hj_solve_noalloc if split else hj.hj_solve)(ctx, *args)
    torch.cuda.synchronize()
    ctx.close()
    phi, v = phi.cpu().numpy(), v.cpu().numpy().astype(np.float64)
    P = oracle_problem(wl.problems[0])
    for i in range(0, nq, 7 if split else 1):
        G = O.functional(P, wl.x[i], float(wl.t[i]), int(wl.n_steps[i]), v[i])
        assert abs(phi[i] + G) <= 1e-12 * (1 + abs(G)), (i, phi[i], -G)


@pytest.mark.parametrize("max_trials", [20, 40])
def test_reseed_budget_runs_in_one_round_from_the_failed_slots(hj, max_trials):
    # cert_tol = 0 fails every start, so every query spends its whole budget:
    # 8 starts, then max_trials - 8 restarts drawn (slot j mod 8, round
    # 1 + j / 8) in one more round (draw rounds 1-2 for 20 trials, 1-4 for
    # 40).  Five descent iterations leave each trial near its start, so the
    # best of the trials, and with it phi, depends on every restart's draw
    # (phi changes on 16 and 20 of the 24 queries against no reseeding).
    # The smooth convex d=10 family keeps these unconverged trajectories
    # well conditioned (the oracle's phi moves by 2e-7 under a 1e-7 change
    # of x; the non-convex family's smoothed |p_i| moves it by 5e-3).
    wl = W.c2_speed_quad(nq_x=16)
    wl.solver.update(cert_tol=0.0, max_iters=5, max_trials=max_trials, max_rounds=3)
    phi, v, st, ref, info = _solve_both(hj, wl, 24)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), err.max()
    assert np.all(st == hj.HJ_ST_RESEEDED | hj.HJ_ST_MAX_ITERS)
    assert np.array_equal(st, ref["status"])
    assert info["n_pairs"] == 24 * max_trials
    assert info["descent_launches"] == 2


@pytest.mark.parametrize("ck", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("quad", ["rk4", "rect", "euler", "euler_rect"])
def test_gradient_checkpoint_intervals_and_quadrature(hj, ck, quad):
    # every checkpoint interval (including ones that do not divide N), both
    # quadratures and both integrators give the oracle's exact gradient of
    # the discretised functional
    spec = _spec(W.FAM_SMOOTH_NONCONVEX, W.HOPF, 20, seed=11, s_eps=1e-2)
    solver = W.solver_constants(quad=quad)
    ctx = hj.hj_create([spec], hj.opts_from_dict(solver, hj.HJ_PREC_FP32, 64), 0)
    hj.hj_set_tuning(ctx, 0, 4, ck)
    n = 33
    x, v, t, N = _rows(n, 20, 21, "fp32")
    N = np.array([1, 2, 5, 17, 64, 100, 255, 256] * 5)[:n].astype(np.int32)
    F, G = hj.hj_grad(ctx, _t(x, torch.float32), _t(t, torch.float32), _t(v, torch.float32), _t(N, torch.int32))
    F, G = F.cpu().numpy(), G.cpu().numpy()
    P = oracle_problem(spec)
    q = QUAD_CODES[quad]
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i], quad=q)
        assert rel_err(F[i], Fo) <= 2e-5
        assert np.abs(G[i] - Go).max() <= 5e-4 * (1 + np.abs(Go).max()), (i, N[i])
    ctx.close()


def test_step_counts_outside_range_give_nan_not_memory_errors(hj):
    spec = _spec(W.FAM_SMOOTH_NONCONVEX, W.HOPF, 20)
    ctx = hj.hj_create([spec], hj.opts_from_dict(W.solver_constants(), hj.HJ_PREC_FP32, 64), 0)
    x, v, t, _ = _rows(4, 20, 3, "fp32")
    N = np.array([0, 257, -5, 1000], dtype=np.int32)
    F, G = hj.hj_grad(ctx, _t(x, torch.float32), _t(t, torch.float32), _t(v, torch.float32), _t(N, torch.int32))
    assert np.all(np.isnan(F.cpu().numpy())) and np.all(np.isnan(G.cpu().numpy()))
    E = hj.hj_eval_functional(ctx, _t(x, torch.float32), _t(t, torch.float32), _t(v, torch.float32),
                              _t(N, torch.int32))
    assert np.all(np.isnan(E.cpu().numpy()))
    ctx.close()


# Tolerances of the tensor-core tile kernel (split-precision BF16x3 stage
# products, relative error ~2^-16 per product, over up to 4 x 128 stages):
# functional 1e-4 relative, gradient 2e-3 of its scale.
TC_TOL_F, TC_TOL_G = 1e-4, 2e-3


@pytest.mark.parametrize("d,m", [(64, 32), (100, 32), (128, 64), (8, 3), (37, 18), (20, 32)])
@pytest.mark.parametrize("prec,path", [("fp32", "tc"), ("fp32", "lanes"), ("fp64", "lanes")])
@pytest.mark.parametrize("principle", [W.LAX, W.HOPF])
def test_linear_quadratic_functional_and_gradient_at_workload_sizes(hj, d, m, prec, path, principle):
    # "tc": the tensor-core tile kernel wherever the problem fits it (d <= 64
    # after padding), "lanes": the lane-group kernels (tuning override)
    spec = _spec(W.FAM_LINEAR_QUAD, principle, d, seed=d + m, m=m)
    dt = torch.float32 if prec == "fp32" else torch.float64
    opts = hj.opts_from_dict(W.lq_solver(), hj.HJ_PREC_FP32 if prec == "fp32" else hj.HJ_PREC_FP64, 100)
    ctx = hj.hj_create([spec], opts, 0)
    if path == "lanes":
        hj.hj_set_tuning(ctx, 0, 32, 0)
    tc = path == "tc" and d <= 64 and 2 * (-(-d // 16) * 16) + (-(-m // 16) * 16) <= 256
    n = 300 if tc else 37  # tiles of 128 rows: two full tiles and a ragged one
    rng = np.random.default_rng(d)
    x = W.f32(rng.normal(size=(n, d)))
    v = W.f32(rng.uniform(-2, 2, (n, d)))
    t = W.f32(rng.uniform(0.1, 2.0, n))
    N = rng.integers(1, 129, n).astype(np.int32)
    F = hj.hj_eval_functional(ctx, _t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32)).cpu().numpy()
    Fg, G = hj.hj_grad(ctx, _t(x, dt), _t(t, dt), _t(v, dt), _t(N, torch.int32))
    Fg, G = Fg.cpu().numpy(), G.cpu().numpy()
    P = oracle_problem(spec)
    tolF = TC_TOL_F if tc else (2e-5 if prec == "fp32" else 1e-11)
    tolG = TC_TOL_G if tc else (5e-4 if prec == "fp32" else 1e-9)
    errs = []
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i])
        scale = 1 + np.abs(Go).max()
        errs.append((rel_err(F[i], Fo), rel_err(Fg[i], Fo), np.abs(G[i] - Go).max() / scale))
    errs = np.array(errs)
    print(f"d={d} m={m} {prec} {path} tc={tc}: max rel err F {errs[:, 0].max():.2e} "
          f"F(grad call) {errs[:, 1].max():.2e} grad {errs[:, 2].max():.2e}")
    assert errs[:, 0].max() <= tolF and errs[:, 1].max() <= tolF
    assert errs[:, 2].max() <= tolG
    ctx.close()


@pytest.mark.parametrize("path", ["tc", "lanes"])
def test_linear_quadratic_step_counts_outside_range_give_nan(hj, path):
    spec = _spec(W.FAM_LINEAR_QUAD, W.LAX, 16, seed=5, m=8)
    ctx = hj.hj_create([spec], hj.opts_from_dict(W.lq_solver(), hj.HJ_PREC_FP32, 64), 0)
    if path == "lanes":
        hj.hj_set_tuning(ctx, 0, 16, 0)
    rng = np.random.default_rng(3)
    x, v = W.f32(rng.normal(size=(6, 16))), W.f32(rng.normal(size=(6, 16)))
    t = np.full(6, 0.5)
    N = np.array([0, 257, -5, 1000, 10, 64], dtype=np.int32)
    F, G = hj.hj_grad(ctx, _t(x, torch.float32), _t(t, torch.float32), _t(v, torch.float32), _t(N, torch.int32))
    F, G = F.cpu().numpy(), G.cpu().numpy()
    assert np.all(np.isnan(F[:4])) and np.all(np.isnan(G[:4]))
    P = oracle_problem(spec)
    for i in (4, 5):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i])
        assert rel_err(F[i], Fo) <= TC_TOL_F
    ctx.close()


@pytest.mark.parametrize("path", ["tc", "lanes"])
def test_solve_linear_quadratic_d64_conjugate_gradients_matches_oracle(hj, path):
    # conjugate directions (100 iterations) on the rank-deficient d=64 problem:
    # phi within the accuracy target of the FP64 oracle running the same rule
    # 136 queries: a full tile of 128 pairs and a ragged one
    phi, v, st, ref, info = _solve_both(hj, W.c4_linear_quad(nq=136), 136, tpp=0 if path == "tc" else 16)
    err = rel_err(phi, ref["phi"])
    print(f"LQ d=64 {path}: max rel err {err.max():.2e}, threads per pair {info['threads_per_pair']}")
    assert info["threads_per_pair"] == (1 if path == "tc" else 16)
    assert np.all(err <= 1e-4), err.max()
    assert np.array_equal(st & 1, ref["status"] & 1)
    assert info["iterations"] == 136 * 100


def test_linear_quadratic_d64_longer_descent_phi_matches_oracle_in_both_precisions(hj):
    # 400 conjugate-gradient iterations instead of the workload's 100: phi
    # within 1e-4 of the oracle in an FP64 context and in binary32 (tile
    # kernel).  The certificate is not compared: at this budget it measures
    # convergence along directions of curvature ~3e-6 that no descent of this
    # length controls, and the decision is decided by rounding (the oracle's
    # own residual on these queries moves between 0.002 and 0.012 under a
    # 1e-7 change of x, across a tolerance of 4.5e-3)
    wl = W.c4_linear_quad(nq=16)
    wl.solver.update(max_iters=400, cert_tol=4.5e-3)
    phi, v, st, ref, info = _solve_both(hj, wl, 16, prec_code=hj.HJ_PREC_FP64)
    assert np.all(rel_err(phi, ref["phi"]) <= 1e-4)
    phi32, v32, st32, ref32, info32 = _solve_both(hj, wl, 16)
    assert np.all(rel_err(phi32, ref["phi"]) <= 1e-4)


def test_solve_speed_quad_d10_with_conjugate_gradients_matches_oracle(hj):
    # smooth state-dependent functional: conjugate directions converge in
    # ~10 iterations (20 gradients) where gradient steps take ~75
    wl = W.c2_speed_quad(nq_x=16)
    wl.solver.update(grad="adjoint_cg", step=0.2, step_max=2.0, max_iters=60)
    phi, v, st, ref, info = _solve_both(hj, wl, 48)
    err = rel_err(phi, ref["phi"])
    assert np.all(err <= 1e-4), err.max()
    assert np.array_equal(st & 1, ref["status"] & 1)


def _mixed_sample(n_pairs=3000, per_problem=14):
    """Rows of the mixed workload covering all twelve problems (families x d)."""
    wl = W.c5_mixed(n_pairs=n_pairs)
    ids = np.concatenate([np.flatnonzero(wl.problem_idx == p)[:per_problem] for p in range(len(wl.problems))])
    return wl.take(np.sort(ids))


def _solve_mixed(hj, w, tune=False):
    from tests.helpers import oracle_opts_list
    ctx = hj.hj_create(w.problems, hj.opts_from_dict(w.solver, hj.HJ_PREC_FP32, 64), 0)
    x, t = _t(w.x, torch.float32), _t(w.t, torch.float32)
    ns, pi = _t(w.n_steps, torch.int32), _t(w.problem_idx, torch.int32)
    chosen = hj.hj_autotune(ctx, x, t, ns, pi, iters=3) if tune else None
    phi, v, st = hj.hj_solve(ctx, x, t, ns, pi)
    info = hj.hj_last_solve_info(ctx)
    ctx.close()
    key = ("mixed", w.nq)
    if key not in _ORACLE_CACHE:
        probs = [oracle_problem(p) for p in w.problems]
        ref = O.solve(probs, oracle_opts_list(w), w.x, w.t, w.n_steps, problem_idx=w.problem_idx)
        # the same solve with x moved twice by 1e-7 (relative): rows whose
        # answer moves, or whose chosen start is not certified, are decided
        # by rounding, not by the problem
        stable = (ref["status"] & 1) == 1
        for seed in (0, 1):
            xp = w.x * (1 + 1e-7 * np.random.default_rng(seed).standard_normal(w.x.shape))
            refp = O.solve(probs, oracle_opts_list(w), xp, w.t, w.n_steps, problem_idx=w.problem_idx)
            stable &= (rel_err(ref["phi"], refp["phi"]) <= 1e-6) & ((refp["status"] & 1) == 1)
        nonconvex = np.array([w.problems[int(i)].family == W.FAM_SMOOTH_NONCONVEX for i in w.problem_idx])
        stable |= ~nonconvex  # the smooth and convex families are checked on every row
        _ORACLE_CACHE[key] = (ref, stable)
    ref, stable = _ORACLE_CACHE[key]
    return phi.cpu().numpy(), st.cpu().numpy(), ref, stable, info, chosen


def _check_mixed(w, phi, st, ref, stable):
    err = rel_err(phi, ref["phi"])
    for p in range(len(w.problems)):
        rows = w.problem_idx == p
        ok = rows & stable
        print(f"problem {p} (family {w.problems[p].family}, d={w.problems[p].d}): {ok.sum()}/{rows.sum()} rows "
              f"checked, max rel err there {err[ok].max() if ok.any() else float('nan'):.2e}")
    assert np.all(err[stable] <= 1e-4), err[stable].max()
    assert np.array_equal(st[stable] & 1, ref["status"][stable] & 1)


def test_solve_mixed_families_and_dimensions_matches_oracle(hj):
    # twelve problems in one batch (speed-quadratic Lax, non-convex Hopf and
    # linear-quadratic Lax at d = 8, 16, 32, 100; t ~ U[0.1, 2] and N per
    # query), each with its own descent constants; the linear-quadratic
    # problems up to d = 32 run on the tensor-core tile kernel, d = 100 on
    # lane groups.  Non-convex Hopf rows at large t or d = 100 often certify
    # no start and their FP64 answer moves under a 1e-7 change of x, so that
    # family is checked on the rows the oracle certifies with an answer that
    # two such changes leave in place; the other families on every row.
    w = _mixed_sample()
    phi, st, ref, stable, info, _ = _solve_mixed(hj, w)
    _check_mixed(w, phi, st, ref, stable)
    assert info["n_pairs"] >= w.n_pairs


def test_mixed_nonconvex_rows_at_small_t_match_oracle_on_every_row(hj):
    # the non-convex Hopf family inside the mixed batch where its answer is
    # reproducible (t <= 0.5, d <= 32: the oracle certifies every such row
    # and its phi stays put under 1e-7 changes of x), 20 rows per dimension
    # beside rows of every other problem: checked on every row, no filter
    from tests.helpers import oracle_opts_list
    wl = W.c5_mixed(n_pairs=20000)
    fam = np.array([wl.problems[int(i)].family for i in wl.problem_idx])
    dd = np.array([wl.problems[int(i)].d for i in wl.problem_idx])
    nc = np.flatnonzero((fam == W.FAM_SMOOTH_NONCONVEX) & (dd <= 32) & (wl.t <= 0.5))
    ids = np.concatenate([nc[dd[nc] == d][:20] for d in (8, 16, 32)])
    others = np.concatenate([np.flatnonzero(wl.problem_idx == p)[:6] for p in range(len(wl.problems))
                             if wl.problems[p].family != W.FAM_SMOOTH_NONCONVEX])
    w = wl.take(np.sort(np.concatenate([ids, others])))
    ctx = hj.hj_create(w.problems, hj.opts_from_dict(w.solver, hj.HJ_PREC_FP32, 64), 0)
    phi, v, st = hj.hj_solve(ctx, _t(w.x, torch.float32), _t(w.t, torch.float32), _t(w.n_steps, torch.int32),
                             _t(w.problem_idx, torch.int32))
    phi, st = phi.cpu().numpy(), st.cpu().numpy()
    ctx.close()
    ref = O.solve([oracle_problem(p) for p in w.problems], oracle_opts_list(w), w.x, w.t, w.n_steps,
                  problem_idx=w.problem_idx)
    rows = np.isin(np.sort(np.concatenate([ids, others])), ids)
    assert rows.sum() == 60
    err = rel_err(phi, ref["phi"])
    assert np.all(err[rows] <= 1e-4), err[rows].max()
    assert np.array_equal(st[rows] & 1, ref["status"][rows] & 1)
    assert np.all(ref["status"][rows] & 1)


def test_autotuned_mixed_solve_still_matches_oracle(hj):
    w = _mixed_sample()
    phi, st, ref, stable, info, chosen = _solve_mixed(hj, w, tune=True)
    print("autotuned threads per pair:", chosen)
    assert len(chosen) == len(w.problems) and all(c in (0, 1, 2, 4, 8, 16, 32) for c in chosen)
    _check_mixed(w, phi, st, ref, stable)


@pytest.mark.parametrize("mixed", [False, True])
def test_solve_through_a_cuda_graph_matches_direct_solves(hj, mixed):
    # hj_set_graph: the first solve records the launch sequence (with the
    # forked per-problem streams of a mixed batch) and launches it, the next
    # one with the same buffers replays it; both equal direct solves bit for bit
    w = _mixed_sample(per_problem=6) if mixed else W.c3_smooth_nonconvex(nq=200)
    opts = hj.opts_from_dict(w.solver, hj.HJ_PREC_FP32, 64)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g_ctx, d_ctx = hj.hj_create(w.problems, opts, 0), hj.hj_create(w.problems, opts, 0)
        hj.hj_set_graph(g_ctx, True)
        x = _t(w.x, torch.float32)
        t, ns = _t(w.t, torch.float32), _t(w.n_steps, torch.int32)
        pi = _t(w.problem_idx, torch.int32) if mixed else None
        out = (torch.empty(w.nq, dtype=torch.float64, device=DEV), torch.zeros_like(x),
               torch.empty(w.nq, dtype=torch.int32, device=DEV))
        rng = np.random.default_rng(1)
        for call in range(3):
            if call:
                x.copy_(_t(W.f32(np.where(w.x != 0, w.x + 0.05 * rng.standard_normal(w.x.shape), 0.0)), torch.float32))
            hj.hj_solve(g_ctx, x, t, ns, pi, 0, out)
            ref = hj.hj_solve(d_ctx, x, t, ns, pi)
            stream.synchronize()
            assert torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[2]) and torch.equal(out[1], ref[1])
            info = hj.hj_last_solve_info(g_ctx)
            assert info["n_queries"] == w.nq and info["total_ms"] > 0
        g_ctx.close()
        d_ctx.close()


@pytest.mark.parametrize("family,prec", [(W.FAM_SMOOTH_NONCONVEX, "fp32"), (W.FAM_SMOOTH_NONCONVEX, "fp64"),
                                         (W.FAM_SPEED_QUAD, "fp64"), (W.FAM_LINEAR_QUAD, "fp32")])
def test_autograd_functional_backward_is_the_adjoint_gradient(hj, family, prec):
    # hj.Functional: forward hj_eval_functional, backward hj_grad; the
    # gradient reaching v equals the upstream weight times the oracle's exact
    # gradient of the discretised functional (the linear-quadratic fp32 case
    # runs on the tensor-core tile kernel)
    d = 20
    spec = _spec(family, W.HOPF if family == W.FAM_SMOOTH_NONCONVEX else W.LAX, d, seed=4, s_eps=1e-2)
    dt = torch.float32 if prec == "fp32" else torch.float64
    ctx = hj.hj_create([spec], hj.opts_from_dict(W.solver_constants(), hj.HJ_PREC_FP32 if prec == "fp32" else
                                                  hj.HJ_PREC_FP64, 32), 0)
    n = 11
    x, v, t, N = _rows(n, d, 7, prec)
    xt, tt, Nt = _t(x, dt), _t(t, dt), _t(N, torch.int32)
    vt = _t(v, dt).requires_grad_(True)
    w = np.random.default_rng(8).uniform(-2, 2, n)
    F = hj.Functional.apply(ctx, xt, tt, vt, Nt)
    (F * _t(w, dt)).sum().backward()
    G = vt.grad.cpu().numpy()
    P = oracle_problem(spec)
    tc = family == W.FAM_LINEAR_QUAD and prec == "fp32"
    tol = TC_TOL_G if tc else (5e-4 if prec == "fp32" else 1e-9)
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i])
        assert np.abs(G[i] - w[i] * Go).max() <= tol * (1 + np.abs(w[i] * Go).max()), i
    if prec == "fp64":
        # finite differences of the forward against the backward
        vs = _t(v[:2], dt).requires_grad_(True)
        assert torch.autograd.gradcheck(lambda vv: hj.Functional.apply(ctx, xt[:2], tt[:2], vv, Nt[:2]), (vs,),
                                        eps=1e-6, atol=1e-5, rtol=1e-4)
    ctx.close()


def test_queries_of_unknown_problems_and_empty_calls(hj):
    # a problem index outside [0, n problems) marks the query invalid (no
    # starts, phi NaN, status HJ_ST_NONFINITE) and leaves the other queries'
    # answers as they are; calls with no rows do nothing
    w = _mixed_sample(per_problem=3)
    ctx = hj.hj_create(w.problems, hj.opts_from_dict(w.solver, hj.HJ_PREC_FP32, 64), 0)
    x, t, ns = _t(w.x, torch.float32), _t(w.t, torch.float32), _t(w.n_steps, torch.int32)
    good = _t(w.problem_idx, torch.int32)
    bad = good.clone()
    bad[3], bad[10] = 99, -1
    phi0, _, st0 = hj.hj_solve(ctx, x, t, ns, good)
    phi1, _, st1 = hj.hj_solve(ctx, x, t, ns, bad)
    phi0, st0, phi1, st1 = phi0.cpu().numpy(), st0.cpu().numpy(), phi1.cpu().numpy(), st1.cpu().numpy()
    keep = np.ones(w.nq, bool)
    keep[[3, 10]] = False
    assert np.isnan(phi1[3]) and np.isnan(phi1[10]) and st1[3] == hj.HJ_ST_NONFINITE and st1[10] == hj.HJ_ST_NONFINITE
    assert np.array_equal(phi1[keep], phi0[keep]) and np.array_equal(st1[keep], st0[keep])
    e = torch.empty(0, w.x.shape[1], dtype=torch.float32, device=DEV)
    et = torch.empty(0, dtype=torch.float32, device=DEV)
    assert hj.hj_eval_functional(ctx, e, et, e).numel() == 0
    assert hj.hj_solve(ctx, e, et, None, torch.empty(0, dtype=torch.int32, device=DEV))[0].numel() == 0
    ctx.close()


def test_caller_supplied_solve_outputs_of_the_wrong_shape_or_type_are_refused(hj):
    wl = W.c3_smooth_nonconvex(nq=8)
    ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, 64), 0)
    x, t = _t(wl.x, torch.float32), _t(wl.t, torch.float32)
    good = (torch.zeros(8, dtype=torch.float64, device=DEV), torch.zeros(8, 20, device=DEV),
            torch.zeros(8, dtype=torch.int32, device=DEV))
    bad = [(torch.zeros(7, dtype=torch.float64, device=DEV),) + good[1:],
           (good[0], torch.zeros(8, 19, device=DEV), good[2]),
           (good[0], torch.zeros(8, 20, dtype=torch.float64, device=DEV), good[2]),
           good[:2] + (torch.zeros(8, dtype=torch.int64, device=DEV),),
           (good[0], torch.zeros(20, 8, device=DEV).t(), good[2])]
    for fn in (hj.hj_solve, hj.hj_solve_noalloc):
        for out in bad:
            with pytest.raises(ValueError):
                fn(ctx, x, t, out=out)
        phi, v, st = fn(ctx, x, t, out=good)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(phi.cpu().numpy()))
    ctx.close()


@pytest.mark.parametrize("d", [2, 5, 8, 13, 16, 20, 27, 32])
def test_one_thread_per_pair_kernels_match_oracle_and_lane_groups(hj, d):
    # the smooth non-convex Hopf family at d <= 32 runs one thread per pair
    # with (u, B) as its state; every instantiated size, exact and padded,
    # against the oracle's functional and adjoint gradient, and against the
    # lane-group kernels forced by a lane-count override
    spec = _spec(W.FAM_SMOOTH_NONCONVEX, W.HOPF, d, seed=d, s_eps=1e-3, n_neg=min(2, d))
    ctx = hj.hj_create([spec], hj.opts_from_dict(W.solver_constants(), hj.HJ_PREC_FP32, 64), 0)
    n = 150  # more than one block, ragged
    x, v, t, N = _rows(n, d, 100 + d, "fp32")
    args = (_t(x, torch.float32), _t(t, torch.float32), _t(v, torch.float32), _t(N, torch.int32))
    E = hj.hj_eval_functional(ctx, *args).cpu().numpy()
    F, G = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
    hj.hj_set_tuning(ctx, 0, 4 if d > 4 else 2, 0)
    F4, G4 = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
    ctx.close()
    P = oracle_problem(spec)
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i])
        assert rel_err(E[i], Fo) <= 2e-5 and rel_err(F[i], Fo) <= 2e-5, (i, E[i], F[i], Fo)
        scale = 1 + np.abs(Go).max()
        assert np.abs(G[i] - Go).max() <= 5e-4 * scale, (i, N[i])
        assert np.abs(G[i] - G4[i]).max() <= 1e-3 * scale
    assert np.all(rel_err(F, F4) <= 4e-5)


def test_one_thread_per_pair_gradient_is_the_same_for_every_checkpoint_interval(hj):
    # the (u, B) checkpoints every K steps with the segment recomputed: the
    # recomputed states repeat the forward arithmetic, so every K (dividing N
    # or not) gives the K = 1 gradient bit for bit, for N across [1, 256]
    spec = _spec(W.FAM_SMOOTH_NONCONVEX, W.HOPF, 20, seed=11, s_eps=1e-2)
    ctx = hj.hj_create([spec], hj.opts_from_dict(W.solver_constants(), hj.HJ_PREC_FP32, 64), 0)
    n = 40
    x, v, t, _ = _rows(n, 20, 21, "fp32")
    N = np.array([1, 2, 5, 17, 64, 100, 255, 256] * 5)[:n].astype(np.int32)
    args = (_t(x, torch.float32), _t(t, torch.float32), _t(v, torch.float32), _t(N, torch.int32))
    F1, G1 = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
    for ck in (2, 3, 8, 16):
        hj.hj_set_tuning(ctx, 0, 0, ck)
        F, G = (a.cpu().numpy() for a in hj.hj_grad(ctx, *args))
        assert np.array_equal(F, F1) and np.array_equal(G, G1), ck
    ctx.close()
    P = oracle_problem(spec)
    for i in range(n):
        Fo, Go = O.gradient(P, x[i], t[i], int(N[i]), v[i])
        assert rel_err(F1[i], Fo) <= 2e-5
        assert np.abs(G1[i] - Go).max() <= 5e-4 * (1 + np.abs(Go).max()), (i, N[i])


def test_d20_hopf_solve_runs_one_thread_per_pair(hj):
    wl = W.c3_smooth_nonconvex(nq=64)
    ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, 64), 0)
    hj.hj_solve(ctx, _t(wl.x, torch.float32), _t(wl.t, torch.float32))
    info = hj.hj_last_solve_info(ctx)
    ctx.close()
    assert info["threads_per_pair"] == 1 and info["comps_per_thread"] == 20
    # nominal work: 64 d per forward step, an adjoint step counted as three more
    assert info["nominal_flops"] == pytest.approx(64 * 20 * (info["rk4_steps"] + 3 * info["adjoint_steps"]),
                                                  rel=0.05)


@pytest.mark.parametrize("split", [[0, 100, 200], [0, 1, 77, 200]])
def test_solve_split_into_query_ranges_equals_the_unsplit_solve(hj, split):
    # the multi-GPU partition on the product path: consecutive query ranges
    # solved by separate hj_solve calls with q_begin = the range's first
    # global query index draw the same Philox starts as one unsplit solve, so
    # phi, v and status agree bit for bit (one GPU here; one range per rank
    # under torchrun)
    wl = W.c3_smooth_nonconvex(nq=200)
    ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, 64), 0)
    x, t = _t(wl.x, torch.float32), _t(wl.t, torch.float32)
    phi, v, st = (a.cpu().numpy() for a in hj.hj_solve(ctx, x, t))
    parts = []
    for a, b in zip(split[:-1], split[1:]):
        parts.append([o.cpu().numpy() for o in hj.hj_solve(ctx, x[a:b].contiguous(), t[a:b].contiguous(), q_begin=a)])
    ctx.close()
    assert np.array_equal(np.concatenate([p[0] for p in parts]), phi)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), v)
    assert np.array_equal(np.concatenate([p[2] for p in parts]), st)


def test_one_and_two_lanes_per_pair_give_identical_solves(hj):
    # the two-lane form splits each pair's components by parity, which is
    # exactly the one-lane form's split of its sums, so both give the same
    # bits; the automatic choice (two lanes for rounds this small) too
    wl = W.c3_smooth_nonconvex(nq=150)
    out = {}
    for tpp in (0, -1, -2):
        ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, 64), 0)
        if tpp:
            hj.hj_set_tuning(ctx, 0, tpp, 0)
        out[tpp] = [a.cpu().numpy() for a in hj.hj_solve(ctx, _t(wl.x, torch.float32), _t(wl.t, torch.float32))]
        info = hj.hj_last_solve_info(ctx)
        ctx.close()
        assert info["threads_per_pair"] == 1 and info["comps_per_thread"] == 20
    for tpp in (-1, -2):
        for a, b in zip(out[tpp], out[0]):
            assert np.array_equal(a, b), tpp
    ref = O.solve(oracle_problem(wl.problems[0]), oracle_opts(wl.solver, 16), wl.x, wl.t, wl.n_steps)
    assert np.all(rel_err(out[0][0], ref["phi"]) <= 1e-4)
    assert np.array_equal(out[0][2] & 1, ref["status"] & 1)


def test_lane_pinning_is_refused_where_it_does_not_apply(hj):
    spec = _spec(W.FAM_SPEED_QUAD, W.LAX, 10)
    ctx = hj.hj_create([spec], hj.opts_from_dict(W.solver_constants(), hj.HJ_PREC_FP32, 64), 0)
    for tpp in (-1, -2):
        with pytest.raises(hj.HJError) as e:
            hj.hj_set_tuning(ctx, 0, tpp, 0)
        assert e.value.status == hj.HJ_EUNSUPPORTED
    with pytest.raises(hj.HJError):
        hj.hj_set_tuning(ctx, 0, -3, 0)
    ctx.close()


def test_plain_cd_fd_d20_solve_matches_oracle_with_the_same_constants(hj):
    # the plain path of the headline comparison: Algorithm 1 (cyclic
    # coordinate descent) with central differences h = 2^-10, per-coordinate
    # step control, at most 100 sweeps, on the d=20 Hopf workload, against the
    # FP64 oracle running the same constants: every row, same certificates.
    # (Against the adjoint descent's answer, the discrete optimum, this plain
    # method misses query 30 here, identically in FP64: h = 2^-10 spans the
    # 1e-3-wide smoothing of |p_i|, the difference quotients' bias leaves the
    # better optimum's starts with residual 1.1e-3 > 1e-3, and the
    # certified-first rule returns the other basin.)
    wl = W.c3_smooth_nonconvex(nq=32)
    wl.solver = W.c3_cd_solver()
    phi, v, st, ref, info = _solve_both(hj, wl, wl.nq)
    err = rel_err(phi, ref["phi"])
    assert info["functional_evals"] > 0 and info["gradient_evals"] == 0
    assert np.all(err <= 1e-4), (err.max(), int(np.argmax(err)))
    assert np.array_equal(st & 1, ref["status"] & 1)


def test_solve_counters_do_not_depend_on_the_lanes_per_pair(hj):
    # the work counters (iterations, gradients, steps) count each pair once,
    # whether it runs on one lane or two
    wl = W.c3_smooth_nonconvex(nq=64)
    infos = []
    for tpp in (-1, -2):
        ctx = hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, 64), 0)
        hj.hj_set_tuning(ctx, 0, tpp, 0)
        hj.hj_solve(ctx, _t(wl.x, torch.float32), _t(wl.t, torch.float32))
        infos.append(hj.hj_last_solve_info(ctx))
        ctx.close()
    for key in ("iterations", "gradient_evals", "rk4_steps", "adjoint_steps", "n_pairs", "nominal_flops"):
        assert infos[0][key] == infos[1][key], key
