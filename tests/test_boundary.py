"""The C-ABI library: it builds, loads, and exports every symbol that
include/hj.h declares (no compute calls, so no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hj_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_02524_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("hj_create", "hj_destroy", "hj_eval_functional", "hj_grad", "hj_certify", "hj_solve",
              "hj_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1704_02524_gb300 import hj
    for name in _declared():
        assert name in hj.EXPORTED and hasattr(hj, name), name


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    # argument validation happens on the host before any CUDA call
    from paper_1704_02524_gb300 import hj
    hj.load_library()
    import numpy as np
    from paper_1704_02524_gb300 import workloads as W
    wl = W.c3_smooth_nonconvex(nq=2)
    spec = wl.problems[0]
    bad = W.ProblemSpec(**{**spec.__dict__, "d": 0})
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([bad], hj.opts_from_dict(wl.solver), 0)
    assert e.value.status == hj.HJ_EINVAL and "d=0" in str(e.value)
    o = hj.opts_from_dict(wl.solver)
    o.n_steps_default = 0
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([spec], o, 0)
    assert e.value.status == hj.HJ_EINVAL
    o = hj.opts_from_dict(wl.solver)
    o.quad = 4  # neither RK4/rectangle nor the Euler flag
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([spec], o, 0)
    assert e.value.status == hj.HJ_EINVAL and "quad" in str(e.value)
    bump = W.bump_ex3(n_side=2).problems[0]
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([W.ProblemSpec(**{**spec.__dict__, "principle": W.HUYGENS})], hj.opts_from_dict(wl.solver), 0)
    assert e.value.status == hj.HJ_EINVAL and "Huygens" in str(e.value)
    ros = W.harmonic_ex2(n_side=2, rosenbrock=True).problems[0]
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([W.ProblemSpec(**{**ros.__dict__, "principle": W.HOPF})], hj.opts_from_dict(wl.solver), 0)
    assert e.value.status == hj.HJ_EINVAL and "Rosenbrock" in str(e.value)
    split = W.split_ex5(n_side=2).problems[0]
    for val in (-1, 3, 0.5):
        with pytest.raises(hj.HJError) as e:
            hj.hj_create([W.ProblemSpec(**{**split.__dict__, "ksplit": val})], hj.opts_from_dict(wl.solver), 0)
        assert e.value.status == hj.HJ_EINVAL and "split k" in str(e.value)
    for field, val, msg in (("hsign", 0.5, "sign"), ("mu", -1.0, "mu"), ("s_eps", -1e-3, "s_eps")):
        with pytest.raises(hj.HJError) as e:
            hj.hj_create([W.ProblemSpec(**{**bump.__dict__, field: val})], hj.opts_from_dict(wl.solver), 0)
        assert e.value.status == hj.HJ_EINVAL and msg in str(e.value)
    neg = W.ProblemSpec(**{**spec.__dict__, "sigma": -np.ones(20)})
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([neg], hj.opts_from_dict(wl.solver), 0)
    assert "sigma" in str(e.value)


def test_create_rejects_a_bad_per_problem_solver_without_a_gpu(lib):
    # a problem's own descent constants are validated on the host, and the
    # message names the problem
    from paper_1704_02524_gb300 import hj
    from paper_1704_02524_gb300 import workloads as W
    hj.load_library()
    wl = W.c3_smooth_nonconvex(nq=2)
    good = wl.problems[0]
    bad = W.ProblemSpec(**{**good.__dict__, "solver": W.solver_constants(n_guesses=16, step=-1.0)})
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([good, bad], hj.opts_from_dict(wl.solver), 0)
    assert e.value.status == hj.HJ_EINVAL and "problem 1 solver" in str(e.value) and "step" in str(e.value)
    cg = W.ProblemSpec(**{**good.__dict__, "solver": W.solver_constants(grad="adjoint_cg", step_max=0.0)})
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([cg], hj.opts_from_dict(wl.solver), 0)
    assert "step_max" in str(e.value)


def test_linear_quadratic_limits_are_checked_without_a_gpu(lib):
    from paper_1704_02524_gb300 import hj
    from paper_1704_02524_gb300 import workloads as W
    import numpy as np
    hj.load_library()
    d = 130
    spec = W.ProblemSpec(d=d, family=W.FAM_LINEAR_QUAD, principle=W.LAX, g_kind=W.G_QUAD_SHIFT,
                         A=np.zeros((d, d)), B=np.zeros((d, 4)), a=np.zeros(d))
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([spec], hj.opts_from_dict(W.lq_solver()), 0)
    assert e.value.status == hj.HJ_EINVAL and "d <= 128" in str(e.value)


def test_mixed_workload_structure():
    # twelve problems (three families x d in {8,16,32,100}) with their own
    # descent constants, N = ceil(64 t), padded rows zero past each row's d
    from paper_1704_02524_gb300 import workloads as W
    import numpy as np
    wl = W.c5_mixed(n_pairs=3000)
    assert len(wl.problems) == 12
    assert wl.n_pairs == 3000
    assert np.array_equal(wl.n_steps, np.ceil(64 * wl.t).astype(np.int32))
    for q in range(0, wl.nq, 37):
        p = wl.problems[int(wl.problem_idx[q])]
        assert np.all(wl.x[q, p.d:] == 0)
        assert p.solver is not None
    lq = [p for p in wl.problems if p.family == W.FAM_LINEAR_QUAD]
    assert all(p.solver["grad"] == "adjoint_cg" and p.n_guesses == 1 for p in lq)


def test_caller_supplied_solve_outputs_are_checked_before_the_call():
    # the solve writes every row of phi, v and status: tensors on the wrong
    # device (or missing) are refused on the host, before the C call
    import torch
    from paper_1704_02524_gb300 import hj
    ctx = hj.Context(None, [type("P", (), {"d": 3})()], hj.hj_solver_opts(precision=hj.HJ_PREC_FP32), 0)
    good_cpu = (torch.zeros(4, dtype=torch.float64), torch.zeros(4, 3), torch.zeros(4, dtype=torch.int32))
    with pytest.raises(ValueError, match="phi must be on cuda"):
        hj._solve_out(ctx, good_cpu, 4)
    with pytest.raises(ValueError, match="out must be"):
        hj._solve_out(ctx, good_cpu[:2], 4)
