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
    neg = W.ProblemSpec(**{**spec.__dict__, "sigma": -np.ones(20)})
    with pytest.raises(hj.HJError) as e:
        hj.hj_create([neg], hj.opts_from_dict(wl.solver), 0)
    assert "sigma" in str(e.value)
