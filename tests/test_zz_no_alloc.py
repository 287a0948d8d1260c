"""hj_solve_noalloc: the solve entry point for callers that cannot allocate
device memory while solving (their GPU memory belongs to another allocator,
or the call sits in a loop that must not risk an allocation).  Its scratch is
one static device array, so it must give the same answers as hj_solve, call
after call, and refuse batches larger than that array.  This file is named to
be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1704_02524_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _ctx(hj, wl):
    return hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, int(wl.n_steps[0])), 0)


def _inputs(wl):
    x = torch.tensor(wl.x, dtype=torch.float32, device=DEV)
    t = torch.tensor(wl.t, dtype=torch.float32, device=DEV)
    ns = torch.tensor(wl.n_steps, dtype=torch.int32, device=DEV)
    return x, t, ns


def _fresh_out(wl, ld):
    # poisoned outputs: every row must be written by the call
    return (torch.full((wl.nq,), np.nan, dtype=torch.float64, device=DEV),
            torch.full((wl.nq, ld), np.nan, dtype=torch.float32, device=DEV),
            torch.full((wl.nq,), -1, dtype=torch.int32, device=DEV))


def test_noalloc_solve_equals_solve_bit_for_bit_on_two_calls_in_a_row():
    # the same kernels on the same pairs with the same starts: hj_solve's
    # answers exactly, and the static scratch left by the first call does not
    # leak into the second
    from paper_1704_02524_gb300 import hj
    wl = W.c3_smooth_nonconvex(nq=300)
    ctx = _ctx(hj, wl)
    x, t, ns = _inputs(wl)
    phi0, v0, st0 = hj.hj_solve(ctx, x, t, ns)
    torch.cuda.synchronize()
    phi0, v0, st0 = phi0.cpu().numpy(), v0.cpu().numpy(), st0.cpu().numpy()
    for _ in range(2):
        phi, v, st = hj.hj_solve_noalloc(ctx, x, t, ns, out=_fresh_out(wl, 20))
        torch.cuda.synchronize()
        phi, v, st = phi.cpu().numpy(), v.cpu().numpy(), st.cpu().numpy()
        assert np.array_equal(phi, phi0)
        assert np.array_equal(v, v0)
        assert np.array_equal(st, st0)
    ctx.close()


def test_noalloc_linear_quadratic_d64_runs_lane_groups():
    # hj_solve runs this problem on the tensor-core tile kernel; the no-alloc
    # entry point runs it on the lane-group kernels (its documented
    # exception).  With the lane groups forced on both, the answers are
    # identical; against the tile kernel each side is within the 1e-4 (1 + |phi|)
    # gate of the FP64 oracle, so they agree within twice that
    from paper_1704_02524_gb300 import hj
    wl = W.c4_linear_quad(nq=256)
    x, t, ns = _inputs(wl)
    for forced in (True, False):
        ctx = _ctx(hj, wl)
        if forced:
            hj.hj_set_tuning(ctx, 0, 16, 0)
        phi0, v0, st0 = hj.hj_solve(ctx, x, t, ns)
        torch.cuda.synchronize()
        phi0, v0, st0 = phi0.cpu().numpy(), v0.cpu().numpy(), st0.cpu().numpy()
        for _ in range(2):
            phi, v, st = hj.hj_solve_noalloc(ctx, x, t, ns, out=_fresh_out(wl, 64))
            torch.cuda.synchronize()
            phi, v, st = phi.cpu().numpy(), v.cpu().numpy(), st.cpu().numpy()
            if forced:
                assert np.array_equal(phi, phi0) and np.array_equal(v, v0) and np.array_equal(st, st0)
            else:
                assert np.all(np.abs(phi - phi0) <= 2e-4 * (1 + np.abs(phi0)))
                assert np.array_equal(st & 1, st0 & 1)
        ctx.close()


def test_noalloc_solve_rejects_batches_beyond_its_static_scratch():
    from paper_1704_02524_gb300 import hj
    wl = W.c3_smooth_nonconvex(nq=20000)  # 320,000 starts: more than the static array holds
    ctx = _ctx(hj, wl)
    x, t, _ = _inputs(wl)
    with pytest.raises(hj.HJError) as e:
        hj.hj_solve_noalloc(ctx, x, t)
    assert e.value.status == hj.HJ_EINVAL and "static array" in str(e.value)
    ctx.close()


def test_noalloc_solve_rejects_a_pair_count_that_would_wrap_before_sizing():
    # a C caller's huge n_queries is refused before n_queries * starts is
    # formed; the pointers are never dereferenced
    from paper_1704_02524_gb300 import hj
    wl = W.c3_smooth_nonconvex(nq=4)
    ctx = _ctx(hj, wl)
    x, t, _ = _inputs(wl)
    phi, v, st = _fresh_out(wl, 20)
    lib = hj.load_library()
    for n in (1 << 40, (1 << 62) + 7, ((1 << 31) - 1) // 16 + 1):
        rc = lib.hj_solve_noalloc(ctx.handle, 0, n, None, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(t.data_ptr()), None, ctypes.c_void_p(phi.data_ptr()),
                                  ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(st.data_ptr()), None)
        assert rc == hj.HJ_EINVAL
        assert "too many" in hj.hj_last_error(ctx)
    torch.cuda.synchronize()
    assert np.all(np.isnan(phi.cpu().numpy())) and np.all(st.cpu().numpy() == -1)  # nothing was enqueued
    ctx.close()
