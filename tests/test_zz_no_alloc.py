"""hj_solve_noalloc: the solve entry point for callers that cannot allocate
device memory while solving (their GPU memory belongs to another allocator,
or the call sits in a loop that must not risk an allocation).  Its scratch is
one static device array, so it must give the same answers as hj_solve, call
after call, and refuse batches larger than that array.  This file is named to
be collected last."""
import numpy as np
import pytest
import torch

from paper_1704_02524_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _ctx(hj, wl):
    return hj.hj_create(wl.problems, hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP32, int(wl.n_steps[0])), 0)


def test_noalloc_solve_matches_solve_on_two_calls_in_a_row():
    from paper_1704_02524_gb300 import hj
    wl = W.c3_smooth_nonconvex(nq=300)
    ctx = _ctx(hj, wl)
    x = torch.tensor(wl.x, dtype=torch.float32, device=DEV)
    t = torch.tensor(wl.t, dtype=torch.float32, device=DEV)
    ns = torch.tensor(wl.n_steps, dtype=torch.int32, device=DEV)
    phi0, v0, st0 = hj.hj_solve(ctx, x, t, ns)
    torch.cuda.synchronize()
    phi0, v0, st0 = phi0.cpu().numpy(), v0.cpu().numpy(), st0.cpu().numpy()
    for _ in range(2):
        out = (torch.full((wl.nq,), np.nan, dtype=torch.float64, device=DEV),
               torch.zeros(wl.nq, 20, dtype=torch.float32, device=DEV),
               torch.full((wl.nq,), -1, dtype=torch.int32, device=DEV))
        phi, v, st = hj.hj_solve_noalloc(ctx, x, t, ns, out=out)
        torch.cuda.synchronize()
        phi, v, st = phi.cpu().numpy(), v.cpu().numpy(), st.cpu().numpy()
        # the solve's tolerance on phi, 1e-4 (1 + |phi|); same certificate decisions
        assert np.all(np.abs(phi - phi0) <= 1e-4 * (1 + np.abs(phi0)))
        assert np.array_equal(st & 1, st0 & 1)
        assert np.allclose(v, v0, rtol=0, atol=1e-3)
    ctx.close()


def test_noalloc_solve_rejects_batches_beyond_its_static_scratch():
    from paper_1704_02524_gb300 import hj
    wl = W.c3_smooth_nonconvex(nq=20000)  # 320,000 starts: more than the static array holds
    ctx = _ctx(hj, wl)
    x = torch.tensor(wl.x, dtype=torch.float32, device=DEV)
    t = torch.tensor(wl.t, dtype=torch.float32, device=DEV)
    with pytest.raises(hj.HJError) as e:
        hj.hj_solve_noalloc(ctx, x, t)
    assert e.value.status == hj.HJ_EINVAL and "static array" in str(e.value)
    ctx.close()
