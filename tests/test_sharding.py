"""Multi-GPU sharding of the solve, exercised on CPU with two gloo ranks.

Queries are independent, so a batch splits into contiguous query ranges,
one per rank, with no exchange on the data path (bench.py's weak scaling).
The Philox counter of a start is the query's global index (hj_solve's
q_begin + row), so the shards together draw exactly the starts of one
unsplit solve.  Here each rank solves its range with the FP64 oracle
(global query ids q_begin + row), the answers are gathered, and rank 0
checks them bit for bit against an unsplit solve; the per-rank step times
are max-reduced the way bench.py reports them.
"""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1704_02524_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import oracle as O
    from tests.helpers import oracle_opts, oracle_problem
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = W.c3_smooth_nonconvex(nq=12)
    n = wl.nq // world
    q_begin = rank * n
    w = wl.take(np.arange(q_begin, q_begin + n))
    P = oracle_problem(wl.problems[0])
    opts = oracle_opts(dict(wl.solver, max_iters=40), wl.problems[0].n_guesses)
    res = O.solve(P, opts, w.x, w.t, w.n_steps, query_ids=np.arange(q_begin, q_begin + n), threads=2)
    parts = [None] * world
    dist.all_gather_object(parts, (rank, res["phi"].tolist(), res["status"].tolist()))
    step_ms = torch.tensor([10.0 + rank], dtype=torch.float64)
    dist.all_reduce(step_ms, op=dist.ReduceOp.MAX)
    if rank == 0:
        parts.sort()
        phi = np.concatenate([np.array(p[1]) for p in parts])
        status = np.concatenate([np.array(p[2]) for p in parts])
        np.savez(os.path.join(out_dir, "shards.npz"), phi=phi, status=status, step_ms=step_ms.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_query_shards_reproduce_the_unsplit_solve():
    import oracle as O
    from tests.helpers import oracle_opts, oracle_problem
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(2, _free_port(), d), nprocs=2, join=True)
        got = np.load(os.path.join(d, "shards.npz"))
    wl = W.c3_smooth_nonconvex(nq=12)
    P = oracle_problem(wl.problems[0])
    opts = oracle_opts(dict(wl.solver, max_iters=40), wl.problems[0].n_guesses)
    ref = O.solve(P, opts, wl.x, wl.t, wl.n_steps, threads=4)
    assert np.array_equal(got["phi"], ref["phi"])
    assert np.array_equal(got["status"], ref["status"])
    assert float(got["step_ms"][0]) == 11.0  # the slowest rank's time
