"""Benchmark: queries/s of the generalized Hopf solve on the d=20 non-convex
workload (65,536 queries x 16 starts, RK4 N=64, t=0.5, certificate and
reseeding), with the adjoint gradient-descent path as the headline and the
plain coordinate-descent / finite-difference path beside it.

One step = one hj_solve over the whole batch with inputs resident in HBM
(guesses, descent, FP64 certificate, reseed rounds, best-of-guesses).
Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload instead (bounded samples per step).

--workload selects another workload of paper_1704_02524_gb300.workloads:
linear_quad_d64_lax (32,768 queries, d=64, the tensor-core tile kernel;
--tpp 16 runs the lane-group kernels instead), speed_quad_d10_lax (49,152
queries, d=10), mixed_persistent (1,048,576 pairs over 12 problems).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1704_02524_gb300 import workloads as W  # noqa: E402

WORKLOAD = "smooth_nonconvex_d20_hopf"
METRIC = "queries/s at 1e-4 rel err (d=20 Hopf), adjoint vs plain CD-FD; % FP32 peak"
# other workloads: builder, default query count, metric, and a one-line description of the descent
WORKLOADS = {
    "smooth_nonconvex_d20_hopf": (lambda nq: W.c3_smooth_nonconvex(nq=nq), 65536, METRIC,
                                  "gradient descent, discrete-adjoint gradient, per-coordinate step control"),
    "linear_quad_d64_lax": (lambda nq: W.c4_linear_quad(nq=nq), 32768,
                            "queries/s at 1e-4 rel err (d=64 linear-quadratic Lax), tensor-core tile kernel",
                            "conjugate gradients (100 iterations), discrete-adjoint gradient on BF16x3 tensor cores"),
    "speed_quad_d10_lax": (lambda nq: W.c2_speed_quad(nq_x=max(1, nq // 3)), 49152,
                           "queries/s at 1e-4 rel err (d=10 state-dependent Lax)",
                           "gradient descent, discrete-adjoint gradient, per-coordinate step control"),
    "mixed_persistent": (lambda nq: W.c5_mixed(n_pairs=nq), 1 << 20,
                         "(query, start) pairs/s (mixed families, d in {8,16,32,100})",
                         "gradient descent (adjoint) for every problem"),
    "bump_norm_d2_plus_lax_paper": (lambda nq: W.bump_ex3(n_side=max(1, int(round(nq ** 0.5)))), 16384,
                                    "points/s (H = c(x)|p|, d=2 cross-section grid, the paper's numerics)",
                                    "Algorithm 1 (cyclic coordinate descent, alpha halving), forward "
                                    "differences, forward Euler with the rectangle rule"),
    "bump_norm_d2_plus_huygens_paper": (lambda nq: W.bump_ex3(n_side=max(1, int(round(nq ** 0.5))),
                                                               principle=W.HUYGENS, ds=0.005), 16384,
                                        "points/s (Example 3 with the Huygens form F^2, d=2 grid, the paper's "
                                        "numerics)",
                                        "Algorithm 1 (alpha halving), forward differences, forward Euler; F^2 = the "
                                        "smallest g over the solver grid"),
    "split_norm_d2_hopf_paper": (lambda nq: W.split_ex5(n_side=max(1, int(round(nq ** 0.5)))), 16384,
                                 "points/s (Example 5 H = c(x)|p_1| - c(-x)|p_2|, d=2 grid, the paper's numerics)",
                                 "Algorithm 1, forward differences, forward Euler with the rectangle rule; 20 starts"),
    "split_norm_d2_hopf_cg": (lambda nq: W.split_ex5(n_side=max(1, int(round(nq ** 0.5))), descent="cg"), 16384,
                              "points/s (Example 5, d=2 grid, conjugate-gradient momentum on the Euler functional)",
                              "conjugate gradients with the discrete adjoint of forward Euler; 20 starts"),
    "harmonic_d2_minus_hopf_paper": (lambda nq: W.harmonic_ex2(n_side=max(1, int(round(nq ** 0.5)))), 16384,
                                     "points/s (Example 2 H = -(|p|^2+|x|^2)/2, d=2 grid, the paper's numerics)",
                                     "Algorithm 1, forward differences, forward Euler with the rectangle rule"),
    "linear_game_d16_hopf": (lambda nq: W.linear_game(nq=nq), 65536,
                             "queries/s (time-dependent linear game, d=16 Hopf, Sec. 3.4 Example 3)",
                             "gradient descent, discrete-adjoint gradient with stage times, coarse-to-fine"),
    "evans_d2_hopf_paper": (lambda nq: W.evans_ex4(n_side=max(1, int(round(nq ** 0.5)))), 16384,
                            "points/s (Example 4 Evans-type H, d=2 grid, the paper's numerics)",
                            "Algorithm 1, forward differences, forward Euler with the rectangle rule"),
    "quad_iso_d2_lax": (lambda nq: W.c1_quad_iso(nq=min(nq, 64)), 64,
                        "queries/s (d=2 Lax, H = |p|^2/2, FP64, the 8x8 grid)",
                        "Algorithm 1 with central differences, exactly 200 sweeps, 4 starts"),
}
CPU_SAMPLE = 64          # queries of the oracle timing sample (cpu_baseline, all host cores)
CPU_SAMPLE_1 = 8         # queries of the one-core oracle timing sample
REF_SAMPLE = 64          # queries per step of the reference arm
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of the dominant descent launch of a smaller case
# (d=20: round 0's fine-level launch; d=64: the tile kernel's launch), from
# ncu captures of the current kernels on a GB300 (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by workload: (queries captured, bytes).  The
# launch's traffic grows with the number of (query, start) pairs, so it is
# scaled by queries / queries captured.  None: not captured for the current
# kernel.
TRAFFIC = {"smooth_nonconvex_d20_hopf": (32768, 17.906e9 + 38.355e9),
           "linear_quad_d64_lax": (4096, 28.598e9 + 42.637e9)}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--nq", type=int, default=0, help="queries (pairs for mixed_persistent); 0: the workload's size")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain CD-FD measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--tpp", type=int, default=0,
                    help="threads per pair of the descent (0: library choice; -1 / -2: one / two lanes per pair "
                         "of the one-pair-per-thread kernels in every round)")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "fp64"],
                    help="arithmetic of the solve (auto: the workload's own)")
    ap.add_argument("--cd-h", type=float, default=0.0, help="plain CD-FD path: difference step (0: the workload's)")
    ap.add_argument("--cd-sweeps", type=int, default=0, help="plain CD-FD path: sweep cap (0: the workload's)")
    ap.add_argument("--cd-precision", default="fp32", choices=["fp32", "fp64"],
                    help="plain CD-FD path: arithmetic (fp64 with --cd-h 1e-5 certifies where binary32 cannot)")
    ap.add_argument("--cd-nq", type=int, default=0,
                    help="plain CD-FD path: time it on every (nq / cd_nq)-th query only (0: all)")
    ap.add_argument("--ck", type=int, default=0, help="adjoint checkpoint interval (0: library choice)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip hj_autotune (launch parameters timed on up to 65,536 queries before the run)")
    return ap.parse_args()


def _oracle_inputs(wl):
    import oracle as O
    from tests.helpers import oracle_opts_list, oracle_problem  # same glue as the tests
    probs = [oracle_problem(p) for p in wl.problems]
    return O, probs, oracle_opts_list(wl)


def _time_oracle(wl, q_ids, threads=None):
    """Oracle on the given query rows of wl (all host cores unless threads is
    given); returns (seconds, result, threads)."""
    O, probs, opts = _oracle_inputs(wl)
    sub = wl.take(q_ids)
    t0 = time.perf_counter()
    res = O.solve(probs, opts, sub.x, sub.t, sub.n_steps, problem_idx=sub.problem_idx,
                  query_ids=np.asarray(q_ids, dtype=np.int64), threads=threads)
    return time.perf_counter() - t0, res, res["threads"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"hj_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


def _workload(a):
    build, default_n, metric, descent = WORKLOADS[a.workload]
    wl = build(a.nq or default_n)
    if a.precision != "auto":
        wl.precision = a.precision
    return wl, metric, descent


def _config(a, wl, descent, nq):
    ps = wl.problems
    cfg = {"workload": wl.name, "d": max(p.d for p in ps), "queries_per_gpu": nq,
           "guesses": sorted({p.n_guesses for p in ps}), "n_steps": [int(wl.n_steps.min()), int(wl.n_steps.max())],
           "t": [float(wl.t.min()), float(wl.t.max())], "descent": descent, "certificate": "fp64",
           "max_trials": wl.solver["max_trials"], "l2": "flushed between timed steps (256 MB write)"}
    if len(ps) > 1:
        cfg["problems"] = len(ps)
        cfg["pairs_per_gpu"] = int(wl.n_pairs)
    return cfg


def run_reference(a):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, metric, descent = _workload(a)
    nq = wl.nq
    rng = np.random.default_rng(0)
    times = []
    threads = 1
    units = 0
    for k in range(a.warmup + a.steps):
        ids = np.sort(rng.choice(nq, REF_SAMPLE, replace=False))
        dt, _, threads = _time_oracle(wl, ids)
        if k >= a.warmup:
            times.append(dt)
            units += _units(wl, ids)
    sec = sum(times)
    val = units / sec
    unit = _unit(wl)
    cfg = _config(a, wl, descent, nq)
    cfg["sample_per_step"] = REF_SAMPLE
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": val, "unit": unit, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sec / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": val, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": f"{REF_SAMPLE} random queries of the workload per step (all their starts)"},
        "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _unit(wl):
    return "pairs/s" if len(wl.problems) > 1 else "queries/s"


def _units(wl, ids=None):
    """Work units of the metric in the given rows: queries, or (query, start) pairs for mixed batches."""
    idx = wl.problem_idx if ids is None else wl.problem_idx[np.asarray(ids)]
    if len(wl.problems) > 1:
        return int(sum(wl.problems[int(i)].n_guesses for i in idx))
    return int(len(idx))


def run_ours(a):
    import torch
    import torch.distributed as dist
    from paper_1704_02524_gb300 import hj

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    wl, metric, descent = _workload(a)
    nq, ld = wl.nq, wl.x.shape[1]
    units = _units(wl)
    q_begin = rank * nq  # weak scaling: every rank solves its own batch of nq queries
    if rank > 0:
        # other ranks draw their own query points from the same distribution
        rng = np.random.default_rng(1000 + rank)
        wl.x = W.f32(np.where(wl.x != 0, rng.uniform(-1, 1, wl.x.shape), 0.0))
    fp64 = wl.precision == "fp64"
    tdt, esz = (torch.float64, 8) if fp64 else (torch.float32, 4)
    x = torch.tensor(wl.x, dtype=tdt, device=dev)
    t = torch.tensor(wl.t, dtype=tdt, device=dev)
    ns = torch.tensor(wl.n_steps, dtype=torch.int32, device=dev)
    multi = len(wl.problems) > 1
    pidx = torch.tensor(wl.problem_idx, dtype=torch.int32, device=dev) if multi else None
    opts = hj.opts_from_dict(wl.solver, hj.HJ_PREC_FP64 if fp64 else hj.HJ_PREC_FP32, int(wl.n_steps.max()))
    ctx = hj.hj_create(wl.problems, opts, local)
    tuning = None
    if a.tpp or a.ck:
        for p in range(len(wl.problems)):
            hj.hj_set_tuning(ctx, p, a.tpp, a.ck)
        tuning = {"threads_per_pair": [a.tpp] * len(wl.problems), "by": "command line"}
    elif all(p_.solver is None for p_ in wl.problems) and wl.solver["grad"].startswith("fd"):
        # Algorithm 1 (coordinate descent): a few capped iterations rank the lane
        # counts wrongly -- on the d=2 paper workloads the timed sample picked 2
        # or 4 lanes per pair, which run 2x and 4x slower over the whole solve
        # than the library's automatic choice (one lane, measured on a GB300)
        tuning = {"threads_per_pair": [0] * len(wl.problems), "by": "automatic (coordinate descent)"}
    elif not a.no_autotune:
        # launch parameters per problem, timed on a sample (outside the timed region).
        # The sample must fill the GPU as the run does: on a batch that fits in
        # one wave the candidates' single-pair latencies decide (more lanes per
        # pair look faster), while the full run is throughput bound.
        ns_ = min(nq, 65536)
        sample = np.sort(np.random.default_rng(7).choice(nq, ns_, replace=False))
        si = torch.tensor(sample, dtype=torch.int64, device=dev)
        chosen = hj.hj_autotune(ctx, x[si].contiguous(), t[si].contiguous(), ns[si].contiguous(),
                                pidx[si].contiguous() if multi else None, iters=3)
        tuning = {"threads_per_pair": chosen, "by": f"hj_autotune on {ns_} queries, 3 iterations (0 = automatic)"}
    phi = torch.empty(nq, dtype=torch.float64, device=dev)
    vout = torch.zeros(nq, ld, dtype=tdt, device=dev)
    status = torch.empty(nq, dtype=torch.int32, device=dev)
    out = (phi, vout, status)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        hj.hj_solve(ctx, x, t, ns, pidx, q_begin, out)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    infos = []
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            flush.fill_(float(k))  # evict L2 between timed steps (outside the timed region)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            infos.append(hj.hj_last_solve_info(ctx))  # synchronises after the end event
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms_steps = [e0.elapsed_time(e1) for e0, e1 in ev]
    ms = sum(ms_steps) / len(ms_steps)
    ms_t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = units * world / (ms_max / 1e3)
    clocks = clk.summary()

    # roofline of the dominant kernel: the descent (FP32 ALU) or, for the
    # linear-quadratic tile kernel, its BF16x3 tensor-core products
    info = infos[-1]
    desc_s = sum(i["descent_ms"] for i in infos) / 1e3
    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    tflops = sum(i["tensor_flops"] for i in infos)
    traffic = TRAFFIC.get(a.workload)
    traffic = None if traffic is None or a.tpp or a.ck else traffic[1] * nq / traffic[0]
    if tflops > 0:
        peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        roof = {"bound": "tensor", "achieved": tflops / desc_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": tflops / desc_s / 1e12 / peak, "traffic": traffic,
                "traffic_note": "DRAM bytes of the descent launch, scaled from a 4,096-query ncu capture",
                "kernel": "k_lq_tc (tensor-core tile kernel, BF16x3 stage products)",
                "peak_note": f"dense BF16, {peak_src} sustained cuBLAS figure; achieved counts the three BF16 "
                             "products of each fp32 product (unpadded d, m)"}
    else:
        # achieved: the descent's work at the fixed per-evaluation counts of
        # the general RK4 form (64 d N flops per functional evaluation of the
        # d=20 family, an adjoint gradient counted as four evaluations, the
        # in-kernel certificate as one) over the descent launches' device time
        flops = sum(i["nominal_flops"] for i in infos)
        flops_lg = sum(i["algorithmic_flops"] for i in infos)
        peak = nsm * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        if fp64:
            peak /= 64.0
        roof = {"bound": "alu", "achieved": flops / desc_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / desc_s / 1e12 / peak, "traffic": traffic,
                "traffic_note": "DRAM bytes of round 0's fine-level descent launch, scaled by queries from a "
                                "smaller ncu capture of the same kernel",
                "kernel": "k_desc (persistent descent)",
                "flops_note": "nominal per-evaluation counts of the general RK4 form (64 d N per functional "
                              "evaluation at d=20, an adjoint gradient as four evaluations, the in-kernel "
                              "certificate as one); the one-pair-per-thread kernel carries the iterate as two "
                              "scalars and executes fewer operations than these counts",
                "achieved_lane_group_model": flops_lg / desc_s / 1e12,
                "frac_lane_group_model": flops_lg / desc_s / 1e12 / peak,
                "peak_note": f"FP32 FMA {nsm} SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                             f"({peak_src} max SM clock)" + ("; FP64 at 1/64 of that" if fp64 else "")}
        # cross-check of that peak: the project's FMA-chain microbenchmark
        # (outside the timed region)
        roof["peak_check_tflops"] = hj.hj_fp32_fma_rate(local)

    # e2e through the C ABI with host buffers: pinned H2D of x, t, N (and the
    # problem index), the solve, D2H of phi, v, status
    hx = torch.tensor(wl.x, dtype=tdt).pin_memory()
    ht = torch.tensor(wl.t, dtype=tdt).pin_memory()
    hn = torch.tensor(wl.n_steps, dtype=torch.int32).pin_memory()
    hp = torch.tensor(wl.problem_idx, dtype=torch.int32).pin_memory() if multi else None
    hphi = torch.empty(nq, dtype=torch.float64).pin_memory()
    hv = torch.empty(nq, ld, dtype=tdt).pin_memory()
    hst = torch.empty(nq, dtype=torch.int32).pin_memory()
    dx, dt_, dn = torch.empty_like(x), torch.empty_like(t), torch.empty_like(ns)
    dp_ = torch.empty_like(pidx) if multi else None
    h2d = hx.numel() * esz + ht.numel() * esz + hn.numel() * 4 + (hp.numel() * 4 if multi else 0)
    d2h = hphi.numel() * 8 + hv.numel() * esz + hst.numel() * 4
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        dx.copy_(hx, non_blocking=True)
        dt_.copy_(ht, non_blocking=True)
        dn.copy_(hn, non_blocking=True)
        if multi:
            dp_.copy_(hp, non_blocking=True)
        hj.hj_solve(ctx, dx, dt_, dn, dp_, q_begin, out)
        hphi.copy_(phi, non_blocking=True)
        hv.copy_(vout, non_blocking=True)
        hst.copy_(status, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / a.steps
    e2e_t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_val = units * world / (float(e2e_t.item()) / 1e3)
    phi_np = hphi.numpy().copy()
    st_np = hst.numpy().copy()

    # plain path: Algorithm 1 (cyclic CD) with central differences, same
    # workload, same kernels' forward functional
    plain = None
    if not a.no_plain and a.workload in (WORKLOAD, "speed_quad_d10_lax"):
        solver_cd = W.plain_cd_solver(wl.solver, max(p_.d for p_ in wl.problems))
        if a.cd_h:
            solver_cd["fd_h"] = a.cd_h
        if a.cd_sweeps:
            solver_cd["max_iters"] = a.cd_sweeps * max(p_.d for p_ in wl.problems)
        cd64 = a.cd_precision == "fp64"
        cdt = torch.float64 if cd64 else torch.float32
        ctx_cd = hj.hj_create(wl.problems, hj.opts_from_dict(solver_cd, hj.HJ_PREC_FP64 if cd64 else hj.HJ_PREC_FP32,
                                                             int(wl.n_steps.max())), local)
        sub = np.arange(nq) if not a.cd_nq or a.cd_nq >= nq else np.arange(0, nq, nq // a.cd_nq)[:a.cd_nq]
        si = torch.tensor(sub, dtype=torch.int64, device=dev)
        xc, tc, nsc = x[si].to(cdt).contiguous(), t[si].to(cdt).contiguous(), ns[si].contiguous()
        m = len(sub)
        phi_cd = torch.empty(m, dtype=torch.float64, device=dev)
        st_cd = torch.empty(m, dtype=torch.int32, device=dev)
        out_cd = (phi_cd, torch.zeros(m, ld, dtype=cdt, device=dev), st_cd)
        hj.hj_solve(ctx_cd, xc, tc, nsc, None, q_begin, out_cd)  # warm-up
        torch.cuda.synchronize()
        flush.fill_(1.0)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        hj.hj_solve(ctx_cd, xc, tc, nsc, None, q_begin, out_cd)
        c1.record(stream)
        torch.cuda.synchronize()
        cd_ms = c0.elapsed_time(c1)
        icd = hj.hj_last_solve_info(ctx_cd)
        sweeps = solver_cd["max_iters"] // max(p_.d for p_ in wl.problems)
        phi_full = np.full(nq, np.nan)
        st_full = np.zeros(nq, dtype=np.int32)
        phi_full[sub] = phi_cd.cpu().numpy()
        st_full[sub] = st_cd.cpu().numpy()
        plain = {"value": m / (cd_ms / 1e3), "unit": "queries/s", "ms_per_step": cd_ms, "queries": m,
                 "dtype": "f64" if cd64 else "f32",
                 "descent": f"cyclic coordinate descent (Algorithm 1), central differences "
                            f"h={solver_cd['fd_h']:.6g}, at most {sweeps} sweeps",
                 "functional_evals": icd["functional_evals"],
                 "functional_evals_per_s": icd["functional_evals"] / (cd_ms / 1e3),
                 "achieved_tflops": icd["nominal_flops"] / (icd["descent_ms"] / 1e3) / 1e12,
                 "certified_frac": float(np.mean(st_cd.cpu().numpy() & 1)),
                 "phi": phi_full, "st": st_full}
        # several times t in one batch: each t's queries solved on their own,
        # the adjoint path and the plain path side by side (speed; the
        # accuracy per t comes from the full runs' sampled rows below)
        tvals = np.unique(wl.t)
        if world == 1 and len(tvals) > 1:
            plain["per_t"] = []
            for tv in tvals:
                rows = torch.tensor(np.flatnonzero(wl.t == tv), dtype=torch.int64, device=dev)
                m = int(rows.numel())
                xs, ts, nss = x[rows].contiguous(), t[rows].contiguous(), ns[rows].contiguous()
                o = (torch.empty(m, dtype=torch.float64, device=dev), torch.zeros(m, ld, dtype=tdt, device=dev),
                     torch.empty(m, dtype=torch.int32, device=dev))
                row = {"t": float(tv), "queries": m}
                for key, c_ in (("adjoint", ctx), ("plain_cd_fd", ctx_cd)):
                    if c_ is ctx_cd and cd64 != fp64:
                        continue  # the plain path in another precision is timed on its own sample only
                    hj.hj_solve(c_, xs, ts, nss, None, 0, o)
                    torch.cuda.synchronize()
                    flush.fill_(2.0)
                    e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0_.record(stream)
                    hj.hj_solve(c_, xs, ts, nss, None, 0, o)
                    e1_.record(stream)
                    torch.cuda.synchronize()
                    row[key + "_queries_per_s"] = m / (e0_.elapsed_time(e1_) / 1e3)
                plain["per_t"].append(row)
        ctx_cd.close()

    # mixed batches: each dimension's slice of the batch (all its families)
    # solved on its own after the timed run, for the per-d throughput
    per_d = None
    if multi and world == 1:
        per_d = []
        dims = sorted({p_.d for p_ in wl.problems})
        pd_arr = np.array([wl.problems[int(i)].d for i in wl.problem_idx])
        for dd in dims:
            rows = np.flatnonzero(pd_arr == dd)
            ri = torch.tensor(rows, dtype=torch.int64, device=dev)
            m = len(rows)
            o = (torch.empty(m, dtype=torch.float64, device=dev), torch.zeros(m, ld, dtype=tdt, device=dev),
                 torch.empty(m, dtype=torch.int32, device=dev))
            xs, ts, nss, ps = x[ri].contiguous(), t[ri].contiguous(), ns[ri].contiguous(), pidx[ri].contiguous()
            flush.fill_(3.0)
            e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0_.record(stream)
            hj.hj_solve(ctx, xs, ts, nss, ps, 0, o)
            e1_.record(stream)
            torch.cuda.synchronize()
            ms_d = e0_.elapsed_time(e1_)
            u_d = _units(wl, rows)
            fam = {f: int(sum(1 for r in rows if wl.problems[int(wl.problem_idx[r])].family == f))
                   for f in sorted({p_.family for p_ in wl.problems})}
            per_d.append({"d": dd, "queries": m, "pairs": u_d, "ms": ms_d, "pairs_per_s": u_d / (ms_d / 1e3),
                          "queries_by_family": fam})

    result = None
    if rank == 0:
        cpu = None
        acc = None
        if not a.no_cpu and world == 1:
            # evenly spread over the batch (a stride that is not a multiple of a
            # batch's period, so a mix of times t is sampled at every t)
            ids = np.unique(np.linspace(0, nq - 1, min(nq, CPU_SAMPLE)).round().astype(np.int64))
            sec, ref, threads = _time_oracle(wl, ids)
            cpu = {"value": _units(wl, ids) / sec, "unit": _unit(wl), "cores": threads, "kind": "oracle",
                   "sample": f"{len(ids)} queries evenly spread over the workload, all their starts, FP64, "
                             f"{sec:.1f} s wall"}
            ids1 = ids[:CPU_SAMPLE_1]
            sec1, _, _ = _time_oracle(wl, ids1, threads=1)
            cpu["one_core"] = {"value": _units(wl, ids1) / sec1, "cores": 1,
                               "sample": f"the first {len(ids1)} of those queries, {sec1:.1f} s wall"}
            err = np.abs(phi_np[ids] - ref["phi"]) / (1 + np.abs(ref["phi"]))
            agree = (st_np[ids] & 1) == (ref["status"] & 1)
            acc = {"sample": len(ids), "max_rel_err": float(err.max()),
                   "frac_within_1e-4": float(np.mean(err <= 1e-4)),
                   "certified_agree": float(np.mean(agree))}
            if sec <= 20.0:
                # the oracle alone, on x moved twice by 1e-7 (relative): queries
                # whose certificate decision or phi moves are decided by
                # rounding, not by the problem (non-convex H: trajectories that
                # pass near the smoothed kinks of |p_i|)
                stable = np.ones(len(ids), bool)
                sub = wl.take(ids)
                O_, probs_, opts_ = _oracle_inputs(wl)
                for seed in (0, 1):
                    xp = sub.x * (1 + 1e-7 * np.random.default_rng(seed).standard_normal(sub.x.shape))
                    rp = O_.solve(probs_, opts_, xp, sub.t, sub.n_steps, problem_idx=sub.problem_idx,
                                  query_ids=np.asarray(ids, dtype=np.int64))
                    stable &= ((rp["status"] & 1) == (ref["status"] & 1)) & \
                        (np.abs(rp["phi"] - ref["phi"]) <= 1e-6 * (1 + np.abs(ref["phi"])))
                acc["oracle_stable"] = int(stable.sum())
                acc["certified_agree_on_stable"] = float(np.mean(agree[stable])) if stable.any() else None
                acc["disagreeing_queries"] = [{"query": int(ids[i]), "oracle_stable": bool(stable[i])}
                                              for i in np.flatnonzero(~agree)]
            if plain is not None:
                # against the oracle's answer (its gradient descent with the
                # adjoint: the discrete optimum)
                have = ~np.isnan(plain["phi"][ids])
                errp = np.abs(plain["phi"][ids] - ref["phi"]) / (1 + np.abs(ref["phi"]))
                plain["accuracy_sample"] = int(have.sum())
                plain["max_rel_err_vs_oracle"] = float(errp[have].max())
                plain["frac_within_1e-4"] = float(np.mean(errp[have] <= 1e-4))
                plain["certified_agree_with_oracle"] = float(np.mean((plain["st"][ids][have] & 1)
                                                                     == (ref["status"][have] & 1)))
                err_ad = np.abs(phi_np[ids] - ref["phi"]) / (1 + np.abs(ref["phi"]))
                for row in plain.get("per_t", []):
                    sel = wl.t[ids] == row["t"]
                    row["sample"] = int(sel.sum())
                    row["adjoint_max_rel_err"] = float(err_ad[sel].max()) if sel.any() else None
                    row["plain_cd_fd_max_rel_err"] = float(errp[sel].max()) if sel.any() else None
                    row["plain_cd_fd_frac_within_1e-4"] = float(np.mean(errp[sel] <= 1e-4)) if sel.any() else None
        if plain is not None:
            plain.pop("phi")
            plain.pop("st")
        result = {
            "metric": metric, "value": value, "unit": _unit(wl), "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": dict(_config(a, wl, descent, nq), tuning=tuning),
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": _unit(wl), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
            "clocks": clocks,
            "detail": {"functional_evals_per_s": sum(i["functional_evals"] + i["n_pairs"] for i in infos)
                       / (sum(ms_steps) / 1e3),
                       "gradients_per_s": sum(i["gradient_evals"] for i in infos) / (sum(ms_steps) / 1e3),
                       "rk4_steps_per_s": sum(i["rk4_steps"] + i["adjoint_steps"] for i in infos)
                       / (sum(ms_steps) / 1e3),
                       "nominal_tflop_per_step": sum(i["nominal_flops"] for i in infos) / len(infos) / 1e12,
                       "descent_ms_per_step": desc_s * 1e3 / len(infos),
                       "descent_round0_ms_per_step": sum(i["descent_ms_round0"] for i in infos) / len(infos),
                       "certify_ms_per_step": sum(i["certify_ms"] for i in infos) / len(infos),
                       "gradients_per_step": info["gradient_evals"], "pairs_per_step": info["n_pairs"],
                       "iterations_per_pair": info["iterations"] / max(1, info["n_pairs"]),
                       "threads_per_pair": info["threads_per_pair"], "comps_per_thread": info["comps_per_thread"],
                       "algorithmic_tflop_per_step": sum(i["algorithmic_flops"] for i in infos) / len(infos) / 1e12,
                       "tensor_tflop_per_step": tflops / len(infos) / 1e12,
                       "certified_frac": float(np.mean(st_np & 1))},
            "plain_cd_fd": plain,
            "per_d": per_d,
            "accuracy_vs_oracle": acc,
            "cpu_baseline": cpu,
        }
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result))


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
