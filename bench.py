"""Benchmark of the QQMC hot path on GB300.

Workload (default): the plain method at scale on the single-level dot --
Gamma = 1, wide band, T = 0, t_max = 10, tau = 1, L = 4096 table nodes,
eps_d in {-1, 0, +1}, orders n = 1..10, N = 2^20 Sobol' points x K = 32
digitally shifted sequences per (eps_d, n), FP64 throughout.

A step is one batch of that workload: all 30 (eps_d, n) integrations over
one contiguous slice of 2^16 Sobol' indices of every shifted sequence, run
as ONE persistent-kernel launch (plus its reduction kernel).  Sixteen steps
cover the whole N = 2^20; step s takes slice s mod 16 (partial sums over
slices add up exactly to the full integration).  L2 is flushed (a 256 MiB
write) between timed steps; the Green-function tables (64 KiB) would
otherwise stay L2-resident.

Metric: integrand evaluations per second (every Sobol' point counts, as in
the paper's N; the line also gives in-domain and Keldysh-determinant rates).
`e2e` runs the same batches through the public C ABI from host parameters:
problem creation (tables built on the device), shift-word upload, launch and
result download inside the timed region.

--impl reference times the CPU oracle (this project's reference arm) on a
bounded sample of the same workload.  Multi-GPU runs are independent
replicas (one full workload per rank, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EPS = (-1.0, 0.0, 1.0)
ORDERS = tuple(range(1, 11))
N_TOTAL = 2 ** 20
SLICE = 2 ** 16
K_SHIFTS = 32
T_MAX, TAU, GAMMA, L_TABLE = 10.0, 1.0, 1.0, 4096
SEED = 2002123720
METRIC = "integrand_evals_per_s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        pg = dist
    return ws, rank, local, pg


def _barrier(pg):
    if pg is not None:
        pg.barrier()


def _max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def aggregate(pg, units: float, seconds: float):
    """Whole-job throughput of independent replicas: the units every rank
    processed divided by the slowest rank's time.  Returns (value, max seconds)."""
    t = _max_over_ranks(pg, seconds)
    return _sum_over_ranks(pg, units) / t, t


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [x for x in sm if mx and x > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def tree_shape(Q, pr, prec: int, n: int):
    """(pair-block tree?, flat depth) that order n of problem pr runs with: the problem's
    elimination order and that tree's tuned flat depth (one-point-per-lane orders resolve
    all n - 1 vertices after the first per lane, with vertex pairs)."""
    pairs = Q.qqmc_elimination(pr, prec) == Q.QQMC_ELIM_PAIRS
    f = Q.qqmc_get_tuning(prec | (Q.QQMC_TUNE_PAIRS if pairs else 0), n)[1]
    return (pairs or f < 2), (f if f >= 2 else n - 1)


def workload_items(Q, problems, s: int, slice_n: int = SLICE):
    """Items of step s: every (eps_d, n) over Sobol' slice s (shift words from the seed)."""
    first = (s % (N_TOTAL // slice_n)) * slice_n
    items = []
    for pr in problems:
        for n in ORDERS:
            items.append((pr, n, K_SHIFTS, slice_n, None, first))
    return items


def run_ours(args, ws, rank, local, pg):
    import torch

    from paper_2002_12372_gb300 import build as b
    from paper_2002_12372_gb300 import perf
    from paper_2002_12372_gb300 import qqmc as Q

    if rank == 0 or ws > 1:
        b.build()
    _barrier(pg)
    torch.cuda.set_device(local)
    Q.load()
    tuned = None
    if args.tuning and os.path.exists(args.tuning):
        from paper_2002_12372_gb300 import autotune
        tuned = autotune.load(args.tuning)
        if tuned:
            autotune.install(tuned)
    prec = Q.QQMC_PREC_FP64 if args.precision == "fp64" else Q.QQMC_PREC_MIXED
    stream = torch.cuda.Stream()
    problems = [Q.qqmc_create_problem(Q.make_params(GAMMA, e, T_MAX, TAU, L_TABLE, SEED)) for e in EPS]
    slice_n = 2 ** args.slice_log2
    n_plans = min(args.steps + args.warmup, N_TOTAL // slice_n)
    plans = [Q.Plan(workload_items(Q, problems, s, slice_n), prec) for s in range(n_plans)]
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    # every item runs with its own order's tuned flat depth on its problem's Keldysh-sum tree
    # (one launch per shape group); one-point-per-lane orders (flat 1) resolve all their
    # vertices per lane with vertex pairs
    shape_of = {(id(pr), n): tree_shape(Q, pr, prec, n) for pr in problems for n in ORDERS}
    pairs0, flat = shape_of[(id(problems[0]), max(ORDERS))]
    wpb = Q.qqmc_get_tuning(prec | (Q.QQMC_TUNE_PAIRS if pairs0 else 0), max(ORDERS))[0]
    flat_of = {n: shape_of[(id(problems[0]), n)][1] for n in ORDERS}

    def step(s):
        p = plans[s % n_plans]
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        p.launch(stream.cuda_stream)
        ev1.record(stream)
        return p, ev0, ev1

    for s in range(args.warmup):
        p, _, _ = step(s)
        p.results()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    _barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step_ms, kern_ms, flops, pts, pts_in, dets, naive = [], [], 0.0, 0, 0, 0.0, 0.0
    for s in range(args.warmup, args.warmup + args.steps):
        p, ev0, ev1 = step(s)
        res = p.results()  # waits for this launch
        km, _ = p.timing()
        step_ms.append(ev0.elapsed_time(ev1))
        kern_ms.append(km)
        items = workload_items(Q, problems, s, slice_n)
        for (r, _S), it in zip(res, items):
            pairs, f = shape_of[(id(it[0]), r.order)]
            pts += r.n_points * r.n_shifts
            pts_in += r.n_in_domain
            dets += r.n_in_domain * 2.0 ** r.order
            flops += r.n_in_domain * perf.flops_per_point(r.order, f, pairs, args.precision)
            naive += r.n_in_domain * perf.w_naive(r.order)
    torch.cuda.synchronize()
    _barrier(pg)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    dev_s = sum(step_ms) / 1e3
    value, dev_s_max = aggregate(pg, pts, dev_s)
    k_s = sum(kern_ms) / 1e3
    launches = args.steps * plans[0].kernel_count()

    # e2e through the public API from host parameters
    e2e_steps = max(1, min(2, args.steps))
    _barrier(pg)
    torch.cuda.synchronize()
    te = time.perf_counter()
    e2e_pts, h2d, d2h = 0, 0, 0
    for s in range(e2e_steps):
        prs = [Q.qqmc_create_problem(Q.make_params(GAMMA, e, T_MAX, TAU, L_TABLE, SEED)) for e in EPS]
        pl = Q.Plan(workload_items(Q, prs, s, slice_n), prec)
        pl.launch(stream.cuda_stream)
        res = pl.results()
        pl.close()
        for pr in prs:
            Q.qqmc_destroy_problem(pr)
        for r, _S in res:
            e2e_pts += r.n_points * r.n_shifts
        # host -> device: item descriptors (128 B each) and shift words; device -> host:
        # per-shift complex sums (16 B) and in-domain counts (8 B)
        h2d += len(res) * 128 + sum(r.n_shifts * r.order * 4 for r, _ in res)
        d2h += sum(r.n_shifts * (16 + 8) for r, _ in res)
    torch.cuda.synchronize()
    e2e_value, e2e_s = aggregate(pg, e2e_pts, time.perf_counter() - te)

    peak = perf.peak_tflops(args.precision)
    achieved = flops / k_s / 1e12 if k_s > 0 else None
    out = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_s_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": "plain QQMC single-level dot: Gamma=1, eps_d in {-1,0,1}, t_max=10, tau=1, "
                               "L=4096, orders 1..10, N=2^20 x 32 shifts (16 batches of 2^16 indices)",
                   "batch": "30 (eps_d, n) integrations x 2^%d indices x 32 shifts per step" % args.slice_log2,
                   "precision": args.precision, "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "tuning": {"warps_per_block": wpb, "flat_vertices": flat,
                              "flat_per_order": flat_of,
                              "source": "autotuner table" if tuned else "built-in defaults"}},
        "in_domain_evals_per_s": _sum_over_ranks(pg, pts_in) / dev_s_max,
        "keldysh_det_evals_per_s": _sum_over_ranks(pg, dets) / dev_s_max,
        "naive_equivalent_tflops": _sum_over_ranks(pg, naive) / dev_s_max / 1e12,
        "wall_s": wall,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d // e2e_steps,
                "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": _launch_traffic(args, slice_n),
                     "kernel": "detsum_kernel<%s,flat> (one launch per tuned flat depth)" % (
                         "double" if args.precision == "fp64" else "float"),
                     "peak_source": "measured: %s FMA throughput of the register-resident microbenchmark "
                                    "(qqmc_fma_peak, bench.py --config peaks) at 2070 MHz; %.4g TFLOP/s derived "
                                    "from unit counts" % (args.precision, perf.derived_tflops(args.precision)),
                     "kernel_ms_per_step": k_s * 1e3 / args.steps},
        "clocks": clk,
    }
    for pl in plans:
        pl.close()
    for pr in problems:
        Q.qqmc_destroy_problem(pr)
    return out


# DRAM bytes (read + write) of the detsum launches of one default benchmark step (one launch per
# tuned flat depth), from a 1-pass ncu capture of this exact command; per step, like the achieved
# rate.  None whenever the determinant kernel has changed since the capture.
MEASURED_LAUNCH_TRAFFIC = {"fp64": 121000000, "mixed": 1610000}


def _launch_traffic(args, slice_n):
    if args.config != "plain" or slice_n != 2 ** 16:
        return None
    return MEASURED_LAUNCH_TRAFFIC.get(args.precision)


def _setup(args, local):
    import torch

    from paper_2002_12372_gb300 import build as b
    from paper_2002_12372_gb300 import qqmc as Q
    b.build()
    torch.cuda.set_device(local)
    Q.load()
    if args.tuning and os.path.exists(args.tuning):
        from paper_2002_12372_gb300 import autotune
        t = autotune.load(args.tuning)
        if t:
            autotune.install(t)
    return Q


def run_batched(args, local):
    """One persistent launch over orders 2..12 with N_n = 2^max(14, 24-n), K = 16 (CUDA graph)."""
    import torch

    Q = _setup(args, local)
    prec = Q.QQMC_PREC_FP64 if args.precision == "fp64" else Q.QQMC_PREC_MIXED
    pr = Q.qqmc_create_problem(Q.make_params(GAMMA, 0.0, T_MAX, TAU, L_TABLE, SEED))
    items = [(pr, n, 16, 2 ** max(14, 24 - n)) for n in range(2, 13)]
    plan = Q.Plan(items, prec)
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        plan.launch(stream.cuda_stream, use_graph=True)
        plan.results()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.launch(stream.cuda_stream, use_graph=True)
        e1.record(stream)
        res = plan.results()
        ms.append(e0.elapsed_time(e1))
    pts = sum(r.n_points * r.n_shifts for r, _ in res)
    dets = sum(r.n_in_domain * 2.0 ** r.order for r, _ in res)
    # the same items as separate launches, one per order (no graph)
    sep = 0.0
    for it in items:
        p1 = Q.Plan([it], prec)
        p1.launch(stream.cuda_stream)
        p1.results()
        p1.launch(stream.cuda_stream)
        p1.results()
        sep += p1.timing()[1]
        p1.close()
    plan.close()
    # where batching pays: many items that each leave most of the GPU idle (a served sweep's small
    # requests): 3 dots x orders 4..10 x 2^12 points x 16 shifts, one batched launch against one
    # plan per item
    probs = [Q.qqmc_create_problem(Q.make_params(GAMMA, e, T_MAX, TAU, L_TABLE, SEED)) for e in EPS]
    small = [(p, n, 16, 2 ** 12) for p in probs for n in range(4, 11)]
    bplan = Q.Plan(small, prec)
    for _ in range(2):
        bplan.launch(stream.cuda_stream, use_graph=True)
        bplan.results()
    sm = []
    for _ in range(max(1, args.steps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bplan.launch(stream.cuda_stream, use_graph=True)
        e1.record(stream)
        bplan.results()
        sm.append(e0.elapsed_time(e1))
    bplan.close()
    small_sep = 0.0
    for it in small:
        p1 = Q.Plan([it], prec)
        p1.launch(stream.cuda_stream)
        p1.results()
        p1.launch(stream.cuda_stream)
        p1.results()
        small_sep += p1.timing()[1]
        p1.close()
    for p in probs:
        Q.qqmc_destroy_problem(p)
    Q.qqmc_destroy_problem(pr)
    t = statistics.median(ms) / 1e3
    return {"metric": "batched_integrand_evals_per_s", "value": pts / t, "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "one persistent launch (CUDA graph) over orders 2..12, N_n = 2^max(14,24-n), "
                                   "16 shifts, Gamma=1, eps_d=0, t=10, tau=1, L=4096", "precision": args.precision},
            "keldysh_det_evals_per_s": dets / t, "separate_launches_ms": sep, "batched_ms": t * 1e3,
            "small_items": {"items": len(small), "batched_ms": statistics.median(sm), "separate_launches_ms": small_sep,
                            "workload": "3 dots (eps_d -1, 0, 1) x orders 4..10 x 2^12 points x 16 shifts"},
            "per_order": {r.order: {"q": r.q_mean, "err": r.q_err, "in_domain": r.n_in_domain} for r, _ in res}}


def run_precision(args, local):
    """Orders 6..12 at N = 2^log2 x 16 shifts: mixed (FP32 tables and Schur updates) against the FP64 path,
    plus the per-point integrand error of the mixed path against the FP64 path on identical points (the FP64
    integrand itself agrees with the CPU oracle to 1e-12 of the Keldysh-sum scale in the parity tests)."""
    import numpy as np
    import torch

    from paper_2002_12372_gb300 import workloads as W

    Q = _setup(args, local)
    N = 2 ** args.precision_log2
    pr = Q.qqmc_create_problem(Q.make_params(GAMMA, 0.0, T_MAX, TAU, L_TABLE, SEED))
    rows = {}
    stream = torch.cuda.Stream()
    t_mixed = t_fp64 = 0.0
    for n in range(6, 13):
        out = {}
        for prec in (Q.QQMC_PREC_MIXED, Q.QQMC_PREC_FP64):
            plan = Q.Plan([(pr, n, 16, N)], prec)
            plan.launch(stream.cuda_stream)
            (r, S), = plan.results()
            out[prec] = (r, plan.timing()[0])
            plan.close()
        rm, km = out[Q.QQMC_PREC_MIXED]
        rf, kf = out[Q.QQMC_PREC_FP64]
        t_mixed += km
        t_fp64 += kf
        u = W.ordered_times(900 + n, 8 if n < 11 else 3, n, T_MAX)
        cm = Q.qqmc_integrand(pr, n, u, Q.QQMC_PREC_MIXED)
        ref = Q.qqmc_integrand(pr, n, u, Q.QQMC_PREC_FP64)
        rows[n] = {"q_mixed": rm.q_mean, "q_fp64": rf.q_mean, "err_bar": rf.q_err,
                   "abs_dev": abs(rm.q_mean - rf.q_mean), "dev_over_err": abs(rm.q_mean - rf.q_mean) / rf.q_err,
                   "rel_dev": abs(rm.q_mean - rf.q_mean) / abs(rf.q_mean),
                   "point_err_rel_max": float(np.max(np.abs(cm - ref) / np.abs(ref))),
                   "point_err_rel_median": float(np.median(np.abs(cm - ref) / np.abs(ref))),
                   "ms_mixed": km, "ms_fp64": kf}
    Q.qqmc_destroy_problem(pr)
    return {"metric": "precision_study", "value": t_fp64 / t_mixed, "unit": "speedup mixed over fp64",
            "config": {"workload": "orders 6..12, N=2^%d x 16 shifts, Gamma=1, eps_d=0, t=10, tau=1, L=4096"
                                   % args.precision_log2}, "per_order": rows}


def run_current(args, local):
    """Current I_n through the dot with semicircular leads under bias (the paper's finite-bias current
    calculations): one plan over orders 1..10 with 2^log2 points x 10 shifts each, alpha at the
    occupation of the tables' level, Im g^<(0) (the shift that cancels the Hartree term)."""
    import numpy as np
    import torch

    from paper_2002_12372_gb300 import workloads as W

    Q = _setup(args, local)
    c = W.CurrentConfig()
    prec = Q.QQMC_PREC_FP64 if args.precision == "fp64" else Q.QQMC_PREC_MIXED
    L = args.current_table

    def params(alpha):
        return Q.make_params(c.gamma, c.E_d, c.t_max, c.tau, L, SEED, alpha=alpha, observable=Q.QQMC_OBS_CURRENT,
                             half_bandwidth=c.half_bandwidth, bias=c.bias)

    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    pr0 = Q.qqmc_create_problem(params(0.0))
    table_s = time.perf_counter() - t0
    alpha = float(np.imag(Q.qqmc_problem_tables(pr0, L)[2]))  # the tables do not depend on alpha
    Q.qqmc_destroy_problem(pr0)
    pr = Q.qqmc_create_problem(params(alpha))
    tree = "pairs" if Q.qqmc_elimination(pr, prec) == Q.QQMC_ELIM_PAIRS else "single"
    N = 2 ** args.current_log2
    plan = Q.Plan([(pr, n, c.n_shifts, N) for n in c.orders], prec)
    for _ in range(args.warmup):
        plan.launch(stream.cuda_stream, use_graph=True)
        plan.results()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.launch(stream.cuda_stream, use_graph=True)
        e1.record(stream)
        res = plan.results()
        ms.append(e0.elapsed_time(e1))
    plan.close()
    _cl, _cg, c0 = Q.qqmc_problem_current_tables(pr, L)
    Q.qqmc_destroy_problem(pr)
    t = sum(ms) / len(ms) / 1e3
    pts = sum(r.n_points * r.n_shifts for r, _ in res)
    return {"metric": "current_integrand_evals_per_s", "value": pts / t, "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "current, semicircular leads D=%g, Gamma=%g, E_d=%g, alpha=Im g<(0)=%.6f, V=%g, "
                                   "t=%g, tau=%g, L=%d, orders %d..%d, N=2^%d x %d shifts, one CUDA-graph launch"
                                   % (c.half_bandwidth, c.gamma, c.E_d, alpha, c.bias, c.t_max, c.tau, L,
                                      c.orders[0], c.orders[-1], args.current_log2, c.n_shifts),
                       "tree": tree,
                       "precision": args.precision, "l2": "flushed (256 MiB write) between timed steps"},
            "table_build_s": table_s, "I_0": -4.0 * c0.real,
            "per_order": {r.order: {"I": r.q_mean, "err": r.q_err, "in_domain": r.n_in_domain} for r, _ in res}}


def run_peaks(args, local):
    """Measured FMA throughput of the FP64 and FP32 pipes (the roofline denominators of the
    determinant kernels), with the SM clocks sampled while it runs."""
    Q = _setup(args, local)
    from paper_2002_12372_gb300 import perf
    clocks = Clocks(local)
    clocks.start()
    runs = {"fp64": [], "fp32": []}
    for _ in range(max(1, args.steps)):
        runs["fp64"].append(Q.qqmc_fma_peak(Q.QQMC_PREC_FP64, 1.0))
        runs["fp32"].append(Q.qqmc_fma_peak(Q.QQMC_PREC_MIXED, 1.0))
    clk = clocks.stop()
    out = {k: {"best_tflops": max(v), "runs": v} for k, v in runs.items()}
    mhz = clk.get("sm_mhz")
    for k in ("fp64", "fp32"):
        derived = perf.derived_tflops("fp64" if k == "fp64" else "mixed", mhz or perf.SM_MAX_MHZ)
        out[k]["derived_tflops_at_sampled_clock"] = derived
        out[k]["fraction_of_derived"] = out[k]["best_tflops"] / derived
    return {"metric": "fma_peak_tflops", "value": out["fp64"]["best_tflops"], "unit": "TFLOP/s (FP64 FMA)",
            "n_gpus": 1, "steps": args.steps, "warmup": 0, "higher_is_better": True, "dtype": "f64",
            "data": "register-resident FMA chains", "config": {"workload": "qqmc_fma_peak: 8 independent FMA chains "
                                                                         "per thread, 64 warps per SM, ~1 s each"},
            "peaks": out, "clocks": clk}


def run_orders(args, local):
    """Integrand evals/s and Keldysh-det evals/s at each order n (the benchmark's per-order metric):
    one single-order plan per n on the paper's long-time dot (Gamma=1, eps_d=0, t=30, tau=0.95, L=4096:
    nearly every point in the domain up to n ~ 20), K = 16 shifts, N a power of two budgeted from the
    algorithmic cost to ~0.3 s (--orders-seconds), the kernel time of the second launch."""
    import torch

    from paper_2002_12372_gb300 import perf

    Q = _setup(args, local)
    prec = Q.QQMC_PREC_FP64 if args.precision == "fp64" else Q.QQMC_PREC_MIXED
    if args.stack_min_order:
        Q.qqmc_set_stack_policy(prec, args.stack_min_order)
    pr = Q.qqmc_create_problem(Q.make_params(GAMMA, 0.0, 30.0, 0.95, L_TABLE, SEED))
    stream = torch.cuda.Stream()
    rows = {}
    rate = 0.7e12 if prec == Q.QQMC_PREC_FP64 else 15e12
    for n in range(args.orders_min, args.orders_max + 1):
        pairs, f = tree_shape(Q, pr, prec, n)
        want = args.orders_seconds * rate / perf.flops_per_point(n, f, pairs, args.precision) / 16
        N = int(2 ** max(6, min(22, math.floor(math.log2(max(want, 1.0))))))
        plan = Q.Plan([(pr, n, 16, N)], prec)
        plan.launch(stream.cuda_stream)
        plan.results()
        plan.launch(stream.cuda_stream)
        (r, _S), = plan.results()
        km = plan.timing()[0]
        plan.close()
        secs = km / 1e3
        rows[n] = {"N": N, "shifts": 16, "kernel_ms": km, "evals_per_s": N * 16 / secs,
                   "in_domain_evals_per_s": r.n_in_domain / secs,
                   "keldysh_det_evals_per_s": r.n_in_domain * 2.0 ** n / secs,
                   "tflops": r.n_in_domain * perf.flops_per_point(n, f, pairs, args.precision) / secs / 1e12,
                   "flat": f,
                   "tree": "pairs" if pairs else "single"}
    Q.qqmc_destroy_problem(pr)
    n_head = min(max(10, args.orders_min), args.orders_max)
    return {"metric": "per_order_integrand_evals_per_s", "value": rows[n_head]["evals_per_s"],
            "unit": "evals/s at order %d" % n_head, "n_gpus": 1, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": "plain dot Gamma=1, eps_d=0, t=30, tau=0.95, L=4096, one plan per order, 16 shifts",
                       "precision": args.precision, "stack_min_order": args.stack_min_order or "default"},
            "per_order": rows}


def run_lattice(args, local):
    """Sobol' against a rank-1 lattice (component-by-component vector, product weights 0.9^d) on the
    plain dot at equal point counts: per order the estimate, its shift error bar, and the time."""
    import numpy as np
    import torch

    Q = _setup(args, local)
    prec = Q.QQMC_PREC_FP64 if args.precision == "fp64" else Q.QQMC_PREC_MIXED
    m, K = args.lattice_log2, 16
    orders = (2, 4, 6, 8, 10)
    gamma = np.array([0.9 ** d for d in range(max(orders))])
    z = Q.qqmc_lattice_cbc(m, max(orders), gamma)
    stream = torch.cuda.Stream()
    rows = {}
    for family in ("sobol", "lattice", "lattice_bakers"):
        pr = Q.qqmc_create_problem(Q.make_params(GAMMA, 0.0, T_MAX, TAU, L_TABLE, SEED))
        if family != "sobol":
            Q.qqmc_set_lattice(pr, m, z, family == "lattice_bakers")
        plan = Q.Plan([(pr, n, K, 1 << m) for n in orders], prec)
        plan.launch(stream.cuda_stream)
        res = plan.results()
        ms = plan.timing()[0]
        plan.close()
        Q.qqmc_destroy_problem(pr)
        for r, _ in res:
            rows.setdefault(r.order, {})[family] = {"q": r.q_mean, "err": r.q_err}
        rows.setdefault("kernel_ms", {})[family] = ms
    ratios = [rows[n]["sobol"]["err"] / rows[n]["lattice_bakers"]["err"] for n in orders]
    return {"metric": "lattice_vs_sobol_error_ratio", "value": float(np.exp(np.mean(np.log(ratios)))),
            "unit": "geometric mean of err(Sobol')/err(lattice with baker's transform)", "n_gpus": 1,
            "config": {"workload": "plain dot Gamma=1, eps_d=0, t=10, tau=1, L=4096, orders %s, N=2^%d x %d shifts"
                                   % (list(orders), m, K), "precision": args.precision,
                       "lattice": "CBC, product weights 0.9^d, z=%s" % list(map(int, z))},
            "per_order": rows}


def run_serving(args, local):
    """Request sweep with Poisson arrivals through qqmc_submit / qqmc_poll (continuous batching)."""
    import torch

    from paper_2002_12372_gb300 import workloads as W

    Q = _setup(args, local)
    prec = Q.QQMC_PREC_FP64 if args.precision == "fp64" else Q.QQMC_PREC_MIXED
    reqs = W.serving_sweep(SEED, args.requests, args.rate, args.serve_log2_min, args.serve_log2_max, 16)
    opts = Q.qqmc_server_opts(device_memory_limit=8 << 30, max_queue=4096, max_batch_items=256, precision=prec,
                              use_graph=0, request_timeout_s=0.0)
    srv = Q.qqmc_server_create(opts)
    handles, done = {}, {}
    t0 = time.perf_counter()
    i = 0
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].arrival_s <= now:
            r = Q.qqmc_request()
            q = reqs[i]
            r.params = Q.make_params(q.gamma, q.eps_d, q.t_max, 1.0 / q.gamma, L_TABLE, SEED + i)
            r.n_max, r.n_shifts, r.n_points, r.U = q.n_max, q.n_shifts, q.n_points, q.U
            handles[Q.qqmc_submit(srv, r)] = i
            i += 1
        for h, k in list(handles.items()):
            rc, out = Q.qqmc_poll(srv, h)
            if rc != Q.QQMC_PENDING:
                done[k] = (rc, out)
                del handles[h]
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    Q.qqmc_server_destroy(srv)
    lat = sorted(out.latency_ms for rc, out in done.values() if rc == Q.QQMC_OK)
    evals = sum(q.n_points * q.n_shifts * q.n_max for q in reqs)
    rel_err = [out.q_err[q.n_max] / max(abs(out.q[q.n_max]), 1e-300) for q, (rc, out) in
               zip(reqs, [done[k] for k in range(len(reqs))]) if rc == Q.QQMC_OK]
    pct = lambda p: lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
    return {"metric": "serving", "value": evals / makespan, "unit": "evals/s", "n_gpus": 1,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "%d requests, eps_d~U[-3,3], U in {1,2,4}, t_max in {5,10,20}, n_max~U{4..10}, "
                                   "N=2^floor(U[%d,%d]), 16 shifts, Poisson arrivals at %g/s"
                                   % (len(reqs), args.serve_log2_min, args.serve_log2_max, args.rate),
                       "precision": args.precision},
            "p50_latency_ms": pct(50), "p99_latency_ms": pct(99), "makespan_s": makespan,
            "completed": len(lat), "failed": len(reqs) - len(lat),
            "median_rel_err_at_nmax": statistics.median(rel_err) if rel_err else None}


def cpu_oracle_sample(seconds_per_order: float = 1.5, orders=ORDERS, shift_seed: int = SEED, threads: int = 0):
    """Time the CPU oracle on a bounded sample of the workload (eps_d = 0, one shift,
    first M points per order with M chosen so each order runs ~seconds_per_order).
    Set-up that is not per-point work stays out of the timed calls: the direction
    words are built once and passed in, and every order runs once untimed first.
    threads = 0: every host core."""
    from oracle import oracle as O

    tabs = O.gf_tables(GAMMA, 0.0, T_MAX, L_TABLE)
    sw = O.shift_words(shift_seed, 1, max(orders))
    V = O.sobol_direction_numbers(max(orders))
    threads = threads or os.cpu_count() or 1
    per_point = {}
    sample = {}
    for n in orders:
        O.estimate(n, 32 * threads, sw, T_MAX, TAU, tabs, T_MAX, V=V, threads=threads, chunk=32)  # warm-up
        M = 64 * threads
        while True:
            t0 = time.perf_counter()
            O.estimate(n, M, sw, T_MAX, TAU, tabs, T_MAX, V=V, threads=threads, chunk=max(1, M // (4 * threads)))
            dt = time.perf_counter() - t0
            if dt > 0.25 * seconds_per_order or M >= 2 ** 20:
                break
            M *= 4
        per_point[n] = dt / M
        sample[n] = M
    # the workload has equal point counts per order: evals/s = n_orders / sum_n t_n
    value = len(orders) / sum(per_point.values())
    return value, threads, sample


def cpu_baseline_entry(seconds_per_order: float = 1.5):
    """The oracle on every host core (the reported value) and on one core."""
    v, threads, sample = cpu_oracle_sample(seconds_per_order)
    v1, _, sample1 = cpu_oracle_sample(seconds_per_order / 2, threads=1)
    return {"value": v, "unit": "evals/s", "cores": threads, "kind": "oracle",
            "single_core_value": v1,
            "sample": "eps_d=0, 1 shift, first points per order " + ",".join(
                "n%d:%d" % (n, m) for n, m in sample.items()) + "; one core: " + ",".join(
                "n%d:%d" % (n, m) for n, m in sample1.items())}


def run_reference(args, ws, rank, pg):
    if rank != 0:
        return None
    for _ in range(args.warmup):
        cpu_oracle_sample(0.05)
    vals = []
    t0 = time.perf_counter()
    threads, sample = 1, {}
    for _ in range(args.steps):
        v, threads, sample = cpu_oracle_sample(0.6)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    desc = "CPU oracle (complex128, naive 2^n pivoted LU), eps_d=0, 1 shift, points per order %s" % (
        ",".join("n%d:%d" % (n, m) for n, m in sample.items()))
    return {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "plain QQMC single-level dot: Gamma=1, eps_d in {-1,0,1}, t_max=10, tau=1, "
                                   "L=4096, orders 1..10, N=2^20 x 32 shifts (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", default=os.path.join(ROOT, "paper_2002_12372_gb300", "tuning_gb300.json"),
                    help="autotuner table (JSON keyed by GPU name); built-in defaults when absent")
    ap.add_argument("--slice-log2", type=int, default=16,
                    help="Sobol' indices per shift in one step (16: the benchmark batch; smaller for profiling)")
    ap.add_argument("--config", choices=["plain", "batched", "precision", "serving", "current", "lattice", "orders",
                                         "peaks"],
                    default="plain",
                    help="plain: the benchmark workload; the others print their own study line")
    ap.add_argument("--precision-log2", type=int, default=22)
    ap.add_argument("--current-log2", type=int, default=16)
    ap.add_argument("--current-table", type=int, default=16384)
    ap.add_argument("--lattice-log2", type=int, default=16)
    ap.add_argument("--orders-min", type=int, default=1)
    ap.add_argument("--orders-max", type=int, default=22)
    ap.add_argument("--orders-seconds", type=float, default=0.3,
                    help="orders: kernel-time budget per order that sets N")
    ap.add_argument("--stack-min-order", type=int, default=0,
                    help="orders: split tree stack from this order on (0: library default)")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--rate", type=float, default=50.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-log2-min", type=int, default=16)
    ap.add_argument("--serve-log2-max", type=int, default=22)
    args = ap.parse_args()
    if args.config != "plain":
        local = int(os.environ.get("LOCAL_RANK", "0"))
        fn = {"batched": run_batched, "precision": run_precision, "serving": run_serving,
              "current": run_current, "lattice": run_lattice, "orders": run_orders, "peaks": run_peaks}[args.config]
        print(json.dumps(fn(args, local)), flush=True)
        return
    ws, rank, local, pg = _dist()
    if args.impl == "reference":
        out = run_reference(args, ws, rank, pg)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out = run_ours(args, ws, rank, local, pg)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_entry(1.5)
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
