#!/usr/bin/env python
"""Benchmark of the batched Bezier edge build + graph search on GB300.

Metric: edge-feasibility checks per second (one check = one candidate pair
(i, j) sharing a free polytope x one duration T) of plan_build_edges, with the
shortest-path query time reported beside it (search_ms_per_query).

Workload (one query per GPU): 3-D triple integrator (|v|<=3, |a|<=6,
|jerk|<=30), 64 free polytopes of 6-12 rows in [0,20]^3, 8192 states, degree-7
Bezier, 16 durations log-uniform in [0.1, 3], FP32; seeded synthetic inputs.
A step = plan_build_edges + plan_search on HBM-resident inputs; each step is
timed with CUDA events on the planner's stream after an L2 flush (a 256 MB
write) outside the events.  N > 1 (torchrun): every rank runs its own query
(seed + rank; weak scaling, no data-path collective), times are max-reduced.
With --shard rows the ranks instead split one query's source rows
(plan_build_edges_shard), all-gather the CSR pieces over NCCL and each
searches the whole graph (strong scaling; the build time includes the
exchange).

--impl reference times the FP64 CPU oracle (the plain definition) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Bezier edge-feasibility checks/sec (+ search ms/query), 1 query per GPU"
UNIT = "checks/s"
WORKLOAD = "triple_integrator_3d N=8192 K=64 rows=6-12 nT=16 p=7 fp32"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-rows", type=int, default=0, help="rows of the oracle sample (0: auto)")
    ap.add_argument("--form", default="plain",
                    choices=["plain", "fp64", "tf32", "bf16", "batched", "refine", "cut", "replan", "planes", "mpc"],
                    help="plain: 3-D FP32 workload (the default line); fp64: 2-D FP64 plain method; tf32/bf16: "
                         "precision form on the 2-D workload; batched: 256 uneven queries in one graph replay; "
                         "refine: 65536-segment forward+backward; cut: keep-out cut of a 5000-state graph "
                         "against 500 obstacles, then the search; replan: the captured replanning tick "
                         "(moving obstacles in, cut + search, path out); planes: closest points and separating "
                         "planes of 5000 nodes x 500 obstacles; mpc: SQP refinement (3 rounds of nearest planes + "
                         "the MPC QP) of a batch of problems in the keep-out scene")
    ap.add_argument("--mpc-batch", type=int, default=1024, help="MPC problems per step (form mpc)")
    ap.add_argument("--queries", type=int, default=256)
    ap.add_argument("--shard", default="queries", choices=["queries", "rows"],
                    help="N > 1: queries -- every rank builds and searches its own query (replicas, weak scaling); "
                         "rows -- the ranks split one query's source rows (plan_build_edges_shard), exchange the CSR "
                         "pieces (all-gather-v over NCCL) and each searches the whole graph (strong scaling)")
    ap.add_argument("--pipeline", type=int, default=-1,
                    help="FP32 pair kernel of the plain line: 0 screened, 1 warp-specialised, 2 unscreened "
                         "(-1: the library default)")
    return ap.parse_args()


PAIR_KERNEL = {0: "k_pairs_sc<3,3,7> (screened)", 1: "k_pairs_ws<3,3,7>",
               2: "k_pairs_fast<3,3,7> (unscreened)"}


def workload(seed):
    from paper_2411_13507_gb300 import synth
    return synth.triple_integrator_3d(seed=seed)


def config(prob, extra=None):
    c = {"workload": WORKLOAD, "N": prob.N, "K": prob.K, "nT": prob.nT, "degree": prob.model.degree,
         "m": prob.model.m, "gamma": prob.model.gamma, "bounds": list(prob.model.bounds),
         "l2": "flushed before every timed step (256 MB write)", "parallelism": "replicas (one query per GPU)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 50 ms around the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def count(self) -> int:
        return len(self.lines)

    def summary(self, since: int = 0):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[since:]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def lane_peaks(dev, fp64=False):
    """FP32 (and FP64) lane-op rates measured on this device (plan_measure_lane_rate) and the nominal figure."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    r = {"sms": sms, "addmax": P.measure_lane_rate(0)["lane_ops_per_s"], "fma": P.measure_lane_rate(1)["lane_ops_per_s"],
         "nominal": sms * 128 * sm_max * 1e6}
    r["note"] = (f"measured: FP32 add + |.|-max register chains on all {sms} SMs (plan_measure_lane_rate) "
                 f"{r['addmax'] / 1e12:.2f} T/s; FMA chains {r['fma'] / 1e12:.2f} T/s; nominal {sms} SMs x 128 lanes "
                 f"x {sm_max:.0f} MHz ({src} clock) = {r['nominal'] / 1e12:.2f} T/s")
    if fp64:
        r["addmax64"] = P.measure_lane_rate(2, 1 << 10)["lane_ops_per_s"]
        r["fma64"] = P.measure_lane_rate(3, 1 << 10)["lane_ops_per_s"]
        r["note64"] = (f"measured: FP64 add + |.|-max register chains on all {sms} SMs (plan_measure_lane_rate) "
                       f"{r['addmax64'] / 1e12:.3f} T/s; FP64 FMA chains {r['fma64'] / 1e12:.3f} T/s")
    return r


def pair_kernel_counters():
    """DRAM traffic of the pair kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    src = os.path.join(ROOT, "paper_2411_13507_gb300", "csrc", "plan_build.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "pair_kernel_counters.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_sha") == h:
            return d, h
    except Exception:
        pass
    return None, h


def cpu_baseline(prob, budget_s=12.0, rows=0):
    """The FP64 oracle as it stands, on a bounded sample of rows of the same query."""
    import oracle
    op = oracle.OracleProblem(prob)
    op.membership()
    cnt = op.candidate_counts()
    nrows = rows
    if nrows <= 0:
        # calibrate on a few rows, then size the sample for ~budget_s of CPU time
        probe = np.arange(0, prob.N, max(1, prob.N // 16), dtype=np.int32)[:16]
        t0 = time.perf_counter()
        op.edges(probe, with_detail=False)
        dt = max(time.perf_counter() - t0, 1e-3)
        per_row = dt / len(probe)
        nrows = int(min(prob.N, max(16, budget_s / per_row)))
    sel = np.linspace(0, prob.N - 1, nrows).astype(np.int32)
    t0 = time.perf_counter()
    checks, reps = 0, 0
    while reps == 0 or time.perf_counter() - t0 < 2.0:   # small workloads: repeat for a stable time
        e = op.edges(sel, with_detail=False)
        checks += int(e["i"].shape[0]) * prob.nT
        reps += 1
    dt = time.perf_counter() - t0
    return {"value": checks / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{nrows} of {prob.N} rows x {reps} ({checks} checks, {dt:.2f} s, FP64 C oracle, OpenMP)",
            "seconds": dt, "checks": checks, "full_checks": int(cnt.sum()) * prob.nT}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = workload(args.seed)
    import oracle
    op = oracle.OracleProblem(prob)
    op.membership()
    # each step: a bounded row sample (~2 s) of the same workload
    rng_rows = [np.arange(s % 37, prob.N, 37 * 4, dtype=np.int32) for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        op.edges(rng_rows[s], with_detail=False)
    tot_checks, tot_t = 0, 0.0
    for s in range(args.steps):
        t0 = time.perf_counter()
        e = op.edges(rng_rows[args.warmup + s], with_detail=False)
        tot_t += time.perf_counter() - t0
        tot_checks += int(e["i"].shape[0]) * prob.nT
    v = tot_checks / tot_t
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config(prob, {"sample": f"{len(rng_rows[0])} rows per step"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"~{len(rng_rows[0])} rows of {prob.N} per step, {args.steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line)
    return 0


def timed(fn, stream, steps, warmup, flush=None):
    """Device time per call (CUDA events on the stream), L2 flushed before each call."""
    import torch
    for _ in range(warmup):
        if flush is not None:
            flush.fill_(1.0)
        fn()
    torch.cuda.synchronize()
    ms = []
    for s in range(steps):
        if flush is not None:
            flush.fill_(float(s))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def clocked(fn, stream, steps, warmup, flush, before=None, after=None):
    """timed() with the nvidia-smi sampler around the timed calls: fn runs
    untimed until a sample has arrived, then the timed calls, then untimed
    again until the next sample; returns (ms, clocks, after())."""
    import torch
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.time()
        while clk.count() < 1 and time.time() - t0 < 10.0:
            fn()
            torch.cuda.synchronize()
        mark = max(0, clk.count() - 1)
        if before:
            before()
        ms = timed(fn, stream, steps, warmup, flush)
        res = after() if after else None
        t0 = time.time()
        while clk.count() < mark + 2 and time.time() - t0 < 5.0:
            fn()
            torch.cuda.synchronize()
    return ms, clk.summary(since=mark), res


def ops_per_check(prob) -> float:
    """Dense separable work per check (every reach, free and cost row)."""
    g, p, m = prob.model.gamma, prob.model.degree, prob.model.m
    n = m * g
    rax = sum(p - k + 1 for k in range(1, g + 1))
    rows_mean = float(np.mean(np.diff(prob.poly_off)))
    return 4 * m * rax + 2 * (p - 1) * rows_mean + p * (2 * n + 2)


def captured_build(pl, dp, graph, stream):
    """The query prepared once as a batch of one (plan_prepare_batched) and its
    build launches (plan_build_edges_batched) captured into one CUDA graph:
    returns the graph (replay() runs one build) and its kernels per replay."""
    import torch
    pl.build_batched([dp], [graph])
    pl.timing(reset=True)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=stream):
        pl.build_batched_async()
    return cg, int(pl.timing(reset=True)["launches"])


def e2e_build_search(pl, dp, prob, graph, sbuf, stream, flush, steps, warmup, np_dtype, build=None):
    """End to end through the C ABI: states and polytopes from pinned host
    memory, the build (the replayed graph when given, else plan_build_edges)
    + plan_search, path and cost back to the host."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    h_states = torch.from_numpy(np.ascontiguousarray(prob.states, dtype=np_dtype)).pin_memory()
    h_off = torch.from_numpy(np.asarray(prob.poly_off, dtype=np.int32)).pin_memory()
    h_A = torch.from_numpy(np.ascontiguousarray(prob.A, dtype=np_dtype)).pin_memory()
    h_b = torch.from_numpy(np.ascontiguousarray(prob.b, dtype=np_dtype)).pin_memory()
    h_path = torch.empty(dp.N, dtype=torch.int32).pin_memory()
    h_cost = torch.empty(1, dtype=torch.float64).pin_memory()
    bi = sum(t.numel() * t.element_size() for t in (h_states, h_off, h_A, h_b))
    ms = []
    for s in range(warmup + steps):
        flush.fill_(2.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dp.states.copy_(h_states, non_blocking=True)
        dp.poly_off.copy_(h_off, non_blocking=True)
        dp.A.copy_(h_A, non_blocking=True)
        dp.b.copy_(h_b, non_blocking=True)
        if build is not None:
            build()
        else:
            pl.build_edges_async(dp, graph)
        pl.search_async(dp, graph, dp.start_pos, dp.goal_pos, sbuf)
        h_path.copy_(sbuf["path"], non_blocking=True)
        h_cost.copy_(sbuf["cost"], non_blocking=True)
        e1.record(stream)
        assert pl.wait() == P.PLAN_OK
        if s >= warmup:
            ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms), bi, h_path.numel() * 4 + 8


def run_form(args):
    """Lines for the other configurations (FP64 plain method, precision,
    batching and differentiation forms), each with clocks, a roofline of its
    dominant kernel, the oracle on the host cores and an end-to-end figure."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "form": args.form}
    with torch.cuda.stream(stream):
        if args.form in ("fp64", "tf32", "bf16"):
            line.update(run_2d_form(args, stream, flush, dev))
        elif args.form == "batched":
            line.update(run_batched_form(args, stream, flush, dev))
        elif args.form == "cut":
            line.update(run_cut_form(args, stream, flush, dev))
        elif args.form == "replan":
            line.update(run_replan_form(args, stream, flush, dev))
        elif args.form == "planes":
            line.update(run_planes_form(args, stream, flush, dev))
        elif args.form == "mpc":
            line.update(run_mpc_form(args, stream, flush, dev))
        elif args.form == "refine":
            line.update(run_refine_form(args, stream, flush, dev))
    return line


def run_2d_form(args, stream, flush, dev):
    """FP64 plain method and the precision form (TF32 / BF16 tensor-core
    halves) on the 2-D double-integrator workload, with the FP64 and FP32 plain
    forms timed on the same inputs."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import synth
    prob = synth.double_integrator_2d(seed=1)
    arith = {"fp64": "f64", "tf32": "tf32", "bf16": "bf16"}[args.form]
    pl = P.Planner.for_problem(prob, arith=arith, input="f64", stream=stream)
    dp = P.to_device(prob, input="f64")
    g = pl.build_edges(dp)
    info = pl.info()
    sbuf = pl.alloc_search(dp.N)
    cg, nrep = captured_build(pl, dp, g, stream)
    bms, clocks, _ = clocked(cg.replay, stream, args.steps, args.warmup, flush)
    assert pl.wait() == P.PLAN_OK
    # the pair kernel's own time and the launched build: the same launches one by one
    pl.set_timing(True)
    pl.timing(reset=True)
    bl = timed(pl.build_batched_async, stream, args.steps, args.warmup, flush)
    tm = pl.timing(reset=True)
    pl.set_timing(False)
    sms = timed(lambda: pl.search_async(dp, g, dp.start_pos, dp.goal_pos, sbuf), stream, args.steps, args.warmup,
                flush)
    assert pl.wait() == P.PLAN_OK
    checks = int(info["checks"])
    build_ms = statistics.mean(bms)
    # the plain forms on the same inputs
    plain = {}
    for ra in ("f64", "f32"):
        if ra == arith:
            continue
        p2 = P.Planner.for_problem(prob, arith=ra, input="f64", stream=stream)
        g2 = p2.build_edges(dp)
        cg2, _ = captured_build(p2, dp, g2, stream)
        ms2 = timed(cg2.replay, stream, args.steps, args.warmup, flush)
        assert p2.wait() == P.PLAN_OK
        plain[ra] = {"build_ms": statistics.mean(ms2), "checks_per_s": checks * 1e3 / statistics.mean(ms2),
                     "speedup_of_this_form": statistics.mean(ms2) / build_ms}
        p2.close()
    e2e_ms, bi, bo = e2e_build_search(pl, dp, prob, g, sbuf, stream, flush, args.steps, args.warmup, np.float64,
                                      build=cg.replay)
    lanes = lane_peaks(dev, fp64=True)
    pair_ms = tm["pair_ms"] / max(1, tm["pair_launches"])
    opc = ops_per_check(prob)
    ach = opc * checks / (pair_ms / 1e3) / 1e12
    canonical = None
    if arith == "f64":
        # default route: FP32 screened pair kernel (bits re-checked in FP64) +
        # canonical FP64 cost pass; beside it the canonical FP64 pair kernel
        peak, pnote, kern = lanes["addmax"] / 1e12, lanes["note"], "k_pairs_sc<2,2,5> (FP64 re-check) + k_cost64"
        p3 = P.Planner.for_problem(prob, arith="f64", input="f64", stream=stream)
        p3.set_tile(0, 0, 0, 3)
        g3 = p3.build_edges(dp)
        cg3, _ = captured_build(p3, dp, g3, stream)
        ms3 = timed(cg3.replay, stream, args.steps, args.warmup, flush)
        assert p3.wait() == P.PLAN_OK
        p3.set_timing(True)
        p3.timing(reset=True)
        timed(p3.build_batched_async, stream, args.steps, args.warmup, flush)
        t3 = p3.timing(reset=True)
        assert p3.wait() == P.PLAN_OK
        k3 = t3["pair_ms"] / max(1, t3["pair_launches"])
        a3 = opc * checks / (k3 / 1e3) / 1e12
        canonical = {"route": "canonical FP64 pair kernel k_pairs_f64<2,2,5> (plan_set_tile pipeline 3)",
                     "build_ms": statistics.mean(ms3), "pair_kernel_ms": k3,
                     "checks_per_s": checks * 1e3 / statistics.mean(ms3),
                     "roofline": {"bound": "alu", "achieved": a3, "peak": lanes["addmax64"] / 1e12, "unit": "TOP/s",
                                  "frac": a3 / (lanes["addmax64"] / 1e12), "peak_note": lanes["note64"],
                                  "fp64_pipe_active": "81% of peak (ncu, profiles/k_pairs_f64_double_integrator_2d.md)"}}
        p3.close()
    else:
        peak, pnote, kern = lanes["addmax"] / 1e12, lanes["note"], f"k_pairs_tc<2,2,5,{arith}>"
    cpu = None if args.no_cpu_baseline else cpu_baseline(prob)
    return {"metric": "edge-feasibility checks/sec, 2-D double integrator (N=512, K=16, nT=8, p=5)",
            "value": checks * 1e3 / build_ms, "unit": UNIT, "dtype": arith,
            "ms_per_step": build_ms + statistics.mean(sms), "build_ms_per_query": build_ms,
            "search_ms_per_query": statistics.mean(sms), "gpu_launches": args.steps * nrep, "clocks": clocks,
            "build_ms_launched": statistics.mean(bl),
            "config": {"workload": "double_integrator_2d seed 1 (|v|<=2, |a|<=4, [0,10]^2, 16 polytopes of 4-8 rows, "
                                   "512 states, p=5, 8 durations in [0.2, 2])", "checks": checks,
                       "rechecks": info["rechecks"], "recheck_frac": info["rechecks"] / max(1, checks),
                       "edges": info["edges"], "l2": "flushed before every timed call (256 MB write)",
                       "build": "the query prepared once as a batch of one, its build launches replayed as one "
                                "captured CUDA graph (every arm)"},
            "vs_plain_forms": plain, **({"canonical_fp64_route": canonical} if canonical else {}),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TOP/s", "frac": ach / peak,
                         "traffic": None, "kernel": kern, "kernel_ms": pair_ms, "ops_per_check": opc,
                         "ops_per_launch": opc * checks,
                         "work_model": "dense separable form per check (all reach, free and cost rows)"
                                       + ("" if arith == "f64" else "; the pair phase runs on the FP32 lanes, the "
                                          "halves on the tensor cores (ncu: profiles/k_pairs_tc_double_integrator_2d.md)"),
                         "peak_note": pnote},
            "e2e": {"value": checks * 1e3 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                    "ms_per_step": e2e_ms},
            "cpu_baseline": ({k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")} if cpu else None)}


def run_batched_form(args, stream, flush, dev):
    """Batching form: the uneven 3-D queries, the edge build in one replay of a
    captured CUDA graph (one persistent pair launch) with autotuned tiles, the
    batched search in another."""
    import torch
    from paper_2411_13507_gb300 import autotune
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import synth
    probs = synth.batched_queries(seed=args.seed, Q=args.queries)
    pl = P.Planner.for_problem(probs[0], arith="f32", input="f32", stream=stream)
    dps = [P.to_device(p, input="f32") for p in probs]
    graphs = pl.build_batched(dps)
    tune = autotune.tune(pl, f"batched{args.queries}", reps=2)
    graphs = pl.build_batched(dps, graphs)      # re-prepare with the tuned tiles
    info = pl.info()
    outs = pl.alloc_search_batched(dps)
    pl.prepare_search_batched(dps, graphs, outs)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=stream):
        pl.build_batched_async()
    sg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(sg, stream=stream):
        pl.search_batched_async()
    bms, clocks, _ = clocked(cg.replay, stream, args.steps, args.warmup, flush)
    sms = timed(sg.replay, stream, args.steps, args.warmup, flush)
    assert pl.wait() == P.PLAN_OK
    # the pair kernel's own time: the same launch outside the graph, with events
    pl.set_timing(True)
    pl.timing(reset=True)
    timed(pl.build_batched_async, stream, max(3, args.steps // 2), 1, flush)
    tm = pl.timing(reset=True)
    pl.set_timing(False)
    assert pl.wait() == P.PLAN_OK
    # end to end: every query's inputs from pinned host memory, the two
    # replays, every query's path length, cost and status back
    hin = []
    for p, dp in zip(probs, dps):
        hin.append([(torch.from_numpy(np.ascontiguousarray(p.states, dtype=np.float32)).pin_memory(), dp.states),
                    (torch.from_numpy(np.asarray(p.poly_off, dtype=np.int32)).pin_memory(), dp.poly_off),
                    (torch.from_numpy(np.ascontiguousarray(p.A, dtype=np.float32)).pin_memory(), dp.A),
                    (torch.from_numpy(np.ascontiguousarray(p.b, dtype=np.float32)).pin_memory(), dp.b)])
    hout = [(torch.empty(1, dtype=torch.int32).pin_memory(), o["path_len"]) for o in outs] + \
           [(torch.empty(1, dtype=torch.float64).pin_memory(), o["cost"]) for o in outs]
    bi = sum(h.numel() * h.element_size() for q in hin for h, _ in q)
    bo = sum(h.numel() * h.element_size() for h, _ in hout)
    e2e = []
    for s in range(args.warmup + args.steps):
        flush.fill_(2.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q in hin:
            for h, d in q:
                d.copy_(h, non_blocking=True)
        cg.replay()
        sg.replay()
        for h, d in hout:
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        assert pl.wait() == P.PLAN_OK
        if s >= args.warmup:
            e2e.append(e0.elapsed_time(e1))
    checks = int(info["checks"])
    build_ms = statistics.mean(bms)
    pair_ms = tm["pair_ms"] / max(1, tm["pair_launches"])
    lanes = lane_peaks(dev)
    # dense work: per-query candidates are not reported separately, so the
    # model's rows use the batch's mean polytope size (every query has p = 7, m = 3)
    rows_mean = float(np.mean(np.concatenate([np.diff(p.poly_off) for p in probs])))
    m, gg, pp = 3, 3, 7
    rax = sum(pp - k + 1 for k in range(1, gg + 1))
    opc = 4 * m * rax + 2 * (pp - 1) * rows_mean + pp * (2 * m * gg + 2)
    ach = opc * checks / (pair_ms / 1e3) / 1e12
    peak = lanes["addmax"] / 1e12
    screened = int(info.get("screened", 0))
    ex_ops = 2 * 3 * m * checks + 2 * (m * rax + (pp - 1) * rows_mean) * screened + pp * (2 * m * gg + 2) * int(info["feasible"])
    cpu = None if args.no_cpu_baseline else batched_cpu_baseline(probs)
    return {"metric": f"edge-feasibility checks/sec, {args.queries} uneven 3-D queries in one captured graph",
            "value": checks * 1e3 / build_ms, "unit": UNIT, "dtype": "f32",
            "ms_per_step": build_ms + statistics.mean(sms), "build_ms_per_batch": build_ms,
            "search_ms_per_query": statistics.mean(sms) / len(probs), "gpu_launches": int(tm["launches"]),
            "clocks": clocks,
            "config": {"workload": f"batched_queries seed {args.seed}: 3-D triple integrator, states log-uniform in "
                                   "512-16384, 8-128 polytopes, 8-16 durations, p=7", "queries": len(probs),
                       "N_total": sum(p.N for p in probs), "checks": checks, "candidates": int(info["candidates"]),
                       "edges": int(info["edges"]), "rechecks": int(info["rechecks"]), "autotune": tune,
                       "l2": "flushed before every timed replay (256 MB write)"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TOP/s", "frac": ach / peak,
                         "hw_frac": ex_ops / (pair_ms / 1e3) / 1e12 / peak, "traffic": None,
                         "kernel": "k_pairs_sc<3,3,7> (one persistent launch for the batch)", "kernel_ms": pair_ms,
                         "ops_per_check": opc, "ops_per_launch": opc * checks,
                         "work_model": "dense separable form per check, rows at the batch's mean polytope size; "
                                       "hw_frac: executed lane-ops (screen rows of every check, all rows of the "
                                       "screened ones, costs of the feasible ones) / measured peak",
                         "peak_note": lanes["note"]},
            "e2e": {"value": checks * 1e3 / statistics.mean(e2e), "unit": UNIT, "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "ms_per_step": statistics.mean(e2e)},
            "cpu_baseline": cpu}


def batched_cpu_baseline(probs, budget_s=12.0):
    """The FP64 oracle on a bounded sample of the batch: every 16th query,
    rows spread over each, until about budget_s of CPU time."""
    import oracle
    t_all, checks = 0.0, 0
    qs = list(range(0, len(probs), 16))
    per_q = budget_s / len(qs)
    rows_used = 0
    for q in qs:
        p = probs[q]
        op = oracle.OracleProblem(p)
        op.membership()
        probe = np.arange(0, p.N, max(1, p.N // 8), dtype=np.int32)[:8]
        t0 = time.perf_counter()
        op.edges(probe, with_detail=False)
        per_row = max(time.perf_counter() - t0, 1e-4) / len(probe)
        n = int(min(p.N, max(8, per_q / per_row)))
        sel = np.linspace(0, p.N - 1, n).astype(np.int32)
        t0 = time.perf_counter()
        e = op.edges(sel, with_detail=False)
        t_all += time.perf_counter() - t0
        checks += int(e["i"].shape[0]) * p.nT
        rows_used += n
    return {"value": checks / t_all, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{rows_used} rows of {len(qs)} queries (every 16th), {checks} checks, {t_all:.1f} s, "
                      "FP64 C oracle, OpenMP"}


def run_refine_form(args, stream, flush, dev):
    """Differentiation form: forward + hand-written backward of the refinement
    objective for 65536 degree-7 3-D segments."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import refine as RF
    from paper_2411_13507_gb300 import synth
    rb = synth.refine_segments(seed=args.seed, S=65536)
    f = lambda x: torch.as_tensor(np.asarray(x, dtype=np.float32)).to(dev).contiguous()
    Pt, Tt, At, bt = f(rb.P), f(rb.T), f(rb.A), f(rb.b)
    nr = torch.as_tensor(rb.nrows, dtype=torch.int32).to(dev)
    refiner = RF.Refiner(stream=stream)
    up = torch.ones(Pt.shape[0], device=dev)
    S = Pt.shape[0]
    res = {}

    def fb():
        res["loss"] = refiner.forward(Pt, Tt, At, bt, nr)
        res["dP"], res["dT"] = refiner.backward(Pt, Tt, At, bt, nr, up)
    refiner.planner.set_timing(True)
    ms, clocks, tm = clocked(fb, stream, args.steps, args.warmup, flush,
                             before=lambda: refiner.planner.timing(reset=True),
                             after=lambda: refiner.planner.timing(reset=True))
    refiner.check()
    # end to end: segments from pinned host memory, forward + backward, loss and gradients back
    hin = [(torch.from_numpy(np.ascontiguousarray(x, dtype=dt)).pin_memory(), d) for x, dt, d in
           ((rb.P, np.float32, Pt), (rb.T, np.float32, Tt), (rb.A, np.float32, At), (rb.b, np.float32, bt),
            (rb.nrows, np.int32, nr))]
    h_loss = torch.empty(S, dtype=torch.float32).pin_memory()
    h_dP = torch.empty(tuple(Pt.shape), dtype=torch.float32).pin_memory()
    h_dT = torch.empty(S, dtype=torch.float32).pin_memory()
    e2e = []
    for s in range(args.warmup + args.steps):
        flush.fill_(2.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h, d in hin:
            d.copy_(h, non_blocking=True)
        fb()
        h_loss.copy_(res["loss"], non_blocking=True)
        h_dP.copy_(res["dP"], non_blocking=True)
        h_dT.copy_(res["dT"], non_blocking=True)
        e1.record(stream)
        refiner.check()
        if s >= args.warmup:
            e2e.append(e0.elapsed_time(e1))
    bi = sum(h.numel() * h.element_size() for h, _ in hin)
    bo = (h_loss.numel() + h_dP.numel() + h_dT.numel()) * 4
    # roofline: HBM bytes of the two launches (each reads the segments; the
    # forward writes the loss, the backward reads the upstream gradient and
    # writes dP, dT)
    rmax = At.shape[1]
    seg_in = (Pt[0].numel() + 1 + rmax * 3 + rmax) * 4 + 4
    bytes_call = S * (2 * seg_in + 4 + 4 + (Pt[0].numel() + 1) * 4)
    step_ms = statistics.mean(ms)
    peaks, src = measured_peaks()
    ach = bytes_call / (step_ms / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import refine as OR
        n = 4096
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 8.0:
            OR.loss_and_grad(rb.P[:n], rb.T[:n], rb.A[:n], rb.b[:n], rb.nrows[:n], rb.bounds)
            reps += 1
        dt = time.perf_counter() - t0
        cpu = {"value": reps * n / dt, "unit": "segments/s", "cores": 1, "kind": "oracle",
               "sample": f"{reps} x {n} segments, {dt:.1f} s (FP64 numpy oracle, loss and gradient)"}
    return {"metric": "refinement segments/sec (forward + backward), 65536 degree-7 3-D segments",
            "value": S * 1e3 / step_ms, "unit": "segments/s", "dtype": "f32", "ms_per_step": step_ms,
            "gpu_launches": int(tm["launches"]), "clocks": clocks,
            "config": {"workload": "refine_segments: 65536 degree-7 3-D segments (end points on a random line, "
                                   "interior points N(0,1) about it, T ~ U[0.2, 2], one polytope of <= 12 rows each)",
                       "segments": S, "l2": "flushed before every timed step (256 MB write)"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": ach / float(peaks["hbm_gbs"]), "traffic": None,
                         "kernel": "k_refine<3,3,7> forward + backward", "kernel_ms": step_ms,
                         "bytes_per_step": bytes_call,
                         "work_model": "segments read by both launches, loss written, upstream gradient read, "
                                       "dP and dT written",
                         "peak_note": f"copy bandwidth ({src})"},
            "e2e": {"value": S * 1e3 / statistics.mean(e2e), "unit": "segments/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "ms_per_step": statistics.mean(e2e)},
            "cpu_baseline": cpu}


def cut_cpu_baseline(prob, obs, budget_s=12.0):
    """The exact keep-out cut oracle as it stands, on a bounded sample of rows."""
    import oracle
    from oracle import cut as OC
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    t0 = time.perf_counter()
    rows, step, units = [], max(1, prob.N // 400), 0
    order = np.arange(0, prob.N, step)
    done = 0
    while done < len(order) and time.perf_counter() - t0 < budget_s:
        r = order[done:done + 8]
        done += len(r)
        OC.cut(op, csr, obs.off, obs.A, obs.b, rows=r)
        rows.extend(r.tolist())
    dt = time.perf_counter() - t0
    e = csr["all"]
    sel = (e["mask"] != 0) & np.isin(e["i"], np.asarray(rows))
    units = int(sum(bin(int(x)).count("1") for x in e["mask"][sel]))
    tests = units * obs.n
    return {"value": tests / dt, "unit": "tests/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(rows)} of {prob.N} rows ({units} (edge, T) x {obs.n} obstacles, {dt:.1f} s, "
                      "numpy margins + exact rational games, one thread)"}


def run_cut_form(args, stream, flush, dev):
    """Keep-out cut (Sec. III-B, Algorithm 2): 2-D double integrator, 5000
    states, one duration, about 46,000 edges, 500 random convex obstacles."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import synth
    prob, obs = synth.keepout_2d(seed=1)
    pl = P.Planner.for_problem(prob, arith="f64", input="f64", stream=stream)
    dp = P.to_device(prob, input="f64")
    g = pl.build_edges(dp)
    E_in = g.E
    do = P.obstacles_to_device(obs, input="f64")
    out = pl.cut_edges(dp, g, do)       # sizes the game lists
    info = pl.info()
    sbuf = pl.alloc_search(dp.N)
    units, n_obst = int(info["cut_units"]), obs.n
    tests = units * n_obst
    pl.set_timing(True)
    pl.timing(reset=True)
    pl.cut_timing(reset=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.time()
        while clk.count() < 1 and time.time() - t0 < 10.0:
            pl.cut_edges_async(dp, g, do, out)
            torch.cuda.synchronize()
        mark = max(0, clk.count() - 1)
        pl.timing(reset=True)
        pl.cut_timing(reset=True)
        cms = timed(lambda: pl.cut_edges_async(dp, g, do, out), stream, args.steps, args.warmup, flush)
        ct = pl.cut_timing(reset=True)
        tm = pl.timing(reset=True)
        t0 = time.time()
        while clk.count() < mark + 2 and time.time() - t0 < 5.0:
            pl.cut_edges_async(dp, g, do, out)
            torch.cuda.synchronize()
    clocks = clk.summary(since=mark)
    assert pl.wait() == P.PLAN_OK
    sms = timed(lambda: pl.search_async(dp, out, dp.start_pos, dp.goal_pos, sbuf), stream, args.steps,
                args.warmup, flush)
    assert pl.wait() == P.PLAN_OK
    E_out = out.E
    # end to end per replanning tick: the obstacles from pinned host memory,
    # the cut, the search, the path and its cost back to the host
    h_off = torch.from_numpy(np.asarray(obs.off, dtype=np.int32)).pin_memory()
    h_A = torch.from_numpy(np.ascontiguousarray(obs.A, dtype=np.float64).reshape(-1)).pin_memory()
    h_b = torch.from_numpy(np.ascontiguousarray(obs.b, dtype=np.float64)).pin_memory()
    h_path = torch.empty(dp.N, dtype=torch.int32).pin_memory()
    h_cost = torch.empty(1, dtype=torch.float64).pin_memory()
    h_len = torch.empty(1, dtype=torch.int32).pin_memory()
    bi = sum(t.numel() * t.element_size() for t in (h_off, h_A, h_b))
    bo = h_path.numel() * 4 + 8 + 4
    e2e = []
    for s in range(args.warmup + args.steps):
        flush.fill_(3.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        do.off.copy_(h_off, non_blocking=True)
        do.A.copy_(h_A, non_blocking=True)
        do.b.copy_(h_b, non_blocking=True)
        pl.cut_edges_async(dp, g, do, out)
        pl.search_async(dp, out, dp.start_pos, dp.goal_pos, sbuf)
        h_path.copy_(sbuf["path"], non_blocking=True)
        h_cost.copy_(sbuf["cost"], non_blocking=True)
        h_len.copy_(sbuf["path_len"], non_blocking=True)
        e1.record(stream)
        st = pl.wait()
        assert st in (P.PLAN_OK, P.PLAN_ERR_NO_PATH)
        if s >= args.warmup:
            e2e.append(e0.elapsed_time(e1))
    # the oracle's bounded sample, after every GPU timing (its host threads
    # must not share the cores with the launches being timed)
    cpu = None if args.no_cpu_baseline else cut_cpu_baseline(prob, obs)
    cut_ms = statistics.mean(cms)
    scan_ms = ct["scan_ms"] / max(1, ct["cuts"])
    # roofline of the screening pass (the bounding-box test of every (edge, T)
    # against every obstacle): ALU-bound, 2m comparisons and 2m - 1 ORs plus
    # the mask bit per test, about 4m FP32 lane operations
    m, NP = prob.model.m, prob.model.degree + 1
    ex_ops = info["cut_tests"] * (4 * m)
    lanes = lane_peaks(dev)
    alu_peak = lanes["addmax"] / 1e12
    achieved = ex_ops / (scan_ms / 1e3) / 1e12
    dense_ops = tests * float(np.mean(np.diff(obs.off))) * NP * (m + 2)
    return {"metric": "keep-out cut decisions/sec ((edge, T) x obstacle), 2-D, 5000 states, 500 obstacles",
            "value": tests * 1e3 / cut_ms, "unit": "tests/s", "dtype": "f32+f64",
            "ms_per_step": cut_ms + statistics.mean(sms), "cut_ms_per_tick": cut_ms,
            "search_ms_per_query": statistics.mean(sms), "gpu_launches": int(tm["launches"]),
            "clocks": clocks,
            "config": {"workload": "keepout_2d seed 1: 2-D double integrator (|v|<=2, |a|<=4, p=5), N=5000 in "
                                   "[0,5]^2, T=0.5, 500 obstacles (boxes of side U[0.025, 0.1] cut by <= 3 planes)",
                       "edges_in": E_in, "edges_out": E_out, "units": units, "obstacles": n_obst, "tests": tests,
                       "box": info["cut_box"], "near": info["cut_near"], "step1": info["cut_step1"],
                       "step2": info["cut_step2"], "games": info["cut_games"], "lp64": info["cut_lp64"],
                       "ties": info["cut_ties"],
                       "l2": "flushed before every timed call (256 MB write)",
                       "paper_context": "cutHeuristic 72.0 ms on an RTX 4090 (Table 1; its graph size is not stated)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TOP/s",
                         "frac": achieved / alu_peak, "traffic": None, "kernel": "k_cut_scan<2,2,5>",
                         "kernel_ms": scan_ms, "ops_per_launch": ex_ops,
                         "work_model": "executed FP32 lane ops: (edge, T, obstacle) box tests x 4m",
                         "dense": {"ops_per_launch": dense_ops, "frac": dense_ops / (scan_ms / 1e3) / 1e12 / alu_peak,
                                   "note": "every control point against every facet of every obstacle, (m+2) ops each"},
                         "peak_note": lanes["note"]},
            "e2e": {"value": tests * 1e3 / statistics.mean(e2e), "unit": "tests/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "ms_per_step": statistics.mean(e2e)},
            "cpu_baseline": cpu}


def run_replan_form(args, stream, flush, dev):
    """The replanning loop (Algorithm 1's cutGraph and findPath every tick on
    the graph its buildGraph made once): 500 obstacles moving by a random walk and a moving start, each
    tick one replay of the captured graph (obstacles and start/goal copied in
    from pinned host memory, cut, search, path copied out), host-timed to the
    path in host memory."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import synth
    prob, obs = synth.keepout_2d(seed=1)
    pl = P.Planner.for_problem(prob, arith="f64", input="f64", stream=stream)
    dp = P.to_device(prob, input="f64")
    g = pl.build_edges(dp)
    rp = P.Replanner(pl, dp, g, n_max=512, rows_max=8)            # warm-started goal-rooted search
    rng = np.random.default_rng(7)
    ticks = args.warmup + args.steps
    A = np.asarray(obs.A).reshape(-1, 2)
    shift = np.zeros((obs.n, 2))
    sets = []
    for k in range(ticks):
        shift += rng.normal(0.0, 0.002, size=shift.shape)     # obstacles drift
        b = np.array(obs.b, dtype=np.float64)
        for o in range(obs.n):
            r0, r1 = obs.off[o], obs.off[o + 1]
            b[r0:r1] += A[r0:r1] @ shift[o]
        sets.append(synth.Obstacles(np.asarray(obs.off), A, b))
    rp.capture(sets[0], prob.start_pos, prob.goal_pos)
    # a goal the start reaches through the cut graph with a path of >= 8
    # vertices; the robot then advances along that first plan, one vertex
    # every few ticks, replanning every tick
    goal, plan0 = prob.goal_pos, None
    for v in rng.permutation(prob.N)[:200]:
        r = rp.tick(sets[0], prob.start_pos, prob.states[v, :2])
        if r["status"] == P.PLAN_OK and len(r["path"]) >= 8:
            goal, plan0 = prob.states[v, :2].copy(), r["path"]
            break
    if plan0 is None:
        plan0 = [int(np.argmin(np.sum((prob.states[:, :2] - prob.start_pos) ** 2, axis=1)))]
    starts = [prob.states[plan0[min(k * len(plan0) // (2 * ticks), len(plan0) - 1)], :2] for k in range(ticks)]
    def loop(rp):
        wall, dev_ms, edges, stats, sweeps, costs = [], [], [], [], [], []
        for k in range(ticks):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(float(k))
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            e0.record(stream)
            rp.tick_async(sets[k], starts[k], goal)
            e1.record(stream)
            r = rp.result()
            h1 = time.perf_counter()
            assert r["status"] in (P.PLAN_OK, P.PLAN_ERR_NO_PATH), r["status"]
            if k >= args.warmup:
                wall.append(1e3 * (h1 - h0))
                dev_ms.append(e0.elapsed_time(e1))
                edges.append(r["edges"])
                stats.append(r["status"])
                sweeps.append(r["info"]["search_iters"])
                costs.append(r["cost"])
        return wall, dev_ms, edges, stats, sweeps, costs

    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.time()
        while clk.count() < 1 and time.time() - t0 < 10.0:
            rp.tick(sets[0], starts[0], goal)
        mark = max(0, clk.count() - 1)
        wall, dev_ms, edges, stats, sweeps, costs = loop(rp)
        t0 = time.time()
        while clk.count() < mark + 2 and time.time() - t0 < 5.0:
            rp.tick(sets[0], starts[0], goal)
    clocks = clk.summary(since=mark)
    # the same ticks searched cold (plan_search_at from the start), for comparison
    rc = P.Replanner(pl, dp, g, n_max=512, rows_max=8, warm=False)
    rc.capture(sets[0], starts[0], goal)
    cwall, cdev, _, cstats, _, ccosts = loop(rc)
    assert cstats == stats
    cost_dev = max((abs(a - b) / max(1.0, abs(b)) for a, b, st in zip(costs, ccosts, stats) if st == P.PLAN_OK),
                   default=0.0)
    bi = sum(t.numel() * t.element_size() for t in (rp.h_off, rp.h_A, rp.h_b, rp.h_ends))
    bo = rp.h_path.numel() * 4 + 4 + 8
    wmed, dmed = statistics.median(wall), statistics.median(dev_ms)
    return {"metric": "replanning ticks/sec (500 moving obstacles in, keep-out cut + search of a 5000-state graph, "
                      "path out)", "value": 1e3 / statistics.mean(wall), "unit": "ticks/s", "higher_is_better": True,
            "dtype": "f32+f64", "ms_per_step": statistics.mean(wall), "tick_ms_median": wmed,
            "tick_ms_max": max(wall), "device_ms_median": dmed, "gpu_launches_per_tick": 8 + 4,
            "search_sweeps_mean": statistics.mean(sweeps),
            "cold_search": {"tick_ms_median": statistics.median(cwall), "device_ms_median": statistics.median(cdev),
                            "max_rel_cost_diff": cost_dev},
            "clocks": clocks,
            "config": {"workload": "keepout_2d seed 1 (N=5000, 45,567 edges, 500 obstacles drifting by a random "
                                   "walk of 0.002 per tick; the start advances along the first plan)",
                       "first_plan_vertices": len(plan0),
                       "captured": "one CUDA graph per tick: 4 host-to-device copies, the cut (7 kernels), the "
                                   "goal-rooted search warm-started from the previous tick (1 launch, one 16-CTA cluster "
                                   "kernel), 3 device-to-host copies",
                       "edges_per_tick": [min(edges), max(edges)], "no_path_ticks": int(sum(s != 0 for s in stats)),
                       "l2": "flushed before every tick (256 MB write)",
                       "paper_context": "graph replanning at 10 Hz with 500 obstacles; cut 10-50 Hz"},
            "e2e": {"value": 1e3 / statistics.mean(wall), "unit": "ticks/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "ms_per_step": statistics.mean(wall)},
            "cpu_baseline": None}


def run_planes_form(args, stream, flush, dev):
    """closestPoint / adjacentHyperplane (Algorithm 2, Sec. III-D) for every
    (node, obstacle) pair: the 5000 states of the keep-out workload against
    its 500 obstacles, FP32, all-pairs outputs plus the nearest obstacle."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import synth
    prob, obs = synth.keepout_2d(seed=1, dtype="f32")
    pl = P.Planner(2, 2, 5, (2.0, 4.0), arith="f32", input="f32", stream=stream)
    pts = torch.as_tensor(np.ascontiguousarray(prob.states[:, :2], dtype=np.float32)).to(dev)
    do = P.obstacles_to_device(obs, input="f32")
    out = pl.obstacle_planes(pts, do)           # sizes scratch, allocates outputs
    Pn, n = pts.shape[0], obs.n
    pairs = Pn * n
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.time()
        while clk.count() < 1 and time.time() - t0 < 10.0:
            pl.obstacle_planes_async(pts, do, out)
            torch.cuda.synchronize()
        mark = max(0, clk.count() - 1)
        ms = timed(lambda: pl.obstacle_planes_async(pts, do, out), stream, args.steps, args.warmup, flush)
        t0 = time.time()
        while clk.count() < mark + 2 and time.time() - t0 < 5.0:
            pl.obstacle_planes_async(pts, do, out)
            torch.cuda.synchronize()
    clocks = clk.summary(since=mark)
    assert pl.wait() == P.PLAN_OK
    # bytes the call must move: the outputs (closest m, plane m + 1, distance
    # per pair; nearest index and distance per point) and the inputs
    out_bytes = pairs * 4 * (2 + 3 + 1) + Pn * 8
    in_bytes = Pn * 8 + int(np.asarray(obs.b).shape[0]) * 16 + (n + 1) * 4
    mean_ms = statistics.mean(ms)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (out_bytes + in_bytes) / (mean_ms / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import planes as OP
        t0 = time.perf_counter()
        k = 0
        A = np.asarray(obs.A, dtype=np.float32).astype(np.float64)
        bb = np.asarray(obs.b, dtype=np.float32).astype(np.float64)
        P32 = np.asarray(prob.states[:, :2], dtype=np.float32).astype(np.float64)
        while time.perf_counter() - t0 < 10.0 and k < Pn:
            OP.planes(P32[k:k + 1], obs.off, A, bb)
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": k * n / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} of {Pn} nodes x {n} obstacles ({dt:.1f} s, numpy FP64 active-set enumeration)"}
    return {"metric": "closest points + separating planes per second ((node, obstacle) pairs), 5000 nodes x 500 "
                      "obstacles", "value": pairs * 1e3 / mean_ms, "unit": "pairs/s", "dtype": "f32",
            "ms_per_step": mean_ms, "gpu_launches": 4, "clocks": clocks,
            "config": {"workload": "keepout_2d seed 1 states (5000) against its 500 obstacles (4-7 rows)",
                       "pairs": pairs,
                       "l2": "flushed before every timed call (256 MB write)",
                       "paper_context": "adjacentHyperplane 0.61 ms on an RTX 4090 (Table 1; counts not stated)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "kernel": "k_planes<2> (whole call)",
                         "bytes_per_launch": out_bytes + in_bytes,
                         "peak_note": f"copy bandwidth ({peak_src})",
                         "note": "algorithmic bytes: 24 B of outputs per pair + 8 B per node + the inputs"},
            "e2e": None, "cpu_baseline": cpu}


def run_mpc_form(args, stream, flush, dev):
    """The MPC refinement of Sec. III-D (Eq. (MPC), solved SQP-style): a batch
    of problems in the keep-out scene (2-D double integrator, degree 5, H = 10
    segments of dt = 0.1, the free box [0, 5]^2 as keep-in polytope, its 500
    obstacles); one step = three rounds of (plane of the nearest obstacle at
    every current node, then the QP of every problem)."""
    import torch
    from paper_2411_13507_gb300 import plan as P
    from paper_2411_13507_gb300 import synth
    B, H, dt, rounds, width = int(args.mpc_batch), 10, 0.1, 3, 5.0
    prob, obs = synth.keepout_2d(seed=1)
    pl = P.Planner(2, 2, 5, (2.0, 4.0), arith="f64", input="f64", stream=stream)
    do = P.obstacles_to_device(obs, input="f64")
    # references whose every node keeps 0.05 from every obstacle (filtered
    # once on the GPU with the nearest distances; untimed)
    kept = []
    for rep in range(8):       # candidate pools until B references keep their clearance
        cand = synth.mpc_references(args.seed + 1000 * rep, 8 * B, H, dt, width)
        pts = torch.tensor(np.ascontiguousarray(cand[:, :, :2].reshape(-1, 2)), dtype=torch.float64, device=dev)
        tmp = torch.empty((pts.shape[0], 3), dtype=torch.float32, device=dev)
        nd = torch.empty(pts.shape[0], dtype=torch.float32, device=dev)
        pl.nearest_planes_async(pts, do, tmp, None, nd)
        assert pl.wait() == P.PLAN_OK
        keep = (nd.view(8 * B, H + 1).min(dim=1).values >= 0.05).cpu().numpy()
        kept.append(cand[keep])
        if sum(k.shape[0] for k in kept) >= B:
            break
    ref_np = np.concatenate(kept)[:B]
    assert ref_np.shape[0] == B, "too few references with clearance"
    Q, F, R, V = [1.0, 1.0, 0.1, 0.1], [0.5, 0.5, 0.05, 0.05], [0.05, 0.05], [2.0, 2.0, 2.0, 2.0]
    KA = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]])
    Kb = np.array([width, 0.0, width, 0.0])
    prm = pl.mpc_params(H, dt, Q, F, R, V, KA, Kb)
    ref = torch.tensor(ref_np, dtype=torch.float64, device=dev)
    x0 = ref[:, 0].contiguous()
    out = pl.alloc_mpc(B, H)
    planes = torch.empty((B, H, 3), dtype=torch.float32, device=dev)
    step = lambda: pl.mpc_refine_async(prm, x0, ref, do, out, sqp_iters=rounds, planes=planes)
    step()
    assert pl.wait() == P.PLAN_OK
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.time()
        while clk.count() < 1 and time.time() - t0 < 10.0:
            step()
            torch.cuda.synchronize()
        mark = max(0, clk.count() - 1)
        ms = timed(step, stream, args.steps, args.warmup, flush)
        qms = timed(lambda: pl.mpc_qp_async(prm, x0, ref, planes, out), stream, args.steps, args.warmup, flush)
        t0 = time.time()
        while clk.count() < mark + 2 and time.time() - t0 < 5.0:
            step()
            torch.cuda.synchronize()
    clocks = clk.summary(since=mark)
    assert pl.wait() == P.PLAN_OK
    st = out["status"].cpu().numpy()
    iters = out["iters"].cpu().numpy()
    # end to end: references and states in from pinned host memory, the
    # refinement, nodes and inputs back to pinned host memory
    h_ref = torch.from_numpy(ref_np.copy()).pin_memory()
    h_x0 = torch.from_numpy(np.ascontiguousarray(ref_np[:, 0])).pin_memory()
    h_x = torch.empty(out["x"].shape, dtype=torch.float64).pin_memory()
    h_u = torch.empty(out["u"].shape, dtype=torch.float64).pin_memory()

    def e2e_step():
        ref.copy_(h_ref, non_blocking=True)
        x0.copy_(h_x0, non_blocking=True)
        step()
        h_x.copy_(out["x"], non_blocking=True)
        h_u.copy_(out["u"], non_blocking=True)
    ems = timed(e2e_step, stream, args.steps, args.warmup, flush)
    bi = h_ref.numel() * 8 + h_x0.numel() * 8
    bo = h_x.numel() * 8 + h_u.numel() * 8
    # FP64 work of the QP kernel (a model from the step counts; the rows are
    # screened in float and do not count): per problem the gradient
    # (8 g (H+1) flops per input) and the unconstrained start (4 nv^2); per
    # active-set step d = J'n (2 nv^2), z (about nv^2), the Householder update
    # (about 2 nv^2), the back substitution and the node states
    # (2 (H+1) n H / 2)
    m_, g_, p_ = 2, 2, 5
    n_ = m_ * g_
    rax = sum(p_ - k + 1 for k in range(1, g_ + 1))
    rows = H * m_ * rax * 2 + H * (p_ + 1) + H * p_ * 4
    nv = m_ * H
    flops = B * (8.0 * g_ * (H + 1) * nv + 4.0 * nv * nv) + float(iters.sum()) * (5.0 * nv * nv + (H + 1) * n_ * H)
    qmean = statistics.mean(qms)
    lanes = lane_peaks(dev, fp64=True)
    fp64_peak = 2.0 * lanes["fma64"] / 1e9   # GFLOP/s: measured FP64 FMA chains, two flops each
    achieved = flops / (qmean / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import mpc as OM
        from oracle import planes as OP
        t0 = time.perf_counter()
        k = 0
        A = np.asarray(obs.A, dtype=np.float64)
        bb = np.asarray(obs.b, dtype=np.float64)
        while time.perf_counter() - t0 < 10.0 and k < B:
            cur = ref_np[k]
            for _ in range(rounds):
                pr = OP.planes(cur[:H, :2], obs.off, A, bb)
                pk = np.stack([pr["plane"][i, pr["nearest"][i]] for i in range(H)])
                r = OM.mpc_qp(2, 2, 5, (2.0, 4.0), dt, ref_np[k, 0], ref_np[k], pk, Q, F, R, V, KA, Kb)
                if r["status"] != OM.OK:
                    break
                cur = r["x"]
            k += 1
        dts = time.perf_counter() - t0
        cpu = {"value": k / dts, "unit": "problems/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} of {B} problems x {rounds} SQP rounds ({dts:.1f} s, numpy FP64: all-pairs planes + "
                         "primal active set)"}
    mean_ms = statistics.mean(ms)
    return {"metric": f"MPC refinements per second ({rounds} SQP rounds of nearest planes + QP), batch of {B} "
                      "problems, keep-out scene", "value": B * 1e3 / mean_ms, "unit": "problems/s", "dtype": "f64",
            "ms_per_step": mean_ms, "qp_ms_per_launch": qmean, "gpu_launches": 7 * rounds, "clocks": clocks,
            "status_counts": {"ok": int((st == 0).sum()), "infeasible": int((st == 1).sum()),
                              "iteration_limit": int((st == 2).sum())},
            "active_set_steps_mean": float(iters.mean()),
            "config": {"workload": f"mpc_references seed {args.seed} (B={B}, H={H}, dt={dt}, nodes 0.05 clear of "
                                   "every obstacle) in keepout_2d seed 1 (500 obstacles, box [0,5]^2 as keep-in)",
                       "rows_per_problem": rows, "inputs_per_problem": nv,
                       "l2": "flushed before every timed step (256 MB write)",
                       "paper_context": "MPC at 200 Hz (one problem, OSQP on a CPU)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s",
                         "frac": achieved / fp64_peak, "traffic": None, "kernel": "k_mpc (one QP launch)",
                         "peak_note": lanes["note64"] + " (x2 flops per FMA); nominal FP64 of the part 1250 GFLOP/s",
                         "note": "FP64 flops modelled from the active-set step counts; comparisons, divisions and "
                                 "square roots also occupy the FP64 pipe, which ncu measures 55% busy while active "
                                 "(profiles/k_mpc_keepout_2d.md)"},
            "e2e": {"value": B * 1e3 / statistics.mean(ems), "unit": "problems/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "ms_per_step": statistics.mean(ems)},
            "cpu_baseline": cpu}


_RESULT = None


def claim_stdout():
    """Keep the process's standard output for the one result line: from here on
    anything else written to fd 1 (NCCL's version banner, library messages)
    goes to stderr, and emit() writes to a duplicate of the original fd 1."""
    global _RESULT
    sys.stdout.flush()
    _RESULT = os.fdopen(os.dup(1), "w")
    os.dup2(2, 1)


def emit(line):
    out = _RESULT or sys.stdout
    out.write(json.dumps(line) + "\n")
    out.flush()


def main():
    args = parse()
    claim_stdout()
    if args.impl == "reference":
        return run_reference(args)
    if args.form != "plain":
        line = run_form(args)
        emit(line)
        return 0
    import torch
    from paper_2411_13507_gb300 import plan as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    shard_rows = args.shard == "rows"
    if world > 1 or shard_rows:
        # --shard rows on one GPU still runs the whole sharded path: one shard,
        # the NCCL exchange with a world of one, the search on the merged graph
        import torch.distributed as dist
        torch.cuda.set_device(local)
        if world == 1:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", str(29500 + (os.getpid() % 1000)))
            dist.init_process_group("nccl", rank=0, world_size=1)
        else:
            dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    assert args.warmup >= 3, "at least 3 warm-up steps"

    # CPU baseline first (before heavy GPU work; threads, no fork)
    prob = workload(args.seed if shard_rows else args.seed + rank)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, rows=args.cpu_sample_rows)

    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        pl = P.Planner.for_problem(prob, arith="f32", input="f32", stream=stream)
        if args.pipeline >= 0:
            pl.set_tile(0, 0, 0, args.pipeline)
        dp = P.to_device(prob, input="f32")
        from paper_2411_13507_gb300 import shard
        if shard_rows:
            graph = pl.build_edges_shard(dp, rank, world)   # sizes scratch and this rank's output CSR
        else:
            graph = pl.build_edges(dp)                      # sizes scratch and the output CSR
        info = pl.info()

        def exchanged():
            """The whole graph from every rank's rows (all-gather-v over NCCL)."""
            st = pl.wait()
            assert st == P.PLAN_OK, f"shard build status {st}"
            i = pl.last_info
            g = shard.exchange(graph.row_off, graph.col, graph.w, graph.mask, graph.tidx, int(graph.count.item()),
                               int(i.shard_lo), int(i.shard_hi), dp.N, dist)
            E = g["count"]
            return P.Graph(dp.N, g["row_off"], g["col"], g["w"], g["tidx"], g["mask"],
                           torch.tensor([E], dtype=torch.int64, device=dev), max(E, 1))

        sgraph = exchanged() if shard_rows else graph
        sres = pl.search(dp, sgraph)
        cap = graph.cap
        # algorithmic work of this query (untimed counting launch)
        pl.set_accounting(True)
        if shard_rows:
            pl.build_edges_shard(dp, rank, world, graph=graph)
        else:
            pl.build_edges(dp, graph=graph)
        work = pl.info()
        pl.set_accounting(False)
        sbuf = pl.alloc_search(dp.N)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        replay, replay_launches = None, 0
        if not shard_rows:
            # the timed build: the query prepared as a batch of one (the same
            # kernels as plan_build_edges, the host work done once) and its
            # launches replayed as one captured CUDA graph
            pl.build_batched([dp], [graph])
            pl.timing(reset=True)
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg, stream=stream):
                pl.build_batched_async()
            replay_launches = int(pl.timing(reset=True)["launches"])
            replay = cg.replay

        def step(evs):
            """build (+ exchange of the row shards) | search; returns the graph searched"""
            evs[0].record(stream)
            if shard_rows:
                pl.build_edges_shard_async(dp, graph, rank, world)
                g = exchanged()
            else:
                replay()
                g = graph
            evs[1].record(stream)
            pl.search_async(dp, g, dp.start_pos, dp.goal_pos, sbuf)
            evs[2].record(stream)
            return g

        for _ in range(args.warmup):
            flush.fill_(1.0)
            step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
            st = pl.wait()
            assert st == P.PLAN_OK, f"warm-up status {st}"
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

        def untimed_until(cond, limit_s):
            t0 = time.time()
            while not cond() and time.time() - t0 < limit_s:
                flush.fill_(1.0)
                step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
                assert pl.wait() == P.PLAN_OK

        with ClockSampler(torch.cuda.current_device()) as clk:
            # the sampler comes up while the same steps run untimed; its samples
            # from the last one before the timed steps to the first one after
            # their start (the steps keep running untimed until it arrives)
            # describe the clocks of the timed region
            untimed_until(lambda: clk.count() >= 1, 10.0)
            mark = max(0, clk.count() - 1)
            pl.set_timing(True)
            pl.timing(reset=True)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            for s in range(args.steps):
                flush.fill_(float(s))
                step(evs[s])
                st = pl.wait()
                assert st == P.PLAN_OK, f"step {s}: status {st}"
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            tm = pl.timing(reset=True)
            pl.set_timing(False)
            untimed_until(lambda: clk.count() >= mark + 2, 5.0)
        clocks = clk.summary(since=mark)
        launches_timed = int(tm["launches"]) + args.steps * replay_launches
        build_launched_ms = None
        if not shard_rows:
            # the pair kernel's own time (events around its launch) and the
            # build's time without the graph: the same launches issued one by one
            pl.set_timing(True)
            pl.timing(reset=True)
            bl = []
            for s in range(max(3, args.steps)):
                flush.fill_(3.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.build_batched_async()
                e1.record(stream)
                assert pl.wait() == P.PLAN_OK
                bl.append(e0.elapsed_time(e1))
            tk = pl.timing(reset=True)
            pl.set_timing(False)
            tm = dict(tm, pair_ms=tk["pair_ms"], pair_launches=tk["pair_launches"])
            build_launched_ms = statistics.mean(bl)
        lanes = lane_peaks(dev)
        build_ms = [a.elapsed_time(b) for a, b, _ in evs]
        search_ms = [b.elapsed_time(c) for _, b, c in evs]
        step_ms = [a.elapsed_time(c) for a, _, c in evs]

        # end to end: host (pinned) inputs -> C ABI -> host result, every step
        h_states = torch.from_numpy(np.ascontiguousarray(prob.states, dtype=np.float32)).pin_memory()
        h_off = torch.from_numpy(np.asarray(prob.poly_off, dtype=np.int32)).pin_memory()
        h_A = torch.from_numpy(np.ascontiguousarray(prob.A, dtype=np.float32)).pin_memory()
        h_b = torch.from_numpy(np.ascontiguousarray(prob.b, dtype=np.float32)).pin_memory()
        h_path = torch.empty(dp.N, dtype=torch.int32).pin_memory()
        h_cost = torch.empty(2, dtype=torch.float64).pin_memory()
        h_E = torch.empty(1, dtype=torch.int64).pin_memory()
        bi = sum(t.numel() * t.element_size() for t in (h_states, h_off, h_A, h_b))
        e2e_ms = []
        for s in range(args.warmup + args.steps):
            flush.fill_(2.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dp.states.copy_(h_states, non_blocking=True)
            dp.poly_off.copy_(h_off, non_blocking=True)
            dp.A.copy_(h_A, non_blocking=True)
            dp.b.copy_(h_b, non_blocking=True)
            if shard_rows:
                pl.build_edges_shard_async(dp, graph, rank, world)
                g = exchanged()
            else:
                replay()
                g = graph
            pl.search_async(dp, g, dp.start_pos, dp.goal_pos, sbuf)
            h_path.copy_(sbuf["path"], non_blocking=True)
            h_cost[:1].copy_(sbuf["cost"], non_blocking=True)
            h_E.copy_(g.count, non_blocking=True)
            e1.record(stream)
            st = pl.wait()
            assert st == P.PLAN_OK
            if s >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
        L = int(sbuf["path_len"].item())
        bo = h_path.element_size() * dp.N + 8 + 8

    checks = int(info["checks"])
    t_build = sum(build_ms) / 1e3
    t_step = sum(step_ms) / 1e3
    t_search = sum(search_ms) / 1e3
    t_e2e = sum(e2e_ms) / 1e3
    from paper_2411_13507_gb300 import shard
    (t_build, t_step, t_search, t_e2e), checks_all = shard.aggregate(
        [t_build, t_step, t_search, t_e2e], float(checks), dist, device=dev)
    value = checks_all * args.steps / t_build
    e2e_value = checks_all * args.steps / t_e2e

    # roofline of the dominant kernel (the pair kernel): ALU-bound.  Algorithmic
    # work per check = the dense separable form: every reach row (add, |.|,
    # compare, min), every free row (add, max), every cost segment (n adds, n
    # FMAs, sqrt, add); times the checks of one launch.
    g, p, m = prob.model.gamma, prob.model.degree, prob.model.m
    n = m * g
    rax = sum(p - k + 1 for k in range(1, g + 1))
    rows_mean = float(np.mean(np.diff(prob.poly_off)))
    ops_per_check = 4 * m * rax + 2 * (p - 1) * rows_mean + p * (2 * n + 2)
    ops_per_launch = ops_per_check * checks
    sc_ops = (2 * work["work_reach_rows"] + 2 * work["work_free_rows"] + work["work_costs"] * p * (2 * n + 2))
    # the dense model restricted to what the screened kernel evaluates: the
    # screen rows (3 reach rows per axis) of every ordered pair in every
    # polytope and duration, every reach and free row of the pairs it passes
    # on, one cost per feasible check (each counted as in the dense model)
    screened = int(info.get("screened", 0))
    ex_ops = (2 * 3 * m * (int(info["slots"]) - int(info["memberships"])) * prob.nT
              + 2 * (m * rax + (p - 1) * rows_mean) * screened + p * (2 * n + 2) * int(info["feasible"]))
    pair_ms = tm["pair_ms"] / max(1, tm["pair_launches"])
    achieved = ops_per_launch / (pair_ms / 1e3) / 1e12
    alu_peak = lanes["addmax"] / 1e12       # measured on this device (add + |.|-max chains)
    ex_frac = ex_ops / (pair_ms / 1e3) / 1e12 / alu_peak
    counters, src_sha = pair_kernel_counters()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True,
        "scaling": "strong" if shard_rows else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config(prob, {"checks_per_query": int(checks_all) if shard_rows else checks,
                                "candidates": int(info["candidates"]),
                                "edges": int(info["edges"]), "rechecks": int(info["rechecks"]),
                                **({"parallelism": f"one query, source rows split over {world} GPUs "
                                                   "(plan_build_edges_shard), CSR pieces all-gathered over NCCL, "
                                                   "search replicated; build_ms includes the exchange"}
                                   if shard_rows else
                                   {"build": "the query prepared once as a batch of one (plan_prepare_batched), "
                                             "its build launches replayed as one captured CUDA graph per step"})}),
        "build_ms_per_query": 1e3 * t_build / args.steps,
        "build_ms_launched": build_launched_ms,
        "search_ms_per_query": 1e3 * t_search / args.steps,
        "path_len": L,
        "gpu_launches": launches_timed,
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TOP/s",
                     "frac": achieved / alu_peak, "hw_frac": ex_frac,
                     "traffic": counters.get("dram_bytes_per_launch") if counters else None,
                     "kernel": PAIR_KERNEL.get(args.pipeline, PAIR_KERNEL[0]), "kernel_ms": pair_ms,
                     "ops_per_check": ops_per_check, "ops_per_launch": ops_per_launch,
                     "work_model": "dense separable form per check (all reach, free and cost rows)",
                     "peak_note": lanes["note"],
                     "hw_frac_note": "the dense model's ops over what the pair kernel evaluates / measured peak "
                                     "(closer to hardware utilisation); frac uses the whole dense separable work model",
                     "executed": {"ops_per_launch": ex_ops, "frac": ex_frac,
                                  "screened_checks": screened,
                                  "note": "the dense model's ops restricted to what the screened kernel evaluates: "
                                          "screen rows of every pair and duration, all reach and free rows of the "
                                          "screened checks, costs of feasible ones"},
                     "short_circuit": {"ops_per_launch": sc_ops, "frac": sc_ops / (pair_ms / 1e3) / 1e12 / alu_peak,
                                       "note": "work left after the early exits (reach rows up to the first violated "
                                               "one, free rows of reach-passing checks, costs of feasible ones)",
                                       **{k: work[k] for k in ("work_reach_rows", "work_free_rows", "work_costs")}}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "ms_per_step": 1e3 * t_e2e / args.steps},
        "cpu_baseline": ({k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")} if cpu else None),
    }
    if rank == 0:
        emit(line)
    if dist:
        dist.destroy_process_group()
    pl.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
