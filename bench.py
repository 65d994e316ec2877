#!/usr/bin/env python3
"""Benchmark of the tensor-product direct solve of -Delta + V1 on one B300 per rank.

Workload (the 3D single large apply): n = 512 per axis (1.34e8 DoF) on [-8,8]^3,
homogeneous Dirichlet, V1 = sum (omega_k x_k)^2 with omega = (1, 1.3, 0.7), shift
sigma = 0.5, right-hand side iid N(0,1) (SplitMix64, seed 2).

One step = one solve of (-Delta_h + V1 + sigma) u = b to relative error <= 1e-10:
mixed-precision iterative refinement (ts_solve_schedule) with split-precision tensor-core
inverses as the preconditioner and FP64 residuals -- u_0 = P b, then refinements
u += P (b - A u).  `value` is GDoF/s = N / step time (summed over ranks).  The same JSON
line carries the plain FP64 apply and a single unrefined BF16X3 apply, each with its error
against the FP64 apply, the roofline of every kernel of the step, the end-to-end rate with
host buffers, and, timed on their own after the main region: the 6D / 9D complex64
Strang steps, the 3D n = 256 shifted inverse iteration, the serving workload (2048
requests per phase, BF16X3 and FP64) with its batched kernel, and the CPU oracle on the
n = 512 workload itself.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain C, FP64, all host cores) on bounded samples
of the same n = 512 workload; multi-GPU launches run one independent replica per rank.
"""
from __future__ import annotations

import argparse
import datetime
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

from paper_2605_20491_b300 import synth  # noqa: E402

WORKLOAD = "3d_n512_apply"
METRIC = "GDoF/s of (-Delta+V1)^-1 apply, FP64 vs mixed at stated err; p50/p99 latency"
UNIT = "GDoF/s"
# Precision of each apply of the refined solve (u_0 = P_0 b, then one refinement per further
# entry).  The error contracts by each apply's relative error; measured at n = 512:
# BF16X3 1.6e-5 per apply, BF16X1 5.6e-3; {3, 3} ends at 7.8e-10 (above the target),
# {3, 3, 3} at 2.2e-14 in 8.79 ms, {3, 3, 1} at 5.2e-12 in 7.91 ms: the last refinement only
# needs a coarse inverse.
SCHEDULE = ("TS_BF16X3", "TS_BF16X3", "TS_BF16X1")
# PCG (V2 = 0) tolerance for the alternative CG-accelerated solve reported beside it.
PCG_TOL = 1e-12
ERR_TARGET = 1e-10
# Fiber fraction of one reference-arm step (a sample of one of the apply's transforms).
REF_FRACTION = 8


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.window = None  # (t0, t1) host wall-clock seconds of the timed region

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), [nm for nm, v in zip(names, f[6:10]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if self.window and self.window[0] <= r[0] <= self.window[1]]
        use = inside or rows  # a region shorter than the sampling period keeps the nearby samples
        sm = [r[1] for r in use]
        mx = [r[2] for r in use]
        reasons = sorted({nm for r in use for nm in r[3]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}


def max_over_ranks(ms, dist=None, device=None):
    """The slowest rank's time (all-reduce MAX over the process group; `dist` None: this
    process alone).  Every rank gets the same value."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(world, dof_per_rank, ms):
    """GDoF/s of `world` independent replicas of dof_per_rank each, timed by the slowest."""
    return world * dof_per_rank / (ms * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# The six transforms of one apply, in the oracle's order: forward along axes 0, 1, 2, then
# backward along axes 0, 1, 2 (the pointwise scale between them is N divisions).
ORACLE_PASSES = [(k, False) for k in range(3)] + [(k, True) for k in range(3)]


def oracle_full_size_plan(n_axis=None):
    """The oracle's plan and right-hand side of the benchmark workload itself (n = 512; a
    smaller n per axis on the same box and potential only when asked for)."""
    import oracle as O
    w = synth.WORKLOADS[WORKLOAD]
    n = (n_axis,) * 3 if n_axis else w["n"]
    P = O.plan(n, w["L"], synth.harmonic(n, w["L"], w["omega"]))
    return O, w, P, synth.normal(w["seed"], P.N)


def time_fiber_sample(O, P, X, Y, k, backward, fraction):
    """Seconds of one oracle transform along axis k restricted to the first 1/fraction of
    its fibers (the same loops as the whole transform)."""
    fibers = P.N // P.n[k]
    t0 = time.perf_counter()
    O.mode_fibers(P, k, X, Y, backward, 0, max(1, fibers // fraction))
    return time.perf_counter() - t0


def cpu_oracle_baseline():
    """The CPU oracle (plain C loops, FP64, OpenMP over fibers, all host cores) timed on the
    benchmark's own workload: one whole inverse apply at n = 512 (six transforms and the
    scale), and, on one core, a 1/64 fiber sample of each of its six transforms."""
    O, w, P, b = oracle_full_size_plan()
    t0 = time.perf_counter()
    u = O.apply_inverse(P, w["sigma"], b)
    full_s = time.perf_counter() - t0
    cores = O.num_threads()
    del u
    frac = 64
    Y = np.empty_like(b)
    O.set_num_threads(1)
    try:
        one = sum(time_fiber_sample(O, P, b, Y, k, bw, frac) for k, bw in ORACLE_PASSES) * frac
    finally:
        O.set_num_threads(cores)
    return {"value": P.N / full_s / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"one whole oracle inverse apply of the benchmark workload (3D n=512, {P.N} DoF, "
                      f"FP64 plain C loops, OpenMP over fibers): {full_s:.1f} s",
            "one_core": {"value": P.N / one / 1e9, "unit": UNIT,
                         "sample": f"the same oracle on 1 thread: the first 1/{frac} of the fibers of each of "
                                   f"the apply's six transforms at n=512, scaled by {frac} ({one:.0f} s "
                                   f"for the six transforms)"}}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    """The reference arm: the CPU oracle on the benchmark's own workload (n = 512).  A whole
    apply takes minutes on the host, so each step is a bounded sample of it: step i runs
    transform i mod 6 of the apply on the first 1/REF_FRACTION of its fibers.  The rate is
    N over the apply time estimated from the per-transform means, scaled by REF_FRACTION
    (the scale between the transforms, N divisions, is left out)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    O, w, P, b = oracle_full_size_plan(args.reference_n)
    Y = np.empty_like(b)
    for i in range(max(args.warmup, 6)):  # every transform at least once before timing
        k, bw = ORACLE_PASSES[i % 6]
        time_fiber_sample(O, P, b, Y, k, bw, REF_FRACTION)
    per = {i: [] for i in range(6)}
    t0 = time.perf_counter()
    for i in range(args.steps):
        k, bw = ORACLE_PASSES[i % 6]
        per[i % 6].append(time_fiber_sample(O, P, b, Y, k, bw, REF_FRACTION))
    el = time.perf_counter() - t0
    for i in range(6):  # fewer than six steps: the missing transforms are timed once more
        if not per[i]:
            k, bw = ORACLE_PASSES[i]
            per[i].append(time_fiber_sample(O, P, b, Y, k, bw, REF_FRACTION))
    apply_s = sum(statistics.mean(v) for v in per.values()) * REF_FRACTION
    value = P.N / apply_s / 1e9
    ms = el / args.steps * 1e3
    sample = (f"each step: one of the six transforms of the n={P.n[0]} oracle apply ({P.N} DoF) on the first "
              f"1/{REF_FRACTION} of its fibers, cycling through the six; the apply time is the sum of the "
              f"per-transform means x {REF_FRACTION} = {apply_s:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": list(P.n), "L": list(w["L"]), "omega": list(w["omega"]),
                       "sigma": w["sigma"], "rhs": "iid N(0,1), SplitMix64 seed 2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """Small fixed case for profiler captures (a few GB on the device): the refined solve
    of the n = 512 workload only (with --profile-n m: on an m^3 grid of the same box and
    potential), or, with --workload 6d_n24_strang / 9d_n8_strang, the complex64 FP32 Strang
    steps only, or, with --workload 3d_n256_pcg, one BF16X3-preconditioned shifted inverse
    iteration; warmup + steps times (not the inverse iteration), nothing else.  With
    --profile-bf16x6 the Strang steps run in TS_BF16X6 (the tensor-core small-n pass)."""
    import torch
    from paper_2605_20491_b300 import tschrod as T
    if args.workload == "3d_n256_pcg":
        # the BF16X3-preconditioned shifted inverse iteration only
        w = synth.WORKLOADS[args.workload]
        n, L = w["n"], w["L"]
        P = T.ts_plan_create(n, L, synth.harmonic(n, L, w["omega"]), 1 << T.TS_BF16X3)
        V2h = synth.v2_cos_bumps(n, L, seed=w["v2_seed"])
        V2 = torch.from_numpy(V2h).cuda()
        shift = sum(T.ts_plan_eigs(P, k)[0] for k in range(3)) + V2h.min() - 1.0
        u = torch.zeros(P.N, dtype=torch.float64, device="cuda")
        T.ts_inverse_iteration(P, shift, V2, u, True, w["lambda_tol"], 400, w["pcg_tol"], 500, T.TS_BF16X3)
        torch.cuda.synchronize()
        print("profile case done", flush=True)
        return 0
    if args.workload == "3d_q2_n1099_table1":
        # the Q^k banded operator (k_banded) alone: Q^20 on 299^3 (213 MB per vector)
        n, k = args.profile_n or 299, 20
        x, _ = T.ts_grid_nodes(n, 8.0, k)
        P = T.ts_plan_create((n,) * 3, (8.0,) * 3, [x ** 2] * 3, 0, order=k)
        u = torch.from_numpy(synth.normal(2, P.N)).cuda()
        y = torch.empty_like(u)
        for _ in range(args.warmup + args.steps):
            T.ts_apply_operator(P, 0.5, None, u, y)
        torch.cuda.synchronize()
        print("profile case done", flush=True)
        return 0
    if args.workload in ("6d_n24_strang", "9d_n8_strang"):
        w = synth.WORKLOADS[args.workload]
        n, L = w["n"], w["L"]
        prec = T.TS_BF16X6 if args.profile_bf16x6 else T.TS_FP32
        P = T.ts_plan_create(n, L, synth.harmonic(n, L, w["omega"]), 1 << prec)
        V2 = torch.from_numpy(synth.v2_soft_coulomb(n, L)).cuda()
        x = torch.from_numpy(synth.sine_state(n, L).astype(np.float32)).cuda()
        T.ts_split_step(P, w["dt"], args.warmup + args.steps, V2, x, T.TS_C64, prec)
        torch.cuda.synchronize()
        print("profile case done", flush=True)
        return 0
    w = synth.WORKLOADS[WORKLOAD]
    n = (args.profile_n,) * 3 if args.profile_n else w["n"]
    P = T.ts_plan_create(n, w["L"], synth.harmonic(n, w["L"], w["omega"]), (1 << T.TS_BF16X3) | (1 << T.TS_BF16X1))
    b = torch.from_numpy(synth.normal(w["seed"], P.N)).cuda()
    x = torch.empty_like(b)
    if args.profile_fp64:
        # the plain FP64 apply (k_rot_fp64 passes) only
        for _ in range(args.warmup + args.steps):
            T.ts_apply_inverse(P, w["sigma"], b, x, T.TS_FP64)
        torch.cuda.synchronize()
        print("profile case done", flush=True)
        return 0
    for _ in range(args.warmup + args.steps):
        T.ts_solve_schedule(P, w["sigma"], b, x, [getattr(T, q) for q in SCHEDULE])
    torch.cuda.synchronize()
    T.ts_device_status()
    print("profile case done", flush=True)
    return 0


def serving_requests_on_device(T, total, seed=4, omega_set=None):
    """The serving workload's request arguments (without the precision): `total` requests of
    3D grids with n_k from {32, 48, 64, 96, 128}, 30% PCG / 50% inverse / 20% exp, their
    right-hand sides and V2 generated on the GPU from the same seeds as the host generators."""
    import torch
    reqs = []
    for sp in synth.serving_requests(total, seed=seed, omega_set=omega_set):
        n, L = sp["n"], sp["L"]
        N = int(np.prod(n))
        kw = dict(n=n, L=L, f=synth.harmonic(n, L, sp["omega"]), sigma=sp["sigma"], tau=sp["tau"])
        if sp["kind"] == "exp":
            kw.update(kind=T.TS_REQ_EXP, inp=synth.complex_normal_torch(sp["rhs_seed"], N),
                      out=torch.empty(2 * N, dtype=torch.float64, device="cuda"), dtype=T.TS_C128)
        else:
            kw.update(inp=synth.normal_torch(sp["rhs_seed"], N),
                      out=torch.zeros(N, dtype=torch.float64, device="cuda"), dtype=T.TS_R64)
            if sp["kind"] == "pcg":
                kw.update(kind=T.TS_REQ_PCG, V2=synth.v2_cos_bumps_torch(n, L, seed=1), tol=1e-10, maxit=200)
            else:
                kw.update(kind=T.TS_REQ_INVERSE)
        reqs.append(kw)
    torch.cuda.synchronize()
    return reqs


def serving_run(T, count, omega_set=None, rate_factor=0.8, seed=4, prec=None, overload_factor=2.0, reqs=None,
                planner_threads=0):
    """The serving workload: `count` requests (3D grids with n_k from {32, 48, 64, 96, 128},
    30% PCG / 50% inverse / 20% exp), first submitted all at once (saturated throughput),
    then again with Poisson arrivals at rate_factor x that throughput, and once more at
    overload_factor x it (an overloaded server: the queue grows while arrivals last);
    returns the stats of each phase.  `reqs` (from serving_requests_on_device, count per
    phase): the requests to serve, so that two precisions can serve the same ones."""
    import torch
    prec = T.TS_BF16X3 if prec is None else prec
    phases = ("saturated", "poisson") + (("overload",) if overload_factor else ())
    # every phase serves its own requests (drawn in one sequence, `count` per phase), so
    # that the plan cache meets new potentials in each phase as a live server would
    if reqs is None:
        reqs = serving_requests_on_device(T, count * len(phases), seed=seed, omega_set=omega_set)
    reqs = [dict(kw, prec=prec) for kw in reqs]
    torch.cuda.synchronize()
    server = T.Server(max_inflight=16, planner_threads=planner_threads)
    out = {}
    for q, phase in enumerate(phases):
        preqs = reqs[q * count:(q + 1) * count]
        torch.cuda.synchronize()
        server.reset_stats()
        if phase == "saturated":
            tickets = [server.submit(**kw) for kw in preqs]
        else:
            factor = rate_factor if phase == "poisson" else overload_factor
            rate = factor * out["saturated"]["completed"] / (out["saturated"]["makespan_ms"] * 1e-3)
            u = synth.uniform(seed + 17, count, 1e-12, 1.0)
            gaps = -np.log(u) / rate
            tickets = []
            t0 = time.perf_counter()
            t_next = 0.0
            for kw, gap in zip(preqs, gaps):
                t_next += gap
                while time.perf_counter() - t0 < t_next:
                    time.sleep(min(1e-4, max(0.0, t_next - (time.perf_counter() - t0))))
                tickets.append(server.submit(**kw))
        fails = 0
        for t in tickets:
            st, _, _ = server.wait(t)
            fails += st != T.TS_OK
        stats = server.stats()
        stats["failed"] = fails
        if phase != "saturated":
            stats["arrival_rate_per_s"] = rate
            stats["rate_factor"] = factor
        out[phase] = stats
    server.close()
    out["requests_per_phase"] = count
    out["mix"] = "30% PCG (V2 = 5 cos cos cos + 8 Gaussian bumps, tol 1e-10) / 50% inverse / 20% exp (tau 0.01)"
    out["grids"] = "3D, n_k iid from {32, 48, 64, 96, 128}"
    out["omega"] = "U[0.5, 2) per axis" if omega_set is None else f"from {list(omega_set)}"
    out["precision"] = ("BF16X3 (PCG: BF16X3 preconditioner, FP64 recurrence)" if prec == T.TS_BF16X3
                        else "FP64 (all applies and the PCG preconditioner)")
    return out


def batched_list_kernel(T, peaks, items=40, reps=5, seed=4):
    """The work-list kernel of a serving batch on its own: `items` inverse requests with the
    serving workload's grids (BF16X3) applied by one ts_apply_batch (one k_rot_tc_list
    launch per pass over all items), timed per launch on the device; achieved FLOP/s and
    algorithmic bytes/s against the bf16 burst peak and the HBM copy rate."""
    import torch
    specs = [sp for sp in synth.serving_requests(4 * items, seed=seed) if sp["kind"] != "exp"][:items]
    batch, dofs = [], 0
    for sp in specs:
        n, L = sp["n"], sp["L"]
        P = T.ts_plan_create(n, L, synth.harmonic(n, L, sp["omega"]), 1 << T.TS_BF16X3)
        x = synth.normal_torch(sp["rhs_seed"], P.N)
        batch.append((P, T.TS_R64, T.TS_BF16X3, sp["sigma"], x, torch.empty_like(x)))
        dofs += P.N
    T.ts_apply_batch(batch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    T.ts_profile_begin()
    e0.record()
    for _ in range(reps):
        T.ts_apply_batch(batch)
    e1.record()
    torch.cuda.synchronize()
    nl, kms, fl, by = T.ts_profile_end(T.PROF_TC_LIST)
    batch_ms = e0.elapsed_time(e1) / reps
    tflops = fl / (kms * 1e-3) / 1e12
    gbs = by / (kms * 1e-3) / 1e9
    f_t, f_h = tflops / peaks["bf16_tflops"], gbs / peaks["hbm_gbs"]
    return {"kernel": "k_rot_tc_list (BF16X3)", "items": len(batch), "dof": dofs, "launches_per_batch": nl / reps,
            "avg_launch_ms": kms / max(1, nl), "batch_ms": batch_ms, "batch_gdofs": dofs / (batch_ms * 1e-3) / 1e9,
            "achieved_tflops": tflops, "achieved_gbs": gbs, "frac_of_bf16_burst": f_t, "frac_of_hbm": f_h,
            "bound": "tensor" if f_t >= f_h else "hbm"}


def strang_run(T, name, peaks, steps=None, prec=None):
    """complex64 Strang steps of the 6D n = 24 or 9D n = 8 workload on the fused small-n
    path (TS_FP32: the FFMA kernels; TS_BF16X6: the tensor-core kernel for axes of 16 or
    24): ms per step, the HBM rate of the fused passes (algorithmic bytes per device time
    of the pass kernels) and, for the tensor-core kernel, its bf16 tensor rate."""
    import torch
    prec = T.TS_FP32 if prec is None else prec
    w = synth.WORKLOADS[name]
    n, L = w["n"], w["L"]
    steps = steps or w["steps"]
    P = T.ts_plan_create(n, L, synth.harmonic(n, L, w["omega"]), 1 << prec)
    V2 = torch.from_numpy(synth.v2_soft_coulomb(n, L)).cuda()
    x = torch.from_numpy(synth.sine_state(n, L).astype(np.float32)).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    T.ts_split_step(P, w["dt"], 3, V2, x, T.TS_C64, prec)
    torch.cuda.synchronize()
    T.ts_profile_begin()
    e0.record()
    T.ts_split_step(P, w["dt"], steps, V2, x, T.TS_C64, prec)
    e1.record()
    torch.cuda.synchronize()
    nl, kms, fl, by = T.ts_profile_end(T.PROF_SMALL_PASS)
    ms = e0.elapsed_time(e1) / steps
    norm = float(torch.linalg.vector_norm(x.double()).item())
    gbs = by / (kms * 1e-3) / 1e9 if kms else None
    tensor = prec == T.TS_BF16X6
    out = {"workload": name, "n": list(n), "dof": P.N, "dtype": "c64",
           "prec": "BF16X6 tensor-core small-n" if tensor else "FP32 fused small-n",
           "steps": steps, "ms_per_step": ms, "gdofs": P.N / (ms * 1e-3) / 1e9,
           "passes_per_step": nl / steps, "pass_ms_per_step": kms / steps, "pass_gbs": gbs,
           "pass_frac_of_hbm": gbs / peaks["hbm_gbs"] if gbs else None,
           "hbm_floor_ms_per_pass": 2.0 * 8.0 * P.N / (peaks["hbm_gbs"] * 1e9) * 1e3,
           "hbm_floor_ms_per_step": nl / steps * 2.0 * 8.0 * P.N / (peaks["hbm_gbs"] * 1e9) * 1e3,
           "norm_after": norm}
    if tensor and kms:
        out["pass_tflops"] = fl / (kms * 1e-3) / 1e12
    del x, V2
    torch.cuda.empty_cache()
    return out


def pcg_inverse_iteration_run(T, prec=None):
    """The 3D n = 256 shifted inverse iteration for V = V1 + V2 (cos + bumps) with the
    split-precision preconditioner: seconds, eigenvalue, outer and PCG iterations, wall time
    per PCG iteration and the device time of the preconditioner's passes per iteration."""
    import torch
    prec = T.TS_BF16X3 if prec is None else prec
    w = synth.WORKLOADS["3d_n256_pcg"]
    n, L = w["n"], w["L"]
    P = T.ts_plan_create(n, L, synth.harmonic(n, L, w["omega"]), 1 << T.TS_BF16X3)
    V2h = synth.v2_cos_bumps(n, L, seed=w["v2_seed"])
    V2 = torch.from_numpy(V2h).cuda()
    shift = sum(T.ts_plan_eigs(P, k)[0] for k in range(3)) + V2h.min() - 1.0
    u = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    T.ts_profile_begin()
    t0 = time.perf_counter()
    lam, outer, pcg = T.ts_inverse_iteration(P, shift, V2, u, True, w["lambda_tol"], 400, w["pcg_tol"], 500, prec)
    el = time.perf_counter() - t0
    pre_ms = sum(T.ts_profile_end(k)[1] for k in (T.PROF_TC_PASS, T.PROF_TC_PASS_OUT))
    out = {"workload": "3d_n256_pcg", "n": list(n), "dof": P.N, "precond": "BF16X3" if prec == T.TS_BF16X3 else "FP64",
           "lambda": lam, "outer_iters": outer, "pcg_iters": pcg, "seconds": el,
           "ms_per_pcg_iter": el * 1e3 / max(1, pcg), "precond_gpu_ms_per_pcg_iter": pre_ms / max(1, pcg),
           "gdofs_per_pcg_iter": P.N * pcg / el / 1e9, "shift": shift}
    del u, V2
    torch.cuda.empty_cache()
    return out


def table1_run(T, n=1099, k=2):
    """The paper's Table 1 3D problem (eq. test_potential) on Q^k SEM: (-Delta + V) u = f on
    [-1, 1]^3, V = 1600 sum sin^2(pi x_k / 4) + (x^2 + 2 y^2 + 3 z^2),
    u* = sin(pi x) sin(2 pi y) sin(3 pi z), f = (14 pi^2 + V) u*, sampled at the GLL nodes.
    Solves it with the FP64 apply and with the split-precision tensor-core applies (single
    and refined) and reports time, GDoF/s and the l2 relative error against u*."""
    import torch
    x, _ = T.ts_grid_nodes(n, 1.0, k)
    xs = torch.from_numpy(x).cuda()
    fx = [1600 * torch.sin(math.pi * xs / 4) ** 2 + (a + 1) * xs ** 2 for a in range(3)]
    P = T.ts_plan_create((n,) * 3, (1.0,) * 3, [v.cpu().numpy() for v in fx],
                         (1 << T.TS_BF16X3) | (1 << T.TS_BF16X1), order=k)
    us = (torch.sin(3 * math.pi * xs)[:, None, None] * torch.sin(2 * math.pi * xs)[None, :, None]
          * torch.sin(math.pi * xs)[None, None, :])
    b = (14 * math.pi ** 2 + fx[2][:, None, None] + fx[1][None, :, None] + fx[0][None, None, :]) * us
    b = b.reshape(-1)
    us = us.reshape(-1)
    u = torch.empty_like(b)
    nus = torch.linalg.vector_norm(us).item()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    N = P.N
    out = {"n": n, "order": k, "dof": N, "data": "synthetic (the paper's manufactured solution)"}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        err = (torch.linalg.vector_norm(u - us) / nus).item()
        return {"ms": ms, "gdofs": N / (ms * 1e-3) / 1e9, "err_vs_exact": err}

    out["fp64"] = timed(lambda: T.ts_apply_inverse(P, 0.0, b, u, T.TS_FP64), 1)
    out["bf16x3"] = timed(lambda: T.ts_apply_inverse(P, 0.0, b, u, T.TS_BF16X3), 5)
    out["bf16x1"] = timed(lambda: T.ts_apply_inverse(P, 0.0, b, u, T.TS_BF16X1), 5)
    sched = [T.TS_BF16X3, T.TS_BF16X3, T.TS_BF16X1]
    out["refined_x3_x3_x1"] = timed(lambda: T.ts_solve_schedule(P, 0.0, b, u, sched), 5)
    out["printed_err"] = {"Q1": 3.66e-6, "Q2": 1.93e-9, "Q10": 7.66e-13}
    return out


def splitting_run(T, n=499, k=10):
    """Table splitting's setup (Q^10, n^3 on [-8, 8]^3, A = -Delta, B = V1 =
    sum (x_k^2 + 100 sin^2(pi x_k / 4)), psi_0 = prod sin(pi (x_k + L) / 2L), T = 0.1): the
    cost of one A-propagation per precision, and the Delta t = 0.1 errors of Strang,
    qHOP (M = 3, 5, 7) and Magnus-2 (M = 1, 3) against the exact propagator."""
    import torch
    L = 8.0
    x, _ = T.ts_grid_nodes(n, L, k)
    v1 = x ** 2 + 100 * np.sin(np.pi * x / 4) ** 2
    mask = (1 << T.TS_BF16X3) | (1 << T.TS_BF16X6)
    PA = T.ts_plan_create((n,) * 3, (L,) * 3, [np.zeros(n)] * 3, mask, order=k)
    PH = T.ts_plan_create((n,) * 3, (L,) * 3, [v1] * 3, 0, order=k)
    xs = torch.from_numpy(x).cuda()
    s1 = torch.sin(np.pi * (xs + L) / (2 * L))
    psi0 = (s1[:, None, None] * s1[None, :, None] * s1[None, None, :]).reshape(-1)
    psi0 = (psi0 / torch.linalg.vector_norm(psi0)).to(torch.complex128)
    v = torch.from_numpy(v1).cuda()
    VB = (v[:, None, None] + v[None, :, None] + v[None, None, :]).reshape(-1).contiguous()
    ref = torch.empty_like(psi0)
    T.ts_apply_exp(PH, 0.1, torch.view_as_real(psi0), torch.view_as_real(ref), T.TS_C128)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"n": n, "order": k, "dof": PA.N, "dtype": "c128"}
    prop = {}
    for label, prec, reps in (("fp64", T.TS_FP64, 1), ("bf16x6", T.TS_BF16X6, 5), ("bf16x3", T.TS_BF16X3, 5)):
        psi = psi0.clone()
        T.ts_apply_exp(PA, 0.01, torch.view_as_real(psi), torch.view_as_real(psi), T.TS_C128, prec)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            T.ts_apply_exp(PA, 0.01, torch.view_as_real(psi), torch.view_as_real(psi), T.TS_C128, prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prop[label] = {"ms_per_A_propagation": ms, "gdofs": PA.N / (ms * 1e-3) / 1e9}
    out["A_propagation"] = prop
    errs = {}
    for name, scheme, M in (("strang", T.TS_STRANG, 1), ("qhop_M3", T.TS_QHOP, 3), ("qhop_M5", T.TS_QHOP, 5),
                            ("qhop_M7", T.TS_QHOP, 7)):
        psi = psi0.clone()
        torch.cuda.synchronize()
        e0.record()
        na = T.ts_propagate(PA, scheme, M, 0.1, 1, VB, torch.view_as_real(psi), T.TS_C128)
        e1.record()
        torch.cuda.synchronize()
        errs[name] = {"err_dt0.1": torch.linalg.vector_norm(psi - ref).item(), "A_propagations": na,
                      "ms": e0.elapsed_time(e1)}
    out["fp64_dt0.1"] = errs
    out["printed_err_dt0.1"] = {"strang": 5.85e-1, "qhop_M3": 1.07e-1, "qhop_M5": 4.25e-2, "qhop_M7": 2.28e-2}
    return out


def run_secondary(args):
    """One JSON line for a workload other than the benchmark's: the 3D n = 256 PCG /
    shifted inverse iteration, the 6D / 9D Strang runs, or the serving workload."""
    import torch
    from paper_2605_20491_b300 import tschrod as T
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    name = args.workload
    line = {"workload": name, "data": "synthetic"}
    if name in ("6d_n24_strang", "9d_n8_strang"):
        w = synth.WORKLOADS[name]
        n, L = w["n"], w["L"]
        P = T.ts_plan_create(n, L, synth.harmonic(n, L, w["omega"]), 1 << T.TS_FP32)
        V2 = torch.from_numpy(synth.v2_soft_coulomb(n, L)).cuda()
        psi0 = synth.sine_state(n, L)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for label, dt_, prec, steps in (("c64_fp32_fused", T.TS_C64, T.TS_FP32, w["steps"]),
                                        ("c128_fp64", T.TS_C128, T.TS_FP64, 5)):
            x = torch.from_numpy(psi0.astype(np.float32) if dt_ == T.TS_C64 else psi0).cuda()
            T.ts_split_step(P, w["dt"], 2, V2, x, dt_, prec)
            torch.cuda.synchronize()
            T.ts_profile_begin()
            e0.record()
            T.ts_split_step(P, w["dt"], steps, V2, x, dt_, prec)
            e1.record()
            torch.cuda.synchronize()
            kind = T.PROF_SMALL_PASS if prec == T.TS_FP32 else T.PROF_FP64_PASS
            nl, kms, fl, by = T.ts_profile_end(kind)
            ms = e0.elapsed_time(e1) / steps
            line[label] = {"ms_per_step": ms, "steps": steps, "gdofs": P.N / (ms * 1e-3) / 1e9,
                           "kernel_launches": nl, "kernel_ms_per_step": kms / steps,
                           "kernel_gbs": by / (kms * 1e-3) / 1e9 if kms else None,
                           "kernel_tflops": fl / (kms * 1e-3) / 1e12 if kms else None}
    elif name == "3d_n256_pcg":
        w = synth.WORKLOADS[name]
        n, L = w["n"], w["L"]
        P = T.ts_plan_create(n, L, synth.harmonic(n, L, w["omega"]), 1 << T.TS_BF16X3)
        V2h = synth.v2_cos_bumps(n, L, seed=w["v2_seed"])
        V2 = torch.from_numpy(V2h).cuda()
        lam1 = sum(T.ts_plan_eigs(P, k)[0] for k in range(3))
        shift = lam1 + V2h.min() - 1.0
        for label, prec in (("precond_bf16x3", T.TS_BF16X3), ("precond_fp64", T.TS_FP64)):
            u = torch.zeros(P.N, dtype=torch.float64, device="cuda")
            t0 = time.perf_counter()
            lam, outer, pcg = T.ts_inverse_iteration(P, shift, V2, u, True, w["lambda_tol"], 400, w["pcg_tol"], 500,
                                                     prec)
            el = time.perf_counter() - t0
            line[label] = {"lambda": lam, "outer_iters": outer, "pcg_iters": pcg, "seconds": el,
                           "gdofs_per_pcg_iter": P.N * pcg / el / 1e9}
        line["shift"] = shift
    elif name == "3d_q2_n1099_table1":
        line.update(table1_run(T))
    elif name == "3d_q10_n499_splitting":
        line.update(splitting_run(T))
    elif name == "serving":
        line["continuous_omega"] = serving_run(T, args.requests)
        line["discrete_omega"] = serving_run(T, args.requests, omega_set=(0.5, 1.0, 1.5, 2.0))
        line["fp64"] = serving_run(T, args.requests, prec=T.TS_FP64)
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2605_20491_b300 import tschrod as T

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = synth.WORKLOADS[WORKLOAD]
    n, L = w["n"], w["L"]
    f = synth.harmonic(n, L, w["omega"])
    mask = (1 << T.TS_BF16X3) | (1 << T.TS_BF16X1)
    P = T.ts_plan_create(n, L, f, mask)
    sched = [getattr(T, q) for q in SCHEDULE]
    N = P.N
    sigma = w["sigma"]
    b_host = torch.from_numpy(synth.normal(w["seed"], N)).pin_memory()
    b = b_host.cuda()
    x = torch.zeros_like(b)
    u64 = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    # FP64 direct apply (plain form) and its time.
    T.ts_apply_inverse(P, sigma, b, u64, T.TS_FP64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    T.ts_apply_inverse(P, sigma, b, u64, T.TS_FP64)
    e1.record()
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    nrm = u64.norm().item()

    # One unrefined split-precision apply and its error.
    um = torch.empty_like(b)
    for _ in range(3):
        T.ts_apply_inverse(P, sigma, b, um, T.TS_BF16X3)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        T.ts_apply_inverse(P, sigma, b, um, T.TS_BF16X3)
    e1.record()
    torch.cuda.synchronize()
    mixed1_ms = e0.elapsed_time(e1) / 5
    mixed1_err = ((um - u64).norm() / nrm).item()
    del um

    # PCG with the same preconditioner (V2 = 0), for comparison.
    x.zero_()
    T.ts_pcg(P, sigma, sigma, None, b, x, PCG_TOL, 20, T.TS_BF16X3)
    torch.cuda.synchronize()
    e0.record()
    x.zero_()
    _, pcg_it, _ = T.ts_pcg(P, sigma, sigma, None, b, x, PCG_TOL, 20, T.TS_BF16X3)
    e1.record()
    torch.cuda.synchronize()
    pcg_ms = e0.elapsed_time(e1)
    pcg_err = ((x - u64).norm() / nrm).item()

    def step():
        T.ts_solve_schedule(P, sigma, b, x, sched)

    clocks = ClockSampler(local)
    clocks.start()  # started before the warm-up so that it samples from the first timed step
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    err = ((x - u64).norm() / nrm).item()

    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    launches0 = T.ts_launch_count()
    T.ts_profile_begin()
    # One event between consecutive steps as well (recording an event costs no GPU time):
    # the whole region gives the mean, the per-step intervals the median.
    ev_steps = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps - 1)]
    e0.record()
    for i in range(args.steps):
        step()
        if i < args.steps - 1:
            ev_steps[i].record()
    e1.record()
    torch.cuda.synchronize()
    clocks.mark(t_wall0, time.time())
    marks = [e0] + ev_steps + [e1]
    step_ms = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
    median_ms = step_ms[len(step_ms) // 2] if len(step_ms) % 2 else 0.5 * sum(step_ms[len(step_ms) // 2 - 1:len(step_ms) // 2 + 1])
    barrier()
    tc_launches, tc_ms, tc_flops, tc_bytes = T.ts_profile_end(T.PROF_TC_PASS)
    out_launches, out_ms, out_flops, out_bytes = T.ts_profile_end(T.PROF_TC_PASS_OUT)
    res_launches, res_ms, _, res_bytes = T.ts_profile_end(T.PROF_RESIDUAL)
    x1_launches, x1_ms, x1_flops, x1_bytes = T.ts_profile_end(T.PROF_TC_PASS_X1)
    launches = T.ts_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    value = whole_job_rate(world, N, ms)

    # End to end through the public API with host buffers: every step copies its right-hand
    # side from pinned host memory, solves, and copies its solution back.  Steps are
    # pipelined over two buffer sets and three streams, as a serving loop would run them:
    # the upload of step k+1 and the download of step k-1 overlap the solve of step k.
    s_h2d, s_cmp, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    bd = [torch.empty_like(b) for _ in range(2)]
    xd = [torch.empty_like(b) for _ in range(2)]
    u_host = [torch.empty_like(b_host).pin_memory() for _ in range(2)]
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("h2d", "cmp", "d2h")}
    for j in range(2):
        for k in ev:
            ev[k][j].record(torch.cuda.current_stream())

    def e2e_run(n_steps):
        for k in range(n_steps):
            j = k % 2
            with torch.cuda.stream(s_h2d):
                s_h2d.wait_event(ev["cmp"][j])  # bd[j] is free once step k-2 has been solved
                bd[j].copy_(b_host, non_blocking=True)
                ev["h2d"][j].record(s_h2d)
            s_cmp.wait_event(ev["h2d"][j])
            s_cmp.wait_event(ev["d2h"][j])  # xd[j] is free once step k-2 has been downloaded
            T.ts_solve_schedule(P, sigma, bd[j], xd[j], sched, stream=s_cmp)
            ev["cmp"][j].record(s_cmp)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(ev["cmp"][j])
                u_host[j].copy_(xd[j], non_blocking=True)
                ev["d2h"][j].record(s_d2h)
        torch.cuda.synchronize()
        return (n_steps - 1) % 2

    e2e_run(2)
    n_e2e = max(4, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    last = e2e_run(n_e2e)
    e2e_ms = (time.perf_counter() - t0) / n_e2e * 1e3
    e2e_err = float(np.linalg.norm(u_host[last].numpy() - u64.cpu().numpy()) / nrm)

    # The floor of that pipeline: the same uploads and downloads with no solve, the two
    # directions concurrent on their own streams (the host link, not the GPU, bounds it).
    def copies_only(n_steps):
        for k in range(n_steps):
            j = k % 2
            with torch.cuda.stream(s_h2d):
                bd[j].copy_(b_host, non_blocking=True)
            with torch.cuda.stream(s_d2h):
                u_host[j].copy_(xd[j], non_blocking=True)
        torch.cuda.synchronize()

    copies_only(1)
    t0 = time.perf_counter()
    copies_only(n_e2e)
    copy_ms = (time.perf_counter() - t0) / n_e2e * 1e3

    peaks, peaks_src = load_peaks()
    avg_launch_ms = tc_ms / max(1, tc_launches)
    achieved = (tc_flops / max(1, tc_launches)) / (avg_launch_ms * 1e-3) / 1e12 if tc_launches else None
    # The timed region lasts well under a second, so the tensor-bound passes are held to the
    # burst bf16 rate (the sustained rate was measured over seconds, at lower clocks).
    peak = peaks["bf16_tflops"]
    roofline = {"bound": "tensor", "kernel": "k_rot_tc, BF16X3 passes writing bf16 planes", "achieved": achieved,
                "peak": peak, "peak_kind": f"bf16 dense burst ({peaks_src})", "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "peak_sustained": peaks.get("bf16_tflops_sustained"),
                "frac_of_sustained": (achieved / peaks["bf16_tflops_sustained"])
                if achieved and peaks.get("bf16_tflops_sustained") else None,
                "traffic": None,
                "traffic_note": "not measured in this run: DRAM bytes per launch come from an ncu capture of the "
                                "same kernel, summarised in profiles/",
                "algorithmic_flops_per_launch": tc_flops / max(1, tc_launches),
                "algorithmic_bytes_per_launch": tc_bytes / max(1, tc_launches),
                "avg_launch_ms": avg_launch_ms, "launches": tc_launches,
                "share_of_step": tc_ms / (ms * args.steps)}

    def hbm_entry(kernel, launches, kms, flops, nbytes):
        gbs = nbytes / max(1e-9, kms * 1e-3) / 1e9
        return {"kernel": kernel, "bound": "hbm", "launches": launches, "avg_launch_ms": kms / max(1, launches),
                "achieved_gbs": gbs, "achieved_tflops": flops / max(1e-9, kms * 1e-3) / 1e12,
                "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
                "algorithmic_bytes_per_launch": nbytes / max(1, launches),
                "share_of_step": kms / max(1e-9, ms * args.steps)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "ms_per_step_median": median_ms, "ms_per_step_min": step_ms[0], "ms_per_step_max": step_ms[-1],
            "vs_baseline": None, "dtype": "bf16 splits (x3, x1) + f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": list(n), "L": list(L), "omega": list(w["omega"]), "sigma": sigma,
                       "rhs": "iid N(0,1), SplitMix64 seed 2",
                       "solve": "split tcgen05 inverses " + " -> ".join(q[3:] for q in SCHEDULE)
                       + " (u_0, then refinements with FP64 residuals)",
                       "l2": "inputs larger than L2 (1.07 GB per vector)",
                       "parallelism": f"replicas x{world}"},
            "err_vs_fp64": err, "err_target": ERR_TARGET,
            "pcg": {"ms": pcg_ms, "iters": pcg_it, "tol": PCG_TOL, "err_vs_fp64": pcg_err,
                    "gdofs": N / (pcg_ms * 1e-3) / 1e9},
            "fp64": {"ms": fp64_ms, "gdofs": N / (fp64_ms * 1e-3) / 1e9, "kernel": "k_rot_fp64 (FFMA64)"},
            "mixed_single_apply": {"prec": "BF16X3", "ms": mixed1_ms, "gdofs": N / (mixed1_ms * 1e-3) / 1e9,
                                   "err_vs_fp64": mixed1_err},
            "speedup_vs_fp64": fp64_ms / ms,
            "roofline": roofline,
            # the last pass of every apply writes the FP64 result (u_0) or adds it (u += delta):
            # the same kernel, HBM-bound
            "fp64_output_passes": hbm_entry("k_rot_tc, passes writing the FP64 result (u_0 store, u += delta)",
                                            out_launches, out_ms, out_flops, out_bytes),
            # the one-plane passes of the last refinement (same kernel, HBM-bound)
            "x1_passes": hbm_entry("k_rot_tc, BF16X1 passes writing one bf16 plane", x1_launches, x1_ms,
                                   x1_flops, x1_bytes),
            # second kernel of the step: the refinement residual (HBM-streaming; x, b in, planes out)
            "residual_kernel": hbm_entry("k_residual_march3", res_launches, res_ms, 0.0, res_bytes),
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": world * N / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N, "err_vs_fp64": e2e_err,
                    "pipelining": "2 buffer sets, 3 streams: upload k+1 and download k-1 overlap solve k",
                    "copy_floor_ms_per_step": copy_ms, "frac_of_copy_floor": copy_ms / e2e_ms}}
    del bd, xd, u_host
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_secondary:
        # the other configurations of the workload family, each timed on its own
        line["strang_6d_n24"] = strang_run(T, "6d_n24_strang", peaks)
        line["strang_6d_n24_bf16x6"] = strang_run(T, "6d_n24_strang", peaks, prec=T.TS_BF16X6)
        line["strang_9d_n8"] = strang_run(T, "9d_n8_strang", peaks)
        line["pcg_3d_n256"] = pcg_inverse_iteration_run(T)
    if rank == 0 and not args.no_serving:
        reqs = serving_requests_on_device(T, 3 * args.requests)
        sv = serving_run(T, args.requests, reqs=reqs)
        line["serving"] = sv
        line["p50_ms"] = sv["poisson"]["p50_ms"]
        line["p99_ms"] = sv["poisson"]["p99_ms"]
        del reqs
        torch.cuda.empty_cache()
        # FP64 serves a second draw of the same distribution: on the first draw's requests its
        # plans would reuse the per-axis tables the BF16X3 run left in the process-wide cache
        reqs = serving_requests_on_device(T, 3 * args.requests, seed=5)
        line["serving_fp64"] = serving_run(T, args.requests, prec=T.TS_FP64, reqs=reqs, seed=5)
        line["serving_fp64"]["requests"] = "a second draw (seed 5) of the same distribution"
        del reqs
        torch.cuda.empty_cache()
        line["serving_batched_kernel"] = batched_list_kernel(T, peaks)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_baseline()
    T.ts_device_status()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="run only the refined solve (for ncu captures); prints no JSON line")
    ap.add_argument("--profile-n", type=int, default=0,
                    help="grid points per axis of the --profile-case refined solve (default: the workload's)")
    ap.add_argument("--profile-fp64", action="store_true",
                    help="with --profile-case: the plain FP64 inverse apply instead of the refined solve")
    ap.add_argument("--profile-bf16x6", action="store_true",
                    help="with --profile-case and a Strang workload: the tensor-core small-n pass (TS_BF16X6)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 6D / 9D Strang and 3D n = 256 inverse-iteration sub-runs")
    ap.add_argument("--requests", type=int, default=2048, help="requests per phase of the serving run")
    ap.add_argument("--reference-n", type=int, default=0,
                    help="grid points per axis of the reference arm (default: the workload's 512; the "
                         "line's config reports the n used)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "3d_n256_pcg", "6d_n24_strang", "9d_n8_strang", "serving",
                             "3d_q2_n1099_table1", "3d_q10_n499_splitting"])
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.workload != WORKLOAD:
        return run_secondary(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
