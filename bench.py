#!/usr/bin/env python3
"""Benchmark of one dual-gradient pass (the hot path) on the c2 workload.

A step is one full dual evaluation through the C ABI (destination prologue,
the edge pass, destination epilogue with the FP64 scalars) on the c2 matching
LP: 1M sources x 10k destinations, Poisson(50) degrees clipped to [1, 500],
Zipf(1.1) destinations, about 50M edges, seeded synthetic data.  The metric is
edges per second per pass; the edge arrays (600 MB) exceed the 129 MB L2, so
no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica (the method is
run on one GPU; there is no sharded path), value = edges of all ranks / max
time.  ``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.

At N = 1 the c2 line also carries

* ``ascent_pass``: the pass timed along the c2 ascent itself (greedy-load
  budgets, every iteration of the solve to the 1e-4 gap) and at the solved
  dual point for gamma 1e-3 and 0.1, where near-ties send sources to the
  multi-pass projection;
* ``forms``: the BF16 and FP32 forms on c3, the batched form on c4 and the
  serving form on c5, each with its pass roofline (CUDA events, measured
  HBM peak), clocks and time to the 1e-4 gap beside the plain FP32 form
  (``--no-forms`` skips them).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s per dual-grad pass"
UNIT = "edges/s"
GAMMA = 1e-3
LAM_SEED = 7


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c3", "c4", "c5", "appb", "hubs"],
                    help="c2: 1M x 10k, ~50M edges (default); c3: 25M x 1M, ~2.0B edges; "
                         "c4: 256 problems in one batched pass, ~3.4B edges; "
                         "c5: a Poisson stream of solve requests through the server; "
                         "appb: the Appendix B generator; hubs: c2 plus 100 hub sources")
    ap.add_argument("--requests", type=int, default=60,
                    help="c5: the first N requests of the seeded trace")
    ap.add_argument("--budget-gib", type=float, default=160.0, help="c5: HBM budget")
    ap.add_argument("--storage", default=None, choices=["f32", "bf16"],
                    help="edge storage (default f32 for c2, bf16 for c3)")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the sources")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the c3/c4/c5 forms that the default c2 line carries")
    ap.add_argument("--form-requests", type=int, default=30,
                    help="forms: requests of the c5 replay")
    return ap.parse_args()


def max_over_ranks(x: float, ws: int) -> float:
    """The largest value of x over the ranks (gloo; every rank gets it)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, steps: int, ws: int, seconds: float) -> float:
    """Units of every rank (independent replicas) per second of the slowest rank."""
    return units_per_rank * steps * ws / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name="c2", scale=1.0):
    import synth

    return synth.config(name, scale=scale)


def lam_for(inst):
    return np.random.default_rng(LAM_SEED).uniform(0.0, 1.0, inst.J).astype(np.float32)


WORKLOADS = {
    "c2": ("c2: matching LP, 1M sources x 10k destinations, Poisson(50) degrees in [1,500], "
           "Zipf(1.1) destinations, c=-LogNormal(0,1), a~U(0.5,1.5), b=0.2*sum(a), int32 dst"),
    "c3": ("c3: matching LP, 25M sources x 1M destinations, Poisson(80) degrees in [1,2000], "
           "Zipf(1.1) destinations, c=-LogNormal(0,1), a~U(0.5,1.5), b=0.2*sum(a), int64 offsets"),
    "c5": ("c5: Poisson(20/s) stream of matching-LP solves, sources LogUniform[10k,5M], "
           "destinations LogUniform[100,200k], degrees Poisson(40) in [1,J], FP32 or BF16 storage "
           "(1/2 each), greedy-load budgets (App. B rule), each solved to a 1e-4 gap"),
    "c4": ("c4: 256 independent matching LPs in one batched pass, sources LogUniform[1k,2M], "
           "destinations LogUniform[10,50k], degrees Uniform[5,100] (<= J), Zipf(1.1) "
           "destinations, c=-LogNormal(0,1), a~U(0.5,1.5), greedy-load budgets (App. B rule)"),
}


def edge_bytes(storage):
    return 8 if storage == "bf16" else 12


def config_dict(inst, name, scale, storage):
    eb = edge_bytes(storage)
    return {
        "workload": WORKLOADS[name] if scale == 1.0 else f"{name} at {scale:g} of the sources",
        "storage": storage, "I": inst.I, "J": inst.J, "E": inst.E, "gamma": GAMMA,
        "lambda": f"U(0,1) seed {LAM_SEED}",
        "edge_bytes": eb * inst.E,
        "l2": f"inputs larger than L2 (edges {eb} B/edge > 129 MB); no flush",
        "parallelism": "replicas",
    }


# DRAM traffic of one pass-kernel launch from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) on a smaller case of each
# workload's recipe (fewer sources, the same destinations), with the hash of
# the kernel source it was taken on.  The per-destination bytes (mu read, A x
# written and read: 12 B each) do not grow with the sources; the rest is scaled
# by the edges processed.  It is reported only while the kernel's code (the
# source without comments and blank lines) is unchanged and, for the batched
# pass, while the autotuner picks the tile shape it was taken at.
PASS_CODE_SHA256 = "fc34354c7c6eab0a0992917b19580f3cbb4ef51819622c0b2179955667d307a0"
PASS_TRAFFIC = {
    # c2 recipe at 0.3 of the sources, FP32 (stored in degree order)
    ("c2", "f32"): {"bytes": 181_435_648 + 3_467_008, "edges": 14_995_720, "J": 10_000},
    # c3 recipe at 0.01 of the sources, BF16 (c, a)
    ("c3", "bf16"): {"bytes": 166_989_824 + 4_261_632, "edges": 20_001_134, "J": 1_000_000},
    # c4 recipe at 0.05 of the sources (degree order), FP32, tiles of 3200 x 128
    ("c4", "f32"): {"bytes": 2_018_348_000 + 11_741_184, "edges": 164_807_481, "J": 1_665_819,
                    "tile_shape": [3200, 128]},
    # the Appendix B generator at 2M requests, FP32 (the small-degree variant)
    ("appb", "f32"): {"bytes": 252_702_208 + 3_992_576, "edges": 20_000_112, "J": 10_000},
}


def kernel_code_hash():
    import hashlib
    import re

    src = os.path.join(ROOT, "paper_2603_04621_gb300", "csrc", "pass.cu")
    with open(src) as f:
        text = f.read()
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def pass_traffic(E, J, name, storage, tile_shape=None):
    cap = PASS_TRAFFIC.get((name, storage))
    if cap is None:
        return None  # no capture of this configuration
    if kernel_code_hash() != PASS_CODE_SHA256:
        return None
    if "tile_shape" in cap and list(tile_shape or []) != cap["tile_shape"]:
        return None
    return (cap["bytes"] - 12 * cap["J"]) * E / cap["edges"] + 12 * J


def algorithmic_bytes(inst, storage="f32"):
    # what one pass must move: 12 B/edge (dst, c, a; 8 B with (c, a) in BF16),
    # a 4 B source offset (the pass streams their low 32 bits), and per
    # destination: mu read, the A x accumulator written and read
    return edge_bytes(storage) * inst.E + 4 * (inst.I + 1) + 12 * inst.J


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        load = [r for r in self.rows if (num(r[3]) or 0) > 0] or self.rows
        sm = [num(r[0]) for r in load if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in load for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(load[0][1]), "reasons": reasons,
                "samples": len(self.rows), "samples_under_load": len(load)}


def cpu_baseline(inst, seconds, d=None, torch=None):
    """The FP64 oracle as it stands, all host cores, on a bounded source sample;
    with the library given, also the error of the GPU evaluation of the same
    sample against it (per result)."""
    import oracle

    n = max(1, min(inst.I, int(inst.I * 0.05)))
    sub = inst.subset_sources(np.arange(n))
    cores = oracle.set_threads(0)
    P = oracle.Problem(sub)
    lam = lam_for(inst).astype(np.float64)
    eo = P.eval(lam, GAMMA)  # warm
    check = None
    if d is not None:
        G = d.Problem.from_instance(sub)
        grad, ev = G.dual_grad(torch.from_numpy(lam.astype(np.float32)).cuda(), GAMMA)
        grad = grad.cpu().numpy().astype(np.float64)
        G.close()
        b = sub.b.astype(np.float64)
        size = np.abs(eo.ax) + np.abs(b)
        err = np.abs(grad - eo.grad)
        terms = float(np.sum(np.abs(lam) * size))
        rel = lambda v, r: abs(v - r) / max(1.0, abs(r))
        check = {"at": "the same lambda and gamma as the pass",
                 "grad_max_err_over_bound": float(np.max(err / (1e-5 * size + 1e-6))),
                 "grad_max_rel_to_scale": float(np.max(err[size > 0] / size[size > 0])),
                 "dual_obj_rel": rel(ev["dual_obj"], eo.dual),
                 "primal_obj_rel": rel(ev["primal_obj"], eo.primal_lin),
                 "reg_rel": rel(ev["reg"], eo.reg),
                 "infeas_l2_rel": rel(ev["infeas_l2"], eo.infeas),
                 "lambda_dot_grad_rel_to_terms": abs(ev["lambda_dot_grad"] - eo.mu_dot_grad) /
                 max(1.0, terms)}
    t0 = time.perf_counter()
    reps = 0
    while True:
        P.eval(lam, GAMMA)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    out = {"value": sub.E * reps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {n} of {inst.I} sources ({sub.E} edges), {reps} FP64 evaluations "
                     f"in {dt:.1f} s"}
    if check is not None:
        out["gpu_error_vs_oracle"] = check
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    inst = workload(args.workload, args.scale)
    import oracle

    n = max(1, min(inst.I, int(inst.I * 0.02)))
    sub = inst.subset_sources(np.arange(n))
    cores = oracle.set_threads(0)
    P = oracle.Problem(sub)
    lam = lam_for(inst).astype(np.float64)
    for _ in range(args.warmup):
        P.eval(lam, GAMMA)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.eval(lam, GAMMA)
    dt = time.perf_counter() - t0
    value = sub.E * args.steps / dt
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": config_dict(inst, args.workload, args.scale, args.storage),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"each step: first {n} sources of {args.workload} "
                                      f"({sub.E} edges)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def load_peak():
    """Measured HBM copy bandwidth (GB/s) and where it came from."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    peak = peaks.get("hbm_gbs")
    if peak:
        return float(peak), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    return 6800.0, "fallback 6.8 TB/s"


def roofline(alg_bytes, pass_ms, peak, note, traffic=None, kernel="dualgrad_pass_kernel"):
    achieved = alg_bytes / (pass_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kernel, "kernel_ms": pass_ms,
            "algorithmic_bytes": alg_bytes, "peak_source": note}


def profiled(d, h, n, step, batch=False):
    """Mean kernel durations (ms) of n evaluations, CUDA events around each kernel."""
    import torch

    (d.dualip_batch_profile_enable if batch else d.dualip_profile_enable)(h, n)
    for _ in range(n):
        step()
    torch.cuda.synchronize()
    prof = (d.dualip_batch_profile_collect if batch else d.dualip_profile_collect)(h)
    c = max(prof["count"], 1)
    return {"prologue": prof["ms_prologue"] / c, "pass": prof["ms_pass"] / c,
            "epilogue": prof["ms_epilogue"] / c, "count": prof["count"]}


def solve_to_gap(d, torch, inst, storage, **kw):
    """dualip_solve to the 1e-4 relative gap (default options), after a short
    warm solve (graph capture, row scale)."""
    P = d.Problem.from_instance(inst, storage=storage)
    P.solve(max_iters=20, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, res = P.solve(**kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return P, lam, {"seconds": dt, "iters": res["iters"], "converged": res["converged"],
                    "gap_rel": res["gap_rel"], "infeas_rel": res["infeas_rel"],
                    "dual_obj": res["dual_obj"], "storage": storage}


def time_to_gap(d, torch, base, name, storage):
    """dualip_solve to the 1e-4 relative gap on the workload's graph and values with
    the paper's greedy-load budgets (the sum-fraction budgets never bind, so
    lambda* = 0 there)."""
    import synth

    inst = synth.greedy_budgets(base)
    P, lam, out = solve_to_gap(d, torch, inst, storage)
    P.close()
    out["workload"] = f"{name} graph and values with greedy-load budgets (App. B rule)"
    if name != "c2":
        return out, lam
    # a recurring solve: costs moved by about 1%, started from this optimum at
    # the final gamma
    rng = np.random.default_rng(17)
    moved = synth.Instance(inst.off, inst.dst,
                           (inst.c * (1.0 + 0.01 * rng.standard_normal(inst.E))).astype(np.float32),
                           inst.a, inst.b, inst.J)
    Q = d.Problem.from_instance(moved, storage=storage)
    wkw = dict(gamma0=1e-3, gamma_final=1e-3, halve_every=0)
    Q.solve(lam0=lam, max_iters=20, **wkw)  # warm: graph capture, row scale
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, wres = Q.solve(lam0=lam, **wkw)
    torch.cuda.synchronize()
    wdt = time.perf_counter() - t0
    Q.close()
    out["warm_recurring"] = {"seconds": wdt, "iters": wres["iters"], "converged": wres["converged"],
                             "change": "c * (1 + 0.01 N(0,1)), from the previous optimum at "
                                       "gamma 1e-3"}
    return out, lam


def ascent_pass(d, torch, base, storage, peak, note):
    """The pass where the ascent runs: every iteration of the solve to the gap
    (CUDA events around each pass, solve without graph capture), then at the
    solved dual point for gamma 1e-3 and 0.1."""
    import synth

    inst = synth.greedy_budgets(base)
    alg = algorithmic_bytes(inst, storage)
    P = d.Problem.from_instance(inst, storage=storage)
    P.solve(max_iters=20, use_graph=0)  # warm
    torch.cuda.synchronize()
    d.dualip_profile_enable(P.h, 5000)
    lam, res = P.solve(use_graph=0)
    torch.cuda.synchronize()
    prof = d.dualip_profile_collect(P.h)
    ms = prof["ms_pass"] / max(prof["count"], 1)
    out = {"workload": "c2 graph and values with greedy-load budgets (App. B rule)",
           "storage": storage, "iters": res["iters"], "converged": res["converged"],
           "solve": {"pass_ms_mean": ms, "edges_per_s": inst.E / (ms / 1e3),
                     "roofline": roofline(alg, ms, peak, note),
                     "epilogue_ms_mean": prof["ms_epilogue"] / max(prof["count"], 1),
                     "passes_timed": prof["count"]}}
    grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
    out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
    sp = int(torch.cuda.current_stream().cuda_stream)
    for gamma in (1e-3, 0.1):
        def step():
            d.dualip_dual_grad_async(P.h, lam.data_ptr(), gamma, grad.data_ptr(),
                                     out_dev.data_ptr(), sp)
        for _ in range(5):
            step()
        k = profiled(d, P.h, 100, step)
        out[f"lambda_star_gamma_{gamma:g}"] = {
            "pass_ms": k["pass"], "edges_per_s": inst.E / (k["pass"] / 1e3),
            "roofline": roofline(alg, k["pass"], peak, note)}
    d.dualip_check_device_status(P.h, sp)
    P.close()
    return out


def pass_form(d, torch, inst, name, storage, steps, warmup, peak, note):
    """One workload's pass on a lone problem: step time and per-kernel CUDA-event
    durations with clocks sampled meanwhile."""
    P = d.Problem.from_instance(inst, storage=storage)
    lam = torch.from_numpy(lam_for(inst)).cuda()
    grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
    out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    def step():
        d.dualip_dual_grad_async(P.h, lam.data_ptr(), GAMMA, grad.data_ptr(), out_dev.data_ptr(),
                                 sp)

    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        k = profiled(d, P.h, steps, step)
    d.dualip_check_device_status(P.h, sp)
    P.close()
    alg = algorithmic_bytes(inst, storage)
    return {"storage": storage, "I": inst.I, "J": inst.J, "E": inst.E, "gamma": GAMMA,
            "ms_per_step": ms, "edges_per_s": inst.E / (ms / 1e3), "kernel_ms": k,
            "roofline": roofline(alg, k["pass"], peak, note,
                                 pass_traffic(inst.E, inst.J, name, storage)),
            "clocks": clk.summary()}


def batch_time_to_gap(d, torch, probs, B):
    """Batched ascent of every problem to the 1e-4 gap, against the lone
    dualip_solve of each problem one after the other (same options)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, res = B.solve()
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    lone = [P.solve()[1] for P in probs]
    torch.cuda.synchronize()
    tl = time.perf_counter() - t0
    return {"workload": "c4 problems, greedy-load budgets", "batched_seconds": tb,
            "batched_converged": sum(r["converged"] for r in res),
            "batched_max_iters": max(r["iters"] for r in res),
            "lone_sequential_seconds": tl,
            "lone_converged": sum(r["converged"] for r in lone), "n": len(probs),
            "speedup_batched_vs_lone": tl / tb}


def batch_form(d, torch, steps, warmup, scale, storage, solve, peak, note):
    """c4: every problem of the batch in one batched pass per step."""
    import synth

    shapes = synth.batch_shapes(256)
    if scale != 1.0:
        shapes = [(max(1, int(I * scale)), J, sd) for I, J, sd in shapes]
    probs, sample = [], None
    I_t = J_t = E_t = 0
    for I, J, sd in shapes:
        inst = synth.greedy_budgets(synth.batch_instance(I, J, sd))
        probs.append(d.Problem.from_instance(inst, storage=storage))
        I_t, J_t, E_t = I_t + inst.I, J_t + inst.J, E_t + inst.E
        if sample is None and inst.I >= 100_000:
            sample = inst
        del inst
    B = d.Batch(probs)
    tune = B.autotune()
    shape = [tune["tile_edges"][tune["chosen"]], tune["tile_sources"][tune["chosen"]]]
    lam_h = np.random.default_rng(LAM_SEED).uniform(0.0, 1.0, J_t).astype(np.float32)
    lam = torch.from_numpy(lam_h).cuda()
    grad = torch.empty_like(lam)
    out_dev = torch.empty(5 * len(probs), dtype=torch.float64, device="cuda")
    gam = [GAMMA] * len(probs)
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    def step():
        d.dualip_batch_dual_grad_async(B.h, lam.data_ptr(), gam, grad.data_ptr(),
                                       out_dev.data_ptr(), sp)

    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        t_end = time.perf_counter() + 1.0
        while time.perf_counter() < t_end:
            for _ in range(5):
                step()
            torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        k = profiled(d, B.h, steps, step, batch=True)
        # end to end with host buffers: lambda in, gradient out, scalars to host
        lam_pin = torch.from_numpy(lam_h).pin_memory()
        grad_pin = torch.empty(J_t, dtype=torch.float32).pin_memory()
        t0 = time.perf_counter()
        for _ in range(steps):
            lam.copy_(lam_pin, non_blocking=True)
            B.dual_grad(lam, gam)
            grad_pin.copy_(grad, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
    ttg = batch_time_to_gap(d, torch, probs, B) if solve else None
    alg = (edge_bytes(storage) * E_t + 8 * (I_t + len(probs)) + 12 * J_t)
    out = {
        "value": E_t * steps / (ms / 1e3), "ms_per_step": ms / steps,
        "config": {"workload": WORKLOADS["c4"] if scale == 1.0 else f"c4 at {scale:g} of the sources",
                   "storage": storage, "problems": len(probs), "I": I_t, "J": J_t, "E": E_t,
                   "gamma": GAMMA, "lambda": f"U(0,1) seed {LAM_SEED}",
                   "l2": "inputs larger than L2; no flush", "parallelism": "replicas",
                   "tile_shape": shape},
        "roofline": roofline(alg, k["pass"], peak, note,
                             pass_traffic(E_t, J_t, "c4", storage, shape),
                             kernel="dualgrad_pass_kernel (batched)"),
        "kernel_ms": k,
        "autotune": {"tile_edges": tune["tile_edges"], "tile_sources": tune["tile_sources"],
                     "ms": tune["ms"], "chosen": tune["chosen"], "lean80": tune["lean80"],
                     "ms_lean80": tune["ms_lean80"]},
        "e2e": {"value": E_t * steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * J_t,
                "d2h_bytes_per_step": 4 * J_t + 40 * len(probs),
                "api": "dualip_batch_dual_grad (lambda and grad through pinned host buffers)"},
        "clocks": clk.summary(),
        "gpu_launches": 3 * steps,
        "time_to_gap": ttg,
    }
    B.close()
    for P in probs:
        P.close()
    return out, sample


def run_batch(args):
    import torch

    torch.cuda.set_device(0)
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    peak, note = load_peak()
    f, sample = batch_form(d, torch, args.steps, args.warmup, args.scale, args.storage,
                           not args.no_solve, peak, note)
    out = {"metric": METRIC, "value": f.pop("value"), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": f.pop("ms_per_step"),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", **f}
    if not args.no_cpu_baseline and sample is not None:
        out["cpu_baseline"] = cpu_baseline(sample, args.cpu_seconds, d, torch)
    print(json.dumps(out), flush=True)
    return 0


def serve_form(d, torch, n, budget_gib):
    """c5: replay the first n requests of the trace in real time through the
    server; then solve each request alone with the plain FP32 form."""
    import synth

    trace = synth.request_trace(400)[:n]
    insts = [synth.greedy_budgets(synth.request_instance(r)) for r in trace]
    srv = d.Server(int(budget_gib * (1 << 30)), max_slots=64, check_every=10)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        tickets = []
        for r, x in zip(trace, insts):
            dt = r["t"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(x, storage=r["storage"]))
        out = [srv.wait(t, 3600.0) for t in tickets]
        span = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    infos = [o[0] for o in out]
    ok = [i for i in infos if i["state"] == d.DUALIP_REQ_DONE]
    conv = [i for i in ok if i["converged"]]
    ttg = np.array([i["t_done"] - i["t_submit"] for i in ok])
    ttg_c = np.array([i["t_done"] - i["t_submit"] for i in conv]) if conv else ttg
    qd = np.array([i["t_admit"] - i["t_submit"] for i in ok])
    work = sum(x.E * i["iters"] for x, i in zip(insts, infos) if i["state"] == d.DUALIP_REQ_DONE)
    # the plain FP32 single-instance form, one request after another
    lone_t, lone_conv = 0.0, 0
    for x in insts:
        P = d.Problem.from_instance(x)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, r1 = P.solve()
        torch.cuda.synchronize()
        lone_t += time.perf_counter() - t1
        lone_conv += r1["converged"]
        P.close()
    return {
        "config": {"workload": WORKLOADS["c5"], "requests": n, "arrival_rate_per_s": 20.0,
                   "budget_gib": budget_gib, "max_slots": 64, "check_every": 10,
                   "E_mean": float(np.mean([x.E for x in insts])),
                   "bf16_requests": sum(r["storage"] == "bf16" for r in trace),
                   "parallelism": "replicas"},
        "serve": {"p50_s": float(np.median(ttg)), "p99_s": float(np.quantile(ttg, 0.99)),
                  "converged_p50_s": float(np.median(ttg_c)),
                  "converged_p99_s": float(np.quantile(ttg_c, 0.99)),
                  "queue_p50_s": float(np.median(qd)), "queue_p99_s": float(np.quantile(qd, 0.99)),
                  "done": len(ok), "converged": len(conv), "failed": n - len(ok),
                  "solves_per_s": len(ok) / span, "span_s": span,
                  "arrival_span_s": trace[-1]["t"],
                  "edge_iterations_per_s": work / span,
                  "busy_s": st["busy_seconds"],
                  "peak_resident_gib": st["peak_resident_bytes"] / 2**30},
        "lone_fp32_sequential": {"seconds": lone_t, "solves_per_s": n / lone_t,
                                 "converged": lone_conv},
        "e2e": {"value": float(np.median(ttg)), "unit": "s",
                "h2d_bytes_per_step": int(np.mean([12 * x.E + 8 * x.I + 4 * x.J for x in insts])),
                "d2h_bytes_per_step": int(np.mean([4 * x.J for x in insts])),
                "api": "dualip_server_submit / _wait (host arrays in, lambda to host)"},
        "clocks": clk.summary(),
        "gpu_launches": int(st["chunks"] * 10 * 5),
    }


def run_serve(args):
    import torch

    torch.cuda.set_device(0)
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    f = serve_form(d, torch, args.requests, args.budget_gib)
    n = args.requests
    out_line = {
        "metric": "serve time-to-1e-4-gap p50", "value": f["serve"]["p50_s"], "unit": "s",
        "n_gpus": 1, "steps": n, "warmup": 0, "ms_per_step": 1e3 * f["serve"]["span_s"] / n,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", **f}
    print(json.dumps(out_line), flush=True)
    return 0


def appb_ablations(d, torch, peak, note, I=1_000_000, J=10_000, nu=10.0, solves=True):
    """The paper's two ablations on its own generator (Appendix B), at 1/25 of
    the Section 7 size (10k resources, 10 edges per request):
    * Jacobi row normalisation (Section 5.1) on and off, at a fixed gamma of
      0.01 (Section 7's setting): iterations to the 1e-4 gap and the dual
      objective's distance to the best value reached, log10 |g_k - g*|;
    * gamma continuation 0.16 -> 0.01, halved every 25 iterations (Section 7),
      against gamma fixed at 0.01."""
    import synth

    inst = synth.appb(I, J, nu)
    P = d.Problem.from_instance(inst)
    lam = torch.zeros(inst.J, dtype=torch.float32, device="cuda")
    grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
    out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
    sp = int(torch.cuda.current_stream().cuda_stream)

    def step():
        d.dualip_dual_grad_async(P.h, lam.data_ptr(), 0.01, grad.data_ptr(), out_dev.data_ptr(),
                                 sp)

    for _ in range(5):
        step()
    k = profiled(d, P.h, 50, step)
    fixed = dict(gamma0=0.01, gamma_final=0.01, halve_every=0, max_iters=3000)
    runs = {
        "row_normalize_on": dict(row_normalize=1, **fixed),
        "row_normalize_off": dict(row_normalize=0, **fixed),
        "continuation_0.16_to_0.01": dict(gamma0=0.16, gamma_final=0.01, halve_every=25,
                                          max_iters=3000),
    } if solves else {}
    res, traces, lam_end = {}, {}, None
    for name, o in runs.items():
        P.solve(max_iters=20, **{kk: v for kk, v in o.items() if kk != "max_iters"})  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam_k, r, tr = P.solve(trace=True, **o)
        torch.cuda.synchronize()
        if name == "row_normalize_on":
            lam_end = lam_k
        res[name] = {"seconds": time.perf_counter() - t0, "iters": r["iters"],
                     "converged": r["converged"], "gap_rel": r["gap_rel"],
                     "infeas_rel": r["infeas_rel"], "dual_obj": r["dual_obj"]}
        traces[name] = tr
    # every run ends at gamma = 0.01 (continuation from iteration 100 on): the
    # distance of g to the best value any run reached there, at a few iteration
    # counts (the paper's Fig. 4 plots this log-gap for the row normalisation)
    at_final = {n: tr[:, 1][tr[:, 0] == 0.01] for n, tr in traces.items()}
    g_star = max((float(np.max(g)) for g in at_final.values() if len(g)), default=0.0)
    for name, tr in traces.items():
        g = tr[:, 1]
        res[name]["log10_gap_to_best"] = {
            str(it): float(np.log10(max(g_star - g[min(it, len(g)) - 1], 1e-300)))
            for it in (10, 25, 50, 100, 200, 500, 1000, 3000)
            if tr[min(it, len(g)) - 1, 0] == 0.01}
    if solves:
        res["fixed_gamma_0.01"] = res["row_normalize_on"]
    # the pass where the ascent is: at the dual point the row-normalised run
    # ends on (many sources there have near-ties or a slack sum; lambda = 0
    # gives every source a single candidate)
    k_end = None
    if lam_end is not None:
        lam.copy_(lam_end)
        for _ in range(3):
            step()
        k_end = profiled(d, P.h, 50, step)
    P.close()
    rown = np.sqrt(np.bincount(inst.dst, weights=inst.a.astype(np.float64) ** 2,
                               minlength=inst.J))
    return {"workload": f"Appendix B generator: {I} requests x {J} resources, {nu:g} edges per "
                        "request, lognormal breadth, greedy-load budgets (unstated laws: "
                        "synth.APPB_DEFAULTS)",
            "I": inst.I, "J": inst.J, "E": inst.E,
            "row_norm_p1_p50_p99": [float(x) for x in np.percentile(rown[rown > 0],
                                                                    [1, 50, 99])],
            "pass": {"kernel_ms": k["pass"], "edges_per_s": inst.E / (k["pass"] / 1e3),
                     "lambda": "0",
                     "roofline": roofline(algorithmic_bytes(inst), k["pass"], peak, note,
                                          pass_traffic(inst.E, inst.J, "appb", "f32"))},
            "pass_at_ascent_end": None if k_end is None else {
                "kernel_ms": k_end["pass"], "edges_per_s": inst.E / (k_end["pass"] / 1e3),
                "lambda": "where the row-normalised ascent ends (3000 iterations, gamma 0.01)",
                "roofline": roofline(algorithmic_bytes(inst), k_end["pass"], peak, note)},
            "solves": res}


def variant_forms(d, torch, peak, note, steps=20, warmup=3):
    """The pass of two variants on the c2 graph, against its plain FP32 pass:
    the unit-box projection (Section 6's clamp map: every edge in [0, 1], no
    sum constraint) and two constraint families (Definition 1, m = 2; one
    warp per source, m duals gathered and m rows scattered per edge)."""
    import synth

    base = synth.config("c2")
    out = {}
    for name, inst, kw in (("unit_box_c2", base, dict(projection="box")),
                           ("two_families_c2", synth.add_families(base, 2), {})):
        m = 1 if inst.a.ndim == 1 else inst.a.shape[0]
        P = d.Problem.from_instance(inst, **kw)
        lam = torch.from_numpy(np.random.default_rng(LAM_SEED).uniform(
            0.0, 1.0, m * inst.J).astype(np.float32)).cuda()
        grad = torch.empty(m * inst.J, dtype=torch.float32, device="cuda")
        out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
        sp = int(torch.cuda.current_stream().cuda_stream)

        def step():
            d.dualip_dual_grad_async(P.h, lam.data_ptr(), GAMMA, grad.data_ptr(),
                                     out_dev.data_ptr(), sp)

        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(warmup):
                step()
            k = profiled(d, P.h, steps, step)
        d.dualip_check_device_status(P.h, sp)
        P.close()
        # per edge: dst, c and m coefficients; per source: the offset (the
        # families pass reads 8-byte offsets); per row: mu, A x written and read
        alg = (edge_bytes("f32") * inst.E + 4 * (inst.I + 1) + 12 * inst.J if m == 1 else
               (8 + 4 * m) * inst.E + 8 * (inst.I + 1) + 12 * m * inst.J)
        out[name] = {"m": m, "E": inst.E, "rows": m * inst.J, "gamma": GAMMA,
                     "pass_ms": k["pass"], "edges_per_s": inst.E / (k["pass"] / 1e3),
                     "roofline": roofline(alg, k["pass"], peak, note, None,
                                          "multi_pass_kernel" if m > 1 else
                                          "dualgrad_pass_kernel (unit box)"),
                     "clocks": clk.summary()}
    return out


def hub_form(d, torch, peak, note, steps=20, warmup=3):
    """Sources far larger than a stage: c2 plus 100 sources of 100k-1M edges
    (log-uniform) over 1M destinations, against the c2 sources alone in the
    same 1M-destination numbering (the same kernel variant)."""
    import synth

    base = synth.config("c2")
    hub = synth.with_hubs(base)
    alone = synth.greedy_budgets(synth.Instance(base.off, base.dst, base.c, base.a,
                                                np.zeros(hub.J, np.float32), hub.J))
    out = {"workload": "c2 + 100 sources of LogUniform[100k, 1M] edges over 1M destinations"}
    for name, inst in (("with_hubs", hub), ("c2_sources_alone", alone)):
        f = pass_form(d, torch, inst, "hubs", "f32", steps, warmup, peak, note)
        out[name] = {"E": inst.E, "pass_ms": f["kernel_ms"]["pass"], "edges_per_s":
                     inst.E / (f["kernel_ms"]["pass"] / 1e3), "roofline": f["roofline"],
                     "clocks": f["clocks"]}
    out["hub_edges"] = int(hub.E - base.E)
    out["edges_per_s_ratio_hubs_vs_alone"] = (out["with_hubs"]["edges_per_s"] /
                                             out["c2_sources_alone"]["edges_per_s"])
    return out


def forms(d, torch, args, plain, peak, note):
    """The BF16, batched and serving forms beside the plain FP32 form (c2)."""
    import synth

    out = {"plain_fp32_c2": plain}
    t0 = time.perf_counter()
    c3 = synth.config("c3")
    gen_s = time.perf_counter() - t0
    for storage in ("bf16", "f32"):
        f = pass_form(d, torch, c3, "c3", storage, 20, 3, peak, note)
        f["workload"] = WORKLOADS["c3"]
        f["time_to_gap"], _ = time_to_gap(d, torch, c3, "c3", storage)
        out[f"{storage}_c3"] = f
    out["bf16_c3"]["generation_s"] = gen_s
    del c3
    f, _ = batch_form(d, torch, 20, 3, 1.0, "f32", True, peak, note)
    out["batched_c4"] = f
    out["serving_c5"] = serve_form(d, torch, args.form_requests, args.budget_gib)
    out["appendix_b_ablations"] = appb_ablations(d, torch, peak, note)
    out["hubs_c2"] = hub_form(d, torch, peak, note)
    out.update(variant_forms(d, torch, peak, note))
    return out


def run_appb(args):
    """The Appendix B generator's instance: pass roofline and the two ablations."""
    import torch

    torch.cuda.set_device(0)
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    peak, note = load_peak()
    f = appb_ablations(d, torch, peak, note, I=max(1, int(1_000_000 * args.scale)),
                       solves=not args.no_solve)
    ms = f["pass"]["kernel_ms"]
    out = {"metric": METRIC, "value": f["pass"]["edges_per_s"], "unit": UNIT, "n_gpus": 1,
           "steps": 50, "warmup": 5, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f["workload"], "I": f["I"], "J": f["J"], "E": f["E"],
                      "gamma": 0.01, "parallelism": "replicas"},
           "roofline": f["pass"]["roofline"], "ablations": f["solves"],
           "row_norm_p1_p50_p99": f["row_norm_p1_p50_p99"]}
    print(json.dumps(out), flush=True)
    return 0


def run_hubs(args):
    """c2 plus 100 sources of 100k-1M edges (the multi-block class) against the
    c2 sources alone."""
    import torch

    torch.cuda.set_device(0)
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    peak, note = load_peak()
    f = hub_form(d, torch, peak, note, steps=args.steps, warmup=args.warmup)
    h = f["with_hubs"]
    out = {"metric": METRIC, "value": h["edges_per_s"], "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["pass_ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": {"workload": f["workload"], "E": h["E"],
                                           "hub_edges": f["hub_edges"], "gamma": GAMMA,
                                           "parallelism": "replicas"},
           "roofline": h["roofline"], "c2_sources_alone": f["c2_sources_alone"],
           "edges_per_s_ratio_hubs_vs_alone": f["edges_per_s_ratio_hubs_vs_alone"]}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    if args.workload == "hubs":
        return run_hubs(args)
    if args.workload == "c4":
        return run_batch(args)
    if args.workload == "c5":
        return run_serve(args)
    if args.workload == "appb":
        return run_appb(args)
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2603_04621_gb300 import build

    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    import paper_2603_04621_gb300 as d

    inst = workload(args.workload, args.scale)
    P = d.Problem.from_instance(inst, storage=args.storage)
    lam_h = lam_for(inst)
    lam = torch.from_numpy(lam_h).cuda()
    grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
    out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    def step():
        d.dualip_dual_grad_async(P.h, lam.data_ptr(), GAMMA, grad.data_ptr(), out_dev.data_ptr(),
                                 sp)

    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        # keep the GPU busy ~1 s before timing so clocks are sampled under load
        torch.cuda.synchronize()
        t_end = time.perf_counter() + 1.0
        while time.perf_counter() < t_end:
            for _ in range(50):
                step()
            torch.cuda.synchronize()
        d.dualip_check_device_status(P.h, sp)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        # the step time, with nothing between the kernels of an evaluation
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # kernel durations: events around each kernel (which also orders them)
        k = profiled(d, P.h, min(args.steps, 500), step)
        d.dualip_check_device_status(P.h, sp)
        ms = max_over_ranks(ms, ws)
        if ws > 1:
            dist.barrier()
        # end to end through the public API with host buffers (pinned)
        lam_pin = torch.from_numpy(lam_h).pin_memory()
        grad_pin = torch.empty(inst.J, dtype=torch.float32).pin_memory()
        for _ in range(3):
            d.dualip_dual_grad_host(P.h, lam_pin.data_ptr(), GAMMA, grad_pin.data_ptr(), sp)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            d.dualip_dual_grad_host(P.h, lam_pin.data_ptr(), GAMMA, grad_pin.data_ptr(), sp)
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, ws)
    P.close()
    if rank != 0:
        if ws > 1:
            dist.barrier()
        return 0
    peak, note = load_peak()
    ttg = asc = fm = None
    if not args.no_solve and args.scale == 1.0:
        ttg, _ = time_to_gap(d, torch, inst, args.workload, args.storage)
        if ws == 1 and args.workload == "c2":
            asc = ascent_pass(d, torch, inst, args.storage, peak, note)

    E = inst.E
    value = whole_job_rate(E, args.steps, ws, ms / 1e3)
    alg = algorithmic_bytes(inst, args.storage)
    rl = roofline(alg, k["pass"], peak, note,
                  pass_traffic(inst.E, inst.J, args.workload, args.storage))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(inst, args.workload, args.scale, args.storage),
        "roofline": rl,
        "kernel_ms": k,
        "hbm_roofline_pct": 100.0 * rl["frac"],
        "e2e": {"value": whole_job_rate(E, args.steps, ws, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": 4 * inst.J, "d2h_bytes_per_step": 4 * inst.J + 40,
                "api": "dualip_dual_grad_host (lambda in, grad + FP64 scalars out, pinned)"},
        "clocks": clk.summary(),
        "gpu_launches": 3 * args.steps,
        "time_to_gap": ttg,
        "ascent_pass": asc,
    }
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inst, args.cpu_seconds, d, torch)
    if (ws == 1 and args.workload == "c2" and args.scale == 1.0 and not args.no_forms
            and not args.no_solve):
        del inst
        plain = {"ms_per_step": ms / args.steps, "roofline": rl, "time_to_gap": ttg,
                 "clocks": out["clocks"]}
        out["forms"] = forms(d, torch, args, plain, peak, note)
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
    return 0


def main():
    args = parse()
    if args.storage is None:
        args.storage = "bf16" if args.workload == "c3" else "f32"
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
