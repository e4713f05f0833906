#!/usr/bin/env python
"""Throughput of the DG rainfall shallow-water stepper on GB300.

Default workload: the coastal wet/dry configuration (seeded jittered Delaunay mesh of ~250k
triangles on 400 km x 300 km, p = 1, SSP(2,2), Roe flux, Manning friction, moving parametric rain,
tide on the open boundary).  A step is one SSP-RK step of the whole mesh: every stage runs the
stage kernel (edge fluxes, area integrals, sources, stage combination, positive-depth operator,
ledger).  ``--workload graded`` (2M triangles, p = 2, SSP(3,3), pressure set-up) and
``--workload hurricane`` (8M triangles, hourly gridded rain) measure the same way.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]

Metric: DOF-updates per second (3 (p+1)(p+2)/2 DOF per triangle, one update per step), FP32-mixed
path; the FP64 path is timed on the same workload and reported beside it.  L2 is flushed (a
256 MiB write) between timed steps, outside the events that time them.  On the coastal workload the
line also carries the batched ensemble (64 scenarios of 20k-400k triangles): scenario-steps/s,
against the same scenarios run one by one on the FP64 path.  With N > 1 (torchrun) each rank runs
an independent replica (the mesh is not sharded; ensemble scenarios are dealt to ranks): value =
all ranks' DOF-updates / the slowest rank's time.  Prints one JSON line on rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per SSP-RK step, FP32-mixed vs FP64, 1 GB300; ensemble steps/s"
UNIT = "DOF-updates/s"
L2_FLUSH_BYTES = 256 << 20
REASONS = ["sw_power_cap", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="0: the workload's default (2000, 1000, 2000)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["coastal", "graded", "hurricane", "basin"], default="coastal",
                    help="coastal 250k p=1 (default); graded 2M p=2; hurricane 8M p=1; basin 400 p=1 (launch-bound: "
                         "CUDA graphs against direct launches)")
    ap.add_argument("--n-tri", type=int, default=0, help="0: the workload's own size")
    ap.add_argument("--subsample-steps", type=int, default=1000, help="graded: steps of the 20k oracle comparison")
    ap.add_argument("--fp64-steps", type=int, default=0, help="0: max(10, min(50, steps // 100))")
    ap.add_argument("--e2e-steps", type=int, default=0, help="0: min(steps, 40)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch", default="", help="block,waves,split of the stage kernels (default: autotuned)")
    ap.add_argument("--fp64-launch", default="", help="block,waves,split of the FP64 leg (default: autotuned)")
    ap.add_argument("--limiter", action="store_true", help="apply the optional slope limiter after every stage")
    ap.add_argument("--sim-hours", type=float, default=0.0,
                    help="hurricane: time the whole run of this many simulated hours (steps from dt) in one "
                         "event pair instead of --steps (the state is several GB, far above L2)")
    ap.add_argument("--ens-scenarios", type=int, default=64, help="ensemble size (0: no ensemble measurement)")
    ap.add_argument("--ens-steps", type=int, default=500)
    ap.add_argument("--ens-fp64-steps", type=int, default=0,
                    help="FP64 steps timed per scenario (0: all --ens-steps steps, no scaling)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing ----
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if os.environ.get("DGSWE_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def whole_job(units_per_rank: float, seconds: float, ws: int, device=None):
    """(total units over all ranks, slowest rank's seconds): max over ranks of time, sum of work."""
    if ws == 1:
        return units_per_rank, seconds
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds, units_per_rank], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    usum = t[1:].clone()
    dist.all_reduce(usum, op=dist.ReduceOp.SUM)
    return float(usum.item()), float(tmax.item())


# ------------------------------------------------------------------------------ clocks ----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"dgswe_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active," + ",".join(
            f"clocks_event_reasons.{r}" for r in REASONS)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        rows = []
        if os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 3 + len(REASONS):
                    try:
                        rows.append(parts)
                    except ValueError:
                        pass
            os.unlink(self.path)
        if not rows:  # timed region shorter than one sample: take one now
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", "--query-gpu=clocks.sm,clocks.max.sm",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
                sm, mx = [float(v) for v in out.stdout.strip().split(",")[:2]]
                return {"sm_mhz": sm, "sm_max_mhz": mx, "reasons": [], "samples": 0}
            except Exception:
                return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({REASONS[k] for r in rows for k in range(len(REASONS)) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------ roofline ----
def step_bytes_per_element(precision: str, p: int) -> float:
    """Algorithmic bytes per element and SSP-RK step, the count of the hot-path scope table: per
    step the state is read three times and written twice (5 x 40 B mixed, 5 x 72 B FP64 at p = 1)
    and the static data is read twice (2 x ~100 B mixed, 2 x ~160 B FP64): 400 B mixed, 680 B
    FP64 at p = 1; p = 2 moves twice as many.  Neighbour records are L2 hits and not counted."""
    return (400.0 if precision == "mixed" else 680.0) * (2.0 if p == 2 else 1.0)


FORM_KERNEL = {0: "stage_kernel (fused)", 1: "edge_kernel + stage_kernel (split)",
               2: "tile_kernel (instantiation specialised to the run's features where one covers them)"}
FORM_PROFILE = {0: "stage_kernel", 1: "stage_kernel", 2: "tile_kernel"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# -------------------------------------------------------------------------- CPU oracle ----
def time_oracle(w, budget_s: float, steps: int | None = None):
    """The FP64 CPU oracle as it stands, single thread, on workload w: (DOF-updates/s, steps, s)."""
    import oracle as O

    o = O.from_workload(w)
    if steps is None:
        t0 = time.perf_counter()
        o.step(1)
        t1 = time.perf_counter() - t0
        steps = max(1, int(budget_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return w.dof * steps / dt, steps, dt


def reference_arm(args, ws, rank):
    """--impl reference: the oracle timed on the host cores, K steps after W, each step one SSP
    step of a mesh of the same workload family sized so the whole run stays within a few
    minutes."""
    if rank != 0:
        return
    from paper_2307_14302_gb300 import workloads as W

    def family(n):
        if args.workload == "coastal":
            return W.coastal_c2(n_tri=n, seed=2)
        if args.workload == "graded":
            return W.graded_c3(n_tri=n)
        if args.workload == "basin":
            return W.basin_c1()
        return W.hurricane_c5(n_tri=n)

    full = args.n_tri or {"coastal": 250_000, "graded": 2_000_000, "hurricane": 8_000_000,
                          "basin": 400}[args.workload]
    # element-step rate of the oracle, from a small calibration mesh
    cal = family(4000)
    rate, _, _ = time_oracle(cal, 0.5)
    elem_rate = rate / (cal.dof / cal.mesh.n_tri)
    budget = 150.0
    n_tri = int(max(2000, min(full, budget * elem_rate / max(1, args.steps + args.warmup))))
    w = family(n_tri)
    import oracle as O

    o = O.from_workload(w)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = w.dof * args.steps / dt
    ssp = "SSP(2,2)" if w.p == 1 else "SSP(3,3)"
    sample = (f"{args.steps} {ssp} steps of the {args.workload} family at {w.mesh.n_tri} triangles "
              f"(the {full}-triangle workload scaled to fit the run budget)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}-{full // 1000}k-p{w.p}", "elements_timed": w.mesh.n_tri, "p": w.p,
                   "ssp": ssp, "flux": "Roe", "impl": "FP64 CPU oracle, single thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------------------- ours ----
WORKLOADS = {
    # name: (generator, default timed steps, ncu summary of its stage kernel)
    "basin": ("basin_c1", 2000, None),
    "coastal": ("coastal_c2", 2000, "stage_kernel_mixed_p1_coastal.md"),
    "graded": ("graded_c3", 1000, "stage_kernel_mixed_p2_graded.md"),
    "hurricane": ("hurricane_c5", 2000, "stage_kernel_mixed_p1_hurricane.md"),
}


def fixed_launch(args, spec=None):
    """Solver keyword arguments for --launch block,waves,split (empty: autotune) and --limiter."""
    spec = args.launch if spec is None else spec
    kw = {"limiter": True} if args.limiter else {}
    if not spec:
        return kw
    block, waves, split = (int(v) for v in spec.split(","))
    kw.update(block=block, waves=waves, split=split)
    return kw


def make_workload(args):
    from paper_2307_14302_gb300 import workloads as W

    gen = getattr(W, WORKLOADS[args.workload][0])
    if args.workload == "coastal":
        return gen(n_tri=args.n_tri, seed=2, steps=args.steps)
    if args.workload == "graded":
        return gen(n_tri=args.n_tri or 2_000_000, steps=args.steps)
    if args.workload == "basin":
        return gen()
    return gen(n_tri=args.n_tri or 8_000_000)


def basin_arm(args, ws, rank, local):
    """The 400-triangle basin fits in L2 and is bound by launch latency: whole runs of K steps
    timed with graph replay (the library default) and with every stage launched directly."""
    import torch

    from paper_2307_14302_gb300 import dgswe as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    w = make_workload(args)
    out = {}
    for mode in ("graphs", "direct"):
        s = D.from_workload(w, precision=D.MIXED, stream=stream.cuda_stream)
        s.set_graphs(mode == "graphs")
        s.step(max(args.warmup, 3))
        s.sync()
        l0 = s.launch_count()
        barrier(ws)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            a.record(stream)
            s.step(args.steps)
            b.record(stream)
            torch.cuda.synchronize(dev)
        t = a.elapsed_time(b) / 1e3
        barrier(ws)
        units, tmax = whole_job(w.dof * args.steps, t, ws, dev)
        out[mode] = {"value": units / tmax, "unit": UNIT, "ms_per_step": 1e3 * tmax / args.steps,
                     "launches": s.launch_count() - l0, "clocks": clk.summary(), "launch": s.launch()}
        led = s.ledger()
        s.close()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, n, secs = time_oracle(w, min(args.cpu_seconds, 5.0))
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} SSP(2,2) steps of the same 400-triangle basin, FP64, one thread ({secs:.1f} s)"}
    if rank == 0:
        g = out["graphs"]
        block, waves, split = g["launch"]
        line = {
            "metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": g["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "elements": w.mesh.n_tri, "p": 1, "dof": w.dof, "ssp": "SSP(2,2)",
                       "flux": "Roe", "l2": "whole problem L2-resident (launch-bound case, not flushed)",
                       "parallelism": f"replicas x{ws}", "launch": {"block": block, "waves": waves, "split": split},
                       "mass_balance_rel_err": led["rel_err"]},
            "roofline": None,
            "roofline_note": "launch-bound: 400 elements per launch, no HBM traffic to speak of",
            "cpu_baseline": cpu,
            "e2e": None,
            "gpu_launches": g["launches"],
            "clocks": g["clocks"],
            "direct_launches": {k: out["direct"][k] for k in ("value", "unit", "ms_per_step", "launches")},
            "graph_speedup": out["direct"]["ms_per_step"] / g["ms_per_step"],
        }
        print(json.dumps(line), flush=True)


def our_arm(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2307_14302_gb300 import dgswe as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a dedicated stream: the library enqueues on it, and the flush and the timing events too
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    w = make_workload(args)
    E = w.mesh.n_tri
    p = w.p
    np_ = (p + 1) * (p + 2) // 2
    stages = 2 if p == 1 else 3
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)

    def timed_steps(solver, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            solver.step(1)
            b.record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3

    # ---- FP32-mixed path (headline)
    s = D.from_workload(w, precision=D.MIXED, stream=stream.cuda_stream, **fixed_launch(args))
    s.step(max(args.warmup, 3))
    s.sync()
    launches0 = s.launch_count()
    barrier(ws)
    torch.cuda.synchronize(dev)
    if args.sim_hours > 0:
        args.steps = int(math.ceil(args.sim_hours * 3600.0 / s.dt()))
    with ClockSampler(local) as clk:
        if args.sim_hours > 0:
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            s.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            t_mixed = ev0.elapsed_time(ev1) / 1e3
        else:
            t_mixed = timed_steps(s, args.steps)
    barrier(ws)
    launches = s.launch_count() - launches0
    s.sync()
    led = s.ledger()
    block, waves, split = s.launch()
    units, t_max = whole_job(w.dof * args.steps, t_mixed, ws, dev)
    value = units / t_max
    clocks = clk.summary()

    # roofline of the stage kernel: algorithmic bytes per launch (scope-table count per element and
    # step, over the stages) / average stage time measured with the events above
    bytes_per_launch = E * step_bytes_per_element("mixed", p) / stages
    launch_s = t_mixed / (args.steps * stages)
    peak, peak_kind = load_peaks()
    achieved = bytes_per_launch / launch_s / 1e9
    summary = f"{FORM_PROFILE[split]}_mixed_p{p}_{args.workload}.md"
    traffic = profiled_traffic(summary, E, split)

    # ---- end to end through the public API, the state crossing the host link both ways every
    # step: each step's input state comes in from pinned host memory and the previous step's
    # result goes out to pinned host memory in one dgswe_exchange_state call, then the step; the
    # last step's result is read after the loop, inside the timed region
    k_e2e = args.e2e_steps or min(args.steps, 40 if E < 1_000_000 else 10)
    zi, xi, yi = (torch.empty((np_, E), dtype=torch.float64).pin_memory().numpy() for _ in range(3))
    zo, xo, yo = (torch.empty((np_, E), dtype=torch.float64).pin_memory().numpy() for _ in range(3))
    s.state_arrays(zi, xi, yi)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        s.exchange(zi, xi, yi, zo, xo, yo)
        s.step(1)
    s.state_arrays(zo, xo, yo)
    t_e2e = time.perf_counter() - t0
    units_e, t_e = whole_job(w.dof * k_e2e, t_e2e, ws, dev)
    e2e = {"value": units_e / t_e, "unit": UNIT, "h2d_bytes_per_step": int(zi.nbytes * 3),
           "d2h_bytes_per_step": int(zo.nbytes * 3), "steps": k_e2e,
           "calls": "per step dgswe_exchange_state (previous result out, this step's input in) and dgswe_step; "
                    "one dgswe_get_state after the last step"}
    s.close()
    del zi, xi, yi, zo, xo, yo

    # ---- FP64 path on the same workload
    k64 = args.fp64_steps or max(10, min(50, args.steps // 100))
    s64 = D.from_workload(w, precision=D.FP64, stream=stream.cuda_stream, **fixed_launch(args, args.fp64_launch))
    s64.step(3)
    s64.sync()
    t64 = timed_steps(s64, k64)
    units64, t64m = whole_job(w.dof * k64, t64, ws, dev)
    b64, w64, sp64 = s64.launch()
    fp64 = {"value": units64 / t64m, "unit": UNIT, "steps": k64, "ms_per_step": 1e3 * t64 / k64,
            "mixed_speedup": value / (units64 / t64m), "launch": {"block": b64, "waves": w64, "split": sp64}}
    # FP64 arithmetic roofline: FP64 FLOPs per element and stage of the launch shape in use (from
    # the committed ncu summary of the FP64 kernels, hash-checked), over the measured time
    fpe = profiled_fp64_flops(sp64) if p == 1 else None
    if fpe is not None:
        ach = fpe * E * stages * k64 / t64 / 1e12
        fp64["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP64_PEAK_TFLOPS, "peak_source": "nominal GB300 FP64 rate (recipe table)",
                            "flops_per_element_stage": fpe}
    s64.close()

    ensemble = None
    if args.workload == "coastal" and args.ens_scenarios > 0:
        ensemble = ensemble_measure(args, ws, rank, dev, stream, flush)
    subsample = None
    if args.workload == "graded" and rank == 0 and args.subsample_steps > 0:
        subsample = graded_subsample_error(args, stream)

    ssp = "SSP(2,2)" if stages == 2 else "SSP(3,3)"
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, n, secs = time_oracle(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} {ssp} steps of the same {E}-triangle workload, FP64, one thread ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "elements": E, "nodes": w.mesh.n_nodes, "p": p, "dof": w.dof,
                       "ssp": ssp, "flux": "Roe", "precision": "FP32 bulk, float-float means, FP64 depth test",
                       "l2": ("inputs larger than L2, whole run timed in one event pair" if args.sim_hours > 0
                              else "flushed (256 MiB write) between timed steps"), "parallelism": f"replicas x{ws}",
                       "launch": {"block": block, "waves": waves, "split": split}, "dt_s": s_dt(led),
                       "simulated_s": led["t"], "mass_balance_rel_err": led["rel_err"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind, "kernel": f"{FORM_KERNEL[split]}, p={p}, Roe, mixed",
                         "bytes_per_launch": bytes_per_launch,
                         "bytes_model": f"{step_bytes_per_element('mixed', p):.0f} B per element and step "
                                        f"(scope table) over {stages} stages",
                         "traffic_source": summary if traffic is not None else None,
                         "avg_launch_us": 1e6 * launch_s},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64": fp64,
        }
        if ensemble is not None:
            line["ensemble"] = ensemble
        if subsample is not None:
            line["subsample_vs_oracle"] = subsample
        print(json.dumps(line), flush=True)


def graded_subsample_error(args, stream):
    """Mixed path against the FP64 oracle on the graded family's 20k-triangle subsample."""
    import numpy as np

    import oracle as O
    from paper_2307_14302_gb300 import dgswe as D
    from paper_2307_14302_gb300 import workloads as W

    w = W.graded_c3(n_tri=20_000, steps=args.subsample_steps)
    ref = O.from_workload(w)
    dt = ref.cfl_dt(w.cfl)
    ref.set_dt(dt)
    dev = D.from_workload(w, precision=D.MIXED, dt=dt, stream=stream.cuda_stream)
    dev64 = D.from_workload(w, precision=D.FP64, dt=dt, stream=stream.cuda_stream)
    out = {"elements": w.mesh.n_tri, "checkpoints": []}
    done = 0
    for n in sorted({min(100, args.subsample_steps), args.subsample_steps}):
        dev.step(n - done)
        dev64.step(n - done)
        ref.step(n - done)
        dev.sync()
        dev64.sync()
        done = n
        got, got64, want = dev.state(), dev64.state(), ref.state()
        out["checkpoints"].append({
            "steps": n,
            "mixed_max_abs_err_zeta_m": float(np.abs(got[:, 0] - want[:, 0]).max()),
            "mixed_max_abs_err_q_m2s": float(np.abs(got[:, 1:] - want[:, 1:]).max()),
            "fp64_max_abs_err_zeta_m": float(np.abs(got64[:, 0] - want[:, 0]).max()),
            "fp64_max_abs_err_q_m2s": float(np.abs(got64[:, 1:] - want[:, 1:]).max()),
            "mass_balance_rel_err": dev.ledger()["rel_err"]})
    out["note"] = ("beyond the first flip of a binary wet/dry edge-closure decision the FP64 device path and the "
                   "oracle separate as well: compare the mixed error with the FP64 one at the same checkpoint")
    dev.close()
    dev64.close()
    return out


def deal_scenarios(sizes, ws):
    """Owner rank of each scenario (the library's dealing: largest first to the least-loaded rank)."""
    from paper_2307_14302_gb300.ensemble import deal_scenarios as deal

    return deal(sizes, ws)


def ensemble_measure(args, ws, rank, dev, stream, flush):
    """Batched ensemble: scenarios of the coastal family on meshes of log-uniform size in
    [20k, 400k] triangles, each with its own rain peak, track heading, Manning field and tidal
    phase, advanced together (one launch per stage over all scenarios, steps replayed from CUDA
    graphs).  Beside it: the same scenarios run one after another, FP32-mixed and plain FP64.
    Scenarios are dealt to ranks largest-first (each rank's own ensemble); the totals are the
    whole job's."""
    import numpy as np
    import torch

    from paper_2307_14302_gb300 import dgswe as D
    from paper_2307_14302_gb300 import workloads as W

    t_gen = time.perf_counter()
    all_w = W.ensemble_c4(n_scen=args.ens_scenarios, steps=args.ens_steps)
    t_gen = time.perf_counter() - t_gen
    owner = deal_scenarios([x.mesh.n_tri for x in all_w], ws)
    mine_idx = [i for i, r in enumerate(owner) if r == rank]
    mine = [all_w[i] for i in mine_idx]
    k = args.ens_steps

    def timed(fn):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / 1e3

    # members (mixed, each autotuned), each also timed solo over the same k steps
    members, solo = [], 0.0
    for w in mine:
        m = D.from_workload(w, precision=D.MIXED, stream=stream.cuda_stream)
        m.step(3)
        flush.zero_()
        solo += timed(lambda: m.step(k))
        members.append(m)
    ens = D.Ensemble(members, device=dev.index, stream=stream.cuda_stream)
    for m in members:
        m.close()
    ens.step(3)
    ens.sync()
    barrier(ws)
    flush.zero_()
    t_ens = timed(lambda: ens.step(k))
    barrier(ws)
    ens.sync()
    # every scenario's ledger gathered on rank 0 (host objects over the process group)
    from paper_2307_14302_gb300.ensemble import gather_results

    gathered = gather_results({i: (None, ens.ledger(j)) for j, i in enumerate(mine_idx)}, ws, rank)
    rel = max(abs(led["rel_err"]) for _, led in gathered) if gathered is not None else None
    block, waves, split = ens.launch()
    ens.close()

    # the same scenarios as sequential plain FP64 GPU runs (the FP64 path's launch form, autotuned)
    k64 = min(k, args.ens_fp64_steps) if args.ens_fp64_steps > 0 else k
    seq64 = 0.0
    for w in mine:
        s64 = D.from_workload(w, precision=D.FP64, stream=stream.cuda_stream)
        s64.step(2)
        flush.zero_()
        seq64 += timed(lambda: s64.step(k64)) * k / k64
        s64.close()

    dof = sum(w.dof for w in mine)
    n_tri = sum(w.mesh.n_tri for w in mine)
    units, t_max = whole_job(len(mine) * k, t_ens, ws, dev)
    dof_units, _ = whole_job(dof * k, t_ens, ws, dev)
    _, t_solo = whole_job(0.0, solo, ws, dev)
    _, t_seq64 = whole_job(0.0, seq64, ws, dev)
    n_all = len(all_w)
    return {
        "metric": "ensemble scenario-steps/s", "value": units / t_max, "unit": "scenario-steps/s",
        "dof_updates_per_s": dof_units / t_max, "steps": k, "scenarios": n_all,
        "elements_total": int(sum(w.mesh.n_tri for w in all_w)), "elements_rank0": n_tri,
        "ms_per_step": 1e3 * t_max / k,
        "sequential_mixed": {"value": n_all * k / t_solo, "unit": "scenario-steps/s",
                             "note": f"each scenario alone (autotuned), all {k} steps timed"},
        "sequential_fp64": {"value": n_all * k / t_seq64, "unit": "scenario-steps/s",
                            "note": (f"each scenario alone on the FP64 path, all {k} steps timed" if k64 == k else
                                     f"each scenario alone on the FP64 path, {k64} steps timed, scaled to {k}")},
        "speedup_vs_sequential_fp64": t_seq64 / t_max,
        "launch": {"block": block, "waves": waves, "split": split},
        "mass_balance_rel_err_max": rel, "mesh_generation_s": t_gen,
        "l2": "inputs larger than L2 (ensemble state and geometry > 1 GB)",
    }


def s_dt(led):
    return led["t"] / max(1, led["steps"])


def profiled_traffic(summary, n_elem, form=0):
    """DRAM bytes per stage launch from a committed ncu summary (dram__bytes_read.sum +
    dram__bytes_write.sum of one capture, scaled to n_elem), or None when the summary is missing
    or was taken on a different kernel source."""
    import re

    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    m_bpe = re.search(r"dram_bytes_per_element_launch:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bpe or m_hash.group(1) != kernel_hash():
        return None
    m_form = re.search(r"launch_form:\s*([0-9])", txt)
    if m_form and int(m_form.group(1)) != form:
        return None
    return float(m_bpe.group(1)) * n_elem


FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 rate of a GB300 (not in the measured peaks)


def profiled_fp64_flops(split):
    """FP64 FLOPs (2 per DFMA, 1 per DADD/DMUL) per element and stage of the FP64 p=1 path in the
    given launch form (split: edge kernel + element kernel; fused: stage kernel), from the committed
    ncu summary, or None when it is missing or was taken on a different kernel source."""
    import re

    path = os.path.join(ROOT, "profiles", "fp64_kernels_p1_coastal.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    key = "fp64_flops_per_element_stage_" + {0: "fused", 1: "split", 2: "tile"}[split]
    m = re.search(key + r":\s*([0-9.eE+]+)", txt)
    if not m_hash or not m or m_hash.group(1) != kernel_hash():
        return None
    return float(m.group(1))


def kernel_hash():
    import hashlib

    h = hashlib.sha256()
    for f in ("stage.cuh", "tile.cuh", "tile_spec.cu", "args.h", "layout.h"):
        h.update(open(os.path.join(ROOT, "paper_2307_14302_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def main(argv=None):
    args = parse_args(argv)
    if args.steps <= 0:
        args.steps = WORKLOADS[args.workload][1]
    if args.workload == "coastal" and args.n_tri <= 0 and args.impl == "ours":
        args.n_tri = 250_000
    ws, rank, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
    elif args.workload == "basin":
        basin_arm(args, ws, rank, local)
    else:
        our_arm(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
