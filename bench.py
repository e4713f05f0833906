#!/usr/bin/env python
"""Throughput of the DG rainfall shallow-water stepper on GB300.

Workload: the coastal wet/dry configuration (seeded jittered Delaunay mesh of ~250k triangles on
400 km x 300 km, p = 1, SSP(2,2), Roe flux, Manning friction, moving parametric rain, tide on the
open boundary).  A step is one SSP-RK step of the whole mesh: every stage runs the fused kernel
(edge fluxes, area integrals, sources, stage combination, positive-depth operator, ledger).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Metric: DOF-updates per second (3 (p+1)(p+2)/2 DOF per triangle, one update per step), FP32-mixed
path; the FP64 path is timed on the same workload and reported beside it.  L2 is flushed (a
256 MiB write) between timed steps, outside the events that time them.  With N > 1 (torchrun) each
rank runs an independent replica (the mesh is not sharded): value = all ranks' DOF-updates / the
slowest rank's time.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
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
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-tri", type=int, default=250_000)
    ap.add_argument("--fp64-steps", type=int, default=0, help="0: max(10, steps // 100)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="0: min(steps, 40)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
def stage_bytes_per_element(precision: str, p: int, rain_from_nodes: bool, nodes_per_elem: float):
    """Algorithmic DRAM bytes one stage launch moves per element: own record in and out, static
    geometry and connectivity, the step-initial record on stages > 0, rain node data.  Neighbour
    records are L2 hits (Hilbert-ordered mesh) and are not counted."""
    np_ = (p + 1) * (p + 2) // 2
    if precision == "mixed":
        rec = 16 * (4 if 3 * np_ + 7 <= 16 else 8)
        static = 16 + 48
        xy = 8
    else:
        rec = 16 * (8 if 3 * np_ + 4 <= 16 else 12)
        static = 16 + 80
        xy = 16
    rain = (16 + xy * nodes_per_elem) if rain_from_nodes else 0.0
    first = rec + static + rain + rec
    later = first + rec
    return first, later


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
    step of a same-family coastal mesh sized so the whole run stays within a few minutes."""
    if rank != 0:
        return
    from paper_2307_14302_gb300 import workloads as W

    # element-step rate of the oracle, from a small calibration mesh
    cal = W.coastal_c2(n_tri=4000, seed=2)
    rate, _, _ = time_oracle(cal, 0.5)
    elem_rate = rate / (cal.dof / cal.mesh.n_tri)
    budget = 150.0
    n_tri = int(max(2000, min(args.n_tri, budget * elem_rate / max(1, args.steps + args.warmup))))
    w = W.coastal_c2(n_tri=n_tri, seed=2)
    import oracle as O

    o = O.from_workload(w)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = w.dof * args.steps / dt
    sample = (f"{args.steps} SSP(2,2) steps of the coastal family at {w.mesh.n_tri} triangles "
              f"(the {args.n_tri}-triangle workload scaled to fit the run budget)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"coastal-{args.n_tri // 1000}k-p1", "elements_timed": w.mesh.n_tri, "p": 1,
                   "ssp": "SSP(2,2)", "flux": "Roe", "impl": "FP64 CPU oracle, single thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------------------- ours ----
def our_arm(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2307_14302_gb300 import dgswe as D
    from paper_2307_14302_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a dedicated stream: the library enqueues on it, and the flush and the timing events too
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    w = W.coastal_c2(n_tri=args.n_tri, seed=2, steps=args.steps)
    E = w.mesh.n_tri
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
    s = D.from_workload(w, precision=D.MIXED, stream=stream.cuda_stream)
    s.step(max(args.warmup, 3))
    s.sync()
    launches0 = s.launch_count()
    barrier(ws)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_mixed = timed_steps(s, args.steps)
    barrier(ws)
    launches = s.launch_count() - launches0
    s.sync()
    led = s.ledger()
    block, waves, split = s.launch()
    units, t_max = whole_job(w.dof * args.steps, t_mixed, ws, dev)
    value = units / t_max
    clocks = clk.summary()

    # roofline of the stage kernel: algorithmic bytes per launch / average launch duration
    nodes_per_elem = w.mesh.n_nodes / E
    b0, b1 = stage_bytes_per_element("mixed", 1, True, nodes_per_elem)
    bytes_per_launch = E * (b0 + b1) / 2
    stages = 2
    launch_s = t_mixed / (args.steps * stages)
    peak, peak_kind = load_peaks()
    achieved = bytes_per_launch / launch_s / 1e9
    traffic = profiled_traffic(E)

    # ---- end to end through the public API: state in from pinned host memory, one step,
    # state back to pinned host memory, every step
    k_e2e = args.e2e_steps or min(args.steps, 40)
    np_ = 3
    zi, xi, yi = (torch.empty((np_, E), dtype=torch.float64).pin_memory().numpy() for _ in range(3))
    zo, xo, yo = (torch.empty((np_, E), dtype=torch.float64).pin_memory().numpy() for _ in range(3))
    s.state_arrays(zi, xi, yi)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        s.load_state(zi, xi, yi)
        s.step(1)
        s.state_arrays(zo, xo, yo)
    t_e2e = time.perf_counter() - t0
    units_e, t_e = whole_job(w.dof * k_e2e, t_e2e, ws, dev)
    e2e = {"value": units_e / t_e, "unit": UNIT, "h2d_bytes_per_step": int(zi.nbytes * 3),
           "d2h_bytes_per_step": int(zo.nbytes * 3), "steps": k_e2e}
    s.close()

    # ---- FP64 path on the same workload
    k64 = args.fp64_steps or max(10, args.steps // 100)
    s64 = D.from_workload(w, precision=D.FP64, stream=stream.cuda_stream)
    s64.step(3)
    s64.sync()
    t64 = timed_steps(s64, k64)
    units64, t64m = whole_job(w.dof * k64, t64, ws, dev)
    fp64 = {"value": units64 / t64m, "unit": UNIT, "steps": k64, "ms_per_step": 1e3 * t64 / k64,
            "mixed_speedup": value / (units64 / t64m)}
    s64.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, n, secs = time_oracle(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} SSP(2,2) steps of the same {E}-triangle workload, FP64, one thread ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "elements": E, "nodes": w.mesh.n_nodes, "p": 1, "dof": w.dof,
                       "ssp": "SSP(2,2)", "flux": "Roe", "precision": "FP32 bulk, float-float means, FP64 depth test",
                       "l2": "flushed (256 MiB write) between timed steps", "parallelism": f"replicas x{ws}",
                       "launch": {"block": block, "waves": waves, "split": split}, "dt_s": s_dt(led),
                       "mass_balance_rel_err": led["rel_err"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind, "kernel": "stage_kernel<1,Roe,Mixed>",
                         "bytes_per_launch": bytes_per_launch, "avg_launch_us": 1e6 * launch_s},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64": fp64,
        }
        print(json.dumps(line), flush=True)


def s_dt(led):
    return led["t"] / max(1, led["steps"])


def profiled_traffic(n_elem):
    """DRAM bytes per stage launch from the committed ncu summary (dram__bytes_read.sum +
    dram__bytes_write.sum of one capture, scaled to n_elem), or None when the summary is missing
    or was taken on a different kernel source."""
    import re

    path = os.path.join(ROOT, "profiles", "stage_kernel_mixed_p1_coastal.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    m_bpe = re.search(r"dram_bytes_per_element_launch:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bpe or m_hash.group(1) != kernel_hash():
        return None
    return float(m_bpe.group(1)) * n_elem


def kernel_hash():
    import hashlib

    h = hashlib.sha256()
    for f in ("stage.cuh", "args.h", "layout.h"):
        h.update(open(os.path.join(ROOT, "paper_2307_14302_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def main(argv=None):
    args = parse_args(argv)
    ws, rank, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
    else:
        our_arm(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
