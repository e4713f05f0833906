"""Scenario ensembles over several ranks (one GPU each).

The scenarios of a batched run are independent problems: they are dealt to the ranks (largest
first, each to the least-loaded rank), every rank advances its own scenarios as one ensemble
(one launch per Runge-Kutta stage over all of them), and rank 0 gathers the per-scenario mass
ledgers and final states on the host.  A scenario's mesh is never split, so ranks exchange
nothing while they step; the gather runs once, after the run.
"""
from __future__ import annotations

from typing import Callable, Sequence

from . import dgswe as D


def deal_scenarios(sizes: Sequence[int], ws: int) -> list[int]:
    """Owner rank of each scenario: largest first, each to the least-loaded rank (ties: lowest)."""
    load = [0] * ws
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(ws), key=lambda k: (load[k], k))
        load[r] += sizes[i]
        owner[i] = r
    return owner


def run_ensemble(workloads, steps: int, precision: int = D.MIXED, device: int = 0, stream=None):
    """Advance the workloads together as one ensemble on this rank's GPU; returns
    [(modal state [E, 3, Np], ledger dict)] in the order given."""
    members = [D.from_workload(w, precision=precision, device=device, stream=stream) for w in workloads]
    ens = D.Ensemble(members, device=device, stream=stream)
    for m in members:
        m.close()
    ens.step(steps)
    ens.sync()
    out = [(ens.state(i), ens.ledger(i)) for i in range(len(workloads))]
    ens.close()
    return out


def gather_results(local: dict, ws: int, rank: int):
    """Rank 0 receives every rank's {scenario index: result} and returns the results in scenario
    order; other ranks return None.  Host objects over torch.distributed (gloo or NCCL)."""
    if ws == 1:
        return [local[i] for i in sorted(local)]
    import torch.distributed as dist

    parts = [None] * ws if rank == 0 else None
    dist.gather_object(local, parts, dst=0)
    if rank != 0:
        return None
    merged = {}
    for p in parts:
        merged.update(p)
    return [merged[i] for i in sorted(merged)]


def run_dealt(workloads, steps: int, ws: int, rank: int, runner: Callable | None = None,
              with_states: bool = True):
    """Deal the workloads to ranks, run this rank's share with runner(workloads, steps) (default:
    run_ensemble on the GPU) and gather every scenario's (state, ledger) on rank 0, in the order of
    workloads.  With with_states False only the ledgers travel (state None)."""
    runner = runner or run_ensemble
    owner = deal_scenarios([w.mesh.n_tri for w in workloads], ws)
    mine = [i for i, r in enumerate(owner) if r == rank]
    res = runner([workloads[i] for i in mine], steps) if mine else []
    local = {i: ((s if with_states else None), led) for i, (s, led) in zip(mine, res)}
    return gather_results(local, ws, rank)
