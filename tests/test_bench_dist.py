"""The benchmark's multi-rank aggregation (replicas: summed work over the slowest rank's time)
and its launch contract, exercised with the gloo backend on CPU at world size 2."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank), DGSWE_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench

    ws, r, local = bench.dist_init()
    units, secs = bench.whole_job(1000.0 * (rank + 1), 0.5 + rank, ws)
    bench.barrier(ws)
    q.put((r, units, secs))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_whole_job_sums_work_and_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    out = sorted(q.get(timeout=10) for _ in range(2))
    for r, units, secs in out:
        assert units == 3000.0 and secs == 1.5
    assert all(p.exitcode == 0 for p in ps)


def test_reference_arm_other_ranks_exit_without_work(tmp_path):
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()), DGSWE_BENCH_BACKEND="gloo")
    # rank 1 alone cannot rendezvous; the reference arm must return before any collective
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reference_arm(bench.parse_args(["--impl", "reference"]), 2, 1) is None


def test_ensemble_scenarios_are_dealt_to_every_rank_once():
    sys.path.insert(0, ROOT)
    import bench

    sizes = [400, 20, 300, 250, 90, 90, 60, 10]
    for ws in (1, 2, 3):
        owner = bench.deal_scenarios(sizes, ws)
        assert sorted(set(owner)) == list(range(ws))
        loads = [sum(s for s, o in zip(sizes, owner) if o == r) for r in range(ws)]
        assert max(loads) - min(loads) <= max(sizes)
    assert bench.deal_scenarios(sizes, 1) == [0] * len(sizes)
