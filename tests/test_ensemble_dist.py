"""Scenarios dealt to two ranks and gathered on rank 0 (gloo, CPU): each rank advances its share
of a small ensemble on the FP64 oracle, rank 0 gathers every scenario's final state and mass
ledger, and the gathered results equal a one-process run bit for bit."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 15


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workloads():
    from paper_2307_14302_gb300 import workloads as W

    return W.ensemble_c4(n_scen=5, lo=2000, hi=6000, seed=11, steps=STEPS)


def _oracle_runner(workloads, steps):
    import oracle as O

    out = []
    for w in workloads:
        o = O.from_workload(w)
        o.step(steps)
        out.append((o.state(), o.ledger()))
    return out


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2307_14302_gb300 import ensemble as EN

    dist.init_process_group("gloo")
    ws = _workloads()
    owner = EN.deal_scenarios([w.mesh.n_tri for w in ws], 2)
    got = EN.run_dealt(ws, STEPS, 2, rank, runner=_oracle_runner)
    q.put((rank, sum(1 for o in owner if o == rank), got))
    dist.barrier()
    dist.destroy_process_group()


def test_dealt_scenarios_gather_to_the_one_process_result():
    sys.path.insert(0, ROOT)
    from paper_2307_14302_gb300 import ensemble as EN

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(2):
        r, n_mine, got = q.get(timeout=300)
        out[r] = (n_mine, got)
    for p in ps:
        p.join(60)
    assert all(p.exitcode == 0 for p in ps)
    assert out[0][0] >= 1 and out[1][0] >= 1  # both ranks did work
    assert out[1][1] is None  # only rank 0 receives the gather
    gathered = out[0][1]
    single = EN.run_dealt(_workloads(), STEPS, 1, 0, runner=_oracle_runner)
    assert len(gathered) == len(single) == 5
    for (sg, lg), (ss, ls) in zip(gathered, single):
        assert np.isfinite(sg).all()
        assert np.array_equal(sg, ss)
        assert lg == ls
        assert lg["rel_err"] < 1e-12
