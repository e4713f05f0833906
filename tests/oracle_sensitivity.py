"""Sensitivity of the FP64 oracle to a one-ulp change of its initial state.

Runs the oracle twice on the graded p = 2 family's 20k-triangle subsample (SSP(3,3), pressure
set-up, moving rain, tide, wet/dry), the second time with every modal coefficient of the initial
state moved by one ulp, and prints the largest differences of zeta and q between the two runs
every 50 steps up to 1000.  The method's binary wet/dry decisions (the edge closure, the dry flag)
amplify rounding-level differences; the numbers bound how closely any other implementation --
including the CUDA paths -- can follow the oracle over that horizon.  Test infrastructure: it
loads only the oracle.  About 3.5 minutes on one core.

    python tests/oracle_sensitivity.py [steps]
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
from paper_2307_14302_gb300 import workloads as W  # noqa: E402


def main(steps=1000, every=50):
    w = W.graded_c3(n_tri=20_000, steps=steps)
    a = O.from_workload(w)
    dt = a.cfl_dt(w.cfl)
    a.set_dt(dt)
    s0 = a.state()
    b = O.from_workload(w)
    b.set_dt(dt)
    a.set_state_modal(s0.copy())
    b.set_state_modal(np.nextafter(s0, np.inf))
    out, done = [], 0
    for n in range(every, steps + 1, every):
        a.step(n - done)
        b.step(n - done)
        done = n
        sa, sb = a.state(), b.state()
        rec = {"steps": n, "max_abs_dzeta_m": float(np.abs(sa[:, 0] - sb[:, 0]).max()),
               "max_abs_dq_m2s": float(np.abs(sa[:, 1:] - sb[:, 1:]).max()),
               "dry_flags_differ": int((a.dry() != b.dry()).sum())}
        out.append(rec)
        print(json.dumps(rec), flush=True)
    return out


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1000)
