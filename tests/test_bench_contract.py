"""The benchmark's reference arm (the FP64 CPU oracle timed on the host) prints one JSON line with
the keys the benchmark contract requires; runs on the CPU with a small mesh."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["coastal", "basin"])
def test_reference_arm_prints_one_contract_line(workload):
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "3",
           "--warmup", "1"]
    if workload == "coastal":
        cmd += ["--n-tri", "3000"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "DOF-updates/s"
    assert d["steps"] == 3 and d["warmup"] == 1 and d["higher_is_better"] is True
    for k in ("metric", "n_gpus", "ms_per_step", "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
