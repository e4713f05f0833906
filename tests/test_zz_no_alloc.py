"""The allocation-free volume entry point (dgswe_volume_sum_noalloc) against dgswe_volume.

Callers that cannot allocate device memory (all of it drawn from their own pool or caching
allocator, or loops that must not stall on cudaFree) get the same total water volume from this
entry point, which keeps its partial sums in a fixed device array.  Two calls in a row reuse that array; each must agree with
dgswe_volume on the same state within the mass-ledger tolerance (1e-12 relative).  This file is
collected last, and passes alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_2307_14302_gb300 import dgswe as D
from paper_2307_14302_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _areas(mesh):
    a, b, c = (mesh.xy[mesh.tri[:, k]] for k in range(3))
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_noalloc_volume_matches_dgswe_volume_on_two_calls(prec):
    import torch

    from paper_2307_14302_gb300 import build as B

    B.build()
    w = W.coastal_c2(n_tri=20_000, seed=17, steps=20)
    s = D.from_workload(w, precision=prec)
    dev = torch.device("cuda", 0)
    area = torch.tensor(_areas(w.mesh), dtype=torch.float64, device=dev)
    z, x, y = (torch.empty((s.np_, s.ne), dtype=torch.float64, device=dev) for _ in range(3))
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):
        s.step(10)
        s.state_device(z.data_ptr(), x.data_ptr(), y.data_ptr())
        s.sync()
        want = s.volume()
        D.volume_sum_noalloc(z[0].data_ptr(), area.data_ptr(), s.ne, out.data_ptr())
        torch.cuda.synchronize(dev)
        got = float(out.item())
        assert abs(got - want) <= 1e-12 * max(abs(want), 1.0), (call, got, want)
        out.fill_(float("nan"))


def test_noalloc_rejects_oversized_and_null_inputs():
    import torch

    dev = torch.device("cuda", 0)
    buf = torch.zeros(4, dtype=torch.float64, device=dev)
    with pytest.raises(D.DgsweError) as ei:
        D.volume_sum_noalloc(buf.data_ptr(), buf.data_ptr(), 16_777_217, buf.data_ptr())
    assert ei.value.code == -1 and "16777216" in str(ei.value)
    with pytest.raises(D.DgsweError):
        D.volume_sum_noalloc(0, buf.data_ptr(), 1, buf.data_ptr())
