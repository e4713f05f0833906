"""The C-ABI boundary's memory paths: element records bound to caller-owned device memory
(dgswe_bind_device) and the state exchanged with page-locked host arrays (dgswe_load_state /
dgswe_get_state read and write them directly), each against the oracle or the staged path."""
import numpy as np
import pytest

import oracle as O
from paper_2307_14302_gb300 import dgswe as D
from paper_2307_14302_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14302_gb300 import build as B

    B.build()
    D.lib()


def _err_ok(got, want, prec):
    if prec == D.FP64:
        return max(np.abs(got[:, v] - want[:, v]).max() / max(1.0, np.abs(want[:, v]).max()) for v in range(3)) <= 1e-11
    return np.abs(got[:, 0] - want[:, 0]).max() <= 1e-4 and np.abs(got[:, 1:] - want[:, 1:]).max() <= 1e-4


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_records_in_torch_memory_step_like_the_oracle(prec):
    import torch

    w = W.coastal_c2(n_tri=6000, seed=21, steps=60)
    ref = O.from_workload(w)
    dt = ref.cfl_dt(w.cfl)
    ref.set_dt(dt)
    ref.step(60)
    dev = D.from_workload(w, precision=prec, dt=dt)
    dev.step(10)
    nbytes = dev.record_bytes()
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    dev.bind_device(buf.data_ptr(), nbytes)
    before = buf.clone()
    dev.step(50)
    dev.sync()
    torch.cuda.synchronize()
    assert not torch.equal(before, buf)  # the steps read and wrote the torch-owned memory
    assert _err_ok(dev.state(), ref.state(), prec)
    assert dev.ledger()["rel_err"] < 1e-12 and dev.ledger()["steps"] == 60
    # unbinding copies the state back into library memory, bit for bit
    s1 = dev.state()
    dev.bind_device(0, 0)
    buf.zero_()
    assert np.array_equal(dev.state(), s1)
    dev.step(1)
    dev.sync()
    # memory that is too small, unaligned or not on the device is refused
    big = torch.zeros(nbytes + 512, dtype=torch.uint8, device="cuda")
    for ptr, n in ((big.data_ptr(), nbytes - 256), (big.data_ptr() + 16, nbytes)):
        with pytest.raises(D.DgsweError) as ei:
            dev.bind_device(ptr, n)
        assert ei.value.code == -1
    host = np.zeros(nbytes, np.uint8)
    with pytest.raises(D.DgsweError):
        dev.bind_device(host.ctypes.data, nbytes)
    dev.close()


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_pinned_state_exchange_matches_the_staged_path(prec):
    import torch

    w = W.coastal_c2(n_tri=5000, seed=3, steps=20)
    a = D.from_workload(w, precision=prec, block=128, split=2)
    b = D.from_workload(w, precision=prec, dt=a.dt(), block=128, split=2)
    a.step(5)
    b.step(5)  # same time in both contexts
    z, x, y = a.state_arrays()  # pageable numpy arrays: the staged path
    pz, px, py = (torch.empty(z.shape, dtype=torch.float64).pin_memory().numpy() for _ in range(3))
    a.state_arrays(pz, px, py)  # page-locked: written by the unpacking kernel directly
    assert np.array_equal(pz, z) and np.array_equal(px, x) and np.array_equal(py, y)
    # the same state loaded through both paths steps to the same bits
    b.load_state(pz, px, py)
    a.load_state(z, x, y)
    for s in (a, b):
        s.step(7)
        s.sync()
    assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
@pytest.mark.parametrize("pinned", [True, False])
def test_exchange_equals_get_then_load(prec, pinned):
    """dgswe_exchange_state (state out, new state in, one call) gives the arrays dgswe_get_state
    gives and leaves the state dgswe_load_state leaves, bit for bit; the following steps agree
    bit for bit too.  Page-locked arrays take the one-pass kernel, pageable ones the two staged
    calls."""
    import torch

    w = W.coastal_c2(n_tri=5000, seed=7, steps=20)
    a = D.from_workload(w, precision=prec, block=128, split=2)
    b = D.from_workload(w, precision=prec, dt=a.dt(), block=128, split=2)
    a.step(6)
    b.step(6)
    c = D.from_workload(w, precision=prec, dt=a.dt(), block=128, split=2)
    c.step(3)
    new = c.state_arrays()  # another valid state of the same mesh
    c.close()

    def arrays(src=None):
        shape = new[0].shape
        if pinned:
            out = [torch.empty(shape, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
        else:
            out = [np.empty(shape) for _ in range(3)]
        if src is not None:
            for o, s_ in zip(out, src):
                o[...] = s_
        return out

    zi, xi, yi = arrays(new)
    zo, xo, yo = arrays()
    a.exchange(zi, xi, yi, zo, xo, yo)
    want = b.state_arrays()
    b.load_state(*new)
    for got, ref in zip((zo, xo, yo), want):
        assert np.array_equal(got, ref)
    assert np.array_equal(a.state(), b.state())
    assert np.array_equal(a.dry(), b.dry())
    for s in (a, b):
        s.step(5)
        s.sync()
    assert np.array_equal(a.state(), b.state())
    # a second exchange hands back what the first put in, advanced by the five steps
    zo2, xo2, yo2 = arrays()
    a.exchange(zi, xi, yi, zo2, xo2, yo2)
    assert np.array_equal(np.stack([zo2.T, xo2.T, yo2.T], axis=1), b.state())
    a.close()
    b.close()
