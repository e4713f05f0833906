"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Bars: FP64 device path within 1e-11 of the oracle (relative to the larger of the variable's
maximum magnitude and 1); mixed path within 1e-4 m in zeta and 1e-4 m^2/s in q; relative mass
balance within 1e-12 in both.  Inputs are the seeded workloads of
paper_2307_14302_gb300.workloads; dt is fixed by the oracle and passed to the device so both
integrate the same steps.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2307_14302_gb300 import dgswe as D
from paper_2307_14302_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14302_gb300 import build as B

    B.build()
    D.lib()


def _pair(w, steps, precision, flux=O.ROE, ssp=None, friction=O.MANNING, cf=0.0, block=0, waves=1, dt=None,
          limiter=False):
    ref = O.from_workload(w, flux=flux, ssp=ssp, friction=friction, cf=cf, dt=dt)
    if limiter:
        ref.set_limiter(True, 1.5, 0.0)
    dt = ref.cfl_dt(w.cfl) if dt is None else dt
    ref.set_dt(dt)
    ref.step(steps)
    dev = D.from_workload(w, precision=precision, flux=flux, ssp_stages=ssp, dt=dt, friction=friction, cf=cf,
                          block=block, waves=waves, limiter=limiter)
    dev.step(steps)
    dev.sync()
    return ref, dev


def _fp64_err(got, want):
    errs = []
    for v in range(3):
        scale = max(1.0, np.abs(want[:, v]).max())
        errs.append(np.abs(got[:, v] - want[:, v]).max() / scale)
    return max(errs)


def _mixed_err(got, want):
    return np.abs(got[:, 0] - want[:, 0]).max(), np.abs(got[:, 1:] - want[:, 1:]).max()


def _vertex(state, p):
    """Vertex values [E, 3, 3] of a modal state from the oracle's (pinned) basis."""
    V = []
    for (r, s) in ((-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0)):
        V.append(O.basis(p, r, s)[0])
    V = np.array(V)  # [3 vertices, Np]
    return np.einsum("evm,im->evi", state, V)


# ----------------------------------------------------------------------- basin (C1) ------
def test_fp64_basin_200_steps_matches_oracle():
    w = W.basin_c1()
    ref, dev = _pair(w, 200, D.FP64)
    assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL
    led = dev.ledger()
    assert led["rel_err"] < 1e-12 and led["steps"] == 200
    assert dev.dt() == O.from_workload(w).cfl_dt(w.cfl)  # the oracle's t = 0 step, passed through


def test_mixed_basin_200_steps_within_tolerance_and_exact_mass():
    w = W.basin_c1()
    ref, dev = _pair(w, 200, D.MIXED)
    ez, eq = _mixed_err(dev.state(), ref.state())
    assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    led = dev.ledger()
    assert led["rel_err"] < 1e-12, led
    lo = ref.ledger()
    assert abs(led["rain_in"] - lo["rain_in"]) / lo["rain_in"] < 1e-6


def test_device_cfl_dt_matches_oracle():
    w = W.basin_c1()
    ref = O.from_workload(w)
    for prec, tol in ((D.FP64, 1e-13), (D.MIXED, 1e-6)):
        dev = D.from_workload(w, precision=prec)
        assert abs(dev.dt() - ref.cfl_dt(w.cfl)) <= tol * dev.dt()


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_lake_at_rest_is_exact(prec):
    w = W.basin_c1(hump=False, rain=False)
    ref, dev = _pair(w, 200, prec)
    s = dev.state()
    assert np.abs(s).max() <= 1e-12
    w = W.basin_c1(hump=False, rain=True)
    ref, dev = _pair(w, 200, prec)
    v = _vertex(dev.state(), 1)
    t = dev.ledger()["t"]
    assert np.abs(v[:, 0] - w.rain_nodal[0] * t).max() < (1e-13 if prec == D.FP64 else 1e-7)
    assert np.abs(v[:, 1:]).max() < 1e-12


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_p2_ssp33_basin(prec):
    w = W.basin_c1()
    w.p = 2
    ref, dev = _pair(w, 100, prec, ssp=3)
    if prec == D.FP64:
        assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL
    else:
        ez, eq = _mixed_err(dev.state(), ref.state())
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_llf_flux(prec):
    w = W.basin_c1()
    ref, dev = _pair(w, 100, prec, flux=O.LLF)
    if prec == D.FP64:
        assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL
    else:
        ez, eq = _mixed_err(dev.state(), ref.state())
        assert ez <= MIXED_TOL and eq <= MIXED_TOL


def test_mirror_symmetric_dam_break_on_device():
    w = W.basin_c1(mirror=True)
    ref, dev = _pair(w, 200, D.FP64)
    assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL


# ------------------------------------------------------------- coastal wet/dry (C2) ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_coastal_wet_dry_small(prec):
    w = W.coastal_c2(n_tri=6000, seed=21, steps=200)
    ref, dev = _pair(w, 200, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
        assert np.array_equal(dev.dry(), ref.dry())
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    led = dev.ledger()
    assert led["rel_err"] < 1e-12, led
    assert led["bdry_in"] != 0.0


def test_coastal_without_rain_dries_like_the_oracle():
    w = W.coastal_c2(n_tri=4000, seed=9, steps=100)
    w.storm = None
    ref, dev = _pair(w, 100, D.FP64)
    assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL
    assert np.array_equal(dev.dry(), ref.dry())
    assert dev.dry().sum() > 100


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_coastal_full_size_short_run(prec):
    """The full 250k-triangle coastal workload in the benchmark's launch configuration
    (autotuned), 10 steps, every element compared."""
    w = W.coastal_c2()
    ref, dev = _pair(w, 10, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12


# ------------------------------------------------------------- graded p=2 (C3) ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_graded_p2_subsample_matches_oracle(prec):
    """The graded p=2 family on its 20k-triangle subsample (same generator, coarser sizing),
    SSP(3,3), pressure set-up, moving rain, tide: 100 steps, every element compared."""
    w = W.graded_c3(n_tri=20_000, steps=100)
    ref, dev = _pair(w, 100, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12
    assert 0 < dev.dry().sum() < w.mesh.n_tri


@pytest.mark.slow
def test_graded_full_size_two_steps():
    """The 2M-triangle graded p=2 workload in the benchmark's launch configuration, mixed path,
    two SSP(3,3) steps against the oracle on every element."""
    w = W.graded_c3()
    ref, dev = _pair(w, 2, D.MIXED)
    ez, eq = _mixed_err(dev.state(), ref.state())
    assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12


# ---------------------------------------------------------- hurricane basin (C5) ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_hurricane_family_small_matches_oracle(prec):
    """The hurricane family (hourly gridded rain on the 0.1 degree grid, 30% dry land, tide) on
    a 20k-triangle mesh of the same basin: 100 steps, every element compared."""
    w = W.hurricane_c5(n_tri=20_000)
    ref, dev = _pair(w, 100, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12


@pytest.mark.slow
def test_hurricane_full_size_two_steps():
    """The 8M-triangle hurricane workload, mixed path, benchmark launch configuration: two
    steps against the oracle on every element."""
    w = W.hurricane_c5()
    ref, dev = _pair(w, 2, D.MIXED)
    ez, eq = _mixed_err(dev.state(), ref.state())
    assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12


# ------------------------------------------------------------------ slope limiter ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
@pytest.mark.parametrize("case", ["basin", "coastal"])
def test_slope_limiter_matches_oracle(prec, case):
    """The optional Cockburn-Shu TVB minmod limiter (after each stage's positive-depth
    operator, then the operator again): dam break on the basin, and the coastal wet/dry
    family; state against the oracle, exact mass."""
    if case == "basin":
        w, steps = W.basin_c1(hump=True, rain=True), 200
    else:
        w, steps = W.coastal_c2(n_tri=4000, seed=23, steps=100), 100
    ref, dev = _pair(w, steps, prec, limiter=True)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12
    assert np.array_equal(dev.dry(), ref.dry())


def test_slope_limiter_rejects_p2():
    with pytest.raises(D.DgsweError):
        D.Solver(p=2, limiter=True)


# ---------------------------------------------------------------- five-stage SSP ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_five_stage_ssp_with_llf_matches_oracle(prec):
    """The five-stage SSP(5,2) stepper with the LLF flux (the pairing of the production runs,
    Sec. 3) on the coastal wet/dry family, at twice the SSP(2,2) CFL number."""
    w = W.coastal_c2(n_tri=4000, seed=19, steps=100)
    w.cfl = 0.6
    ref, dev = _pair(w, 100, prec, flux=O.LLF, ssp=5)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12 and dev.ledger()["steps"] == 100


# ------------------------------------------------------------------------- rivers ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
@pytest.mark.parametrize("wet", [True, False])
def test_river_boundaries_match_oracle(prec, wet):
    """Eq. river_bc: two ramped river inflows into the walled basin (wet, and onto dry land):
    state against the oracle and the boundary inflow against the prescribed discharge."""
    w = W.river_basin(q=(2.0, 0.5) if wet else (0.05, 0.0), ramp_s=600.0 if wet else 60.0, wet=wet)
    steps = 200
    ref, dev = _pair(w, steps, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    led, rl = dev.ledger(), ref.ledger()
    assert led["rel_err"] < 1e-12
    # prescribed inflow: exact in FP64; the mixed path carries edge lengths in FP32 (6e-8)
    tol = 1e-9 if prec == D.FP64 else 1e-6
    assert abs(led["bdry_in"] - rl["bdry_in"]) <= tol * abs(rl["bdry_in"])
    assert np.array_equal(dev.dry(), ref.dry())


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_internal_river_boundary_matches_oracle(prec):
    """Sec. 2.3 internal river boundaries: two wall rivers and one river on interior edges of the
    basin (entering the triangles north of its line); state, dry flags and the booked inflow
    against the oracle."""
    w = W.river_basin(q=(2.0, 0.5, 1.5), ramp_s=600.0, internal=True)
    ref, dev = _pair(w, 200, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    led, rl = dev.ledger(), ref.ledger()
    assert led["rel_err"] < 1e-12
    tol = 1e-9 if prec == D.FP64 else 1e-6
    assert abs(led["bdry_in"] - rl["bdry_in"]) <= tol * abs(rl["bdry_in"])
    assert np.array_equal(dev.dry(), ref.dry())


# ---------------------------------------------------------- rain on a flume (Sec. 3.2) --
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_inclined_plane_runoff_matches_oracle(prec):
    """Initially dry flume (condition B: three slopes and rain rates, H0 = 0.1 mm), gridded rain
    stopping after 1 s, free outfall: 1500 steps of 1 ms against the oracle."""
    w = W.inclined_plane("B", duration=1.0)
    ref, dev = _pair(w, 1500, prec, dt=1e-3)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    led, rl = dev.ledger(), ref.ledger()
    assert abs(led["V"] - led["V0"] - led["rain_in"] - led["bdry_in"]) < 1e-12
    assert abs(led["bdry_in"] - rl["bdry_in"]) <= 1e-6 * abs(rl["rain_in"])


# -------------------------------------------------------------------- forcing paths ------
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_gridded_rain_and_pressure_setup(prec):
    w = W.coastal_c2(n_tri=3000, seed=31, steps=50)
    w.storm = None
    rng = np.random.default_rng(3)
    nx, ny, nt = 12, 9, 3
    w.rain_grid = W.RainGrid(nx, ny, nt, 0.0, 0.0, 400_000.0 / (nx - 1), 300_000.0 / (ny - 1), 0.0, 60.0,
                             rng.uniform(0, 80, (nt, ny, nx)).astype(np.float32))
    w.pressure = (320_000.0, 150_000.0, 50_000.0, 1.0)
    ref, dev = _pair(w, 50, prec)
    got, want = dev.state(), ref.state()
    if prec == D.FP64:
        assert _fp64_err(got, want) <= FP64_TOL
    else:
        ez, eq = _mixed_err(got, want)
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (ez, eq)
    assert dev.ledger()["rel_err"] < 1e-12


def test_quadratic_friction_bathtub_short():
    w = W.bathtub()
    ref, dev = _pair(w, 500, D.FP64, friction=O.QUADRATIC, cf=0.001, dt=5.0)
    assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL


# ----------------------------------------------------------- launch shapes, edge cases ----
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_launch_shapes_give_identical_bits(prec):
    """Block size and waves do not change a single bit; the fused, split and tile forms agree to
    rounding."""
    w = W.coastal_c2(n_tri=5000, seed=5, steps=30)
    both = []
    for split in (0, 1, 2):
        outs = []
        for block, waves in ((64, 1), (128, 2), (256, 1), (256, 2)):
            if split == 2 and block == 256 and prec == D.FP64:
                continue  # the FP64 tile form's shared memory does not fit 8 warps in one block
            dev = D.from_workload(w, precision=prec, block=block, waves=waves, split=split)
            dev.step(30)
            dev.sync()
            assert dev.launch() == (block, waves, split)
            outs.append(dev.state())
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        both.append(outs[0])
    tol = 1e-13 if prec == D.FP64 else 1e-5
    for other in both[1:]:
        assert np.abs(both[0] - other).max() <= tol * max(1.0, np.abs(both[0]).max())


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_direct_launches_match_graph_replay(prec):
    """Steps replayed from CUDA graphs and steps launched kernel by kernel give identical bits
    (13 steps: one 8-step graph, five 1-step graphs)."""
    w = W.coastal_c2(n_tri=3000, seed=17, steps=13)
    a = D.from_workload(w, precision=prec, block=128, split=2)
    b = D.from_workload(w, precision=prec, block=128, split=2)
    b.set_graphs(False)
    a.step(13)
    b.step(13)
    a.sync()
    b.sync()
    assert np.array_equal(a.state(), b.state())
    assert a.ledger() == b.ledger()
    assert b.launch_count() > 0


def test_ragged_and_tiny_meshes():
    # 2 triangles (one partial tile) and a mesh whose size is not a multiple of any block
    for w in (W.basin_c1(nx=1, ny=1), W.basin_c1(nx=13, ny=7)):
        ref, dev = _pair(w, 50, D.FP64)
        assert _fp64_err(dev.state(), ref.state()) <= FP64_TOL


def test_modal_state_round_trip_and_nonfinite_rejected():
    w = W.basin_c1()
    dev = D.from_workload(w, precision=D.FP64)
    s = dev.state()
    dev2 = D.Solver(precision=D.FP64, H0=w.h0, cfl=w.cfl)
    dev2.set_mesh(w.mesh)
    dev2.set_fields(w.hb, w.manning)
    dev2.set_rain_nodal(w.rain_nodal)
    dev2.set_state(np.ascontiguousarray(s[:, 0].T), np.ascontiguousarray(s[:, 1].T),
                   np.ascontiguousarray(s[:, 2].T), layout=D.LAYOUT_MODAL)
    assert np.array_equal(dev2.state(), s)
    bad = w.zeta0.copy()
    bad[3] = np.nan
    with pytest.raises(D.DgsweError) as ei:
        dev2.set_state(bad)
    assert ei.value.code == -1


def test_negative_mean_depth_is_reported_not_trapped():
    w = W.basin_c1()
    z = w.zeta0.copy()
    z[:] = -w.hb - 0.5  # every element well below its bed: a host-made invalid state
    dev = D.Solver(precision=D.MIXED, H0=w.h0, cfl=0.0, dt=1.0)
    dev.set_mesh(w.mesh)
    dev.set_fields(w.hb, w.manning)
    dev.set_state(z)
    with pytest.raises(D.DgsweError) as ei:
        dev.sync()
    assert ei.value.code == -5


# --------------------------------------------------------------------------- ensemble ----
@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
@pytest.mark.parametrize("split", [0, 1, 2])
def test_ensemble_members_match_solo_runs(prec, split):
    """Batching does not change a bit: each member of an ensemble, run with the same kernels
    (launch shape fixed on both sides), ends bit-identical to its solo run."""
    ws = W.ensemble_c4(n_scen=3, lo=1500, hi=6000, seed=8, steps=40)
    solos, members = [], []
    for w in ws:
        s = D.from_workload(w, precision=prec, block=128, split=split)
        members.append(s)
        solo = D.from_workload(w, precision=prec, block=128, split=split)
        solo.step(40)
        solo.sync()
        solos.append((solo.state(), solo.ledger()))
    ens = D.Ensemble(members)
    ens.set_launch(128, 1, split)
    ens.step(40)
    ens.sync()
    for i, (st, led) in enumerate(solos):
        assert np.array_equal(ens.state(i), st)
        le = ens.ledger(i)
        assert le["rel_err"] < 1e-12 and le["steps"] == 40
        assert abs(le["t"] - led["t"]) == 0.0
    # and the FP64 members against the oracle
    if prec == D.FP64:
        w = ws[0]
        ref = O.from_workload(w)
        ref.step(40)
        assert _fp64_err(ens.state(0), ref.state()) <= FP64_TOL


@pytest.mark.slow
def test_ensemble_full_size_sampled_members_match_oracle():
    """The 64-scenario ensemble at the benchmark's size (about 10M triangles in all, members
    built with the benchmark's launch shape, the ensemble autotuned), 10 mixed-precision steps;
    the three smallest members are compared element by element with the oracle run alone on the
    same scenario and dt."""
    ws = W.ensemble_c4()
    sample = set(np.argsort([w.mesh.n_tri for w in ws])[:3].tolist())
    members, refs = [], {}
    for i, w in enumerate(ws):
        dt = 0.0
        if i in sample:
            ref = O.from_workload(w)
            dt = ref.cfl_dt(w.cfl)
            ref.set_dt(dt)
            refs[i] = ref
        members.append(D.from_workload(w, precision=D.MIXED, dt=dt, block=64, waves=1, split=0))
    ens = D.Ensemble(members)
    for m in members:
        m.close()
    ens.step(10)
    ens.sync()
    for i, ref in refs.items():
        ref.step(10)
        ez, eq = _mixed_err(ens.state(i), ref.state())
        assert ez <= MIXED_TOL and eq <= MIXED_TOL, (i, ez, eq)
        assert ens.ledger(i)["rel_err"] < 1e-12 and ens.ledger(i)["steps"] == 10


@pytest.mark.parametrize("prec", [D.FP64, D.MIXED])
def test_load_state_round_trip_and_restart(prec):
    """Checkpoint/restart through the public API (also the e2e benchmark's per-step exchange).
    Modes >= 1 round-trip bit for bit; mode 0 is sqrt(2) times the element mean, so it is rounded
    once on the way out and once on the way in (a few ulps).  The continued run stays within the
    path's tolerance of the uninterrupted one."""
    w = W.coastal_c2(n_tri=4000, seed=13, steps=40)
    a = D.from_workload(w, precision=prec)
    a.step(20)
    z, x, y = a.state_arrays()
    a.step(20)
    a.sync()
    b = D.from_workload(w, precision=prec)
    b.step(20)
    b.load_state(z, x, y)
    got = b.state()
    want = np.stack([z.T, x.T, y.T], axis=1)
    assert np.array_equal(got[:, :, 1:], want[:, :, 1:])
    assert np.abs(got[:, :, 0] - want[:, :, 0]).max() <= 4e-16 * max(1.0, np.abs(want[:, :, 0]).max())
    b.step(20)
    b.sync()
    if prec == D.FP64:
        assert _fp64_err(b.state(), a.state()) <= 1e-13
    else:
        ez, eq = _mixed_err(b.state(), a.state())
        assert ez <= 1e-6 and eq <= 1e-5, (ez, eq)
