"""Pins of the oracle's wet/dry edge closure (Sec. 2.4: the element flag decides how an element
interacts with its neighbours; the reading taken here: an edge whose mass flux would take water
out of a dry element is closed, each side then seeing a wall built from its own state).

After the positive-depth operator a dry element is flat and still (its mean depth is at most H0,
every vertex takes that depth and the momentum is zero), so water can leave it only where the
other side's state pulls it: a wet neighbour whose water moves away from the edge faster than its
surface excess pushes back, or an open boundary whose tide lies below the dry element's film.
Each case first shows, with the oracle's stand-alone numerical flux (Roe, evaluated here on the
traces), that the open edge would drain the dry element; the closure must then leave the dry
element's mass right-hand side exactly zero, while the same geometry with a wet film does lose
water through the edge."""
import math

import numpy as np

import oracle as O
from paper_2307_14302_gb300 import workloads as W

H0 = 0.01


def _square(btype):
    """A 1000 m x 800 m square split along the diagonal from (0, 0) to (1000, 800): element 0
    below the diagonal, element 1 above; outer edges bottom, right, top, left."""
    xy = np.array([[0.0, 0.0], [1000.0, 0.0], [1000.0, 800.0], [0.0, 800.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    be = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)
    return W.Mesh(xy, tri, be, np.asarray(btype, np.int32), np.zeros(4, np.int32))


def _modal_p1(vertex_values):
    """p = 1 modal coefficients of the linear field with the given vertex values."""
    V = np.array([O.basis(1, r, s)[0] for r, s in ((-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0))])
    return np.linalg.solve(V, np.asarray(vertex_values, float))


def _oracle_with(mesh, hb, w, tide=None):
    o = O.Oracle(mesh, hb, p=1, friction=O.NOFRICTION, h0=H0)
    if tide is not None:
        o.set_tide(tide)
    o.set_state_modal(w)
    o.set_dt(1e-9)
    o.step(1)  # the positive-depth operator runs and sets the element flags; the state moves by ~1e-9
    return o


def test_dry_element_keeps_its_water_against_a_receding_neighbour():
    n = np.array([-800.0, 1000.0]) / math.hypot(800.0, 1000.0)  # outward normal of element 0 on the diagonal
    hb = np.full(4, 1.0)
    HL, HR, u = 0.005, 0.02, 0.6  # element 0 dry and still; element 1 wet, flowing away at 0.6 m/s
    wl = np.array([HL - 1.0, 0.0, 0.0])
    wr = np.array([HR - 1.0, u * HR * n[0], u * HR * n[1]])
    f = O.numflux(O.ROE, wl, 1.0, wr, 1.0, n, h0=H0)
    assert f[0] > 1e-5  # the open edge would carry water out of the dry element

    def run(film):
        w = np.zeros((2, 3, 3))
        w[0, 0] = _modal_p1(film - hb[[0, 1, 2]])
        w[1, 0] = _modal_p1(HR - hb[[0, 2, 3]])
        w[1, 1] = _modal_p1(np.full(3, u * HR * n[0]))
        w[1, 2] = _modal_p1(np.full(3, u * HR * n[1]))
        return _oracle_with(_square([O.BT_LAND] * 4), hb, w)

    o = run(HL)
    assert list(o.dry()) == [1, 0]
    L = o.rhs()
    assert abs(L[0, 0, 0]) <= 1e-15  # no water leaves the dry element (walls elsewhere)
    assert abs(L[1, 0, 0]) <= 1e-15  # and none enters the wet one through the closed edge
    assert o.ledger()["rel_err"] < 1e-12
    # with a wet film (2 H0) the same flow drains element 0 through the open edge
    o2 = run(2 * H0)
    assert list(o2.dry()) == [0, 0]
    L2 = o2.rhs()
    assert L2[0, 0, 0] < -1e-8 and L2[1, 0, 0] > 1e-8
    assert abs(L2[0, 0, 0] * math.sqrt(2) + L2[1, 0, 0] * math.sqrt(2)) <= 1e-12 * abs(L2[0, 0, 0])


def test_dry_element_keeps_its_water_against_a_low_tide():
    hb = np.full(4, -1.0)  # land 1 m above the datum
    tide = W.Tide(np.array([0.2]), np.array([1e9]), np.array([-0.5 * math.pi]))  # zeta_bc = -0.2 m
    film = 0.005
    zl = film + 1.0
    f = O.numflux(O.ROE, np.array([zl, 0.0, 0.0]), -1.0, np.array([-0.2, 0.0, 0.0]), -1.0,
                  np.array([0.0, -1.0]), h0=H0)
    assert f[0] > 1e-3  # the open edge (bottom, outward normal -y) would drain the film

    def run(H):
        w = np.zeros((2, 3, 3))
        w[0, 0] = _modal_p1(np.full(3, H + 1.0))
        w[1, 0] = _modal_p1(np.full(3, H + 1.0))
        return _oracle_with(_square([O.BT_OCEAN, O.BT_LAND, O.BT_LAND, O.BT_LAND]), hb, w, tide)

    o = run(film)
    assert list(o.dry()) == [1, 1]
    L = o.rhs()
    assert np.abs(L[:, 0]).max() <= 1e-15
    # a wet film of the same geometry runs out through the open edge
    o2 = run(2 * H0)
    assert list(o2.dry()) == [0, 0]
    assert o2.rhs()[0, 0, 0] < -1e-6


def test_rain_on_a_dry_flat_floodplain_wets_it_at_the_threshold():
    """A flat floodplain 2 m above the datum under a 5 mm film (below H0, every element dry) and
    uniform rain R, walls all round: rain falls on dry elements too (Sec. 2.3), nothing moves, so
    the depth is 5 mm + R t exactly, the elements stay dry while it is below H0 and are all wet
    once it is above, and the mass ledger balances."""
    mesh = W.structured_mesh(4000.0, 2000.0, 10, 5)
    hb = np.full(mesh.n_nodes, -2.0)
    R, film, dt = 1.0e-5, 0.005, 10.0  # the film reaches H0 at t = 500 s
    o = O.Oracle(mesh, hb, np.full(mesh.n_tri, 0.03), p=1, h0=H0)
    o.set_rain_nodal(np.full(mesh.n_nodes, R))
    o.set_state_nodal(np.full(mesh.n_nodes, film + 2.0))
    o.set_dt(dt)
    for n, wet in ((49, False), (2, True)):  # t = 490 s, then 510 s
        o.step(n)
        t = o.ledger()["t"]
        s = o.state()
        H = s[:, 0, 0] / math.sqrt(2) - 2.0
        assert np.abs(H - (film + R * t)).max() <= 1e-13, t
        assert np.abs(s[:, 0, 1:]).max() <= 1e-13 and np.abs(s[:, 1:]).max() <= 1e-12  # flat, at rest
        assert (o.dry() == (0 if wet else 1)).all(), t
        assert o.ledger()["rel_err"] < 1e-12
