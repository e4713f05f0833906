"""Pins of the oracle's friction laws, tidal boundary and pressure set-up forcing.

Each check compares the oracle with something it does not compute itself: the closed-form
solution of a scalar ODE, an independent numpy eigen-decomposition of the Roe flux, a
high-order quadrature written here, or the quasi-static limit of a tidal basin.

* Friction (Sec. 3.1 and the production runs' Manning law): a spatially uniform flow on a flat
  bed loses momentum only to friction, so away from the walls (beyond the dependency cone of
  the explicit stages) every element follows the ODE  dq/dt = -tau_b(q) q  integrated by the
  same SSP(2,2) steps; the ODE's exact solution is approached at second order in dt.
* Tide (Sec. 2.1, specified elevation on the open boundary): a lake at rest at the constant
  tidal level stays at rest; a slow tide drives the basin mean quasi-statically; the ghost
  state of an ocean edge is (zeta_bc(t), interior q), checked against the Roe flux of that
  ghost on a single element.
* Pressure set-up (F of Eq. SWE): F = g H grad(eta_p) is checked against a 12x12 Gauss
  integral of the same field on a small element, and the residual of zeta = P_h eta_p at rest
  falls under refinement (the surface at rest follows the set-up).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2307_14302_gb300 import workloads as W

G = 9.81


def _element_hops_to_boundary(mesh):
    """Graph distance (edge-sharing steps) from each triangle to the nearest triangle that has
    a boundary edge."""
    tri = mesh.tri
    E = len(tri)
    key = {}
    for e in range(E):
        for j in range(3):
            a, b = tri[e, j], tri[e, (j + 1) % 3]
            key.setdefault((min(a, b), max(a, b)), []).append(e)
    nbrs = [[] for _ in range(E)]
    dist = np.full(E, -1)
    front = []
    for lst in key.values():
        if len(lst) == 2:
            nbrs[lst[0]].append(lst[1])
            nbrs[lst[1]].append(lst[0])
        else:
            if dist[lst[0]] < 0:
                dist[lst[0]] = 0
                front.append(lst[0])
    d = 0
    while front:
        nxt = []
        for e in front:
            for n in nbrs[e]:
                if dist[n] < 0:
                    dist[n] = d + 1
                    nxt.append(n)
        front, d = nxt, d + 1
    return dist


def _tri_area(a, b, c):
    return 0.5 * np.abs((b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) - (c[..., 0] - a[..., 0]) * (b[..., 1] - a[..., 1]))


def _ssp22(f, y, dt, n):
    for _ in range(n):
        y1 = y + dt * f(y)
        y = 0.5 * y + 0.5 * (y1 + dt * f(y1))
    return y


# ------------------------------------------------------------------------------ friction ---
@pytest.mark.parametrize("law", ["manning", "quadratic"])
def test_friction_decay_of_a_uniform_flow_follows_the_closed_form(law):
    H, n_man, cf = 2.0, 0.05, 0.003
    q0 = np.array([0.6, 0.8])  # |u0| = 0.5 m/s at H = 2 m
    if law == "manning":
        k = G * n_man ** 2 / H ** (4.0 / 3.0)   # du/dt = -k |u| u
        fr, cfv = O.MANNING, 0.0
    else:
        k = cf / H                              # du/dt = -(Cf / H) |u| u
        fr, cfv = O.QUADRATIC, cf

    def f(q):  # in discharge: dq/dt = -k |q|/H q
        return -k * np.hypot(q[0], q[1]) / H * q

    T = 160.0
    results = []
    for nsteps, nx in ((16, 40), (32, 72)):
        dt = T / nsteps
        mesh = W.structured_mesh(1000.0 * nx, 1000.0 * nx, nx, nx)
        o = O.Oracle(mesh, np.full(mesh.n_nodes, H), np.full(mesh.n_tri, n_man), p=1, friction=fr, cf=cfv)
        o.set_state_nodal(np.zeros(mesh.n_nodes), np.full(mesh.n_nodes, q0[0]), np.full(mesh.n_nodes, q0[1]))
        o.set_dt(dt)
        o.step(nsteps)
        s = o.state()
        hops = _element_hops_to_boundary(mesh)
        far = hops >= 2 * nsteps  # no wall has reached these elements after 2 stages per step
        assert far.sum() >= 20
        mean_q = s[far, 1:, 0] / math.sqrt(2.0)
        # the same SSP(2,2) steps applied to the scalar ODE
        want = _ssp22(f, q0.copy(), dt, nsteps)
        assert np.abs(mean_q - want).max() <= 1e-13 * np.abs(q0).max(), (law, mean_q[:2], want)
        assert np.abs(s[far, 0, :]).max() <= 1e-12           # zeta untouched
        assert np.abs(s[far, 1:, 1:]).max() <= 1e-12         # no slopes appear
        # the ODE's exact solution u(t) = u0 / (1 + k |u0| t)
        u0 = np.hypot(*q0) / H
        exact = q0 / (1.0 + k * u0 * T)
        results.append(np.abs(mean_q[0] - exact).max())
    # SSP(2,2) is second order: halving dt divides the error by about four
    assert 3.0 < results[0] / results[1] < 5.0, results


def test_friction_laws_differ_only_by_their_depth_power():
    """Manning at depth H with n^2 g = Cf H^(1/3) gives the quadratic law's decay."""
    H, n_man = 3.0, 0.04
    cf = G * n_man ** 2 / H ** (1.0 / 3.0)
    out = []
    for fr, c in ((O.MANNING, 0.0), (O.QUADRATIC, cf)):
        mesh = W.structured_mesh(30_000.0, 30_000.0, 30, 30)
        o = O.Oracle(mesh, np.full(mesh.n_nodes, H), np.full(mesh.n_tri, n_man), p=1, friction=fr, cf=c)
        o.set_state_nodal(np.zeros(mesh.n_nodes), np.full(mesh.n_nodes, 0.9), np.full(mesh.n_nodes, -0.3))
        o.set_dt(10.0)
        o.step(5)
        far = _element_hops_to_boundary(mesh) >= 10
        out.append(o.state()[far, 1:, 0])
    assert np.abs(out[0] - out[1]).max() <= 1e-13
    assert np.abs(out[0][:, 0] / math.sqrt(2) - 0.9).max() > 1e-3  # friction did act


# ---------------------------------------------------------------------------------- tide ---
def test_lake_at_rest_at_a_constant_tidal_level_stays_at_rest():
    mesh = W.structured_mesh(2000.0, 1000.0, 20, 10, ocean_side="x0")
    x = mesh.xy[:, 0]
    hb = 5.0 + 0.004 * x + 0.5 * np.sin(mesh.xy[:, 1] / 200.0)
    A, phase = 0.3, 0.7
    level = A * math.sin(phase)
    o = O.Oracle(mesh, hb, np.full(mesh.n_tri, 0.03), p=1)
    o.set_tide(W.Tide(np.array([A]), np.array([1e15]), np.array([phase])))
    o.set_state_nodal(np.full(mesh.n_nodes, level))
    o.set_dt(o.cfl_dt(0.3))
    o.step(200)
    s = o.state()
    depth = hb[mesh.tri].mean(axis=1) + level
    assert np.abs(s[:, 1:]).max(axis=(1, 2)).__truediv__(depth).max() <= 1e-12  # velocity, m/s
    assert np.abs(s[:, 0, 0] / math.sqrt(2) - level).max() <= 1e-12 and np.abs(s[:, 0, 1:]).max() <= 1e-12
    # the wrong level (e.g. a cosine instead of a sine) would drive a flow
    o2 = O.Oracle(mesh, hb, np.full(mesh.n_tri, 0.03), p=1)
    o2.set_tide(W.Tide(np.array([A]), np.array([1e15]), np.array([phase])))
    o2.set_state_nodal(np.full(mesh.n_nodes, A * math.cos(phase)))
    o2.set_dt(o.cfl_dt(0.3))
    o2.step(20)
    assert np.abs(o2.state()[:, 1:]).max() > 1e-3


def _tidal_basin_mean_error(period, A=0.2, h=10.0, L=2000.0):
    mesh = W.structured_mesh(L, 400.0, 10, 2, ocean_side="x0")
    o = O.Oracle(mesh, np.full(mesh.n_nodes, h), p=1, friction=O.NOFRICTION)
    # zeta_bc = A sin(2 pi t / T + pi/2) = A cos(2 pi t / T): start at the crest, at rest
    o.set_tide(W.Tide(np.array([A]), np.array([period]), np.array([0.5 * math.pi])))
    o.set_state_nodal(np.full(mesh.n_nodes, A))
    dt = o.cfl_dt(0.3)
    n_total = int(round(0.5 * period / dt))
    dt = 0.5 * period / n_total
    o.set_dt(dt)
    area = _tri_area(mesh.xy[mesh.tri[:, 0]], mesh.xy[mesh.tri[:, 1]], mesh.xy[mesh.tri[:, 2]])
    err, done = 0.0, 0
    for frac in (0.125, 0.25, 0.375, 0.5):
        n = int(round(frac * period / dt))
        o.step(n - done)
        done = n
        zbar = (o.state()[:, 0, 0] / math.sqrt(2) * area).sum() / area.sum()
        err = max(err, abs(zbar - A * math.cos(2 * math.pi * done * dt / period)))
    return err / A


def test_slow_tide_drives_the_basin_mean_quasi_statically():
    """A basin much shorter than the tidal wavelength follows the open-boundary elevation
    A sin(2 pi t / T + phi); the lag falls as (L / (c T))^2 when T grows."""
    e1 = _tidal_basin_mean_error(4 * 3600.0)
    e2 = _tidal_basin_mean_error(8 * 3600.0)
    assert e1 < 0.02, e1
    assert e2 < e1 / 2.5, (e1, e2)


def _roe_np(wl, wr, hb, n):
    """Roe flux written from its definition with a numpy eigen-decomposition."""
    def phys(w):
        H = w[0] + hb
        un = (w[1] * n[0] + w[2] * n[1]) / H
        P = 0.5 * G * (H * H - hb * hb)
        return np.array([w[1] * n[0] + w[2] * n[1], w[1] * un + P * n[0], w[2] * un + P * n[1]])

    HL, HR = wl[0] + hb, wr[0] + hb
    sL, sR = math.sqrt(HL), math.sqrt(HR)
    ut = (sL * wl[1] / HL + sR * wr[1] / HR) / (sL + sR)
    vt = (sL * wl[2] / HL + sR * wr[2] / HR) / (sL + sR)
    c = math.sqrt(G * 0.5 * (HL + HR))
    un = ut * n[0] + vt * n[1]
    # Roe matrix: the Jacobian of the normal flux in (zeta, qx, qy) at the Roe state
    Jm = np.array([[0.0, n[0], n[1]],
                   [c * c * n[0] - ut * un, un + ut * n[0], ut * n[1]],
                   [c * c * n[1] - vt * un, vt * n[0], un + vt * n[1]]])
    lam, R = np.linalg.eig(Jm)
    absA = (R * np.abs(lam.real)) @ np.linalg.inv(R)
    return 0.5 * (phys(wl) + phys(wr)) - 0.5 * absA.real @ (np.asarray(wr) - np.asarray(wl))


def test_ocean_edge_ghost_is_the_tide_with_the_interior_discharge():
    xy = np.array([[0.0, 0.0], [300.0, 40.0], [60.0, 250.0]])
    tri = np.array([[0, 1, 2]], np.int32)
    bedge = np.array([[0, 1], [1, 2], [2, 0]], np.int32)
    btype = np.array([O.BT_LAND, O.BT_OCEAN, O.BT_LAND], np.int32)
    mesh = W.Mesh(xy, tri, bedge, btype, np.zeros(3, np.int32))
    hb, A, per, pha = 8.0, 0.4, 3600.0, 0.3
    w = np.array([0.05, 0.7, -0.4])
    o = O.Oracle(mesh, np.full(3, hb), p=1, friction=O.NOFRICTION)
    o.set_tide(W.Tide(np.array([A]), np.array([per]), np.array([pha])))
    o.set_state_nodal(np.full(3, w[0]), np.full(3, w[1]), np.full(3, w[2]))
    t = 1234.5
    o.set_time(t)
    L = o.rhs()[0, :, 0]
    zbc = A * math.sin(2 * math.pi * t / per + pha)
    total = np.zeros(3)
    for j, kind in enumerate(btype):
        a, b = xy[tri[0, j]], xy[tri[0, (j + 1) % 3]]
        ln = np.array([b[1] - a[1], -(b[0] - a[0])])
        length = np.hypot(*ln)
        n = ln / length
        if kind == O.BT_OCEAN:
            f = _roe_np(w, np.array([zbc, w[1], w[2]]), hb, n)
        else:
            qn = w[1] * n[0] + w[2] * n[1]
            f = _roe_np(w, np.array([w[0], w[1] - 2 * qn * n[0], w[2] - 2 * qn * n[1]]), hb, n)
            f[0] = 0.0
        total += length * f
    area = float(_tri_area(xy[0], xy[1], xy[2]))
    want = -math.sqrt(2.0) / area * total  # mode-0 rate of the orthonormal basis (phi_0 = 1/sqrt 2)
    assert np.allclose(L, want, rtol=1e-12, atol=1e-14), (L, want)
    # a ghost with zero discharge, or the mirrored one, gives another mass flux
    for ghost in ([zbc, 0.0, 0.0], [zbc, -w[1], -w[2]]):
        j = 1
        a, b = xy[tri[0, j]], xy[tri[0, (j + 1) % 3]]
        ln = np.array([b[1] - a[1], -(b[0] - a[0])])
        f2 = _roe_np(w, np.array(ghost), hb, ln / np.hypot(*ln))
        assert abs(-math.sqrt(2.0) / area * np.hypot(*ln) * f2[0] - L[0]) > 1e-6


# ------------------------------------------------------------------------ pressure set-up ---
def _collapsed_rule(n=12):
    x, w = np.polynomial.legendre.leggauss(n)
    A, B = np.meshgrid(x, x, indexing="ij")
    WA, WB = np.meshgrid(w, w, indexing="ij")
    r = 0.5 * (1 + A) * (1 - B) - 1
    return r.ravel(), B.ravel(), (WA * WB * 0.5 * (1 - B)).ravel()


def test_pressure_setup_forcing_is_g_H_grad_eta():
    """On a fluid at rest (zeta = 0, q = 0) over a sloping bed the only momentum source is the
    set-up forcing; its moments on a 10 m triangle equal a 12x12 Gauss integral of
    g H d(eta_p)/dx with eta_p = peak exp(-r^2 / (2 sigma^2))."""
    xy = np.array([[1000.0, 800.0], [1010.0, 801.0], [1002.0, 809.0]])
    tri = np.array([[0, 1, 2]], np.int32)
    bedge = np.array([[0, 1], [1, 2], [2, 0]], np.int32)
    mesh = W.Mesh(xy, tri, bedge, np.zeros(3, np.int32), np.zeros(3, np.int32))
    hbf = lambda x, y: 10.0 + 0.002 * x + 0.001 * y  # noqa: E731
    hb = hbf(xy[:, 0], xy[:, 1])
    x0, y0, sig, peak = 700.0, 1100.0, 300.0, 2.0
    o = O.Oracle(mesh, hb, p=1, friction=O.NOFRICTION)
    o.set_pressure(x0, y0, sig, peak)
    o.set_state_nodal(np.zeros(3))
    L = o.rhs()[0]
    r, s, wq = _collapsed_rule()
    lam = np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=-1)
    X = lam @ xy
    eta = peak * np.exp(-((X[:, 0] - x0) ** 2 + (X[:, 1] - y0) ** 2) / (2 * sig ** 2))
    H = hbf(X[:, 0], X[:, 1])
    Fx = G * H * eta * (-(X[:, 0] - x0) / sig ** 2)
    Fy = G * H * eta * (-(X[:, 1] - y0) / sig ** 2)
    phi = np.array([O.basis(1, ri, si)[0] for ri, si in zip(r, s)])
    # M^{-1} with M = detJ I: the moments in reference coordinates
    wantx, wanty = phi.T @ (wq * Fx), phi.T @ (wq * Fy)
    assert np.allclose(L[1], wantx, rtol=1e-4, atol=1e-6 * abs(wantx[0])), (L[1], wantx)
    assert np.allclose(L[2], wanty, rtol=1e-4, atol=1e-6 * abs(wanty[0])), (L[2], wanty)
    assert np.abs(L[0]).max() == 0.0
    assert abs(wantx[0]) > 1e-3  # the forcing is not negligible here


def _project_gaussian(mesh, p, x0, y0, sig, peak):
    r, s, w = _collapsed_rule(8)
    lam = np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=-1)
    B = np.array([O.basis(p, ri, si)[0] for ri, si in zip(r, s)])
    out = np.zeros((mesh.n_tri, 3, B.shape[1]))
    for e, v in enumerate(mesh.tri):
        X = lam @ mesh.xy[v]
        z = peak * np.exp(-((X[:, 0] - x0) ** 2 + (X[:, 1] - y0) ** 2) / (2 * sig ** 2))
        out[e, 0] = B.T @ (w * z)
    return out


@pytest.mark.parametrize("p,rate", [(1, 0.85), (2, 2.5)])
def test_surface_at_rest_follows_the_setup(p, rate):
    """zeta = P_h eta_p, q = 0 balances g H grad(zeta) against the forcing up to the
    projection error: the momentum residual falls with the mesh size at order about p.  The
    opposite sign of F, or a missing g or H, leaves an O(1) residual."""
    lx = 4000.0
    x0 = y0 = 2000.0
    sig, peak = 600.0, 0.5
    res = []
    for n in (16, 32, 64):
        mesh = W.structured_mesh(lx, lx, n, n)
        o = O.Oracle(mesh, np.full(mesh.n_nodes, 10.0), p=p, friction=O.NOFRICTION)
        o.set_pressure(x0, y0, sig, peak)
        o.set_state_modal(_project_gaussian(mesh, p, x0, y0, sig, peak))
        L = o.rhs()
        res.append(np.abs(L[:, 1:, 0]).max())
        if n == 8:
            scale = G * 10.0 * peak / sig  # size of each of the two balancing terms
            o2 = O.Oracle(mesh, np.full(mesh.n_nodes, 10.0), p=p, friction=O.NOFRICTION)
            o2.set_pressure(x0, y0, sig, -peak)
            o2.set_state_modal(_project_gaussian(mesh, p, x0, y0, sig, peak))
            assert np.abs(o2.rhs()[:, 1:, 0]).max() > 0.5 * scale
    rates = -np.diff(np.log(res)) / math.log(2.0)
    assert rates.min() > rate, (res, rates)
