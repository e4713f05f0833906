"""Seeded synthetic inputs for the DG rainfall shallow-water solver.

This module only draws inputs: meshes, bathymetry, Manning fields, initial states and forcing
parameters.  It holds none of the method's arithmetic (no basis, quadrature, flux, source,
positivity or time stepping), so both the CUDA library and the CPU oracle can be driven from it.

Every generator takes an integer seed and uses numpy's PCG64 (``numpy.random.default_rng``).
The workloads stand in for the paper's ADCIRC/Harvey inputs (Sec. 3.3), which are not
available: shapes, sizes, bathymetry families and forcing magnitudes follow the paper's
experiments and the configurations stated in the build notes, the values are synthetic.

Conventions shared with the C interface:
  * ``xy``  [N, 2] float64 node coordinates in metres;
  * ``tri`` [E, 3] int32 counter-clockwise node indices;
  * ``bedge`` [B, 2] int32 node pairs of boundary edges, ``btype`` [B] (0 land, 1 ocean),
    ``bseg`` [B] tidal segment of ocean edges;
  * ``hb`` [N] bathymetry, positive downward (Sec. 2.1, Fig. 1);
  * rain in m/s, Manning n per element.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G = 9.81
MMH = 1.0 / 3.6e6  # (mm/h) -> (m/s)
LAND, OCEAN, RIVER = 0, 1, 2


@dataclasses.dataclass
class Mesh:
    xy: np.ndarray
    tri: np.ndarray
    bedge: np.ndarray
    btype: np.ndarray
    bseg: np.ndarray

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])


@dataclasses.dataclass
class Storm:
    """Moving radially symmetric rain cell; the field shape is applied by the solver."""
    x0: float
    y0: float
    heading: float  # radians, direction of travel
    speed: float  # m/s
    rpeak: float  # m/s, peak rain rate
    rm: float  # m, radius of the peak
    re: float  # m, e-folding length outside rm
    t0: float = 0.0


@dataclasses.dataclass
class RainGrid:
    nx: int
    ny: int
    nt: int
    x0: float
    y0: float
    dx: float
    dy: float
    t0: float
    dt_rec: float
    mm_per_h: np.ndarray  # float32 [nt, ny, nx]


@dataclasses.dataclass
class Tide:
    amp: np.ndarray
    period: np.ndarray
    phase: np.ndarray


@dataclasses.dataclass
class River:
    """Specified normal discharge (m^2/s, positive into the domain) per river segment: nt records
    from t0 every dt, linear in time (nt = 1: constant); q is [nt, nseg]."""
    q: np.ndarray
    t0: float = 0.0
    dt: float = 3600.0


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    hb: np.ndarray
    manning: np.ndarray
    zeta0: np.ndarray  # nodal initial elevation
    p: int
    steps: int
    cfl: float
    rain_nodal: np.ndarray | None = None
    storm: Storm | None = None
    rain_grid: RainGrid | None = None
    tide: Tide | None = None
    pressure: tuple | None = None  # (x0, y0, sigma, peak)
    river: River | None = None
    h0: float = 0.01
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def dof(self) -> int:
        return 3 * (self.p + 1) * (self.p + 2) // 2 * self.mesh.n_tri


# --------------------------------------------------------------------------------------------
# meshes


def _ccw(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    a = xy[tri[:, 0]]
    b = xy[tri[:, 1]]
    c = xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])
    tri = tri.copy()
    flip = cross < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    return tri.astype(np.int32)


def _boundary_edges(tri: np.ndarray) -> np.ndarray:
    """Edges used by exactly one triangle, oriented as in that (CCW) triangle."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    key = np.sort(e, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return e[cnt[inv.ravel()] == 1].astype(np.int32)


def _tag_rect(xy, bedge, lx, ly, ocean_side):
    """Boundary types on a rectangle [0,lx]x[0,ly]: one side ocean (segment 0), rest land."""
    mid = 0.5 * (xy[bedge[:, 0]] + xy[bedge[:, 1]])
    tol = 1e-6 * max(lx, ly)
    if ocean_side is None:
        ocean = np.zeros(len(bedge), bool)
    elif ocean_side == "x0":
        ocean = mid[:, 0] < tol
    elif ocean_side == "y0":
        ocean = mid[:, 1] < tol
    elif ocean_side == "x1":
        ocean = mid[:, 0] > lx - tol
    else:
        raise ValueError(ocean_side)
    btype = np.where(ocean, OCEAN, LAND).astype(np.int32)
    bseg = np.zeros(len(bedge), np.int32)
    return btype, bseg


def structured_mesh(lx, ly, nx, ny, mirror=False, ocean_side=None) -> Mesh:
    """nx*ny squares, each split into 2 triangles.  With ``mirror`` the diagonals of the upper
    half of the rows are the reflections of the lower half's across y = ly/2, so the mesh is
    symmetric under that reflection."""
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)

    def nid(i, j):
        return j * (nx + 1) + i

    tris = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)
            up = mirror and (2 * j >= ny)
            if not up:  # diagonal a-c
                tris += [(a, b, c), (a, c, d)]
            else:  # diagonal b-d (mirror image of a-c)
                tris += [(a, b, d), (b, c, d)]
    tri = _ccw(xy, np.array(tris, np.int64))
    bedge = _boundary_edges(tri)
    btype, bseg = _tag_rect(xy, bedge, lx, ly, ocean_side)
    return Mesh(xy, tri, bedge, btype, bseg)


def jittered_delaunay(lx, ly, n_tri_target, seed, jitter=0.35, ocean_side="x0", density=None) -> Mesh:
    """Seeded jittered-point Delaunay mesh of the rectangle [0,lx]x[0,ly].

    Points: a jittered lattice (interior) plus evenly spaced points on the four sides, so the
    convex hull is the rectangle.  ``density`` (optional) maps (x, y) -> relative point density
    in (0, 1]; lattice points are thinned by rejection against it (graded meshes)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    n_pts = max(n_tri_target // 2, 16)
    if density is not None:  # oversample, then thin
        n_pts = int(n_pts / max(density_mean(density, lx, ly), 1e-3))
    h = math.sqrt(lx * ly / n_pts)
    nx = max(int(round(lx / h)), 2)
    ny = max(int(round(ly / h)), 2)
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(1, nx), np.arange(1, ny), indexing="xy")
    px = (ii.ravel() + rng.uniform(-jitter, jitter, ii.size)) * hx
    py = (jj.ravel() + rng.uniform(-jitter, jitter, jj.size)) * hy
    if density is not None:
        keep = rng.uniform(0.0, 1.0, px.size) < density(px, py)
        px, py = px[keep], py[keep]
    bx = np.concatenate([np.arange(nx + 1) * hx, np.arange(nx + 1) * hx, np.zeros(ny - 1), np.full(ny - 1, lx)])
    by = np.concatenate([np.zeros(nx + 1), np.full(nx + 1, ly), np.arange(1, ny) * hy, np.arange(1, ny) * hy])
    xy = np.stack([np.concatenate([bx, px]), np.concatenate([by, py])], axis=1)
    xy[:, 0] = np.clip(xy[:, 0], 0.0, lx)
    xy[:, 1] = np.clip(xy[:, 1], 0.0, ly)
    tri = Delaunay(xy).simplices
    tri = _ccw(xy, tri)
    # drop slivers of (numerically) zero area along the straight boundary
    a = xy[tri[:, 0]]
    b = xy[tri[:, 1]]
    c = xy[tri[:, 2]]
    area = 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))
    tri = tri[area > 1e-9 * hx * hy]
    used = np.unique(tri)
    remap = -np.ones(len(xy), np.int64)
    remap[used] = np.arange(len(used))
    xy = xy[used]
    tri = remap[tri].astype(np.int32)
    bedge = _boundary_edges(tri)
    btype, bseg = _tag_rect(xy, bedge, lx, ly, ocean_side)
    return Mesh(np.ascontiguousarray(xy), tri, bedge, btype, bseg)


def jittered_grid_mesh(lx, ly, n_tri_target, seed, jitter=0.2, ocean_side="x0", xs=None) -> Mesh:
    """Seeded jittered structured mesh: an (nx+1) x (ny+1) node lattice, interior nodes moved by up
    to ``jitter`` of the local spacing, boundary nodes moved along their side only, each cell split
    along its shorter diagonal.  ``xs`` (optional, increasing from 0 to lx) fixes the node columns,
    which grades the mesh in x.  Linear in the node count, so meshes of millions of triangles are
    drawn in seconds."""
    rng = np.random.default_rng(seed)
    if xs is None:
        h = math.sqrt(2.0 * lx * ly / max(n_tri_target, 2))
        nx = max(int(round(lx / h)), 1)
        xs = np.linspace(0.0, lx, nx + 1)
    else:
        xs = np.asarray(xs, float)
        nx = len(xs) - 1
    ny = max(int(round(n_tri_target / (2 * nx))), 1)
    ys = np.linspace(0.0, ly, ny + 1)
    dxl = np.diff(xs)
    hxl = np.minimum(np.r_[dxl[0], dxl], np.r_[dxl, dxl[-1]])  # local x spacing per column
    hy = ly / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    HX = np.broadcast_to(hxl, X.shape)
    jx = rng.uniform(-jitter, jitter, X.shape) * HX
    jy = rng.uniform(-jitter, jitter, X.shape) * hy
    jx[:, 0] = jx[:, -1] = 0.0
    jy[0, :] = jy[-1, :] = 0.0
    X = X + jx
    Y = Y + jy
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    a = (jj * (nx + 1) + ii).ravel()
    b, c, d = a + 1, a + nx + 2, a + nx + 1
    # split each jittered cell along its shorter diagonal (the Delaunay choice for a convex
    # quadrilateral with near-equal angles), which keeps slivers out of large meshes
    dac = np.hypot(*(xy[a] - xy[c]).T)
    dbd = np.hypot(*(xy[b] - xy[d]).T)
    flip = dbd < dac
    t1 = np.where(flip[:, None], np.stack([a, b, d], 1), np.stack([a, b, c], 1))
    t2 = np.where(flip[:, None], np.stack([b, c, d], 1), np.stack([a, c, d], 1))
    tri = _ccw(xy, np.concatenate([t1, t2]))
    bedge = _boundary_edges(tri)
    btype, bseg = _tag_rect(xy, bedge, lx, ly, ocean_side)
    return Mesh(np.ascontiguousarray(xy), tri, bedge, btype, bseg)


def _graded_h(x, x_coast, hmin, hmax, width):
    return hmin + (hmax - hmin) * np.minimum(1.0, np.abs(x - x_coast) / width) ** 2


def _graded_columns(lx, ly, x_coast, hmin, hmax, width):
    """Column abscissae with spacing h(x) and the cell count of each column (ly / h)."""
    xf = np.linspace(0.0, lx, 400_001)
    hh = _graded_h(xf, x_coast, hmin, hmax, width)
    cells = np.concatenate([[0.0], np.cumsum(np.diff(xf) / (0.5 * (hh[1:] + hh[:-1])))])
    nx = max(int(round(cells[-1])), 2)
    xs = np.interp(np.linspace(0.0, cells[-1], nx + 1), cells, xf)
    xs[0], xs[-1] = 0.0, lx
    ny = np.maximum(1, np.round(ly / _graded_h(xs, x_coast, hmin, hmax, width))).astype(np.int64)
    return xs, ny


def graded_strip_mesh(lx, ly, x_coast, hmin, hmax, n_tri_target, seed, jitter=0.2, ocean_side="x0") -> Mesh:
    """Seeded mesh graded in x: node columns spaced by h(x) = hmin + (hmax - hmin) min(1,
    |x - x_coast| / width)^2, each column holding ly / h(x) nodes, neighbouring columns joined by
    merging their nodes in y order (a strip triangulation).  Element sizes are roughly isotropic
    and follow h.  ``width`` is chosen by bisection so the mesh has about n_tri_target
    triangles; interior nodes are jittered by up to ``jitter`` of the local spacing."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(1e2), math.log(1e8)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        _, ny = _graded_columns(lx, ly, x_coast, hmin, hmax, math.exp(mid))
        if int(np.sum(ny[:-1] + ny[1:])) < n_tri_target:
            lo = mid
        else:
            hi = mid
    xs, ny = _graded_columns(lx, ly, x_coast, hmin, hmax, math.exp(hi))
    ncol = len(xs)
    gap = np.diff(xs)
    xgap = np.minimum(np.r_[gap[0], gap], np.r_[gap, gap[-1]])
    start = np.concatenate([[0], np.cumsum(ny + 1)])
    xy = np.empty((int(start[-1]), 2))
    for i in range(ncol):
        n = int(ny[i])
        y = np.linspace(0.0, ly, n + 1)
        y[1:-1] += rng.uniform(-jitter, jitter, n - 1) * (ly / n)
        x = np.full(n + 1, xs[i])
        if 0 < i < ncol - 1:
            x += rng.uniform(-jitter, jitter, n + 1) * xgap[i]
        xy[start[i]:start[i + 1], 0] = x
        xy[start[i]:start[i + 1], 1] = y
    tris = []
    for i in range(ncol - 1):
        a0, na = int(start[i]), int(ny[i]) + 1
        b0, nb = int(start[i + 1]), int(ny[i + 1]) + 1
        ya, yb = xy[a0 + 1:a0 + na, 1], xy[b0 + 1:b0 + nb, 1]
        # advance events in y order: moving up column A (kind 0) or column B (kind 1)
        key = np.concatenate([ya, yb])
        kind = np.concatenate([np.zeros(na - 1, np.int64), np.ones(nb - 1, np.int64)])
        o = np.lexsort((kind, key))
        kind = kind[o]
        ia = np.cumsum(kind == 0) - (kind == 0)  # A index before the event
        ib = np.cumsum(kind == 1) - (kind == 1)
        t = np.where((kind == 0)[:, None],
                     np.stack([a0 + ia, a0 + ia + 1, b0 + ib], 1),
                     np.stack([a0 + ia, b0 + ib + 1, b0 + ib], 1))
        tris.append(t)
    tri = _ccw(xy, np.concatenate(tris).astype(np.int64))
    bedge = _boundary_edges(tri)
    btype, bseg = _tag_rect(xy, bedge, lx, ly, ocean_side)
    return Mesh(np.ascontiguousarray(xy), tri, bedge, btype, bseg)


def density_mean(density, lx, ly, n=64):
    xs = (np.arange(n) + 0.5) / n * lx
    ys = (np.arange(n) + 0.5) / n * ly
    X, Y = np.meshgrid(xs, ys)
    return float(np.mean(density(X, Y)))


def element_mean(mesh: Mesh, nodal: np.ndarray) -> np.ndarray:
    return nodal[mesh.tri].mean(axis=1)


# --------------------------------------------------------------------------------------------
# configurations


def basin_c1(seed=1, hump=True, rain=True, mirror=False, nx=20, ny=10) -> Workload:
    """Rectangular basin 10 km x 5 km, 20x10 squares split into 400 triangles, p=1.

    Depth 5 m to 20 m on a linear slope in x with a 1 m sinusoidal bump (shallower), an
    initial 0.5 m Gaussian hump (sigma 800 m, seeded centre), uniform 50 mm/h rain, Manning
    0.025, reflective walls, CFL 0.3, 200 steps.  With ``mirror`` the mesh is symmetric
    about y = 2.5 km and the hump is centred on that line."""
    lx, ly = 10_000.0, 5_000.0
    mesh = structured_mesh(lx, ly, nx, ny, mirror=mirror, ocean_side=None)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    hb = 5.0 + 15.0 * x / lx - 1.0 * np.sin(np.pi * x / lx) * np.sin(np.pi * y / ly)
    rng = np.random.default_rng(seed)
    xc = rng.uniform(0.3, 0.7) * lx
    yc = 0.5 * ly if mirror else rng.uniform(0.3, 0.7) * ly
    zeta0 = 0.5 * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (2 * 800.0**2)) if hump else np.zeros_like(x)
    rain_nodal = np.full(mesh.n_nodes, 50.0 * MMH) if rain else None
    return Workload(
        name="basin-400tri-p1", mesh=mesh, hb=hb, manning=np.full(mesh.n_tri, 0.025), zeta0=zeta0,
        p=1, steps=200, cfl=0.3, rain_nodal=rain_nodal, meta={"seed": seed, "hump_centre": (xc, yc)},
    )


def river_basin(q=(2.0, 0.5), ramp_s=600.0, nx=20, ny=10, wet=True, seed=7, internal=False) -> Workload:
    """The basin of ``basin_c1`` (no hump, no rain) with two river inflow segments on its walls:
    segment 0 on the x = 0 wall for 1 km <= y <= 3 km, segment 1 on the y = 5 km wall for
    6 km <= x <= 8 km.  With ``internal`` a third segment (q gives its discharge as a third value)
    lies inside the basin, on the interior edges of the line y = 2.5 km for 4 km <= x <= 6 km,
    listed west to east so that the river enters the triangles north of the line (an internal
    river boundary).  Discharge per unit width ramps linearly from 0 to q over ramp_s seconds
    (records every ramp_s / 4 s).  With wet=False the bathymetry rises above the geoid near the
    x = 0 river so that the river first flows onto dry land; the CFL number is then 0.04, since
    explicit Manning friction on films of about H0 (tau ~ 3/s) needs dt * tau < 1."""
    w = basin_c1(seed=seed, hump=False, rain=False, nx=nx, ny=ny)
    m = w.mesh
    mid = 0.5 * (m.xy[m.bedge[:, 0]] + m.xy[m.bedge[:, 1]])
    btype = m.btype.copy()
    bseg = m.bseg.copy()
    r0 = (mid[:, 0] < 1e-6) & (mid[:, 1] > 1000.0) & (mid[:, 1] < 3000.0)
    r1 = (mid[:, 1] > 5000.0 - 1e-6) & (mid[:, 0] > 6000.0) & (mid[:, 0] < 8000.0)
    btype[r0 | r1] = RIVER
    bseg[r0] = 0
    bseg[r1] = 1
    bedge = m.bedge
    if internal:
        lx, ly = 10_000.0, 5_000.0
        dx = lx / nx
        j = int(round(0.5 * ly / (ly / ny)))
        inner = np.array([(j * (nx + 1) + i, j * (nx + 1) + i + 1) for i in range(nx + 1)
                          if 4000.0 - 1e-6 <= i * dx and (i + 1) * dx <= 6000.0 + 1e-6], np.int32)
        bedge = np.concatenate([bedge, inner])
        btype = np.concatenate([btype, np.full(len(inner), RIVER, np.int32)])
        bseg = np.concatenate([bseg, np.full(len(inner), 2, np.int32)])
    w.mesh = Mesh(m.xy, m.tri, bedge, btype, bseg)
    if not wet:
        x = m.xy[:, 0]
        w.hb = w.hb - 8.0 * np.clip(1.0 - x / 2500.0, 0.0, None)
        w.zeta0 = _initial_dry(w.hb, w.h0)
        w.cfl = 0.04
    tq = np.linspace(0.0, 1.0, 5)[:, None] * np.asarray(q, float)[None, :]
    w.river = River(q=tq, t0=0.0, dt=ramp_s / 4.0)
    w.name = f"river-basin-{m.n_tri}tri-p1"
    return w


def inclined_plane(condition="A", duration=10.0, nx=240, ny=2, h0=1e-4, sim_s=86.4) -> Workload:
    """Rain on an initially dry inclined flume, after the set-up of Sec. 3.2: 24 m long, 19.6 cm
    wide; condition A: slope sin(theta) = 0.015, rain 0.0833 cm/s; condition B: three 8 m
    segments (top to bottom) with slopes 0.020, 0.015, 0.010 and rain 0.1080, 0.0638, 0.0800
    cm/s.  Rain falls for ``duration`` seconds (10, 20 or 30), Manning n = 0.009, dt = 1 ms.
    The flume walls are land; its downstream end (x = 24 m, bed at the geoid) is an open
    boundary held at the bed level (free outfall).  Mesh: nx x ny squares, mirrored about the
    flume axis.  The rain is a gridded field (5 cm cells, records every 0.1 s) so that it stops
    within one record after ``duration``."""
    lx, ly = 24.0, 0.196
    mesh = structured_mesh(lx, ly, nx, ny, mirror=True, ocean_side="x1")
    x = mesh.xy[:, 0]
    if condition == "A":
        slope = lambda xx: np.full_like(xx, 0.015)
        rate = lambda xx: np.full_like(xx, 0.0833e-2)
    else:
        slope = lambda xx: np.where(xx < 8.0, 0.020, np.where(xx < 16.0, 0.015, 0.010))
        rate = lambda xx: np.where(xx < 8.0, 0.1080e-2, np.where(xx < 16.0, 0.0638e-2, 0.0800e-2))
    # bed elevation above the outlet: integral of the slope from x to the downstream end
    xf = np.linspace(0.0, lx, 24001)
    zf = np.concatenate([[0.0], np.cumsum(0.5 * (slope(xf[1:]) + slope(xf[:-1])) * np.diff(xf))])
    zf = zf[-1] - zf
    hb = -np.interp(x, xf, zf)
    zeta0 = _initial_dry(hb, h0)
    gdx, gdt = 0.05, 0.1
    gx = np.arange(0.0, lx + 1e-9, gdx)
    nt = int(np.ceil(sim_s / gdt)) + 1
    tr = np.arange(nt) * gdt
    on = (tr <= duration + 1e-9).astype(np.float64)
    field = (on[:, None, None] * rate(gx)[None, None, :] * 3.6e6 * np.ones((1, 2, 1))).astype(np.float32)
    grid = RainGrid(len(gx), 2, nt, 0.0, 0.0, gdx, ly, 0.0, gdt, field)
    tide = Tide(np.array([0.0]), np.array([3600.0]), np.array([0.0]))
    return Workload(
        name=f"plane-{condition}-{int(duration)}s", mesh=mesh, hb=hb, manning=np.full(mesh.n_tri, 0.009),
        zeta0=zeta0, p=1, steps=int(round(sim_s / 1e-3)), cfl=0.0, rain_grid=grid, tide=tide, h0=h0,
        meta={"dt": 1e-3, "condition": condition, "duration": duration},
    )


def bathtub(nx=25, ny=4) -> Workload:
    """Bathtub of Sec. 3.1: 50 km x 8 km, 25x4 squares -> 200 triangles, bump bathymetry with
    x read in kilometres (the printed formula is unit-garbled), walls, quadratic friction
    0.001, dt 5 s, 1 inch/h rain for 24 h then 48 h dry."""
    lx, ly = 50_000.0, 8_000.0
    mesh = structured_mesh(lx, ly, nx, ny)
    x = mesh.xy[:, 0]
    hb = 5.0 - np.exp(-100.0 * (x / 1000.0 - 25.0) ** 2)
    return Workload(
        name="bathtub-200tri", mesh=mesh, hb=hb, manning=np.zeros(mesh.n_tri), zeta0=np.zeros(mesh.n_nodes),
        p=1, steps=72 * 3600 // 5, cfl=0.0, rain_nodal=np.full(mesh.n_nodes, 7.0556e-6),
        meta={"dt": 5.0, "rain_hours": 24.0, "cf": 0.001},
    )


def _coastal_bathymetry(x, y, lx, ly, land_top, rng_phase):
    """Offshore depth 3000 m (ocean side x=0) tapering across a shelf to a floodplain that rises
    above the geoid (negative h_b) near x = lx; a gentle seeded alongshore undulation."""
    s = x / lx
    deep = 3000.0
    shelf = 200.0
    wob = 0.02 * np.sin(2 * np.pi * (y / ly) * 3 + rng_phase)
    s = s + wob
    hb = np.where(
        s < 0.45,
        deep - (deep - shelf) * 0.5 * (1 - np.cos(np.pi * np.clip(s / 0.45, 0, 1))),
        np.where(
            s < 0.78,
            shelf * (1 - (s - 0.45) / 0.33),
            -land_top * np.clip((s - 0.78) / 0.22, 0.0, None),
        ),
    )
    return hb


def _initial_dry(hb, h0):
    """Nodal initial elevation: 0 over water; on land (hb < h0) a film of depth h0/2, so dry
    land starts clearly below the wet/dry threshold h0 instead of exactly on it (where the last
    bit of roundoff would pick the element's flag)."""
    return np.where(hb < h0, 0.5 * h0 - hb, 0.0)


def coastal_c2(n_tri=250_000, seed=2, steps=2000, fast_mesh=False) -> Workload:
    """Coastal wet/dry workload: jittered Delaunay mesh (~n_tri triangles) on 400 km x 300 km,
    p=1, 3000 m offshore depth tapering across a shelf to a floodplain rising to +2 m (about
    20% initially dry), Manning n ~ U[0.02, 0.06] per element, a moving radially symmetric rain
    cell (30 mm/h peak at 50 km radius, exponential decay, 5 m/s straight track) and a 0.5 m,
    12.42 h tide on the open (x = 0) side."""
    lx, ly = 400_000.0, 300_000.0
    rng = np.random.default_rng(seed)
    mesh = jittered_grid_mesh(lx, ly, n_tri, seed) if fast_mesh else jittered_delaunay(lx, ly, n_tri, seed)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    hb = _coastal_bathymetry(x, y, lx, ly, 2.0, rng.uniform(0, 2 * np.pi))
    manning = rng.uniform(0.02, 0.06, mesh.n_tri)
    h0 = 0.01
    zeta0 = _initial_dry(hb, h0)
    storm = Storm(x0=0.55 * lx, y0=rng.uniform(0.3, 0.7) * ly, heading=rng.uniform(-0.3, 0.3), speed=5.0,
                  rpeak=30.0 * MMH, rm=50_000.0, re=100_000.0)
    tide = Tide(np.array([0.5]), np.array([12.42 * 3600.0]), np.array([rng.uniform(0, 2 * np.pi)]))
    return Workload(
        name=f"coastal-{mesh.n_tri // 1000}k-p1", mesh=mesh, hb=hb, manning=manning, zeta0=zeta0, p=1,
        steps=steps, cfl=0.3, storm=storm, tide=tide, h0=h0, meta={"seed": seed},
    )


def graded_c3(n_tri=2_000_000, seed=3, steps=1000) -> Workload:
    """p=2 graded mesh: element sizes graded from 100 m at the coastline (x = 0.78 lx) to 5 km
    offshore and inland (a strip mesh; smaller n_tri scale both sizes by sqrt(2M / n_tri), the
    same generator at coarser sizing), same bathymetry/forcing families as the coastal workload
    with a new seed, plus a Gaussian pressure-driven set-up of 2 m peak at the coast; SSP(3,3)."""
    lx, ly = 400_000.0, 300_000.0
    rng = np.random.default_rng(seed)
    f = max(1.0, math.sqrt(2_000_000 / n_tri))
    mesh = graded_strip_mesh(lx, ly, 0.78 * lx, 100.0 * f, 5000.0 * f, n_tri, seed)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    hb = _coastal_bathymetry(x, y, lx, ly, 2.0, rng.uniform(0, 2 * np.pi))
    manning = rng.uniform(0.02, 0.06, mesh.n_tri)
    zeta0 = _initial_dry(hb, 0.01)
    storm = Storm(x0=0.55 * lx, y0=rng.uniform(0.3, 0.7) * ly, heading=rng.uniform(-0.3, 0.3), speed=5.0,
                  rpeak=30.0 * MMH, rm=50_000.0, re=100_000.0)
    tide = Tide(np.array([0.5]), np.array([12.42 * 3600.0]), np.array([rng.uniform(0, 2 * np.pi)]))
    pressure = (0.78 * lx, rng.uniform(0.35, 0.65) * ly, 60_000.0, 2.0)
    return Workload(
        name=f"graded-{mesh.n_tri // 1000}k-p2", mesh=mesh, hb=hb, manning=manning, zeta0=zeta0, p=2,
        steps=steps, cfl=0.3, storm=storm, tide=tide, pressure=pressure, meta={"seed": seed},
    )


def ensemble_c4(n_scen=64, lo=20_000, hi=400_000, seed=4, steps=500, fast_mesh=True) -> list[Workload]:
    """Ensemble of coastal scenarios on seeded meshes with log-uniform sizes in [lo, hi]; each
    has its own rain peak (10..80 mm/h), track heading, Manning field and tidal phase.  Meshes are
    jittered grids (``fast_mesh``) or jittered-point Delaunay triangulations."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_scen)).astype(int)
    out = []
    for s, n in enumerate(sizes):
        w = coastal_c2(int(n), seed=1000 * seed + s, steps=steps, fast_mesh=fast_mesh)
        w.storm.rpeak = rng.uniform(10.0, 80.0) * MMH
        w.storm.heading = rng.uniform(0.0, 2 * np.pi)
        w.tide.phase = np.array([rng.uniform(0, 2 * np.pi)])
        w.name = f"ens{s}-{w.mesh.n_tri}"
        out.append(w)
    return out


def hurricane_c5(n_tri=8_000_000, seed=5, hours=24.0) -> Workload:
    """Hurricane-scale basin: 1500 km x 1000 km, ~n_tri triangles, p=1, about 30% initially
    dry land rising to +10 m, hourly gridded rain on a 0.1 degree (~11.1 km) grid from a
    seeded smooth log-normal field clipped to [0, 100] mm/h.  Steps follow from 24 h at CFL
    0.3 once the solver has fixed dt (``steps`` is filled in by the caller)."""
    lx, ly = 1_500_000.0, 1_000_000.0
    rng = np.random.default_rng(seed)
    mesh = jittered_grid_mesh(lx, ly, n_tri, seed)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    s = x / lx + 0.02 * np.sin(2 * np.pi * 2 * y / ly + rng.uniform(0, 2 * np.pi))
    hb = np.where(s < 0.4, 3000.0 - 2800.0 * 0.5 * (1 - np.cos(np.pi * np.clip(s / 0.4, 0, 1))),
                  np.where(s < 0.7, 200.0 * (1 - (s - 0.4) / 0.3), -10.0 * np.clip((s - 0.7) / 0.3, 0, None)))
    manning = rng.uniform(0.02, 0.06, mesh.n_tri)
    zeta0 = _initial_dry(hb, 0.01)
    dx = 11_100.0
    nxg = int(math.ceil(lx / dx)) + 1
    nyg = int(math.ceil(ly / dx)) + 1
    nt = int(hours) + 1
    field = _smooth_lognormal(rng, nt, nyg, nxg)
    grid = RainGrid(nxg, nyg, nt, 0.0, 0.0, dx, dx, 0.0, 3600.0, field)
    tide = Tide(np.array([0.5]), np.array([12.42 * 3600.0]), np.array([rng.uniform(0, 2 * np.pi)]))
    return Workload(
        name=f"hurricane-{mesh.n_tri // 1000}k-p1", mesh=mesh, hb=hb, manning=manning, zeta0=zeta0, p=1,
        steps=0, cfl=0.3, rain_grid=grid, tide=tide, meta={"seed": seed, "hours": hours},
    )


def _smooth_lognormal(rng, nt, ny, nx):
    """Smooth log-normal rain field (mm/h) clipped to [0, 100]: Gaussian-filtered white noise in
    log space with a slow drift between hourly records."""
    from scipy.ndimage import gaussian_filter

    base = gaussian_filter(rng.standard_normal((ny, nx)), sigma=6.0, mode="wrap")
    out = np.empty((nt, ny, nx), np.float32)
    for k in range(nt):
        pert = gaussian_filter(rng.standard_normal((ny, nx)), sigma=6.0, mode="wrap")
        f = base + 0.3 * pert
        f = f / (f.std() + 1e-12)
        out[k] = np.clip(np.exp(1.0 + 1.2 * f), 0.0, 100.0)
    return out


def mms_square(n, lx=1.0, ly=1.0) -> Mesh:
    """Unit-square structured mesh for manufactured-solution refinement studies."""
    return structured_mesh(lx, ly, n, n)
