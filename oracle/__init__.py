"""ctypes binding of the FP64 CPU oracle (``dgswe_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs are the only callers.  The CUDA library never
imports, links or calls anything here, and nothing here imports the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgswe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ROE, LLF = 0, 1
MANNING, QUADRATIC, NOFRICTION = 0, 1, 2
BT_LAND, BT_OCEAN, BT_EXACT = 0, 1, 3

_d = C.POINTER(C.c_double)
_i = C.POINTER(C.c_int32)
_u8 = C.POINTER(C.c_uint8)
_f = C.POINTER(C.c_float)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, -O2, no vectorisation flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_mesh.argtypes = [C.c_void_p, C.c_int, _d, C.c_int, _i, C.c_int, _i, _i, _i]
        L.orc_set_fields.argtypes = [C.c_void_p, _d, _d]
        L.orc_set_rain_nodal.argtypes = [C.c_void_p, _d]
        L.orc_set_rain_parametric.argtypes = [C.c_void_p] + [C.c_double] * 8
        L.orc_set_rain_grid.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int] + [C.c_double] * 6 + [_f]
        L.orc_set_tide.argtypes = [C.c_void_p, C.c_int, _d, _d, _d]
        L.orc_set_river.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, _d]
        L.orc_set_limiter.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
        L.orc_apply_limiter.argtypes = [C.c_void_p]
        L.orc_set_pressure.argtypes = [C.c_void_p] + [C.c_double] * 4
        L.orc_set_exact_wave.argtypes = [C.c_void_p] + [C.c_double] * 5
        L.orc_set_exact_linear.argtypes = [C.c_void_p, _d]
        L.orc_set_state_nodal.argtypes = [C.c_void_p, _d, _d, _d]
        L.orc_set_state_modal.argtypes = [C.c_void_p, _d]
        L.orc_get_state.argtypes = [C.c_void_p, _d]
        L.orc_get_vertex_values.argtypes = [C.c_void_p, _d]
        L.orc_get_dry.argtypes = [C.c_void_p, _u8]
        L.orc_cfl_dt.restype = C.c_double
        L.orc_cfl_dt.argtypes = [C.c_void_p, C.c_double]
        L.orc_set_dt.argtypes = [C.c_void_p, C.c_double]
        L.orc_set_time.argtypes = [C.c_void_p, C.c_double]
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_rhs.argtypes = [C.c_void_p, _d]
        L.orc_get_ledger.argtypes = [C.c_void_p, _d]
        L.orc_l2_error_exact.restype = C.c_double
        L.orc_l2_error_exact.argtypes = [C.c_void_p, C.c_int]
        L.orc_basis.argtypes = [C.c_int, C.c_double, C.c_double, _d, _d, _d]
        L.orc_area_rule.restype = C.c_int
        L.orc_area_rule.argtypes = [C.c_int, _d, _d, _d]
        L.orc_edge_rule.restype = C.c_int
        L.orc_edge_rule.argtypes = [C.c_int, _d, _d]
        L.orc_numflux.argtypes = [C.c_int, C.c_double, C.c_double, _d, C.c_double, _d, C.c_double, C.c_double,
                                  C.c_double, _d]
        L.orc_positivity_vertex.restype = C.c_int
        L.orc_positivity_vertex.argtypes = [C.c_double, _d, _d, _d, _d, _d, _d, _u8]
        L.orc_positivity_modal.restype = C.c_int
        L.orc_positivity_modal.argtypes = [C.c_int, C.c_double, _d, _d]
        L.orc_ssp_amplification.restype = C.c_double
        L.orc_ssp_amplification.argtypes = [C.c_int, C.c_double]
        _lib = L
    return _lib


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Oracle:
    """One oracle instance: a mesh, its fields, forcing, state and ledger."""

    def __init__(self, mesh, hb, manning=None, p=1, flux=ROE, ssp=None, g=9.81, h0=0.01, friction=MANNING,
                 cf=0.0):
        L = lib()
        self.p = p
        self.np_ = (p + 1) * (p + 2) // 2
        ssp = ssp if ssp is not None else min(p + 1, 3)
        self.h = L.orc_create(p, flux, ssp, g, h0, friction, cf)
        if not self.h:
            raise ValueError("invalid oracle parameters")
        self._keep = []
        xy = _f64(mesh.xy)
        tri = _i32(mesh.tri)
        be, bt, bs = _i32(mesh.bedge), _i32(mesh.btype), _i32(mesh.bseg)
        rc = L.orc_set_mesh(self.h, xy.shape[0], _p(xy), tri.shape[0], _p(tri, _i), be.shape[0], _p(be, _i),
                            _p(bt, _i), _p(bs, _i))
        if rc < 0:
            raise ValueError(f"orc_set_mesh failed ({rc})")
        self.ne = tri.shape[0]
        self.nn = xy.shape[0]
        man = _f64(manning if manning is not None else np.zeros(self.ne))
        L.orc_set_fields(self.h, _p(_f64(hb)), _p(man))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # forcing -------------------------------------------------------------------------------
    def set_rain_nodal(self, r):
        lib().orc_set_rain_nodal(self.h, _p(_f64(r)))

    def set_storm(self, s):
        lib().orc_set_rain_parametric(self.h, s.x0, s.y0, s.heading, s.speed, s.rpeak, s.rm, s.re, s.t0)

    def set_rain_grid(self, g):
        a = np.ascontiguousarray(g.mm_per_h, dtype=np.float32)
        self._keep.append(a)
        lib().orc_set_rain_grid(self.h, g.nx, g.ny, g.nt, g.x0, g.y0, g.dx, g.dy, g.t0, g.dt_rec, _p(a, _f))

    def set_tide(self, t):
        lib().orc_set_tide(self.h, len(t.amp), _p(_f64(t.amp)), _p(_f64(t.period)), _p(_f64(t.phase)))

    def set_limiter(self, on=True, nu=1.5, M=0.0):
        lib().orc_set_limiter(self.h, 1 if on else 0, nu, M)

    def apply_limiter(self):
        lib().orc_apply_limiter(self.h)

    def set_river(self, r):
        q = np.ascontiguousarray(np.atleast_2d(np.asarray(r.q, dtype=np.float64)))
        lib().orc_set_river(self.h, q.shape[1], q.shape[0], r.t0, r.dt, _p(q))

    def set_pressure(self, x0, y0, sigma, peak):
        lib().orc_set_pressure(self.h, x0, y0, sigma, peak)

    def set_exact_wave(self, a, k, l, c, h0):
        lib().orc_set_exact_wave(self.h, a, k, l, c, h0)

    def set_exact_linear(self, coef9):
        lib().orc_set_exact_linear(self.h, _p(_f64(coef9)))

    # state ---------------------------------------------------------------------------------
    def set_state_nodal(self, zeta, qx=None, qy=None):
        z = _f64(zeta)
        qx = _f64(qx if qx is not None else np.zeros_like(z))
        qy = _f64(qy if qy is not None else np.zeros_like(z))
        lib().orc_set_state_nodal(self.h, _p(z), _p(qx), _p(qy))

    def set_state_modal(self, w):
        lib().orc_set_state_modal(self.h, _p(_f64(w)))

    def state(self) -> np.ndarray:
        """Modal state as [E, 3, Np] (variables zeta, qx, qy)."""
        w = np.empty((self.ne, 3, self.np_))
        lib().orc_get_state(self.h, _p(w))
        return w

    def vertex_values(self) -> np.ndarray:
        v = np.empty((self.ne, 3, 3))
        lib().orc_get_vertex_values(self.h, _p(v))
        return v

    def dry(self) -> np.ndarray:
        d = np.empty(self.ne, np.uint8)
        lib().orc_get_dry(self.h, _p(d, _u8))
        return d

    def rhs(self) -> np.ndarray:
        L = np.empty((self.ne, 3, self.np_))
        lib().orc_rhs(self.h, _p(L))
        return L

    def cfl_dt(self, cfl):
        return lib().orc_cfl_dt(self.h, cfl)

    def set_dt(self, dt):
        lib().orc_set_dt(self.h, dt)

    def set_time(self, t):
        lib().orc_set_time(self.h, t)

    def step(self, n):
        lib().orc_step(self.h, int(n))

    def ledger(self) -> dict:
        o = np.empty(8)
        lib().orc_get_ledger(self.h, _p(o))
        keys = ["t", "V0", "V", "rain_in", "bdry_in", "VH0", "rel_err", "wet_frac"]
        return dict(zip(keys, o.tolist()))

    def l2_error_exact(self, var=0):
        return lib().orc_l2_error_exact(self.h, var)


def from_workload(w, flux=ROE, ssp=None, dt=None, friction=MANNING, cf=0.0) -> Oracle:
    """Oracle set up with a workload's mesh, fields, forcing and initial (nodal) state."""
    o = Oracle(w.mesh, w.hb, w.manning, p=w.p, flux=flux, ssp=ssp, h0=w.h0, friction=friction, cf=cf)
    if w.rain_nodal is not None:
        o.set_rain_nodal(w.rain_nodal)
    if w.storm is not None:
        o.set_storm(w.storm)
    if w.rain_grid is not None:
        o.set_rain_grid(w.rain_grid)
    if w.tide is not None:
        o.set_tide(w.tide)
    if w.pressure is not None:
        o.set_pressure(*w.pressure)
    if getattr(w, "river", None) is not None:
        o.set_river(w.river)
    o.set_state_nodal(w.zeta0)
    o.set_dt(dt if dt is not None else o.cfl_dt(w.cfl))
    return o


# component hooks ---------------------------------------------------------------------------
def basis(p, r, s):
    n = (p + 1) * (p + 2) // 2
    phi, dr, ds = np.empty(n), np.empty(n), np.empty(n)
    lib().orc_basis(p, r, s, _p(phi), _p(dr), _p(ds))
    return phi, dr, ds


def area_rule(p):
    r, s, w = np.empty(16), np.empty(16), np.empty(16)
    n = lib().orc_area_rule(p, _p(r), _p(s), _p(w))
    return r[:n], s[:n], w[:n]


def edge_rule(p):
    x, w = np.empty(4), np.empty(4)
    n = lib().orc_edge_rule(p, _p(x), _p(w))
    return x[:n], w[:n]


def numflux(kind, wl, hbl, wr, hbr, n, g=9.81, h0=0.01):
    f = np.empty(3)
    lib().orc_numflux(kind, g, h0, _p(_f64(wl)), hbl, _p(_f64(wr)), hbr, n[0], n[1], _p(f))
    return f


def positivity_vertex(H, qx, qy, h0=0.01):
    Ho, qxo, qyo = np.empty(3), np.empty(3), np.empty(3)
    dry = np.empty(3, np.uint8)
    c = lib().orc_positivity_vertex(h0, _p(_f64(H)), _p(Ho), _p(_f64(qx)), _p(_f64(qy)), _p(qxo), _p(qyo),
                                    _p(dry, _u8))
    return c, Ho, qxo, qyo, dry


def positivity_modal(p, w, hbv, h0=0.01):
    """M Pi_h on one element: w [3][Np] modal (zeta, qx, qy) -> (new modes, dry)."""
    out = np.ascontiguousarray(np.array(w, dtype=np.float64).reshape(3, -1))
    rc = lib().orc_positivity_modal(p, h0, _p(_f64(hbv)), _p(out))
    if rc < 0:
        raise ValueError("p must be 0, 1 or 2")
    return out, bool(rc)


def ssp_amplification(stages, z):
    return lib().orc_ssp_amplification(stages, z)
