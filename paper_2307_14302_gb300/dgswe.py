"""Python binding of libdgswe (include/dgswe.h): the same entry points, argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays to pointers and
return codes to exceptions.  Importing it does not load the library; the first call does, and
raises ``DgsweUnavailable`` when ``libdgswe.so`` is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgswe.so")

FLUX_ROE, FLUX_LLF = 0, 1
FP64, MIXED = 0, 1
MANNING, QUADRATIC, NOFRICTION = 0, 1, 2
LAYOUT_MODAL, LAYOUT_NODAL = 0, 1
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ENEGDEPTH", -6: "ETIMEOUT",
          -7: "ESTATE", -8: "ENOLIB"}


class DgsweUnavailable(RuntimeError):
    pass


class DgsweError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("flux", C.c_int32), ("ssp_stages", C.c_int32), ("precision", C.c_int32),
                ("g", C.c_double), ("H0", C.c_double), ("cfl", C.c_double), ("dt", C.c_double),
                ("friction", C.c_int32), ("cf", C.c_double), ("limiter", C.c_int32), ("lim_nu", C.c_double),
                ("lim_M", C.c_double)]


class Storm(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("x0", "y0", "heading", "speed", "rpeak", "rm", "re", "t0")]


class GaussSetup(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("x0", "y0", "sigma", "peak")]


class Ledger(C.Structure):
    _fields_ = [("t", C.c_double), ("steps", C.c_int64), ("V0", C.c_double), ("V", C.c_double),
                ("rain_in", C.c_double), ("bdry_in", C.c_double), ("VH0", C.c_double), ("rel_err", C.c_double),
                ("wet_frac", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = [
    "dgswe_create", "dgswe_set_params", "dgswe_set_mesh", "dgswe_set_fields", "dgswe_set_rain_nodal",
    "dgswe_set_rain_parametric", "dgswe_set_rain_grid", "dgswe_set_tide", "dgswe_set_river", "dgswe_set_pressure_setup",
    "dgswe_set_state", "dgswe_load_state", "dgswe_exchange_state", "dgswe_step", "dgswe_sync", "dgswe_get_dt", "dgswe_get_state", "dgswe_get_state_device",
    "dgswe_get_dry", "dgswe_get_ledger", "dgswe_volume", "dgswe_record_bytes", "dgswe_bind_device", "dgswe_volume_sum_noalloc", "dgswe_ensemble_create", "dgswe_ensemble_step",
    "dgswe_ensemble_get_state", "dgswe_ensemble_get_ledger", "dgswe_set_launch", "dgswe_get_launch", "dgswe_get_tile_features",
    "dgswe_set_graphs", "dgswe_launch_count", "dgswe_destroy", "dgswe_last_error",
]

_lib = None
_d = C.POINTER(C.c_double)
_i = C.POINTER(C.c_int32)
_f = C.POINTER(C.c_float)
_u8 = C.POINTER(C.c_uint8)
_h = C.c_void_p


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise DgsweUnavailable(f"{LIB_PATH} is missing: build it with paper_2307_14302_gb300.build.build()")
    try:
        L = C.CDLL(LIB_PATH)
    except OSError as e:
        raise DgsweUnavailable(f"cannot load {LIB_PATH}: {e}") from e
    sig = {
        "dgswe_create": ([C.POINTER(_h), C.c_int, C.c_void_p], C.c_int),
        "dgswe_set_params": ([_h, C.POINTER(Params)], C.c_int),
        "dgswe_set_mesh": ([_h, C.c_int32, _d, C.c_int32, _i, C.c_int32, _i, _i, _i], C.c_int),
        "dgswe_set_fields": ([_h, _d, _d, C.c_int32], C.c_int),
        "dgswe_set_rain_nodal": ([_h, _d], C.c_int),
        "dgswe_set_rain_parametric": ([_h, C.POINTER(Storm)], C.c_int),
        "dgswe_set_rain_grid": ([_h, C.c_int32, C.c_int32, C.c_int32] + [C.c_double] * 6 + [_f], C.c_int),
        "dgswe_set_tide": ([_h, C.c_int32, _d, _d, _d], C.c_int),
        "dgswe_set_river": ([_h, C.c_int32, C.c_int32, C.c_double, C.c_double, _d], C.c_int),
        "dgswe_set_pressure_setup": ([_h, C.POINTER(GaussSetup)], C.c_int),
        "dgswe_set_state": ([_h, _d, _d, _d, C.c_int32, C.c_double], C.c_int),
        "dgswe_load_state": ([_h, _d, _d, _d], C.c_int),
        "dgswe_exchange_state": ([_h, _d, _d, _d, _d, _d, _d], C.c_int),
        "dgswe_step": ([_h, C.c_int64], C.c_int),
        "dgswe_sync": ([_h], C.c_int),
        "dgswe_get_dt": ([_h, _d], C.c_int),
        "dgswe_get_state": ([_h, _d, _d, _d], C.c_int),
        "dgswe_get_state_device": ([_h, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
        "dgswe_get_dry": ([_h, _u8], C.c_int),
        "dgswe_get_ledger": ([_h, C.POINTER(Ledger)], C.c_int),
        "dgswe_volume": ([_h, _d], C.c_int),
        "dgswe_record_bytes": ([_h, C.POINTER(C.c_uint64)], C.c_int),
        "dgswe_bind_device": ([_h, C.c_void_p, C.c_uint64], C.c_int),
        "dgswe_volume_sum_noalloc": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
        "dgswe_ensemble_create": ([C.POINTER(_h), C.c_int32, C.POINTER(_h), C.c_int, C.c_void_p], C.c_int),
        "dgswe_ensemble_step": ([_h, C.c_int64], C.c_int),
        "dgswe_ensemble_get_state": ([_h, C.c_int32, _d, _d, _d], C.c_int),
        "dgswe_ensemble_get_ledger": ([_h, C.c_int32, C.POINTER(Ledger)], C.c_int),
        "dgswe_set_launch": ([_h, C.c_int32, C.c_int32, C.c_int32], C.c_int),
        "dgswe_get_launch": ([_h, _i, _i, _i], C.c_int),
        "dgswe_get_tile_features": ([_h, _i, _i], C.c_int),
        "dgswe_launch_count": ([_h], C.c_int64),
        "dgswe_set_graphs": ([_h, C.c_int32], C.c_int),
        "dgswe_destroy": ([_h], None),
        "dgswe_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise DgsweError(rc, lib().dgswe_last_error().decode())


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Solver:
    """One library context (dgswe_create ... dgswe_destroy)."""

    def __init__(self, p=1, flux=FLUX_ROE, ssp_stages=None, precision=MIXED, g=9.81, H0=0.01, cfl=0.3, dt=0.0,
                 friction=MANNING, cf=0.0, device=0, stream=None, limiter=False, lim_nu=1.5, lim_M=0.0):
        L = lib()
        h = _h()
        _check(L.dgswe_create(C.byref(h), device, C.c_void_p(stream) if stream else None))
        self.h = h
        self.p = p
        self.np_ = (p + 1) * (p + 2) // 2
        self.prm = Params(p, flux, ssp_stages if ssp_stages else min(p + 1, 3), precision, g, H0, cfl, dt, friction, cf,
                          1 if limiter else 0, lim_nu, lim_M)
        _check(L.dgswe_set_params(self.h, C.byref(self.prm)))
        self.ne = 0
        self._members = []

    def close(self):
        if getattr(self, "h", None):
            lib().dgswe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mesh(self, mesh):
        xy, tri = _f64(mesh.xy), _i32(mesh.tri)
        be, bt, bs = _i32(mesh.bedge), _i32(mesh.btype), _i32(mesh.bseg)
        _check(lib().dgswe_set_mesh(self.h, xy.shape[0], _p(xy), tri.shape[0], _p(tri, _i), be.shape[0],
                                    _p(be, _i), _p(bt, _i), _p(bs, _i)))
        self.ne = tri.shape[0]
        self.nn = xy.shape[0]

    def set_fields(self, hb, manning=None, manning_nodal=False):
        man = None if manning is None else _f64(manning)
        _check(lib().dgswe_set_fields(self.h, _p(_f64(hb)), None if man is None else _p(man), int(manning_nodal)))

    def set_rain_nodal(self, r):
        _check(lib().dgswe_set_rain_nodal(self.h, _p(_f64(r))))

    def set_storm(self, s):
        st = Storm(s.x0, s.y0, s.heading, s.speed, s.rpeak, s.rm, s.re, s.t0)
        _check(lib().dgswe_set_rain_parametric(self.h, C.byref(st)))

    def set_rain_grid(self, g):
        a = np.ascontiguousarray(g.mm_per_h, dtype=np.float32)
        _check(lib().dgswe_set_rain_grid(self.h, g.nx, g.ny, g.nt, g.x0, g.y0, g.dx, g.dy, g.t0, g.dt_rec,
                                         _p(a, _f)))

    def set_tide(self, t):
        _check(lib().dgswe_set_tide(self.h, len(t.amp), _p(_f64(t.amp)), _p(_f64(t.period)), _p(_f64(t.phase))))

    def set_river(self, r):
        """River discharge series (workloads.River: q [nt, nseg] m^2/s into the domain)."""
        q = np.ascontiguousarray(np.atleast_2d(np.asarray(r.q, dtype=np.float64)))
        _check(lib().dgswe_set_river(self.h, q.shape[1], q.shape[0], float(r.t0), float(r.dt), _p(q)))

    def set_pressure_setup(self, x0, y0, sigma, peak):
        gs = GaussSetup(x0, y0, sigma, peak)
        _check(lib().dgswe_set_pressure_setup(self.h, C.byref(gs)))

    def set_state(self, zeta, qx=None, qy=None, layout=LAYOUT_NODAL, t0=0.0):
        z = _f64(zeta)
        qx = _f64(qx if qx is not None else np.zeros_like(z))
        qy = _f64(qy if qy is not None else np.zeros_like(z))
        _check(lib().dgswe_set_state(self.h, _p(z), _p(qx), _p(qy), layout, t0))

    def load_state(self, z, x, y):
        """Modal arrays [Np][E] (caller order), e.g. from state_arrays()."""
        _check(lib().dgswe_load_state(self.h, _p(z), _p(x), _p(y)))

    def exchange(self, zi, xi, yi, zo=None, xo=None, yo=None):
        """The current modal state out (filled in place when given, e.g. pinned) and (zi, xi, yi)
        in as the new state, in one call; returns the outputs."""
        if zo is None:
            zo, xo, yo = (np.empty((self.np_, self.ne)) for _ in range(3))
        _check(lib().dgswe_exchange_state(self.h, _p(zi), _p(xi), _p(yi), _p(zo), _p(xo), _p(yo)))
        return zo, xo, yo

    def step(self, n):
        _check(lib().dgswe_step(self.h, int(n)))

    def sync(self):
        _check(lib().dgswe_sync(self.h))

    def state_arrays(self, z=None, x=None, y=None):
        """Modal state as three [Np][E] arrays (filled in place when given, e.g. pinned)."""
        if z is None:
            z, x, y = (np.empty((self.np_, self.ne)) for _ in range(3))
        _check(lib().dgswe_get_state(self.h, _p(z), _p(x), _p(y)))
        return z, x, y

    def dt(self):
        v = C.c_double()
        _check(lib().dgswe_get_dt(self.h, C.byref(v)))
        return v.value

    def state(self) -> np.ndarray:
        """Modal state as [E, 3, Np] (caller element order), like the oracle's layout."""
        z, x, y = (np.empty((self.np_, self.ne)) for _ in range(3))
        _check(lib().dgswe_get_state(self.h, _p(z), _p(x), _p(y)))
        return np.stack([z.T, x.T, y.T], axis=1)

    def state_device(self, z_ptr, x_ptr, y_ptr):
        _check(lib().dgswe_get_state_device(self.h, z_ptr, x_ptr, y_ptr))

    def dry(self) -> np.ndarray:
        d = np.empty(self.ne, np.uint8)
        _check(lib().dgswe_get_dry(self.h, _p(d, _u8)))
        return d

    def ledger(self) -> dict:
        led = Ledger()
        _check(lib().dgswe_get_ledger(self.h, C.byref(led)))
        return led.as_dict()

    def volume(self) -> float:
        v = C.c_double()
        _check(lib().dgswe_volume(self.h, C.byref(v)))
        return v.value

    def record_bytes(self) -> int:
        v = C.c_uint64()
        _check(lib().dgswe_record_bytes(self.h, C.byref(v)))
        return v.value

    def bind_device(self, ptr, nbytes):
        """Element records in caller-owned device memory (e.g. a torch tensor's storage); ptr 0 unbinds."""
        _check(lib().dgswe_bind_device(self.h, C.c_void_p(ptr) if ptr else None, int(nbytes)))

    def set_launch(self, block, waves=1, split=1):
        _check(lib().dgswe_set_launch(self.h, block, waves, split))

    def launch(self):
        b, w, sp = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().dgswe_get_launch(self.h, C.byref(b), C.byref(w), C.byref(sp)))
        return b.value, w.value, sp.value

    def tile_features(self):
        """(features of the run, features compiled into the tile kernel it launches) as bit sets."""
        r, k = C.c_int32(), C.c_int32()
        _check(lib().dgswe_get_tile_features(self.h, C.byref(r), C.byref(k)))
        return r.value, k.value

    def launch_count(self) -> int:
        return int(lib().dgswe_launch_count(self.h))

    def set_graphs(self, on: bool):
        """Replay steps from CUDA graphs (default) or launch every stage directly."""
        _check(lib().dgswe_set_graphs(self.h, 1 if on else 0))


def volume_sum_noalloc(w0_ptr, area_ptr, n, out_ptr, stream=None):
    """dgswe_volume_sum_noalloc on caller-owned device pointers (allocates nothing)."""
    _check(lib().dgswe_volume_sum_noalloc(C.c_void_p(w0_ptr), C.c_void_p(area_ptr), int(n), C.c_void_p(out_ptr),
                                          C.c_void_p(stream) if stream else None))


class Ensemble:
    """dgswe_ensemble_create over already set-up Solvers (their data is copied)."""

    def __init__(self, members, device=0, stream=None):
        L = lib()
        arr = (_h * len(members))(*[m.h for m in members])
        h = _h()
        _check(L.dgswe_ensemble_create(C.byref(h), len(members), arr, device, C.c_void_p(stream) if stream else None))
        self.h = h
        self.sizes = [(m.ne, m.np_) for m in members]

    def close(self):
        if getattr(self, "h", None):
            lib().dgswe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n):
        _check(lib().dgswe_ensemble_step(self.h, int(n)))

    def sync(self):
        _check(lib().dgswe_sync(self.h))

    def state(self, i) -> np.ndarray:
        ne, npm = self.sizes[i]
        z, x, y = (np.empty((npm, ne)) for _ in range(3))
        _check(lib().dgswe_ensemble_get_state(self.h, i, _p(z), _p(x), _p(y)))
        return np.stack([z.T, x.T, y.T], axis=1)

    def ledger(self, i) -> dict:
        led = Ledger()
        _check(lib().dgswe_ensemble_get_ledger(self.h, i, C.byref(led)))
        return led.as_dict()

    def set_launch(self, block, waves=1, split=1):
        _check(lib().dgswe_set_launch(self.h, block, waves, split))

    def launch(self):
        b, w, s = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().dgswe_get_launch(self.h, C.byref(b), C.byref(w), C.byref(s)))
        return b.value, w.value, s.value

    def launch_count(self) -> int:
        return int(lib().dgswe_launch_count(self.h))

    def set_graphs(self, on: bool):
        _check(lib().dgswe_set_graphs(self.h, 1 if on else 0))


def from_workload(w, precision=MIXED, flux=FLUX_ROE, ssp_stages=None, dt=0.0, friction=MANNING, cf=0.0, device=0,
                  stream=None, block=0, waves=1, split=1, limiter=False, lim_nu=1.5, lim_M=0.0) -> Solver:
    """A Solver set up with a workload's mesh, fields, forcing and nodal initial state."""
    s = Solver(p=w.p, flux=flux, ssp_stages=ssp_stages, precision=precision, H0=w.h0, cfl=w.cfl, dt=dt,
               friction=friction, cf=cf, device=device, stream=stream, limiter=limiter, lim_nu=lim_nu, lim_M=lim_M)
    s.set_launch(block, waves, split)
    s.set_mesh(w.mesh)
    s.set_fields(w.hb, w.manning if friction == MANNING else None)
    if w.rain_nodal is not None:
        s.set_rain_nodal(w.rain_nodal)
    if w.storm is not None:
        s.set_storm(w.storm)
    if w.rain_grid is not None:
        s.set_rain_grid(w.rain_grid)
    if w.tide is not None:
        s.set_tide(w.tide)
    if w.pressure is not None:
        s.set_pressure_setup(*w.pressure)
    if getattr(w, "river", None) is not None:
        s.set_river(w.river)
    s.set_state(w.zeta0)
    return s
