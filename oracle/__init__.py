"""FP64 CPU oracle of the FullSWOF_2D time step -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
arm may import this package.  The product path (paper_1307_4839_gb300) never
does; the two share no code.

`build()` compiles swof_oracle.c (plain C, -O2 -ffp-contract=off, OpenMP over
rows) into oracle/_build/liboracle.so; `Oracle` drives it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swof_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleParams(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("cfl", ctypes.c_double),
                ("h_dry", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("t_end", ctypes.c_double), ("cfl_mode", ctypes.c_int),
                ("bc", ctypes.c_int * 4), ("friction", ctypes.c_int),
                ("fric_coef", ctypes.c_double), ("rain_rate", ctypes.c_double),
                ("rain_t_on", ctypes.c_double), ("rain_t_off", ctypes.c_double),
                ("infiltration", ctypes.c_int), ("ks", ctypes.c_double),
                ("psi", ctypes.c_double), ("dtheta", ctypes.c_double),
                ("check_cfl", ctypes.c_int), ("dt_fixed", ctypes.c_double),
                ("order", ctypes.c_int), ("bc_h", ctypes.c_double * 4),
                ("bc_q", ctypes.c_double * 4)]


_D = ctypes.POINTER(ctypes.c_double)


def load_library(path: str):
    """Load an oracle shared library and declare its C signatures."""
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _declare(L):
    L.oracle_create.restype = ctypes.c_void_p
    L.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, _D, ctypes.POINTER(OracleParams),
                                _D, _D]
    L.oracle_destroy.argtypes = [ctypes.c_void_p]
    for f in ("oracle_set_state", "oracle_get_state"):
        getattr(L, f).argtypes = [ctypes.c_void_p, _D, _D, _D]
    L.oracle_set_vinf.argtypes = [ctypes.c_void_p, _D]
    L.oracle_get_vinf.argtypes = [ctypes.c_void_p, _D]
    L.oracle_set_time.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.oracle_set_dt_sequence.argtypes = [ctypes.c_void_p, _D, ctypes.c_int]
    L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
    L.oracle_step.restype = ctypes.c_int
    L.oracle_diag.argtypes = [ctypes.c_void_p, _D]
    L.oracle_lambda.argtypes = [ctypes.c_void_p, _D, _D]
    L.oracle_minmod.restype = ctypes.c_double
    L.oracle_minmod.argtypes = [ctypes.c_double, ctypes.c_double]
    L.oracle_icbrt.restype = ctypes.c_double
    L.oracle_icbrt.argtypes = [ctypes.c_double]
    L.oracle_hll.argtypes = [ctypes.c_double] * 7 + [_D]
    L.oracle_threads.restype = ctypes.c_int
    L.oracle_friction_cf.restype = ctypes.c_double
    L.oracle_friction_cf.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.oracle_inflow_celerity.restype = ctypes.c_double
    L.oracle_inflow_celerity.argtypes = [ctypes.c_double, ctypes.c_double]
    L.oracle_imposed_state.argtypes = ([ctypes.c_double, ctypes.c_double, ctypes.c_int]
                                       + [ctypes.c_double] * 5 + [_D])
    L.oracle_track_max.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.oracle_get_max.argtypes = [ctypes.c_void_p, _D]
    L.oracle_get_max.restype = ctypes.c_int
    L.oracle_set_gauges.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                    ctypes.c_int]
    L.oracle_set_gauges.restype = ctypes.c_int
    L.oracle_get_gauges.argtypes = [ctypes.c_void_p, _D, ctypes.c_int]
    L.oracle_get_gauges.restype = ctypes.c_int
    L.oracle_d8.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_float, ctypes.POINTER(ctypes.c_uint8)]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def minmod(a: float, b: float) -> float:
    return lib().oracle_minmod(a, b)


def icbrt(x: float) -> float:
    return lib().oracle_icbrt(x)


def hll(g, hL, unL, utL, hR, unR, utR) -> np.ndarray:
    F = np.zeros(3)
    lib().oracle_hll(g, hL, unL, utL, hR, unR, utR, _ptr(F))
    return F


def threads() -> int:
    return lib().oracle_threads()


def friction_cf(law: int, g: float, coef: float) -> float:
    """C_f of Sec. 2.1 for law 1 Manning n, 2 Strickler K, 3 Darcy-Weisbach f, 4 Chezy C."""
    return lib().oracle_friction_cf(int(law), g, coef)


def inflow_celerity(R: float, Q: float) -> float:
    """Positive root c of 2c^3 + R c^2 - Q (imposed-discharge boundary state, Sec. 2.2)."""
    return lib().oracle_inflow_celerity(R, Q)


def imposed_state(g, h_dry, kind, hset, qset, h1, qn1, qt1) -> np.ndarray:
    """Boundary state (h, normal q inwards, tangential q) of an imposed edge."""
    out = np.zeros(3)
    lib().oracle_imposed_state(g, h_dry, int(kind), hset, qset, h1, qn1, qt1, _ptr(out))
    return out


def d8(z, nodata: float | None = None) -> np.ndarray:
    """D8 flow-direction codes (uint8, 0 = no lower neighbour) of a float32
    DEM [ny][nx]; neighbours with z <= nodata are no candidates (None: no
    no-data value)."""
    z = np.ascontiguousarray(z, dtype=np.float32)
    ny, nx = z.shape
    out = np.zeros((ny, nx), dtype=np.uint8)
    lib().oracle_d8(z.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nx, ny, int(nodata is not None),
                    float(nodata if nodata is not None else 0.0),
                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle run: grid, topography, parameters, state and diagnostics."""

    DIAG_KEYS = ("t", "last_dt", "steps", "volume", "rain_in", "infiltrated",
                 "outflow", "min_h", "cfl_viol")

    def __init__(self, nx, ny, dx, dy, z, *, g=9.81, cfl=0.5, h_dry=1e-6,
                 dt_max=0.1, t_end=1e30, cfl_mode=0, bc=(0, 0, 0, 0),
                 friction=0, manning_n=0.0, n_map=None, rain_rate=0.0,
                 rain_t_on=0.0, rain_t_off=0.0, infiltration=0, ks=0.0,
                 ks_map=None, psi=0.0, dtheta=0.0, check_cfl=0, dt_fixed=0.0,
                 friction_coef=None, order=2, bc_h=(0.0,) * 4, bc_q=(0.0,) * 4,
                 library=None):
        """friction: 0 none, 1 Manning, 2 Strickler, 3 Darcy-Weisbach, 4 Chezy,
        with its coefficient in friction_coef (manning_n is the same value
        under its older name); n_map is then a per-cell map of that
        coefficient.  bc: 0 wall, 1 outflow, 2 imposed h (bc_h), 3 imposed
        discharge (bc_q, into the domain), 4 both.  order 1: first order."""
        self._L = library if library is not None else lib()
        self.nx, self.ny = int(nx), int(ny)
        p = OracleParams()
        p.g, p.cfl, p.h_dry, p.dt_max, p.t_end = g, cfl, h_dry, dt_max, t_end
        p.cfl_mode = cfl_mode
        for k in range(4):
            p.bc[k] = int(bc[k])
        p.friction = int(friction)
        p.fric_coef = manning_n if friction_coef is None else friction_coef
        p.order = int(order)
        for k in range(4):
            p.bc_h[k], p.bc_q[k] = float(bc_h[k]), float(bc_q[k])
        p.rain_rate, p.rain_t_on, p.rain_t_off = rain_rate, rain_t_on, rain_t_off
        p.infiltration, p.ks, p.psi, p.dtheta = int(infiltration), ks, psi, dtheta
        p.check_cfl, p.dt_fixed = int(check_cfl), dt_fixed
        self._keep = [_c(z)]
        nm = None if n_map is None else _c(n_map)
        km = None if ks_map is None else _c(ks_map)
        self._o = self._L.oracle_create(self.nx, self.ny, dx, dy, _ptr(self._keep[0]),
                                      ctypes.byref(p),
                                      None if nm is None else _ptr(nm),
                                      None if km is None else _ptr(km))
        if not self._o:
            raise OracleError("oracle_create rejected its arguments")

    @classmethod
    def from_workload(cls, w, **over):
        kw = dict(cfl=w.cfl, h_dry=w.h_dry, dt_max=w.dt_max, t_end=w.t_end,
                  bc=w.bc, friction=w.friction, manning_n=w.manning_n,
                  rain_rate=w.rain_rate, rain_t_on=w.rain_t_on,
                  rain_t_off=w.rain_t_off, infiltration=w.infiltration,
                  ks_map=w.ks, psi=w.psi, dtheta=w.dtheta)
        kw.update(over)
        o = cls(w.nx, w.ny, w.dx, w.dy, w.z, **kw)
        o.set_state(w.h, w.qx, w.qy)
        return o

    def __del__(self):
        if getattr(self, "_o", None):
            self._L.oracle_destroy(self._o)
            self._o = None

    def set_state(self, h, qx, qy):
        h, qx, qy = _c(h), _c(qx), _c(qy)
        assert h.shape == (self.ny, self.nx)
        self._L.oracle_set_state(self._o, _ptr(h), _ptr(qx), _ptr(qy))

    def state(self):
        h = np.empty((self.ny, self.nx))
        qx = np.empty_like(h)
        qy = np.empty_like(h)
        self._L.oracle_get_state(self._o, _ptr(h), _ptr(qx), _ptr(qy))
        return h, qx, qy

    def vinf(self):
        v = np.empty((self.ny, self.nx))
        self._L.oracle_get_vinf(self._o, _ptr(v))
        return v

    def set_vinf(self, v):
        v = _c(v)
        self._L.oracle_set_vinf(self._o, _ptr(v))

    def set_time(self, t):
        self._L.oracle_set_time(self._o, float(t))

    def set_dt_sequence(self, dts):
        d = _c(dts)
        self._dts = d
        self._L.oracle_set_dt_sequence(self._o, _ptr(d), int(d.size))

    def step(self, n: int) -> np.ndarray:
        dts = np.zeros(max(int(n), 1))
        st = self._L.oracle_step(self._o, int(n), _ptr(dts))
        if st != 0:
            raise OracleError(f"oracle_step failed with status {st}")
        return dts[:n]

    def run_to(self, t_end: float, max_steps: int = 10 ** 7) -> np.ndarray:
        dts = []
        for _ in range(max_steps):
            if self.diag()["t"] >= t_end:
                break
            dts.append(self.step(1)[0])
        return np.array(dts)

    def lam(self):
        lx = ctypes.c_double()
        ly = ctypes.c_double()
        self._L.oracle_lambda(self._o, ctypes.byref(lx), ctypes.byref(ly))
        return lx.value, ly.value

    def track_max(self, on: bool = True):
        self._L.oracle_track_max(self._o, int(bool(on)))

    def max_depth(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        if self._L.oracle_get_max(self._o, _ptr(out)) != 0:
            raise OracleError("maximum depth not tracked")
        return out

    def set_gauges(self, cells, capacity: int):
        ij = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 2))
        self._gauges = ij
        st = self._L.oracle_set_gauges(self._o, ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       int(ij.shape[0]), int(capacity))
        if st != 0:
            raise OracleError("gauge outside the grid")

    def gauges(self) -> np.ndarray:
        """Records [n][1 + 3G]: t, then h, qx, qy at each gauge."""
        G = self._gauges.shape[0]
        cap = 1 << 20
        buf = np.zeros((cap, 1 + 3 * G)) if G else np.zeros((0, 1))
        n = self._L.oracle_get_gauges(self._o, _ptr(buf), cap) if G else 0
        return buf[:n].copy()

    def diag(self) -> dict:
        out = np.zeros(10)
        self._L.oracle_diag(self._o, _ptr(out))
        return {k: float(out[i]) for i, k in enumerate(self.DIAG_KEYS)}
