"""Python binding of libswof (include/swof.h): argument marshalling only.

Every step of the shallow-water time step runs in the CUDA kernels of
libswof.so; this module loads that library through ctypes, mirrors its
structs, exposes the C entry points under the same names, and wraps them in
a small `Solver` class.  There is no CPU fallback: if the library is not
built (see `build()`), or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB as _LIB_RELEASE
from .build import LIB_DEBUG as _LIB_DEBUG
from .build import build

# SWOF_LIB_VARIANT=debug selects the index-checking build (build(debug=True))
_LIB_PATH = _LIB_DEBUG if os.environ.get("SWOF_LIB_VARIANT", "") == "debug" else _LIB_RELEASE

__all__ = ["build", "load", "Solver", "SwofError", "SwofParams", "SwofDiag", "SwofStepInfo",
           "FP64", "FP32", "BC_WALL", "BC_OUTFLOW", "BC_IMPOSED_H", "BC_IMPOSED_Q", "BC_IMPOSED_HQ",
           "FRIC_NONE", "FRIC_MANNING", "FRIC_STRICKLER", "FRIC_DARCY", "FRIC_CHEZY", "ORDER_1",
           "ORDER_2", "flow_directions"]

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ENEGATIVE, ECFL, EDTSEQ, ETIMEOUT, EDTUNDERFLOW, ESTATE, EBOUNDS = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10, -11)
FP64, FP32 = 0, 1
CFL_SUM, CFL_MIN = 0, 1
BC_WALL, BC_OUTFLOW, BC_IMPOSED_H, BC_IMPOSED_Q, BC_IMPOSED_HQ = 0, 1, 2, 3, 4
FRIC_NONE, FRIC_MANNING, FRIC_STRICKLER, FRIC_DARCY, FRIC_CHEZY = 0, 1, 2, 3, 4
ORDER_2, ORDER_1 = 0, 1
NOALLOC_MAX_ROWS = 65536

_D = ctypes.POINTER(ctypes.c_double)


class SwofParams(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("cfl", ctypes.c_double), ("h_dry", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("dt_min", ctypes.c_double), ("t_end", ctypes.c_double),
                ("precision", ctypes.c_int), ("cfl_mode", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("friction", ctypes.c_int), ("friction_coef", ctypes.c_double),
                ("friction_map", _D), ("rain_rate", ctypes.c_double),
                ("rain_t_on", ctypes.c_double), ("rain_t_off", ctypes.c_double),
                ("infiltration", ctypes.c_int), ("ks", ctypes.c_double), ("ks_map", _D),
                ("psi", ctypes.c_double), ("dtheta", ctypes.c_double), ("check_cfl", ctypes.c_int),
                ("dt_fixed", ctypes.c_double), ("stream", ctypes.c_void_p), ("order", ctypes.c_int),
                ("bc_h", ctypes.c_double * 4), ("bc_q", ctypes.c_double * 4)]


class SwofStepInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("steps", ctypes.c_longlong),
                ("status", ctypes.c_int)]


class SwofDiag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("last_dt", ctypes.c_double), ("steps", ctypes.c_longlong),
                ("volume", ctypes.c_double), ("rain_in", ctypes.c_double),
                ("infiltrated", ctypes.c_double), ("outflow", ctypes.c_double),
                ("min_h", ctypes.c_double), ("cfl_viol", ctypes.c_longlong)]


class SwofScenario(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("z", _D), ("h", _D), ("hu", _D), ("hv", _D), ("manning_n", ctypes.c_double),
                ("rain_rate", ctypes.c_double), ("rain_t_on", ctypes.c_double),
                ("rain_t_off", ctypes.c_double), ("bc", ctypes.c_int * 4),
                ("bc_h", ctypes.c_double * 4), ("bc_q", ctypes.c_double * 4)]


class SwofError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib.swof_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_SIGS = {
    "swof_default_params": (None, [ctypes.POINTER(SwofParams)]),
    "swof_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D,
                                   ctypes.POINTER(SwofParams), ctypes.POINTER(ctypes.c_void_p)]),
    "swof_destroy": (None, [ctypes.c_void_p]),
    "swof_set_state": (ctypes.c_int, [ctypes.c_void_p, _D, _D, _D]),
    "swof_get_state": (ctypes.c_int, [ctypes.c_void_p, _D, _D, _D]),
    "swof_set_state_device": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 3 + [ctypes.c_int]),
    "swof_get_state_device": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 3 + [ctypes.c_int]),
    "swof_get_infiltrated": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "swof_set_infiltrated": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "swof_set_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "swof_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(SwofStepInfo)]),
    "swof_set_dt_sequence": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int]),
    "swof_get_dt_history": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "swof_get_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SwofDiag)]),
    "swof_enable_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_get_timing": (ctypes.c_int, [ctypes.c_void_p, _D, _D, _D, ctypes.POINTER(ctypes.c_int)]),
    "swof_use_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_set_fp64_contraction": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_volume_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "swof_tile_shapes": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "swof_set_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_set_tile_shapes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "swof_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]),
    "swof_ensemble_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(SwofScenario),
                                            ctypes.POINTER(SwofParams), ctypes.POINTER(ctypes.c_void_p)]),
    "swof_ensemble_destroy": (None, [ctypes.c_void_p]),
    "swof_ensemble_size": (ctypes.c_int, [ctypes.c_void_p]),
    "swof_ensemble_member": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "swof_ensemble_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "swof_ensemble_shapes": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "swof_ensemble_set_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_ensemble_set_member_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "swof_ensemble_get_member_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_ensemble_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
    "swof_ensemble_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int]),
    "swof_gemm_bf16_nt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "swof_unet_create": (ctypes.c_int, [ctypes.c_int] * 6 + [ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_void_p)]),
    "swof_unet_destroy": (None, [ctypes.c_void_p]),
    "swof_unet_param_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "swof_unet_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "swof_unet_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "swof_unet_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "swof_unet_get_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "swof_unet_set_norm": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "swof_unet_forward_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "swof_unet_grads_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "swof_unet_adamw": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_float] * 5 + [ctypes.c_void_p]),
    "swof_unet_activation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_longlong]),
    "swof_surrogate_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                 ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.c_void_p]),
    "swof_surrogate_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "swof_set_infiltrated_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "swof_get_infiltrated_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "swof_coarsen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "swof_coarsen_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p]),
    "swof_batch_stats": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5 + [ctypes.c_double] * 2
                         + [ctypes.c_void_p, ctypes.c_void_p]),
    "swof_surrogate_rollout": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 8),
    "swof_track_max_depth": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_get_max_depth": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "swof_set_gauges": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int]),
    "swof_get_gauges": (ctypes.c_int, [ctypes.c_void_p, _D, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "swof_set_dry_tile_skip": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "swof_get_tile_activity": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                              ctypes.POINTER(ctypes.c_longlong)]),
    "swof_flow_directions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_float), ctypes.c_void_p, ctypes.c_void_p]),
    "swof_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "swof_version": (ctypes.c_char_p, []),
    "swof_debug_build": (ctypes.c_int, []),
    "swof_debug_probe_index": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
}


def declared_symbols() -> list[str]:
    return sorted(_SIGS)


def library_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Load libswof.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libswof is not built ({p} missing); call "
                                   "paper_1307_4839_gb300.build() first -- there is no CPU fallback")
            L = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(code: int, what: str):
    if code != OK:
        raise SwofError(code, what)


def default_params(**kw) -> SwofParams:
    p = SwofParams()
    load().swof_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("bc", "bc_h", "bc_q"):
            arr = getattr(p, k)
            for i in range(4):
                arr[i] = int(v[i]) if k == "bc" else float(v[i])
        else:
            setattr(p, k, v)
    return p


class Solver:
    """One libswof context.  Arrays are numpy float64 [ny][nx] on the host,
    or torch CUDA tensors for the *_device methods."""

    def __init__(self, nx, ny, dx, dy, z, *, precision=FP64, g=9.81, cfl=0.5, h_dry=1e-6,
                 dt_max=0.1, dt_min=0.0, t_end=1e30, cfl_mode=CFL_SUM, bc=(0, 0, 0, 0),
                 friction=FRIC_NONE, manning_n=0.0, friction_map=None, rain_rate=0.0,
                 rain_t_on=0.0, rain_t_off=0.0, infiltration=0, ks=0.0, ks_map=None, psi=0.0,
                 dtheta=0.0, check_cfl=0, dt_fixed=0.0, stream=None, friction_coef=None,
                 order=ORDER_2, bc_h=(0.0,) * 4, bc_q=(0.0,) * 4):
        """friction: FRIC_* with its coefficient in friction_coef (manning_n
        is the same value under its older name); friction_map is a per-cell
        map of that coefficient.  bc: BC_* per edge W, E, S, N with bc_h /
        bc_q for the imposed ones.  order: ORDER_2 or ORDER_1."""
        L = load()
        coef = manning_n if friction_coef is None else friction_coef
        self.nx, self.ny, self.precision = int(nx), int(ny), int(precision)
        self.fp64_contraction = False
        self._ctx = None
        keep = []
        fm = km = None
        if friction_map is not None:
            fm = _f64(friction_map)
            keep.append(fm)
        if ks_map is not None:
            km = _f64(ks_map)
            keep.append(km)
        p = default_params(g=g, cfl=cfl, h_dry=h_dry, dt_max=dt_max, dt_min=dt_min, t_end=t_end,
                           precision=int(precision), cfl_mode=int(cfl_mode), bc=bc,
                           friction=int(friction), friction_coef=float(coef),
                           order=int(order), bc_h=bc_h, bc_q=bc_q,
                           rain_rate=float(rain_rate), rain_t_on=float(rain_t_on),
                           rain_t_off=float(rain_t_off), infiltration=int(infiltration),
                           ks=float(ks), psi=float(psi), dtheta=float(dtheta),
                           check_cfl=int(check_cfl), dt_fixed=float(dt_fixed))
        p.friction_map = _ptr(fm) if fm is not None else None
        p.ks_map = _ptr(km) if km is not None else None
        p.stream = stream
        z = _f64(z)
        if z.shape != (self.ny, self.nx):
            raise ValueError("z must have shape (ny, nx)")
        ctx = ctypes.c_void_p()
        _check(L.swof_create(self.nx, self.ny, float(dx), float(dy), _ptr(z), ctypes.byref(p),
                             ctypes.byref(ctx)), "swof_create")
        self._ctx = ctx

    @classmethod
    def from_workload(cls, w, precision=FP64, **over):
        kw = dict(cfl=w.cfl, h_dry=w.h_dry, dt_max=w.dt_max, t_end=w.t_end, bc=w.bc,
                  friction=w.friction, manning_n=w.manning_n, rain_rate=w.rain_rate,
                  rain_t_on=w.rain_t_on, rain_t_off=w.rain_t_off, infiltration=w.infiltration,
                  ks_map=w.ks, psi=w.psi, dtheta=w.dtheta)
        kw.update(over)
        s = cls(w.nx, w.ny, w.dx, w.dy, w.z, precision=precision, **kw)
        s.set_state(w.h, w.qx, w.qy)
        return s

    def close(self):
        if self._ctx:
            load().swof_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, h, qx, qy):
        h, qx, qy = _f64(h), _f64(qx), _f64(qy)
        _check(load().swof_set_state(self._ctx, _ptr(h), _ptr(qx), _ptr(qy)), "swof_set_state")

    def state(self, out=None):
        """(h, hu, hv) as float64 [ny][nx] host arrays; `out` = three
        caller arrays (e.g. views of pinned memory) to fill instead."""
        if out is None:
            h = np.empty((self.ny, self.nx))
            qx = np.empty_like(h)
            qy = np.empty_like(h)
        else:
            h, qx, qy = out
            for a in out:
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != self.nx * self.ny:
                    raise ValueError("out arrays must be contiguous float64 [ny][nx]")
        _check(load().swof_get_state(self._ctx, _ptr(h), _ptr(qx), _ptr(qy)), "swof_get_state")
        return h, qx, qy

    def set_state_device(self, h, qx, qy):
        """torch CUDA tensors (float64 or float32), contiguous [ny][nx]."""
        dt = FP64 if str(h.dtype) == "torch.float64" else FP32
        _check(load().swof_set_state_device(self._ctx, h.data_ptr(), qx.data_ptr(), qy.data_ptr(), dt),
               "swof_set_state_device")

    def get_state_device(self, h, qx, qy):
        dt = FP64 if str(h.dtype) == "torch.float64" else FP32
        _check(load().swof_get_state_device(self._ctx, h.data_ptr(), qx.data_ptr(), qy.data_ptr(), dt),
               "swof_get_state_device")

    def infiltrated(self):
        v = np.empty((self.ny, self.nx))
        _check(load().swof_get_infiltrated(self._ctx, _ptr(v)), "swof_get_infiltrated")
        return v

    def set_infiltrated(self, v):
        v = _f64(v)
        _check(load().swof_set_infiltrated(self._ctx, _ptr(v)), "swof_set_infiltrated")

    def set_infiltrated_device(self, v):
        """torch CUDA tensor (float64 or float32), contiguous [ny][nx]."""
        dt = FP64 if str(v.dtype) == "torch.float64" else FP32
        _check(load().swof_set_infiltrated_device(self._ctx, ctypes.c_void_p(v.data_ptr()), dt),
               "swof_set_infiltrated_device")

    def get_infiltrated_device(self, v):
        dt = FP64 if str(v.dtype) == "torch.float64" else FP32
        _check(load().swof_get_infiltrated_device(self._ctx, ctypes.c_void_p(v.data_ptr()), dt),
               "swof_get_infiltrated_device")

    def set_time(self, t):
        _check(load().swof_set_time(self._ctx, float(t)), "swof_set_time")

    def step(self, n: int = 1, sync: bool = True) -> SwofStepInfo | None:
        if not sync:
            _check(load().swof_step(self._ctx, int(n), None), "swof_step")
            return None
        info = SwofStepInfo()
        _check(load().swof_step(self._ctx, int(n), ctypes.byref(info)), "swof_step")
        return info

    def track_max_depth(self, on: bool = True):
        _check(load().swof_track_max_depth(self._ctx, int(bool(on))), "swof_track_max_depth")

    def max_depth(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        _check(load().swof_get_max_depth(self._ctx, _ptr(out)), "swof_get_max_depth")
        return out

    def set_gauges(self, cells, capacity: int):
        ij = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 2))
        n = int(ij.shape[0])
        _check(load().swof_set_gauges(self._ctx, ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      n, int(capacity)), "swof_set_gauges")
        self._n_gauges = n                  # (a rejected call keeps the earlier gauges)
        self._gauge_cap = int(capacity)

    def gauges(self) -> np.ndarray:
        """Records [n][1 + 3G]: t, then h, hu, hv at each gauge."""
        G = getattr(self, "_n_gauges", 0)
        cap = getattr(self, "_gauge_cap", 0)
        buf = np.zeros((max(cap, 1), 1 + 3 * G))
        cnt = ctypes.c_int()
        _check(load().swof_get_gauges(self._ctx, _ptr(buf), cap, ctypes.byref(cnt)), "swof_get_gauges")
        return buf[:cnt.value].copy()

    def set_dry_tile_skip(self, on: bool = True):
        _check(load().swof_set_dry_tile_skip(self._ctx, int(bool(on))), "swof_set_dry_tile_skip")

    def tile_activity(self):
        """(tiles processed, tiles offered) since skipping was switched on."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().swof_get_tile_activity(self._ctx, ctypes.byref(a), ctypes.byref(b)),
               "swof_get_tile_activity")
        return a.value, b.value

    def set_dt_sequence(self, dts):
        d = _f64(dts).ravel()
        _check(load().swof_set_dt_sequence(self._ctx, _ptr(d) if d.size else None, int(d.size)),
               "swof_set_dt_sequence")

    def dt_history(self, max_n: int | None = None) -> np.ndarray:
        n = max_n if max_n is not None else int(self.diagnostics()["steps"])
        out = np.zeros(max(n, 1))
        cnt = ctypes.c_int()
        _check(load().swof_get_dt_history(self._ctx, _ptr(out), int(n), ctypes.byref(cnt)),
               "swof_get_dt_history")
        return out[:cnt.value]

    def debug_probe_index(self, i: int, j: int) -> int:
        """Debug build only: form the padded index of cell (i, j) through the
        checked path (swof_debug_probe_index); returns the status code."""
        return int(load().swof_debug_probe_index(self._ctx, int(i), int(j)))

    def diagnostics(self) -> dict:
        d = SwofDiag()
        _check(load().swof_get_diagnostics(self._ctx, ctypes.byref(d)), "swof_get_diagnostics")
        return {k: getattr(d, k) for k, _ in SwofDiag._fields_}

    def enable_timing(self, on=True):
        _check(load().swof_enable_timing(self._ctx, int(bool(on))), "swof_enable_timing")

    def timing(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int()
        _check(load().swof_get_timing(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                      ctypes.byref(n)), "swof_get_timing")
        return {"lambda_ms": a.value, "stage1_ms": b.value, "stage2_ms": c.value, "launches": n.value}

    def coarsen(self, f: int, out):
        """Block means of (h, hu, hv, V_inf) over f x f cells into the torch
        tensor out [4][ny/f][nx/f] (float32, CUDA), on the context's stream."""
        _check(load().swof_coarsen(self._ctx, int(f), ctypes.c_void_p(out.data_ptr())), "swof_coarsen")

    def use_graph(self, on=True):
        _check(load().swof_use_graph(self._ctx, int(bool(on))), "swof_use_graph")

    def set_fp64_contraction(self, on=True):
        """FP64 kernels with multiply-add contraction (within 1e-12 of the
        oracle under its dt sequence) instead of the bit-exact ones."""
        _check(load().swof_set_fp64_contraction(self._ctx, int(bool(on))), "swof_set_fp64_contraction")
        self.fp64_contraction = bool(on)

    def set_tile_shape(self, shape: int, shape2: int | None = None):
        """Tile shape of both stage kernels, or of stage 1 and stage 2."""
        if shape2 is None:
            _check(load().swof_set_tile_shape(self._ctx, int(shape)), "swof_set_tile_shape")
        else:
            _check(load().swof_set_tile_shapes(self._ctx, int(shape), int(shape2)), "swof_set_tile_shapes")

    def autotune(self, reps: int = 5, cache: str | None = None, key: str | None = None) -> dict:
        """Pick the fastest stage-kernel tile shape for this grid and
        precision.  With `cache`, a JSON file maps "<gpu>|<nx>x<ny>|<prec>"
        to the chosen shape so later runs skip the timing (and the number of
        shapes the library has: a cache written by a build with another
        shape table is not used)."""
        import json
        if key is None:
            prec = "fp32" if self.precision == FP32 else ("fp64c" if self.fp64_contraction else "fp64")
            key = f"{_gpu_name()}|{self.nx}x{self.ny}|{prec}"
        key = f"{key}|{len(tile_shapes())} shapes"
        data = {}
        if cache and os.path.exists(cache):
            try:
                data = json.load(open(cache))
            except (OSError, ValueError):
                data = {}
        if key in data:
            self.set_tile_shape(int(data[key]["shape"][0]), int(data[key]["shape"][1]))
            return dict(data[key], cached=True)
        n = tile_shapes()
        ms = (ctypes.c_double * (2 * len(n)))()
        best = (ctypes.c_int * 2)()
        _check(load().swof_autotune(self._ctx, int(reps), ms, best), "swof_autotune")
        rec = {"shape": [best[0], best[1]], "stage1": list(n[best[0]]), "stage2": list(n[best[1]]),
               "ms_stage1": [ms[k] for k in range(len(n))],
               "ms_stage2": [ms[len(n) + k] for k in range(len(n))]}
        if cache:
            data[key] = rec
            tmp = cache + ".tmp"
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(rec, cached=False)


def ensemble_shapes() -> list[tuple[int, int]]:
    """Member tile shapes (CTA width, rows) of the ensemble launch."""
    L = load()
    n = L.swof_ensemble_shapes(None, None, 0)
    a = (ctypes.c_int * n)()
    b = (ctypes.c_int * n)()
    L.swof_ensemble_shapes(a, b, n)
    return [(a[k], b[k]) for k in range(n)]


def flow_directions(z, out=None, nodata: float | None = None, stream=None):
    """D8 flow-direction codes (uint8 torch tensor [ny][nx], 0 = no lower
    neighbour, 1..8 = E, NE, N, NW, W, SW, S, SE) of a float32 CUDA DEM
    tensor [ny][nx] (Sec. 5.2's eight-neighbour example), in one kernel;
    neighbours at z <= nodata are no candidates (None: no no-data value)."""
    import torch
    if z.dtype != torch.float32 or not z.is_cuda or z.dim() != 2 or not z.is_contiguous():
        raise ValueError("z must be a contiguous float32 CUDA tensor [ny][nx]")
    ny, nx = z.shape
    if out is None:
        out = torch.empty((ny, nx), dtype=torch.uint8, device=z.device)
    s = stream if stream is not None else torch.cuda.current_stream(z.device).cuda_stream
    nd = None if nodata is None else ctypes.byref(ctypes.c_float(nodata))
    _check(load().swof_flow_directions(ctypes.c_void_p(z.data_ptr()), int(nx), int(ny), nd,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s)),
           "swof_flow_directions")
    return out


def tile_shapes() -> list[tuple[int, int]]:
    """(threads along x, rows) of each stage-kernel shape."""
    L = load()
    n = L.swof_tile_shapes(None, None, 0)
    a = (ctypes.c_int * n)()
    b = (ctypes.c_int * n)()
    L.swof_tile_shapes(a, b, n)
    return [(a[k], b[k]) for k in range(n)]


def tile_shape_forms() -> list[str]:
    """How each stage-kernel shape brings in its input rows: "ring" (TMA
    ring with the dry fast path) for the first half of the shapes, "reg"
    (one-row register prefetch) for the second half."""
    n = len(tile_shapes())
    return ["ring"] * (n // 2) + ["reg"] * (n - n // 2)


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "gpu"


class _Member(Solver):
    """A member context borrowed from an Ensemble (not destroyed here)."""

    def __init__(self, ctx, nx, ny, precision):
        self._ctx = ctx
        self.nx, self.ny, self.precision = nx, ny, precision

    def close(self):
        self._ctx = None


class Ensemble:
    """A batch of independent grids advanced by one persistent kernel.

    `workloads` are swof_inputs.Workload objects (z, initial state, Manning
    n, rain, boundaries are taken from each); the remaining parameters are
    common to all members."""

    def __init__(self, workloads, precision=FP32, cfl=0.5, h_dry=1e-6, dt_max=0.1, t_end=1e30,
                 stream=None):
        L = load()
        self._e = None
        self._keep = []
        specs = (SwofScenario * len(workloads))()
        for k, w in enumerate(workloads):
            arrs = [_f64(a) for a in (w.z, w.h, w.qx, w.qy)]
            self._keep.extend(arrs)
            sc = specs[k]
            sc.nx, sc.ny, sc.dx, sc.dy = w.nx, w.ny, w.dx, w.dy
            sc.z, sc.h, sc.hu, sc.hv = (_ptr(a) for a in arrs)
            sc.manning_n = w.manning_n if w.friction else 0.0
            sc.rain_rate, sc.rain_t_on, sc.rain_t_off = w.rain_rate, w.rain_t_on, w.rain_t_off
            bh = getattr(w, "bc_h", None) or (0.0,) * 4     # imposed edge values (optional attributes)
            bq = getattr(w, "bc_q", None) or (0.0,) * 4
            for b in range(4):
                sc.bc[b] = int(w.bc[b])
                sc.bc_h[b] = float(bh[b])
                sc.bc_q[b] = float(bq[b])
        p = default_params(precision=int(precision), cfl=cfl, h_dry=h_dry, dt_max=dt_max, t_end=t_end)
        p.stream = stream
        e = ctypes.c_void_p()
        _check(L.swof_ensemble_create(len(workloads), specs, ctypes.byref(p), ctypes.byref(e)),
               "swof_ensemble_create")
        self._e = e
        self._keep = None
        self.precision = int(precision)
        self.sizes = [(w.nx, w.ny) for w in workloads]
        self.cells = sum(nx * ny for nx, ny in self.sizes)

    def close(self):
        if self._e:
            load().swof_ensemble_destroy(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.sizes)

    def member(self, k: int) -> Solver:
        c = ctypes.c_void_p()
        _check(load().swof_ensemble_member(self._e, int(k), ctypes.byref(c)), "swof_ensemble_member")
        nx, ny = self.sizes[k]
        return _Member(c, nx, ny, self.precision)

    def step(self, n: int = 1, sync: bool = True) -> int | None:
        if not sync:
            _check(load().swof_ensemble_step(self._e, int(n), None), "swof_ensemble_step")
            return None
        st = ctypes.c_int()
        _check(load().swof_ensemble_step(self._e, int(n), ctypes.byref(st)), "swof_ensemble_step")
        return st.value

    def set_shape(self, shape: int):
        _check(load().swof_ensemble_set_shape(self._e, int(shape)), "swof_ensemble_set_shape")

    def member_shapes(self) -> list[int]:
        L = load()
        return [int(L.swof_ensemble_get_member_shape(self._e, k)) for k in range(len(self.sizes))]

    def set_member_shapes(self, shapes):
        """Member shapes (indices into ensemble_shapes(), one launch width)."""
        shapes = [int(x) for x in shapes]
        self.set_shape(shapes[0])
        for k, sh in enumerate(shapes):
            if sh != shapes[0]:
                _check(load().swof_ensemble_set_member_shape(self._e, k, sh), "swof_ensemble_set_member_shape")

    def autotune(self, steps: int = 2, cache: str | None = None) -> dict:
        """Launch width and per-size-class tile heights (swof_ensemble_autotune).
        With `cache`, a JSON file maps "<gpu>|<precision>|<member sizes>" to
        the member shapes, so later runs skip the timing."""
        import json
        import hashlib
        key = None
        if cache:
            sizes = ",".join(f"{nx}x{ny}" for nx, ny in self.sizes)
            key = (f"{_gpu_name()}|{'fp64' if self.precision == FP64 else 'fp32'}|"
                   f"{hashlib.sha1(sizes.encode()).hexdigest()[:16]}|{len(ensemble_shapes())} shapes")
            data = {}
            if os.path.exists(cache):
                try:
                    data = json.load(open(cache))
                except (OSError, ValueError):
                    data = {}
            if key in data:
                self.set_member_shapes(data[key]["member_shapes"])
                return dict(data[key], cached=True)
        L = load()
        ms = (ctypes.c_double * 2)()
        best = ctypes.c_int()
        mem = (ctypes.c_int * len(self.sizes))()
        _check(L.swof_ensemble_autotune(self._e, int(steps), ms, ctypes.byref(best), mem), "swof_ensemble_autotune")
        shp = ensemble_shapes()
        rec = {"shape": best.value, "ntx": shp[best.value][0], "rows": shp[best.value][1],
               "member_shapes": [int(mem[k]) for k in range(len(self.sizes))],
               "ms_per_step_width": {"128": ms[0], "64": ms[1]}}
        by_size = {}
        for (nx, ny), sh in zip(self.sizes, rec["member_shapes"]):
            by_size[f"{nx}x{ny}"] = list(shp[sh])
        rec["by_size"] = by_size
        if cache:
            data[key] = rec
            tmp = cache + ".tmp"
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(rec, cached=False)

    def set_wait_limit(self, polls: int, block_member: int = -1):
        _check(load().swof_ensemble_set_wait_limit(self._e, int(polls), int(block_member)),
               "swof_ensemble_set_wait_limit")


class UNet:
    """The learned surrogate's network (libswof swof_unet_*): BF16 tcgen05
    convolutions with FP32 accumulation and FP32 AdamW master weights.
    Device arrays are torch CUDA tensors."""

    def __init__(self, base=32, in_ch=4, out_ch=3, H=256, W=256, max_batch=8, seed=0):
        L = load()
        self._u = None
        u = ctypes.c_void_p()
        _check(L.swof_unet_create(int(base), int(in_ch), int(out_ch), int(H), int(W), int(max_batch),
                                  int(seed), ctypes.byref(u)), "swof_unet_create")
        self._u = u
        self.base, self.in_ch, self.out_ch, self.H, self.W, self.max_batch = base, in_ch, out_ch, H, W, max_batch
        self.nparam = int(L.swof_unet_param_count(u))

    def close(self):
        if self._u:
            load().swof_unet_destroy(self._u)
            self._u = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        out = []
        k = 0
        while True:
            info = (ctypes.c_int * 9)()
            n = load().swof_unet_layout(self._u, k, info)
            if n < 0:
                break
            out.append(dict(zip(("kind", "cin", "cin_p", "cout", "ncols", "Kp", "woff", "boff", "act"), info)))
            k += 1
            if k >= n:
                break
        return out

    def params(self) -> np.ndarray:
        a = np.empty(self.nparam, dtype=np.float32)
        _check(load().swof_unet_get_params(self._u, a.ctypes.data), "swof_unet_get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.nparam
        _check(load().swof_unet_set_params(self._u, a.ctypes.data), "swof_unet_set_params")

    def grads(self) -> np.ndarray:
        a = np.empty(self.nparam, dtype=np.float32)
        _check(load().swof_unet_get_grads(self._u, a.ctypes.data), "swof_unet_get_grads")
        return a

    def set_norm(self, mean, scale_in, scale_out):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        si_ = np.ascontiguousarray(scale_in, dtype=np.float32)
        so = np.ascontiguousarray(scale_out, dtype=np.float32)
        _check(load().swof_unet_set_norm(self._u, m.ctypes.data, si_.ctypes.data, so.ctypes.data),
               "swof_unet_set_norm")

    @staticmethod
    def _s(stream):
        return None if stream is None else ctypes.c_void_p(stream)

    def forward_raw(self, x, y, stream=None):
        B = x.shape[0] // (self.H * self.W)
        _check(load().swof_unet_forward_raw(self._u, ctypes.c_void_p(x.data_ptr()), B,
                                            ctypes.c_void_p(y.data_ptr()), self._s(stream)), "swof_unet_forward_raw")

    def grads_raw(self, x, tgt, stream=None) -> float:
        B = x.shape[0] // (self.H * self.W)
        loss = ctypes.c_double()
        _check(load().swof_unet_grads_raw(self._u, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(tgt.data_ptr()),
                                          B, ctypes.byref(loss), self._s(stream)), "swof_unet_grads_raw")
        return loss.value

    def activation(self, which: int, level: int, shape) -> np.ndarray:
        a = np.empty(int(np.prod(shape)), dtype=np.float32)
        _check(load().swof_unet_activation(self._u, int(which), int(level), a.ctypes.data, a.size),
               "swof_unet_activation")
        return a.reshape(shape)

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        _check(load().swof_unet_adamw(self._u, lr, beta1, beta2, eps, weight_decay, self._s(stream)),
               "swof_unet_adamw")

    def train_step(self, state_in, state_next, lr, weight_decay=0.0, stream=None) -> float:
        loss = ctypes.c_double()
        _check(load().swof_surrogate_train_step(self._u, ctypes.c_void_p(state_in.data_ptr()),
                                                ctypes.c_void_p(state_next.data_ptr()), int(state_in.shape[0]),
                                                float(lr), float(weight_decay), ctypes.byref(loss), self._s(stream)),
               "swof_surrogate_train_step")
        return loss.value

    def predict(self, state_in, out, stream=None):
        _check(load().swof_surrogate_predict(self._u, ctypes.c_void_p(state_in.data_ptr()), int(state_in.shape[0]),
                                             ctypes.c_void_p(out.data_ptr()), self._s(stream)),
               "swof_surrogate_predict")


def coarsen_static(z, ks, dx, dy, f, out, snap_stride, nsnap, ks_const=0.0, stream=None):
    """The surrogate's static channels (bed slopes dz/dx, dz/dy of the f x f
    block-mean bed, block-mean K_s) from device float64 tensors z and ks
    [ny][nx] (ks None: ks_const) into the float32 CUDA tensor `out` (channel
    0 of snapshot 0; snapshots snap_stride floats apart), swof_coarsen_static."""
    ny, nx = z.shape
    _check(load().swof_coarsen_static(ctypes.c_void_p(z.data_ptr()),
                                      None if ks is None else ctypes.c_void_p(ks.data_ptr()), float(ks_const),
                                      int(nx), int(ny), float(dx), float(dy), int(f),
                                      ctypes.c_void_p(out.data_ptr()), int(snap_stride), int(nsnap),
                                      None if stream is None else ctypes.c_void_p(stream)), "swof_coarsen_static")


def batch_stats(states, out, outmask=0, dx=1.0, dy=1.0, stream=None):
    """Per-member {sum h, sum min(h, 0), discharge out [m^3/s], sum V_inf,
    min h} of states [B][C][H][W] (float32 CUDA) into out [B][5] (float64
    CUDA); outmask bits 1 W, 2 E, 4 S, 8 N."""
    B, C, H, W = states.shape
    _check(load().swof_batch_stats(ctypes.c_void_p(states.data_ptr()), int(B), int(C), int(H), int(W), int(outmask),
                                   float(dx), float(dy), ctypes.c_void_p(out.data_ptr()),
                                   None if stream is None else ctypes.c_void_p(stream)),
           "swof_batch_stats")


class RolloutOpts(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int), ("fallback_steps", ctypes.c_int), ("span", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("tol", ctypes.c_double),
                ("h_dry", ctypes.c_double), ("rain_channel", ctypes.c_int), ("outflow_mask", ctypes.c_int),
                ("inject_member", ctypes.c_int), ("inject_call", ctypes.c_int), ("inject_dh", ctypes.c_double)]


def rollout(net, states, t, rain, fallback, fallback_of, *, calls, span, fallback_steps, dx, dy, tol=1e-3,
            h_dry=1e-6, rain_channel=-1, outflow_mask=0, inject=None, stream=None):
    """swof_surrogate_rollout: advance the members in `states` (float32 CUDA
    [B][in_ch][H][W], updated in place) by `calls` network calls with the
    positivity / mass check and per-member fallback to the solvers in
    `fallback` (Solver list; fallback_of[b] indexes it).  t (float64 [B]) is
    advanced in place; rain is [B][3] (rate, t_on, t_off).  Returns
    (accepted [calls][B] int, checks [calls][B][2] float64)."""
    B = states.shape[0]
    t = np.ascontiguousarray(t, dtype=np.float64)
    rain = np.ascontiguousarray(rain, dtype=np.float64).reshape(B, 3)
    fb = (ctypes.c_void_p * max(len(fallback), 1))(*[f._ctx.value for f in fallback])
    fo = np.ascontiguousarray(fallback_of, dtype=np.int32)
    o = RolloutOpts(int(calls), int(fallback_steps), float(span), float(dx), float(dy), float(tol), float(h_dry),
                    int(rain_channel), int(outflow_mask), -1, -1, 0.0)
    if inject is not None:
        o.inject_member, o.inject_call, o.inject_dh = int(inject[0]), int(inject[1]), float(inject[2])
    acc = np.zeros((max(calls, 1), B), dtype=np.int32)
    chk = np.zeros((max(calls, 1), B, 2))
    st = load().swof_surrogate_rollout(net._u, ctypes.c_void_p(states.data_ptr()), int(B), t.ctypes.data,
                                       rain.ctypes.data, fb, fo.ctypes.data, ctypes.byref(o), acc.ctypes.data,
                                       chk.ctypes.data, None if stream is None else ctypes.c_void_p(stream))
    _check(st, "swof_surrogate_rollout")
    return acc[:calls], chk[:calls], t
