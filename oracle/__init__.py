"""FP64 CPU oracle for elevation-map fusion (arXiv 2204.12876, Section II).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2204_12876_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``em_oracle.c`` (plain C loops in double precision,
each step citing the paper).  This module only builds that file with gcc and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "em_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_em.so")

NORMALS, SMOOTH, INPAINT, MEDIAN, GAUSS, UPPER = 1, 2, 4, 8, 16, 32
ST_NONFINITE, ST_RANGE, ST_OUTSIDE, ST_ACCEPT, ST_REJECT, ST_WALL = range(6)
PF_BIN, PF_GATE, PF_WALL, PF_RANGE = 1, 2, 4, 8
CF_VALUE, CF_MARK = 1, 2
FP32_UNIT = 2.0 ** -24


def build(force: bool = False) -> str:
    """Compile em_oracle.c into liboracle_em.so (gcc, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("resolution", ctypes.c_double),
                ("noise_a0", ctypes.c_double), ("noise_a1", ctypes.c_double), ("noise_a2", ctypes.c_double),
                ("var_min", ctypes.c_double),
                ("min_range", ctypes.c_double), ("max_range", ctypes.c_double),
                ("mahalanobis_k", ctypes.c_double), ("outlier_variance", ctypes.c_double),
                ("wall_num_thresh", ctypes.c_int32),
                ("time_variance", ctypes.c_double),
                ("ray_step", ctypes.c_double),
                ("cleanup_min_age", ctypes.c_int32),
                ("cleanup_normal_thresh", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("drift_flatness", ctypes.c_double),
                ("excl_b", ctypes.c_double), ("excl_c", ctypes.c_double), ("excl_theta", ctypes.c_double),
                ("excl_d", ctypes.c_double), ("overlap_radius", ctypes.c_double), ("overlap_dz", ctypes.c_double)]


class _Cloud(ctypes.Structure):
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int32),
                ("pose", ctypes.c_float * 12)]


class _Trace(ctypes.Structure):
    _fields_ = [("ix", ctypes.c_void_p), ("iy", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("pflags", ctypes.c_void_p), ("mark", ctypes.c_void_p), ("cleared", ctypes.c_void_p),
                ("cflags", ctypes.c_void_p), ("counts", ctypes.c_int64 * 8),
                ("unit", ctypes.c_double), ("abs_band", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [ctypes.POINTER(_Params)]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_origin.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.orc_t_now.restype = ctypes.c_int32
        lib.orc_t_now.argtypes = [vp]
        lib.orc_get_shift.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        lib.orc_get.argtypes = [vp] + [vp] * 8
        lib.orc_set.argtypes = [vp] + [vp] * 6 + [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
        lib.orc_update.restype = ctypes.c_int
        lib.orc_update.argtypes = [vp, ctypes.POINTER(_Cloud), ctypes.c_int32, ctypes.POINTER(_Trace)]
        lib.orc_shift.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        lib.orc_filters.argtypes = [vp, ctypes.c_uint32]
        lib.orc_get_upper.argtypes = [vp, vp]
        lib.orc_last_drift.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double)]
        lib.orc_set_upper.argtypes = [vp, vp]
        _lib = lib
    return _lib


@dataclass
class Params:
    """Map and method parameters (names follow the paper's notation where it has one)."""
    width: int = 100
    height: int = 100
    resolution: float = 0.04
    noise_a0: float = 0.0
    noise_a1: float = 0.0
    noise_a2: float = 0.0
    var_min: float = 1e-8
    min_range: float = 0.0
    max_range: float = 1e9
    mahalanobis_k: float = 0.0
    outlier_variance: float = 0.0
    wall_num_thresh: int = 0
    time_variance: float = 0.0
    ray_step: float = 0.0
    cleanup_min_age: int = 0
    cleanup_normal_thresh: float = 0.0
    flags: int = 0
    drift_flatness: float = 0.0
    excl_b: float = 0.0
    excl_c: float = 0.0
    excl_theta: float = 0.0
    excl_d: float = 0.0
    overlap_radius: float = 0.0
    overlap_dz: float = 0.0

    def _c(self) -> _Params:
        return _Params(**{f.name: getattr(self, f.name) for f in fields(self)})


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


@dataclass
class Trace:
    ix: np.ndarray
    iy: np.ndarray
    status: np.ndarray
    pflags: np.ndarray
    mark: np.ndarray
    cleared: np.ndarray
    cflags: np.ndarray
    counts: dict


class OracleMap:
    """One elevation map held by the FP64 oracle (logical row-major [iy][ix] layout)."""

    def __init__(self, params: Params):
        self.params = params
        self._lib = _load()
        self._cp = params._c()
        self._h = self._lib.orc_create(ctypes.byref(self._cp))
        if not self._h:
            raise ValueError("invalid oracle parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.params.height, self.params.width)

    @property
    def t_now(self) -> int:
        return int(self._lib.orc_t_now(self._h))

    def origin(self):
        x0, y0 = ctypes.c_double(), ctypes.c_double()
        self._lib.orc_origin(self._h, ctypes.byref(x0), ctypes.byref(y0))
        return x0.value, y0.value

    def state(self) -> dict:
        H, W = self.shape
        out = {k: np.empty((H, W), np.float64) for k in ("h", "var", "nx", "ny", "nz", "smooth", "inpaint")}
        out["t_last"] = np.empty((H, W), np.int32)
        self._lib.orc_get(self._h, _ptr(out["h"]), _ptr(out["var"]), _ptr(out["t_last"]), _ptr(out["nx"]),
                          _ptr(out["ny"]), _ptr(out["nz"]), _ptr(out["smooth"]), _ptr(out["inpaint"]))
        out["upper"] = np.empty((H, W), np.float64)
        self._lib.orc_get_upper(self._h, _ptr(out["upper"]))
        return out

    def last_drift(self):
        """(mean height error added by the last update, points that entered it)."""
        return self.last_drift_band()[:2]

    def last_drift_band(self):
        """(mean, points, marginal band of the mean in metres; 0 without marginal bands)."""
        d, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        self._lib.orc_last_drift(self._h, ctypes.byref(d), ctypes.byref(n), ctypes.byref(b))
        return d.value, n.value, b.value

    def set_upper(self, upper):
        a = np.ascontiguousarray(upper, dtype=np.float64).reshape(-1)
        if a.size != self.params.width * self.params.height:
            raise ValueError("layer size mismatch")
        self._lib.orc_set_upper(self._h, _ptr(a))

    def set_state(self, h=None, var=None, t_last=None, nx=None, ny=None, nz=None, t_now=None, shift=None):
        """Overwrite layers (None keeps a layer).  Empty cells are those with non-finite variance."""
        conv = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt).reshape(-1)
        arrs = [conv(h, np.float64), conv(var, np.float64), conv(t_last, np.int32),
                conv(nx, np.float64), conv(ny, np.float64), conv(nz, np.float64)]
        n = self.params.width * self.params.height
        for a in arrs:
            if a is not None and a.size != n:
                raise ValueError("layer size mismatch")
        sx, sy = self._shift() if shift is None else shift
        self._lib.orc_set(self._h, *[_ptr(a) for a in arrs], int(self.t_now if t_now is None else t_now),
                          int(sx), int(sy))
        self._keep = arrs

    def _shift(self):
        sx, sy = ctypes.c_int64(), ctypes.c_int64()
        self._lib.orc_get_shift(self._h, ctypes.byref(sx), ctypes.byref(sy))
        return sx.value, sy.value

    @property
    def shift_xy(self):
        return self._shift()

    def shift(self, dx: int, dy: int):
        self._lib.orc_shift(self._h, int(dx), int(dy))

    def filters(self, which: int):
        self._lib.orc_filters(self._h, int(which))

    def update(self, clouds, trace: bool = False, unit: float = 0.0, abs_band: float = 1e-6):
        """Fuse one update made of one or more clouds [(pts (n,3|4) float32, pose float32[12]), ...]."""
        if isinstance(clouds, tuple):
            clouds = [clouds]
        keep, carr = [], (_Cloud * max(1, len(clouds)))()
        total = 0
        for i, (pts, pose) in enumerate(clouds):
            pts = np.ascontiguousarray(pts, dtype=np.float32)
            if pts.ndim != 2 or pts.shape[1] not in (3, 4):
                raise ValueError("points must be (n, 3) or (n, 4)")
            pose = np.ascontiguousarray(pose, dtype=np.float32).reshape(12)
            keep.append(pts)
            carr[i].pts = pts.ctypes.data
            carr[i].n = pts.shape[0]
            carr[i].stride = pts.shape[1]
            for k in range(12):
                carr[i].pose[k] = float(pose[k])
            total += pts.shape[0]
        tr = None
        trp = None
        if trace:
            H, W = self.shape
            tr = Trace(ix=np.empty(total, np.int32), iy=np.empty(total, np.int32),
                       status=np.empty(total, np.uint8), pflags=np.empty(total, np.uint8),
                       mark=np.empty((H, W), np.uint8), cleared=np.empty((H, W), np.uint8),
                       cflags=np.empty((H, W), np.uint8), counts={})
            ct = _Trace(ix=_ptr(tr.ix), iy=_ptr(tr.iy), status=_ptr(tr.status), pflags=_ptr(tr.pflags),
                        mark=_ptr(tr.mark), cleared=_ptr(tr.cleared), cflags=_ptr(tr.cflags),
                        unit=float(unit), abs_band=float(abs_band))
            trp = ctypes.byref(ct)
        rc = self._lib.orc_update(self._h, carr, len(clouds), trp)
        if rc != 0:
            raise RuntimeError(f"orc_update failed: {rc}")
        if trace:
            names = ("in", "valid", "in_map", "accepted", "rejected", "wall", "cells_updated", "cleared")
            tr.counts = {k: int(ct.counts[i]) for i, k in enumerate(names)}
        return tr
