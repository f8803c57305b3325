"""ctypes binding of libem.so (include/em.h).  Argument marshalling only: every
step of the fusion runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.

The library must have been built (``paper_2204_12876_gb300.build.build()``);
importing this module without it raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libem.so")

EM_OK = 0
EM_ERR_INVALID_ARG, EM_ERR_OOM, EM_ERR_CUDA, EM_ERR_TIMEOUT, EM_ERR_REJECTED, EM_ERR_BUSY, EM_ERR_CAPACITY = \
    -1, -2, -3, -4, -5, -6, -7
F_NORMALS, F_SMOOTH, F_INPAINT, F_MEDIAN, F_GAUSS, F_UPPER, F_TRACE = 1, 2, 4, 8, 16, 32, 256
LAYER_ELEVATION, LAYER_VARIANCE, LAYER_TIME = 1, 2, 4
LAYER_NORMAL_X, LAYER_NORMAL_Y, LAYER_NORMAL_Z = 8, 16, 32
LAYER_SMOOTH, LAYER_INPAINT, LAYER_VALID, LAYER_VARIANCE_NOW, LAYER_UPPER = 64, 128, 256, 512, 1024
PROF_SLOTS = ("count", "ray", "alloc", "scatter", "fuse", "clear", "normals", "smooth", "inpaint", "drift",
              "overlap", "persist")
KERNEL_NAMES = {"count": "k_count", "ray": "k_ray", "alloc": "k_alloc", "scatter": "k_scatter", "fuse": "k_fuse",
                "clear": "k_clear", "normals": "k_normals", "smooth": "k_smooth", "inpaint": "k_inpaint",
                "drift": "k_drift", "overlap": "k_overlap", "persist": "k_persist"}
LAYER_NAMES = {LAYER_ELEVATION: "h", LAYER_VARIANCE: "var", LAYER_TIME: "t_last", LAYER_NORMAL_X: "nx",
               LAYER_NORMAL_Y: "ny", LAYER_NORMAL_Z: "nz", LAYER_SMOOTH: "smooth", LAYER_INPAINT: "inpaint",
               LAYER_VALID: "valid", LAYER_VARIANCE_NOW: "var_now", LAYER_UPPER: "upper"}


class EMError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_str(code)} ({code}) {last_cuda_error()}")


class _Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("resolution", ctypes.c_float),
                ("noise_a0", ctypes.c_float), ("noise_a1", ctypes.c_float), ("noise_a2", ctypes.c_float),
                ("var_min", ctypes.c_float), ("min_range", ctypes.c_float), ("max_range", ctypes.c_float),
                ("mahalanobis_k", ctypes.c_float), ("outlier_variance", ctypes.c_float),
                ("wall_num_thresh", ctypes.c_int32), ("time_variance", ctypes.c_float),
                ("ray_step", ctypes.c_float), ("cleanup_min_age", ctypes.c_int32),
                ("cleanup_normal_thresh", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("drift_flatness", ctypes.c_float), ("excl_b", ctypes.c_float), ("excl_c", ctypes.c_float),
                ("excl_theta", ctypes.c_float), ("excl_d", ctypes.c_float), ("overlap_radius", ctypes.c_float),
                ("overlap_dz", ctypes.c_float)]


class _Cloud(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int32),
                ("pose", ctypes.c_float * 12)]


class _Info(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("resolution", ctypes.c_float),
                ("t_now", ctypes.c_int32), ("shift_x", ctypes.c_int64), ("shift_y", ctypes.c_int64),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("point_capacity", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("updates", "points_in", "points_valid", "points_in_map",
                                             "points_accepted", "points_rejected", "points_wall",
                                             "cells_updated", "cells_cleared", "ray_samples",
                                             "drift_points")] + [("drift_last", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2204_12876_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "em_create": ([ctypes.POINTER(_Params), ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "em_destroy": ([vp], ctypes.c_int),
        "em_reserve": ([vp, i64], ctypes.c_int),
        "em_update": ([vp, vp, i64, i32, ctypes.POINTER(ctypes.c_float), vp], ctypes.c_int),
        "em_update_multi": ([vp, ctypes.POINTER(_Cloud), i32, vp], ctypes.c_int),
        "em_update_host": ([vp, ctypes.POINTER(_Cloud), i32, vp], ctypes.c_int),
        "em_shift": ([vp, i32, i32, vp], ctypes.c_int),
        "em_get_layers": ([vp, ctypes.c_uint32, vp, ctypes.c_int, vp], ctypes.c_int),
        "em_set_layers": ([vp, ctypes.c_uint32, vp, ctypes.c_int, vp], ctypes.c_int),
        "em_set_time": ([vp, i32], ctypes.c_int),
        "em_get_info": ([vp, ctypes.POINTER(_Info)], ctypes.c_int),
        "em_get_stats": ([vp, ctypes.POINTER(_Stats)], ctypes.c_int),
        "em_sync": ([vp], ctypes.c_int),
        "em_get_trace": ([vp, vp, vp, vp, i64], ctypes.c_int),
        "em_profile": ([vp, ctypes.c_int], ctypes.c_int),
        "em_profile_read": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "em_update_noalloc": ([ctypes.POINTER(_Params), i64, i64, i32, vp, vp, vp, vp, vp, vp,
                               ctypes.POINTER(_Cloud), i32, vp], ctypes.c_int),
        "em_status_str": ([ctypes.c_int], ctypes.c_char_p),
        "em_last_cuda_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def status_str(code: int) -> str:
    return lib.em_status_str(int(code)).decode()


def last_cuda_error() -> str:
    return lib.em_last_cuda_error().decode()


def _check(rc: int, what: str):
    if rc != EM_OK:
        raise EMError(rc, what)


@dataclass
class Params:
    """em_params (include/em.h); float fields are float32 in the library."""
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


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _torch():
    import torch  # imported on first use (the module loads without it)
    return torch


_F12 = ctypes.c_float * 12


def _pose(pose) -> ctypes.Array:
    return _F12.from_buffer_copy(np.ascontiguousarray(pose, dtype=np.float32).reshape(12))


def _cloud_struct(pts, pose, host: bool, any_device: bool = False) -> _Cloud:
    if host:
        n, stride = pts.shape
        ptr = pts.ctypes.data
    else:
        if pts.dtype is not _torch().float32 or not (pts.is_cuda or any_device) or not pts.is_contiguous():
            raise ValueError("points must be a contiguous float32 CUDA tensor of shape (n, 3) or (n, 4)")
        n, stride = pts.shape
        ptr = pts.data_ptr()
    return _Cloud(ptr, n, stride, _pose(pose))


class Map:
    """One elevation map resident on a CUDA device."""

    def __init__(self, params: Params, device: int = 0):
        self.params = params
        self._cp = params._c()
        h = ctypes.c_void_p()
        _check(lib.em_create(ctypes.byref(self._cp), int(device), ctypes.byref(h)), "em_create")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            lib.em_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def shape(self):
        return (self.params.height, self.params.width)

    def reserve(self, max_points: int):
        _check(lib.em_reserve(self._h, int(max_points)), "em_reserve")

    def update(self, points, pose, stream=None):
        """Fuse one device cloud: points is a float32 CUDA tensor (n, 3|4)."""
        if points.dtype.__str__() != "torch.float32" or not points.is_cuda or not points.is_contiguous():
            raise ValueError("points must be a contiguous float32 CUDA tensor of shape (n, 3) or (n, 4)")
        n, stride = points.shape
        _check(lib.em_update(self._h, points.data_ptr(), n, stride, _pose(pose), _stream_handle(stream)),
               "em_update")

    def update_multi(self, clouds, stream=None):
        """One update from several device clouds [(tensor, pose), ...]."""
        arr = (_Cloud * len(clouds))(*[_cloud_struct(p, q, False) for p, q in clouds])
        _check(lib.em_update_multi(self._h, arr, len(clouds), _stream_handle(stream)), "em_update_multi")

    def update_host(self, clouds, stream=None):
        """One update from host clouds [(np.ndarray float32 (n,3|4), pose), ...]."""
        keep = [np.ascontiguousarray(p, dtype=np.float32) for p, _ in clouds]
        arr = (_Cloud * len(clouds))(*[_cloud_struct(k, q, True) for k, (_, q) in zip(keep, clouds)])
        _check(lib.em_update_host(self._h, arr, len(clouds), _stream_handle(stream)), "em_update_host")

    def shift(self, dx: int, dy: int, stream=None):
        _check(lib.em_shift(self._h, int(dx), int(dy), _stream_handle(stream)), "em_shift")

    def get_layers(self, mask: int, out=None, stream=None):
        """Layers in ascending bit order.  out=None: host numpy (k, H, W); else a CUDA tensor."""
        k = bin(mask).count("1")
        H, W = self.shape
        if out is None:
            host = np.empty((k, H, W), np.float32)
            _check(lib.em_get_layers(self._h, mask, host.ctypes.data, 1, _stream_handle(stream)), "em_get_layers")
            return host
        if out.numel() != k * H * W:
            raise ValueError("output tensor has the wrong size")
        _check(lib.em_get_layers(self._h, mask, out.data_ptr(), 0, _stream_handle(stream)), "em_get_layers")
        return out

    def state(self) -> dict:
        """All layers as host float32 arrays keyed by name (t_last as int32)."""
        mask = sum(LAYER_NAMES) & ~LAYER_VALID
        arr = self.get_layers(mask)
        out = {}
        for i, bit in enumerate(b for b in sorted(LAYER_NAMES) if mask & b):
            out[LAYER_NAMES[bit]] = arr[i]
        out["t_last"] = out["t_last"].astype(np.int32)
        return out

    def set_layers(self, mask: int, src, stream=None):
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.float32)
            _check(lib.em_set_layers(self._h, mask, src.ctypes.data, 1, _stream_handle(stream)), "em_set_layers")
        else:
            _check(lib.em_set_layers(self._h, mask, src.data_ptr(), 0, _stream_handle(stream)), "em_set_layers")

    def set_state(self, h=None, var=None, t_last=None, nx=None, ny=None, nz=None, t_now=None, upper=None):
        layers, mask = [], 0
        for bit, a in ((LAYER_ELEVATION, h), (LAYER_VARIANCE, var), (LAYER_TIME, t_last), (LAYER_NORMAL_X, nx),
                       (LAYER_NORMAL_Y, ny), (LAYER_NORMAL_Z, nz), (LAYER_UPPER, upper)):
            if a is not None:
                mask |= bit
                layers.append(np.asarray(a, np.float32))
        if mask:
            self.set_layers(mask, np.stack(layers))
        if t_now is not None:
            _check(lib.em_set_time(self._h, int(t_now)), "em_set_time")

    def info(self) -> dict:
        i = _Info()
        _check(lib.em_get_info(self._h, ctypes.byref(i)), "em_get_info")
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def stats(self) -> dict:
        s = _Stats()
        _check(lib.em_get_stats(self._h, ctypes.byref(s)), "em_get_stats")
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def sync(self):
        _check(lib.em_sync(self._h), "em_sync")

    def profile(self, enable: bool = True):
        _check(lib.em_profile(self._h, 1 if enable else 0), "em_profile")

    def profile_read(self) -> dict:
        ms = (ctypes.c_double * len(PROF_SLOTS))()
        n = (ctypes.c_int64 * len(PROF_SLOTS))()
        _check(lib.em_profile_read(self._h, ms, n), "em_profile_read")
        return {k: (ms[i], n[i]) for i, k in enumerate(PROF_SLOTS)}

    def trace(self, n: int):
        ix = np.empty(n, np.int32)
        iy = np.empty(n, np.int32)
        st = np.empty(n, np.uint8)
        _check(lib.em_get_trace(self._h, ix.ctypes.data, iy.ctypes.data, st.ctypes.data, int(n)), "em_get_trace")
        return ix, iy, st


NOALLOC_MAX_CELLS, NOALLOC_MAX_POINTS, NOALLOC_MAX_CLOUDS = 65536, 327680, 8


def _check_layers(layers, cells: int, device):
    """Caller layers the kernels read or write whole, as (name, tensor, dtype):
    each must be a contiguous tensor of its dtype with exactly `cells`
    elements, on the CUDA device of the points (the library cannot check
    sizes; a wrong one would be written out of bounds)."""
    for name, t, dtype in layers:
        if not hasattr(t, "is_cuda") or str(t.dtype) != dtype:
            raise ValueError(f"{name} must be a {dtype} tensor, got {getattr(t, 'dtype', type(t))}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() != cells:
            raise ValueError(f"{name} must hold width * height = {cells} elements, got {t.numel()}")
    for name, t, _ in layers:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if device is not None and t.device != device:
            raise ValueError(f"{name} is on {t.device}, the points on {device}")


def update_noalloc(params: Params, h, var, t_last, clouds, t_now: int, shift=(0, 0), normals=None, stream=None):
    """em_update_noalloc: one update of caller-owned layers (CUDA tensors: h, var
    float32 (H, W), t_last int32 (H, W), optional normals (nx, ny, nz) float32
    (H, W)) that allocates no device memory.  Every layer is checked (dtype,
    size, contiguity, device) before the call: ValueError otherwise."""
    cells = int(params.width) * int(params.height)
    device = clouds[0][0].device if clouds and hasattr(clouds[0][0], "device") else None
    layers = [("h", h, "torch.float32"), ("var", var, "torch.float32"), ("t_last", t_last, "torch.int32")]
    if normals is not None:
        if len(normals) != 3:
            raise ValueError("normals must be (nx, ny, nz)")
        layers += [(k, t, "torch.float32") for k, t in zip(("nx", "ny", "nz"), normals)]
    _check_layers(layers, cells, device)
    cp = params._c()
    arr = (_Cloud * len(clouds))(*[_cloud_struct(p, q, False) for p, q in clouds])
    nx, ny, nz = (None, None, None) if normals is None else (n.data_ptr() for n in normals)
    _check(lib.em_update_noalloc(ctypes.byref(cp), int(shift[0]), int(shift[1]), int(t_now), h.data_ptr(),
                                 var.data_ptr(), t_last.data_ptr(), nx, ny, nz, arr, len(clouds),
                                 _stream_handle(stream)), "em_update_noalloc")


BATCH_GRAPH = 1
BATCH_PERSISTENT = 2


class _Tuning(ctypes.Structure):
    _fields_ = [("ray_group", ctypes.c_int32), ("fuse_chunk", ctypes.c_int32), ("big_thresh", ctypes.c_int32)]


def _bind_batch():
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "em_batch_create": ([ctypes.c_int, i32, i32, i64, i32, ctypes.c_uint32, ctypes.POINTER(vp)], ctypes.c_int),
        "em_batch_destroy": ([vp], ctypes.c_int),
        "em_update_batch": ([vp, ctypes.POINTER(vp), ctypes.POINTER(_Cloud), i32, vp], ctypes.c_int),
        "em_batch_set_tuning": ([vp, ctypes.POINTER(_Tuning)], ctypes.c_int),
        "em_batch_get_tuning": ([vp, ctypes.POINTER(_Tuning)], ctypes.c_int),
        "em_batch_autotune": ([vp, ctypes.POINTER(vp), ctypes.POINTER(_Cloud), i32, vp, i32,
                               ctypes.POINTER(_Tuning)], ctypes.c_int),
        "em_wait_selftest": ([ctypes.c_int, i32], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


_bind_batch()


def wait_selftest(device: int = 0, wait_us: int = 20000) -> int:
    """em_wait_selftest: the persistent launch's bounded wait on a word that nothing
    sets; returns the status code (EM_ERR_TIMEOUT when the wait ran out, as it must)."""
    return int(lib.em_wait_selftest(int(device), int(wait_us)))


class Batch:
    """em_batch: many maps updated by one kernel sequence (optionally one CUDA graph launch)."""

    def __init__(self, max_maps: int, max_clouds: int, max_points: int, max_cells: int, graph: bool = True,
                 device: int = 0, persistent: bool = False):
        h = ctypes.c_void_p()
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_PERSISTENT if persistent else 0)
        _check(lib.em_batch_create(int(device), int(max_maps), int(max_clouds), int(max_points), int(max_cells),
                                   flags, ctypes.byref(h)), "em_batch_create")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            lib.em_batch_destroy(self._h)
            self._h = None

    __del__ = close

    @staticmethod
    def _pairs(pairs):
        maps = (ctypes.c_void_p * len(pairs))(*[m.handle.value for m, _, _ in pairs])
        clouds = (_Cloud * len(pairs))(*[_cloud_struct(p, q, False) for _, p, q in pairs])
        return maps, clouds

    def update(self, pairs, stream=None):
        """pairs: [(Map, points CUDA tensor (n,3|4), pose), ...]; a map may repeat."""
        maps, clouds = self._pairs(pairs)
        _check(lib.em_update_batch(self._h, maps, clouds, len(pairs), _stream_handle(stream)), "em_update_batch")

    def autotune(self, pairs, reps: int = 3, stream=None) -> dict:
        maps, clouds = self._pairs(pairs)
        t = _Tuning()
        _check(lib.em_batch_autotune(self._h, maps, clouds, len(pairs), _stream_handle(stream), int(reps),
                                     ctypes.byref(t)), "em_batch_autotune")
        return {f: getattr(t, f) for f, _ in _Tuning._fields_}

    def tuning(self) -> dict:
        t = _Tuning()
        _check(lib.em_batch_get_tuning(self._h, ctypes.byref(t)), "em_batch_get_tuning")
        return {f: getattr(t, f) for f, _ in _Tuning._fields_}

    def set_tuning(self, ray_group: int, fuse_chunk: int, big_thresh: int):
        t = _Tuning(ray_group, fuse_chunk, big_thresh)
        _check(lib.em_batch_set_tuning(self._h, ctypes.byref(t)), "em_batch_set_tuning")


SERVE_BATCHED, SERVE_PLAIN = 0, 1
SERVE_RECORD_BYTES = 16  # admission accounting per point (EM_SERVE_RECORD_BYTES)


class _ServerCfg(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_batch_maps", ctypes.c_int32),
                ("max_batch_points", ctypes.c_int64), ("max_map_cells", ctypes.c_int32), ("mode", ctypes.c_uint32),
                ("batch_flags", ctypes.c_uint32), ("fail_alloc_at", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("map_id", ctypes.c_int32), ("points", ctypes.c_int64),
                ("batch_size", ctypes.c_int32), ("t_submit_ns", ctypes.c_int64), ("t_start_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class _Request(ctypes.Structure):
    _fields_ = [("map_id", ctypes.c_int32), ("n_clouds", ctypes.c_int32), ("clouds", ctypes.POINTER(_Cloud)),
                ("read_mask", ctypes.c_uint32), ("read_to_host", ctypes.c_int32), ("read_dst", ctypes.c_void_p),
                ("clouds_on_host", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "rejected", "cancelled", "batches",
                                             "batched_requests", "max_batch_size", "bytes_in_use", "peak_bytes",
                                             "slots_in_use")]


def _bind_server():
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "em_server_create": ([ctypes.POINTER(_ServerCfg), ctypes.POINTER(vp)], ctypes.c_int),
        "em_server_add_map": ([vp, ctypes.POINTER(_Params), ctypes.POINTER(i32)], ctypes.c_int),
        "em_server_map": ([vp, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "em_server_submit": ([vp, i32, ctypes.POINTER(_Cloud), i32, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "em_server_submit_after": ([vp, i32, ctypes.POINTER(_Cloud), i32, vp, ctypes.POINTER(ctypes.c_uint64)],
                                   ctypes.c_int),
        "em_server_submit_many": ([vp, ctypes.POINTER(_Request), i32, vp, ctypes.POINTER(ctypes.c_uint64)],
                                  ctypes.c_int),
        "em_server_wait": ([vp, ctypes.c_uint64, i64, ctypes.POINTER(_Result)], ctypes.c_int),
        "em_server_wait_many": ([vp, ctypes.POINTER(ctypes.c_uint64), i32, i64, ctypes.POINTER(_Result)],
                                ctypes.c_int),
        "em_server_cancel": ([vp, ctypes.c_uint64], ctypes.c_int),
        "em_server_drain": ([vp, i64], ctypes.c_int),
        "em_server_get_stats": ([vp, ctypes.POINTER(_ServerStats)], ctypes.c_int),
        "em_server_destroy": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


_bind_server()


class _MapView(Map):
    """A resident map owned by a server (not destroyed by Python)."""

    def __init__(self, handle, params):
        self.params = params
        self._h = handle
        self.device = 0

    def close(self):
        self._h = None

    __del__ = close


class Server:
    """em_server: continuous-batching request loop over resident maps."""

    def __init__(self, budget_bytes: int, max_slots: int = 256, n_streams: int = 2, max_batch_maps: int = 32,
                 max_batch_points: int = 8_000_000, max_map_cells: int = 250_000, mode: int = SERVE_BATCHED,
                 graph: bool = True, device: int = 0, fail_alloc_at: int = 0):
        self._cfg = _ServerCfg(device, int(budget_bytes), max_slots, n_streams, max_batch_maps,
                               int(max_batch_points), max_map_cells, mode, BATCH_GRAPH if graph else 0,
                               fail_alloc_at)
        h = ctypes.c_void_p()
        _check(lib.em_server_create(ctypes.byref(self._cfg), ctypes.byref(h)), "em_server_create")
        self._h = h
        self._keep = {}
        self._params = []

    def close(self):
        if getattr(self, "_h", None):
            lib.em_server_destroy(self._h)
            self._h = None

    __del__ = close

    def add_map(self, params: Params) -> int:
        cp = params._c()
        mid = ctypes.c_int32()
        _check(lib.em_server_add_map(self._h, ctypes.byref(cp), ctypes.byref(mid)), "em_server_add_map")
        self._params.append(params)
        return mid.value

    def map(self, map_id: int) -> Map:
        h = ctypes.c_void_p()
        _check(lib.em_server_map(self._h, int(map_id), ctypes.byref(h)), "em_server_map")
        return _MapView(h, self._params[map_id])

    def submit(self, map_id: int, clouds, ready=None) -> int:
        """clouds: [(points CUDA tensor, pose), ...]; tensors are kept alive until the ticket is waited.
        ready: optional torch.cuda.Event recorded after the points were written."""
        arr = (_Cloud * len(clouds))(*[_cloud_struct(p, q, False) for p, q in clouds])
        tk = ctypes.c_uint64()
        if ready is None:
            _check(lib.em_server_submit(self._h, int(map_id), arr, len(clouds), ctypes.byref(tk)), "em_server_submit")
        else:
            _check(lib.em_server_submit_after(self._h, int(map_id), arr, len(clouds), ready.cuda_event,
                                              ctypes.byref(tk)), "em_server_submit_after")
        self._keep[tk.value] = (clouds, ready)
        return tk.value

    def submit_many(self, requests, ready=None) -> list:
        """requests: [(map_id, [(points, pose), ...], read), ...]: points contiguous float32
        (n, 3|4) tensors, all on the CUDA device or all in pinned CPU memory (then the server
        copies them to the device itself); read None or (layer_mask, out): out a contiguous
        float32 tensor (CUDA, or pinned CPU memory) that receives the map's layers right after
        this update.  One call queues them all (they reach the same batch when they fit);
        ready as in submit.  Returns the tickets."""
        n = len(requests)
        reqs = (_Request * n)()
        keep = []
        f32 = _torch().float32
        for q, (map_id, clouds, read) in enumerate(requests):
            on_host = not clouds[0][0].is_cuda
            cs = []
            for p, pose in clouds:
                if p.is_cuda == on_host or p.dtype is not f32 or not p.is_contiguous() or \
                        p.dim() != 2 or p.shape[1] not in (3, 4) or (on_host and not p.is_pinned()):
                    raise ValueError("points: contiguous float32 (n, 3|4) tensors, all CUDA or all pinned CPU")
                cs.append(_Cloud(p.data_ptr(), p.shape[0], p.shape[1], _pose(pose)))
            arr = (_Cloud * len(cs))(*cs)
            keep.append((arr, clouds, read))
            r = reqs[q]
            r.map_id = int(map_id)
            r.n_clouds = len(cs)
            r.clouds = arr
            r.clouds_on_host = 1 if on_host else 0
            if read is not None:
                mask, out = read
                if out.dtype is not f32 or not out.is_contiguous():
                    raise ValueError("read-back buffer must be a contiguous float32 tensor")
                r.read_mask = int(mask)
                r.read_to_host = 0 if out.is_cuda else 1
                r.read_dst = out.data_ptr()
        tks = (ctypes.c_uint64 * n)()
        _check(lib.em_server_submit_many(self._h, reqs, n, ready.cuda_event if ready is not None else None, tks),
               "em_server_submit_many")
        for q in range(n):
            self._keep[tks[q]] = (keep[q], ready)
        return list(tks)

    def wait_many(self, tickets, timeout_us: int = -1, results: bool = False):
        """Wait for all tickets in one call.  Returns their statuses (or result dicts)."""
        n = len(tickets)
        tks = (ctypes.c_uint64 * n)(*tickets)
        res = (_Result * n)()
        _check(lib.em_server_wait_many(self._h, tks, n, int(timeout_us), res), "em_server_wait_many")
        for t in tickets:
            self._keep.pop(t, None)
        if results:
            return [{f: getattr(r, f) for f, _ in _Result._fields_} for r in res]
        return [r.status for r in res]

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        r = _Result()
        _check(lib.em_server_wait(self._h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(r)),
               "em_server_wait")
        self._keep.pop(ticket, None)
        return {f: getattr(r, f) for f, _ in _Result._fields_}

    def cancel(self, ticket: int):
        _check(lib.em_server_cancel(self._h, ctypes.c_uint64(ticket)), "em_server_cancel")

    def drain(self, timeout_us: int = -1):
        _check(lib.em_server_drain(self._h, int(timeout_us)), "em_server_drain")

    def stats(self) -> dict:
        s = _ServerStats()
        _check(lib.em_server_get_stats(self._h, ctypes.byref(s)), "em_server_get_stats")
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}


def _bind_extra():
    vp = ctypes.c_void_p
    sig = {
        "em_batch_profile": ([vp, ctypes.c_int], ctypes.c_int),
        "em_batch_profile_read": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "em_server_set_tuning": ([vp, ctypes.POINTER(_Tuning)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


_bind_extra()


def _batch_profile(self, enable: bool = True):
    _check(lib.em_batch_profile(self._h, 1 if enable else 0), "em_batch_profile")


def _batch_profile_read(self) -> dict:
    ms = (ctypes.c_double * len(PROF_SLOTS))()
    n = (ctypes.c_int64 * len(PROF_SLOTS))()
    _check(lib.em_batch_profile_read(self._h, ms, n), "em_batch_profile_read")
    return {k: (ms[i], n[i]) for i, k in enumerate(PROF_SLOTS)}


def _server_set_tuning(self, ray_group: int, fuse_chunk: int, big_thresh: int):
    """Call while the server is idle (after drain)."""
    t = _Tuning(ray_group, fuse_chunk, big_thresh)
    _check(lib.em_server_set_tuning(self._h, ctypes.byref(t)), "em_server_set_tuning")


Batch.profile = _batch_profile
Batch.profile_read = _batch_profile_read
Server.set_tuning = _server_set_tuning
