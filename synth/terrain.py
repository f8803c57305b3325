"""Terrain and range-sensor simulation (seeded, numpy, float64 inside, float32 out).

Workloads (all sizes are those of the fusion workloads this repository
measures; every recipe is seeded):

* ``single_update``: 20,000 points over a 4.4 m square of wave terrain seen from
  0.5 m above, identity pose (single-update workload).
* ``depth_stream``: four 320x240 pinhole depth cameras on a walking robot, ~5 %
  invalid pixels, terrain with random boxes, random-walk pose.
* ``lidar_stream``: 128 beams x 2,048 azimuths out to 30 m over stairs and a
  ramp.
* ``batch_clouds``: many independent maps of uneven size and point count.
* ``random_prior``: a seeded map state of the kind a stream leaves behind.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

F32 = np.float32


def pose_matrix(R: np.ndarray, t) -> np.ndarray:
    """Row-major 3x4 [R | t] as float32[12]."""
    P = np.zeros((3, 4))
    P[:, :3] = R
    P[:, 3] = t
    return P.astype(F32).reshape(12)


def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


class Terrain:
    """Three sinusoids (amplitudes summing to ``amplitude``, wavelengths 0.5-4 m)
    plus one ``step``-high step along a seeded line, plus optional flat-topped
    boxes of height 0.05-0.4 m."""

    def __init__(self, seed: int, amplitude: float = 0.2, step: float = 0.15, n_boxes: int = 0,
                 box_extent: float = 5.0):
        rng = np.random.default_rng(seed)
        self.amp = amplitude * rng.dirichlet(np.ones(3))
        lam = rng.uniform(0.5, 4.0, 3)
        ang = rng.uniform(0.0, 2 * math.pi, 3)
        self.kx = 2 * math.pi * np.cos(ang) / lam
        self.ky = 2 * math.pi * np.sin(ang) / lam
        self.phase = rng.uniform(0.0, 2 * math.pi, 3)
        a = rng.uniform(0.0, 2 * math.pi)
        self.sn = np.array([math.cos(a), math.sin(a)])
        self.sc = rng.uniform(-1.5, 1.5)
        self.step = step
        self.lip = float(np.sum(self.amp * np.hypot(self.kx, self.ky)))
        self.faces = [(self.sn[0], self.sn[1], self.sc)] if step != 0 else []
        self.boxes = []
        for _ in range(n_boxes):
            cx, cy = rng.uniform(-box_extent, box_extent, 2)
            hx, hy = rng.uniform(0.05, 0.3, 2)
            yaw = rng.uniform(0.0, math.pi)
            hb = rng.uniform(0.05, 0.4)
            top = float(self.ground(np.array([cx]), np.array([cy]))[0]) + hb
            self.boxes.append((cx, cy, hx, hy, yaw, top))

    def smooth(self, x, y):
        z = np.zeros_like(np.asarray(x, dtype=np.float64))
        for k in range(3):
            z = z + self.amp[k] * np.sin(self.kx[k] * x + self.ky[k] * y + self.phase[k])
        return z

    def ground(self, x, y):
        return self.smooth(x, y) + self.step * ((self.sn[0] * x + self.sn[1] * y) > self.sc)

    def height(self, x, y):
        z = self.ground(x, y)
        for (cx, cy, hx, hy, yaw, top) in self.boxes:
            c, s = math.cos(yaw), math.sin(yaw)
            lx = c * (x - cx) + s * (y - cy)
            ly = -s * (x - cx) + c * (y - cy)
            inside = (np.abs(lx) <= hx) & (np.abs(ly) <= hy)
            z = np.where(inside, np.maximum(z, top), z)
        return z


class StairsTerrain(Terrain):
    """Ten stairs (0.17 m rise, 0.30 m run) up along +x, a 15 degree ramp, and
    low waves (amplitude 0.03 m)."""

    def __init__(self, seed: int):
        super().__init__(seed, amplitude=0.03, step=0.0)
        rng = np.random.default_rng(seed + 1000)
        self.x_st = rng.uniform(1.5, 3.0)
        self.y_st = rng.uniform(-1.0, 1.0)
        self.rise, self.run, self.nst = 0.17, 0.30, 10
        self.x_ramp, self.y_ramp = -2.0 - rng.uniform(0.0, 1.0), rng.uniform(3.0, 4.0)
        self.slope = math.tan(math.radians(15.0))
        faces = [(1.0, 0.0, self.x_st + j * self.run) for j in range(self.nst + 1)]
        faces += [(1.0, 0.0, self.x_st + self.nst * self.run + 2.0)]
        faces += [(0.0, 1.0, self.y_st - 1.5), (0.0, 1.0, self.y_st + 1.5)]
        faces += [(0.0, 1.0, self.y_ramp), (0.0, 1.0, self.y_ramp + 4.0), (1.0, 0.0, self.x_ramp - 8.0)]
        self.faces = faces
        self.lip += self.slope

    def ground(self, x, y):
        z = self.smooth(x, y)
        in_strip = np.abs(y - self.y_st) <= 1.5
        k = np.floor((x - self.x_st) / self.run) + 1
        top = self.x_st + self.nst * self.run + 2.0
        st = np.where((x >= self.x_st) & (x < top), self.rise * np.clip(k, 0, self.nst), 0.0)
        z = z + np.where(in_strip, st, 0.0)
        in_ramp = (y >= self.y_ramp) & (y <= self.y_ramp + 4.0)
        rl = np.clip(self.x_ramp - x, 0.0, 6.0) * self.slope
        rl = np.where(x < self.x_ramp - 8.0, 0.0, rl)
        return z + np.where(in_ramp, rl, 0.0)


def _box_hits(terrain: Terrain, o: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Exact ray / box intersection (slabs; a box extends down to -inf)."""
    t_best = np.full(o.shape[0], np.inf)
    for (cx, cy, hx, hy, yaw, top) in terrain.boxes:
        c, s = math.cos(yaw), math.sin(yaw)
        lox = c * (o[:, 0] - cx) + s * (o[:, 1] - cy)
        loy = -s * (o[:, 0] - cx) + c * (o[:, 1] - cy)
        ldx = c * d[:, 0] + s * d[:, 1]
        ldy = -s * d[:, 0] + c * d[:, 1]
        t0 = np.full(o.shape[0], -np.inf)
        t1 = np.full(o.shape[0], np.inf)
        with np.errstate(divide="ignore", invalid="ignore"):
            for lo, ld, h in ((lox, ldx, hx), (loy, ldy, hy)):
                ta = (-h - lo) / ld
                tb = (h - lo) / ld
                near = np.where(ld != 0, np.minimum(ta, tb), np.where(np.abs(lo) <= h, -np.inf, np.inf))
                far = np.where(ld != 0, np.maximum(ta, tb), np.where(np.abs(lo) <= h, np.inf, -np.inf))
                t0 = np.maximum(t0, near)
                t1 = np.minimum(t1, far)
            tz = (top - o[:, 2]) / d[:, 2]
            near = np.where(d[:, 2] < 0, tz, np.where(d[:, 2] > 0, -np.inf, np.where(o[:, 2] <= top, -np.inf, np.inf)))
            far = np.where(d[:, 2] > 0, tz, np.where(d[:, 2] < 0, np.inf, np.where(o[:, 2] <= top, np.inf, -np.inf)))
        t0 = np.maximum(t0, near)
        t1 = np.minimum(t1, far)
        hit = (t0 <= t1) & (t1 >= 0)
        t_best = np.where(hit, np.minimum(t_best, np.maximum(t0, 0.0)), t_best)
    return t_best


def raycast(terrain: Terrain, o: np.ndarray, d: np.ndarray, t_max: float, dt_min: float = 0.004,
            dt_max: float = 0.5) -> np.ndarray:
    """Distance along unit rays (o + t d) to the first terrain / box surface, NaN if none within t_max.

    Ground: march with steps bounded by the slope bound of the smooth part, stop
    at every discontinuity line, then bisect the bracketing interval.
    """
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    n = o.shape[0]
    out = np.full(n, np.nan)
    idx = np.arange(n)
    t = np.zeros(n)
    L = terrain.lip + 1e-3
    g = o[:, 2] - terrain.ground(o[:, 0], o[:, 1])
    out[g <= 0] = 0.0
    keep = g > 0
    idx, t, g = idx[keep], t[keep], g[keep]
    it = 0
    while idx.size and it < 2000:
        it += 1
        oo, dd = o[idx], d[idx]
        dxy = np.hypot(dd[:, 0], dd[:, 1])
        denom = L * dxy - dd[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(denom > 1e-9, g / denom, dt_max)
        s = np.clip(s, dt_min, dt_max)
        for (a, b, c) in terrain.faces:  # stop just past the next discontinuity line
            den = a * dd[:, 0] + b * dd[:, 1]
            with np.errstate(divide="ignore", invalid="ignore"):
                tc = (c - a * oo[:, 0] - b * oo[:, 1]) / den
            cross = (tc > t + 1e-9) & (tc < t + s)
            s = np.where(cross, tc - t + 1e-7, s)
        tn = t + s
        p = oo + tn[:, None] * dd
        gn = p[:, 2] - terrain.ground(p[:, 0], p[:, 1])
        hit = gn <= 0
        if hit.any():
            lo, hi = t[hit], tn[hit]
            oh, dh = oo[hit], dd[hit]
            for _ in range(30):
                mid = 0.5 * (lo + hi)
                pm = oh + mid[:, None] * dh
                below = pm[:, 2] - terrain.ground(pm[:, 0], pm[:, 1]) <= 0
                hi = np.where(below, mid, hi)
                lo = np.where(below, lo, mid)
            out[idx[hit]] = hi
        live = ~hit & (tn <= t_max)
        idx, t, g = idx[live], tn[live], gn[live]
    if terrain.boxes:
        tb = _box_hits(terrain, o, d)
        out = np.where(np.isfinite(tb) & ~(out <= tb), tb, out)
    out[out > t_max] = np.nan
    return out


def single_update(seed: int = 1, n: int = 20000, half: float = 2.2, sensor_height: float = 0.5):
    """Points (x, y) ~ U[-half, half]^2 on wave terrain 0.5 m below the sensor,
    z noise sigma = 0.005 + 0.002 z^2; identity pose.  Returns (pts (n,3) f32, pose f32[12])."""
    rng = np.random.default_rng(seed)
    terr = Terrain(seed)
    x = rng.uniform(-half, half, n)
    y = rng.uniform(-half, half, n)
    z = -sensor_height + terr.height(x, y)
    z = z + rng.normal(0.0, 1.0, n) * (0.005 + 0.002 * z * z)
    pts = np.stack([x, y, z], axis=1).astype(F32)
    return pts, pose_matrix(np.eye(3), [0.0, 0.0, 0.0])


@dataclass
class DepthRig:
    """Four pinhole depth cameras (front, left, back, right) pitched down 40 deg."""
    width: int = 320
    height: int = 240
    fx: float = 200.0
    fy: float = 200.0
    pitch_deg: float = 40.0
    mount: float = 0.3
    max_depth: float = 8.0
    dropout: float = 0.05

    def cam_to_body(self, k: int) -> tuple[np.ndarray, np.ndarray]:
        th = math.radians(self.pitch_deg)
        # optical frame: x right, y down, z forward; forward pitched down by th
        zf = np.array([math.cos(th), 0.0, -math.sin(th)])
        xr = np.array([0.0, -1.0, 0.0])
        yd = np.cross(zf, xr)
        Rb = rot_z(k * math.pi / 2) @ np.stack([xr, yd, zf], axis=1)
        tb = rot_z(k * math.pi / 2) @ np.array([self.mount, 0.0, 0.0])
        return Rb, tb

    def pixel_dirs(self) -> np.ndarray:
        u, v = np.meshgrid(np.arange(self.width) + 0.5, np.arange(self.height) + 0.5)
        return np.stack([(u - self.width / 2) / self.fx, (v - self.height / 2) / self.fy,
                         np.ones_like(u)], axis=-1).reshape(-1, 3)


def _camera_cloud(terr, rig, R_wc, t_wc, rng):
    dirs = rig.pixel_dirs()
    norm = np.linalg.norm(dirs, axis=1)
    dw = (dirs / norm[:, None]) @ R_wc.T
    o = np.broadcast_to(t_wc, dw.shape)
    rng_t = raycast(terr, o, dw, rig.max_depth * 1.8)
    depth = rng_t / norm
    bad = ~np.isfinite(depth) | (depth > rig.max_depth) | (rng.random(depth.shape) < rig.dropout)
    depth = depth + rng.normal(0.0, 1.0, depth.shape) * (0.005 + 0.002 * np.nan_to_num(depth) ** 2)
    pts = dirs * depth[:, None]
    pts[bad] = np.nan
    return pts.astype(F32), pose_matrix(R_wc, t_wc)


def depth_stream(seed: int = 2, frames: int = 100, rig: DepthRig | None = None, n_boxes: int = 30,
                 step_xy: float = 0.02, step_yaw_deg: float = 1.0, base_height: float = 0.5):
    """Yield per frame a dict with ``clouds`` = [(pts (76800,3) f32, pose f32[12]) x 4] and the
    robot's ``xy``.  Random-walk pose: N(0, step_xy) per axis, N(0, step_yaw_deg) yaw; the body
    height follows the terrain + base_height."""
    rig = rig or DepthRig()
    rng = np.random.default_rng(seed)
    terr = Terrain(seed, n_boxes=n_boxes)
    xy = np.zeros(2)
    yaw = 0.0
    for _ in range(frames):
        xy = xy + rng.normal(0.0, step_xy, 2)
        yaw = yaw + math.radians(rng.normal(0.0, step_yaw_deg))
        zb = float(terr.ground(np.array([xy[0]]), np.array([xy[1]]))[0]) + base_height
        R_wb = rot_z(yaw)
        t_wb = np.array([xy[0], xy[1], zb])
        clouds = []
        for k in range(4):
            Rb, tb = rig.cam_to_body(k)
            clouds.append(_camera_cloud(terr, rig, R_wb @ Rb, t_wb + R_wb @ tb, rng))
        yield {"clouds": clouds, "xy": xy.copy(), "yaw": yaw}


@dataclass
class LidarRig:
    beams: int = 128
    azimuths: int = 2048
    el_min_deg: float = -45.0
    el_max_deg: float = 15.0
    max_range: float = 30.0
    height: float = 0.6

    def dirs(self) -> np.ndarray:
        el = np.radians(np.linspace(self.el_min_deg, self.el_max_deg, self.beams))
        az = np.linspace(0.0, 2 * math.pi, self.azimuths, endpoint=False)
        E, A = np.meshgrid(el, az, indexing="ij")
        return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1).reshape(-1, 3)


def lidar_stream(seed: int = 3, frames: int = 1000, rig: LidarRig | None = None, step_xy: float = 0.03,
                 step_yaw_deg: float = 1.0):
    """Yield per frame {"clouds": [(pts (beams*azimuths,3) f32, pose)], "xy"}: range noise
    sigma = 0.01 + 0.001 r^2, no return (NaN) beyond max_range, stairs + ramp terrain."""
    rig = rig or LidarRig()
    rng = np.random.default_rng(seed)
    terr = StairsTerrain(seed)
    dirs = rig.dirs()
    xy = np.zeros(2)
    yaw = 0.0
    for _ in range(frames):
        xy = xy + rng.normal(0.0, step_xy, 2)
        yaw = yaw + math.radians(rng.normal(0.0, step_yaw_deg))
        zb = float(terr.ground(np.array([xy[0]]), np.array([xy[1]]))[0]) + rig.height
        R = rot_z(yaw)
        t = np.array([xy[0], xy[1], zb])
        dw = dirs @ R.T
        r = raycast(terr, np.broadcast_to(t, dw.shape), dw, rig.max_range)
        bad = ~np.isfinite(r)
        r = r + rng.normal(0.0, 1.0, r.shape) * (0.01 + 0.001 * np.nan_to_num(r) ** 2)
        pts = dirs * r[:, None]
        pts[bad] = np.nan
        yield {"clouds": [(pts.astype(F32), pose_matrix(R, t))], "xy": xy.copy(), "yaw": yaw}


def scattered_cloud(seed: int, n: int, half: float, sensor_height: float = 0.5, yaw: float = 0.0,
                    nan_frac: float = 0.0):
    """n points uniform over a (2*half)^2 square of wave terrain, seen from a sensor
    ``sensor_height`` above the map centre with heading ``yaw``; depth-style noise."""
    rng = np.random.default_rng(seed)
    terr = Terrain(seed)
    x = rng.uniform(-half, half, n)
    y = rng.uniform(-half, half, n)
    z = terr.height(x, y)
    dz = sensor_height - z
    z = z + rng.normal(0.0, 1.0, n) * (0.005 + 0.002 * dz * dz)
    pw = np.stack([x, y, z], axis=1)
    R = rot_z(yaw)
    t = np.array([0.0, 0.0, sensor_height])
    ps = (pw - t) @ R  # sensor frame: R^T (p - t)
    if nan_frac > 0:
        ps[rng.random(n) < nan_frac] = np.nan
    return ps.astype(F32), pose_matrix(R, t)


def batch_clouds(seed: int = 4, maps: int = 64, side_min: int = 100, side_max: int = 500,
                 n_min: int = 10000, n_max: int = 400000, resolution: float = 0.04):
    """Independent maps of uneven size and load: side ~ U{side_min..side_max} cells,
    N ~ U[n_min, n_max] points, per-map seeded terrain.  Returns a list of dicts
    {"side", "clouds": [(pts, pose)]}."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(maps):
        side = int(rng.integers(side_min, side_max + 1))
        n = int(rng.integers(n_min, n_max + 1))
        half = 0.5 * side * resolution * 1.05
        pts, pose = scattered_cloud(seed * 1000 + j, n, half, yaw=float(rng.uniform(0, 2 * math.pi)))
        out.append({"side": side, "clouds": [(pts, pose)]})
    return out


def random_prior(seed: int, width: int, height: int, resolution: float = 0.04, t_now: int = 10,
                 invalid_frac: float = 0.15, obstacle_frac: float = 0.03, with_normals: bool = True,
                 base: float = 0.0):
    """A seeded map state: terrain heights at cell centres plus noise, variances
    10^U(-5,-3) m^2, a fraction of empty cells (variance inf), a few raised stale
    'obstacle' cells, last-update indices in [t_now-10, t_now-1], unit normals
    (some NaN).  Arrays are logical row-major [iy][ix] float32 / int32."""
    rng = np.random.default_rng(seed)
    terr = Terrain(seed)
    xs = (np.arange(width) + 0.5 - width / 2) * resolution
    ys = (np.arange(height) + 0.5 - height / 2) * resolution
    X, Y = np.meshgrid(xs, ys)
    h = base + terr.ground(X, Y) + rng.normal(0.0, 0.01, X.shape)
    obst = rng.random(X.shape) < obstacle_frac
    h = np.where(obst, h + rng.uniform(0.1, 0.5, X.shape), h)
    var = 10.0 ** rng.uniform(-5, -3, X.shape)
    empty = rng.random(X.shape) < invalid_frac
    var[empty] = np.inf
    h[empty] = np.nan
    t_last = rng.integers(max(0, t_now - 10), max(1, t_now), X.shape).astype(np.int32)
    out = {"h": h.astype(F32), "var": var.astype(F32), "t_last": t_last, "t_now": t_now}
    if with_normals:
        tilt = rng.normal(0.0, 0.3, (2,) + X.shape)
        n = np.stack([tilt[0], tilt[1], np.ones_like(X)])
        n = n / np.linalg.norm(n, axis=0)
        nan = rng.random(X.shape) < 0.1
        n[:, nan | empty] = np.nan
        out.update(nx=n[0].astype(F32), ny=n[1].astype(F32), nz=n[2].astype(F32))
    return out
