"""Pins of the oracle's marginal bands (CPU only).

The parity tests compare decisions bit for bit except where the oracle flags a
decision as marginal: its exact FP64 value lies so close to the threshold that
float32 arithmetic may decide it the other way.  Those bands decide what the
parity tests skip, so each is pinned here from both sides:

  * sound: inputs are placed around the threshold (cell edges, the range
    limits, the Mahalanobis gate, the wall rule, the Eq. 3 ray threshold, the
    Eq. 4 guard, the exclusion ramp), the decision is recomputed in float32 by
    two evaluation orders written out here (an FMA chain and plain float32
    operations), and every input on which either differs from the oracle must
    be flagged; each test also checks that such inputs exist, so it is not
    vacuous;
  * tight: inputs far from the threshold (beyond a stated distance, well above
    the band) are never flagged, and inputs within the absolute band (1e-6) are
    always flagged.

The drift band (Section II-D) is pinned by brute force: every way the
float32 path may assign the marginal points of a tiny map is enumerated, and
the deviation of each resulting mean must stay within the band.
"""
import itertools
import math

import numpy as np
import pytest

U = 2.0 ** -24
AB = 1e-6
f32 = np.float32


def fma32(a, b, c):
    """float32 fused multiply-add (the product of two float32 is exact in float64)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def mul32(a, b):
    return (np.asarray(a, f32) * np.asarray(b, f32)).astype(f32)


def add32(a, b):
    return (np.asarray(a, f32) + np.asarray(b, f32)).astype(f32)


def sub32(a, b):
    return (np.asarray(a, f32) - np.asarray(b, f32)).astype(f32)


def make(oracle_mod, **kw):
    return oracle_mod.OracleMap(oracle_mod.Params(**kw))


def pose12(R, t):
    P = np.zeros((3, 4))
    P[:, :3] = R
    P[:, 3] = t
    return P.astype(f32).reshape(12)


def rot(yaw, pitch):
    cz, sz, cy, sy = math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch)
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    return Rz @ Ry


def transform32(pose, pts, fused):
    """Map-frame coordinates of float32 sensor points in float32: the FMA chain
    R0 px + (R1 py + R2 pz), or plain float32 products and sums."""
    P = np.asarray(pose, f32).reshape(3, 4)
    px, py, pz = (pts[:, i].astype(f32) for i in range(3))
    out = []
    for r in range(3):
        if fused:
            v = fma32(P[r, 0], px, fma32(P[r, 1], py, mul32(P[r, 2], pz)))
        else:
            v = add32(add32(mul32(P[r, 0], px), mul32(P[r, 1], py)), mul32(P[r, 2], pz))
        out.append((v, add32(v, P[r, 3])))
    return out  # [(v_r, x_r)] for r = x, y, z


def dist32(pts, fused):
    px, py, pz = (pts[:, i].astype(f32) for i in range(3))
    if fused:
        d2 = fma32(px, px, fma32(py, py, mul32(pz, pz)))
    else:
        d2 = add32(add32(mul32(px, px), mul32(py, py)), mul32(pz, pz))
    return np.sqrt(d2.astype(f32)).astype(f32)


def cells32(x, y, x0, y0, r, fused):
    """floor((x - x0) / r) in float32, as a product with the rounded 1/r or as a quotient."""
    if fused:
        inv = f32(1.0 / float(f32(r)))
        qx, qy = mul32(sub32(x, f32(x0)), inv), mul32(sub32(y, f32(y0)), inv)
    else:
        qx = (sub32(x, f32(x0)) / f32(r)).astype(f32)
        qy = (sub32(y, f32(y0)) / f32(r)).astype(f32)
    return np.floor(qx).astype(np.int64), np.floor(qy).astype(np.int64)


def sensor_points(pose, pm):
    """float32 sensor-frame points whose exact map-frame image is pm (FP64)."""
    P = np.asarray(pose, np.float64).reshape(3, 4)
    return ((pm - P[:, 3]) @ P[:, :3]).astype(f32)


def exact_map(pose, pts):
    P = np.asarray(pose, np.float64).reshape(3, 4)
    return pts.astype(np.float64) @ P[:, :3].T + P[:, 3]


def trace(m, oracle_mod, clouds):
    return m.update(clouds, trace=True, unit=oracle_mod.FP32_UNIT, abs_band=AB)


# ------------------------------------------------------------------- binning

@pytest.mark.parametrize("far", [False, True])
def test_bin_band(oracle_mod, far):
    """Cell indices (Section II-A binning): every float32 index that differs is
    flagged PF_BIN; points farther than a few times the band from a cell edge
    never are; points within 1e-6 m always are.  Far: the map and the sensor
    80 m from the origin, where float32 rounding exceeds the 1e-6 m floor."""
    r = 0.04
    m = make(oracle_mod, width=100, height=100, resolution=r, noise_a0=0.01)
    m.shift(2037 if far else 37, -1977 if far else -23)
    x0, y0 = m.origin()
    off = np.array([81.5, -79.1, 0.0]) if far else np.zeros(3)
    pose = pose12(rot(0.7, 0.1), np.array([1.3, -0.7, 0.8]) + off)
    rng = np.random.default_rng(11)
    n = 60000
    ix = rng.integers(-2, 102, n)
    iy = rng.integers(-2, 102, n)
    spread = 1.5e-4 if far else 3e-5
    dx = rng.uniform(-spread, spread, n)
    dy = np.where(rng.random(n) < 0.5, rng.uniform(-spread, spread, n), rng.uniform(0.002, 0.038, n))
    pm = np.column_stack([x0 + ix * r + dx, y0 + iy * r + dy, rng.uniform(-0.5, 0.5, n)])
    pts = sensor_points(pose, pm)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.pflags & oracle_mod.PF_BIN) != 0
    diffs = 0
    for fused in (True, False):
        (_, x), (_, y), _ = transform32(pose, pts, fused)
        gx, gy = cells32(x, y, x0, y0, r, fused)
        bad = (gx != tr.ix) | (gy != tr.iy)
        assert not (bad & ~flagged).any(), f"unflagged float32 cell change on {(bad & ~flagged).sum()} points"
        diffs += int(bad.sum())
    assert diffs > 20
    xe = exact_map(pose, pts)
    qx, qy = (xe[:, 0] - x0) / r, (xe[:, 1] - y0) / r
    ed = np.minimum(np.minimum(qx - np.floor(qx), np.ceil(qx) - qx), np.minimum(qy - np.floor(qy), np.ceil(qy) - qy)) * r
    assert not (flagged & (ed > (1e-4 if far else 2e-5))).any()
    assert flagged[ed < AB].all() and (ed < AB).sum() > 20


@pytest.mark.parametrize("rmax", [7.3, 39.3])
def test_range_band(oracle_mod, rmax):
    """d against min_range and max_range (Section II-C): float32 distance
    decisions that differ are flagged PF_RANGE; none farther than 5e-5 m.
    A 39.3 m limit (a LiDAR range) puts float32 rounding above the 1e-6 floor."""
    m = make(oracle_mod, width=50, height=50, resolution=0.04, noise_a0=0.01, min_range=0.7, max_range=rmax)
    pose = pose12(np.eye(3), [0.0, 0.0, 0.0])
    rng = np.random.default_rng(12)
    n = 40000
    lim = np.where(rng.random(n) < 0.5, 0.7, rmax).astype(np.float64)
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = (dirs * (lim + rng.uniform(-4e-6, 4e-6, n) * lim / 7.3)[:, None]).astype(f32)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.pflags & oracle_mod.PF_RANGE) != 0
    o_valid = tr.status != oracle_mod.ST_RANGE
    diffs = 0
    for fused in (True, False):
        d = dist32(pts, fused)
        g_valid = (d >= f32(0.7)) & (d <= f32(rmax))
        bad = g_valid != o_valid
        assert not (bad & ~flagged).any()
        diffs += int(bad.sum())
    assert diffs > 20
    de = np.linalg.norm(pts.astype(np.float64), axis=1)
    far = np.minimum(np.abs(de - 0.7), np.abs(de - rmax))
    assert not (flagged & (far > 5e-5)).any()
    assert flagged[far < AB].all()


# --------------------------------------------------------- gate and wall rule

def _prior(oracle_mod, m, h, var, t_last, t_now):
    m.set_state(h=h, var=var, t_last=t_last, t_now=t_now)


def test_gate_band(oracle_mod):
    """Mahalanobis gate |z - h| / sqrt(var_eff + var_p) > k (Section II-C), with
    time variance: float32 decisions in the squared and in the quotient form
    that differ are flagged PF_GATE; none farther than 1e-3 in distance units;
    all within 1e-6."""
    W = H = 40
    r = 0.05
    k = 2.5
    P = dict(width=W, height=H, resolution=r, noise_a0=0.004, noise_a1=0.0, noise_a2=0.003, var_min=1e-8,
             mahalanobis_k=k, time_variance=float(f32(3e-6)))
    m = make(oracle_mod, **P)
    rng = np.random.default_rng(13)
    h = rng.uniform(-0.3, 0.3, (H, W)).astype(f32)
    var = (10 ** rng.uniform(-5, -3, (H, W))).astype(f32)
    t_last = rng.integers(1, 9, (H, W)).astype(np.int32)
    m.set_state(h=h.astype(np.float64), var=var.astype(np.float64), t_last=t_last, t_now=9)
    x0, y0 = m.origin()
    pose = pose12(rot(0.3, 0.05), [0.2, -0.1, 0.9])
    n = 40000
    cx, cy = rng.integers(0, W, n), rng.integers(0, H, n)
    pm = np.column_stack([x0 + (cx + rng.uniform(0.1, 0.9, n)) * r, y0 + (cy + rng.uniform(0.1, 0.9, n)) * r,
                          np.zeros(n)])
    # place z so that the Mahalanobis distance is k + delta, using the exact d of a first guess
    ve = var[cy, cx].astype(np.float64) + float(f32(3e-6)) * (10 - t_last[cy, cx])
    for _ in range(2):
        pts = sensor_points(pose, pm)
        d = np.linalg.norm(pts.astype(np.float64), axis=1)
        vp = np.maximum((0.004 + 0.003 * d * d) ** 2, 1e-8)
        md = k + rng.uniform(-2e-5, 2e-5, n) if _ == 0 else md
        sign = np.where(rng.random(n) < 0.5, 1.0, -1.0) if _ == 0 else sign
        pm[:, 2] = h[cy, cx] + sign * md * np.sqrt(ve + vp)
    pts = sensor_points(pose, pm)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.pflags & oracle_mod.PF_GATE) != 0
    o_rej = tr.status == oracle_mod.ST_REJECT
    inmap = tr.status >= oracle_mod.ST_ACCEPT
    diffs = 0
    for fused in (True, False):
        d32 = dist32(pts, fused)
        (_, _), (_, _), (_, z32) = transform32(pose, pts, fused)
        s = fma32(fma32(f32(0.003), d32, f32(0.0)), d32, f32(0.004)) if fused else \
            add32(mul32(mul32(f32(0.003), d32), d32), f32(0.004))
        vp32 = np.maximum(mul32(s, s), f32(1e-8))
        ii, jj = np.clip(tr.iy, 0, H - 1), np.clip(tr.ix, 0, W - 1)
        ve32 = fma32(f32(3e-6), (9 + 1 - t_last[ii, jj]).astype(f32), var[ii, jj])
        dz = sub32(z32, h[ii, jj])
        if fused:
            g_rej = mul32(dz, dz) > mul32(mul32(f32(k), f32(k)), add32(ve32, vp32))
        else:
            g_rej = (np.abs(dz) / np.sqrt(add32(ve32, vp32)).astype(f32)).astype(f32) > f32(k)
        bad = inmap & (g_rej != o_rej)
        assert not (bad & ~flagged).any(), f"unflagged gate change on {(bad & ~flagged).sum()} points"
        diffs += int(bad.sum())
    assert diffs > 20
    xe = exact_map(pose, pts)
    de = np.linalg.norm(pts.astype(np.float64), axis=1)
    ii, jj = np.clip(tr.iy, 0, H - 1), np.clip(tr.ix, 0, W - 1)
    ve = var[ii, jj].astype(np.float64) + float(f32(3e-6)) * (10 - t_last[ii, jj])
    mde = np.abs(xe[:, 2] - h[ii, jj]) / np.sqrt(ve + np.maximum((0.004 + 0.003 * de * de) ** 2, 1e-8))
    assert not (flagged & inmap & (np.abs(mde - k) > 1e-3)).any()
    assert flagged[inmap & (np.abs(mde - k) < AB)].all()


def test_wall_band(oracle_mod):
    """Wall rule z < h in a cell with more than N points (Section II-C): float32
    comparisons that differ are flagged PF_WALL; none farther than 1e-5 m."""
    W = H = 20
    r = 0.05
    m = make(oracle_mod, width=W, height=H, resolution=r, noise_a0=0.01, wall_num_thresh=3)
    rng = np.random.default_rng(14)
    h = rng.uniform(-0.4, 0.4, (H, W)).astype(f32)
    m.set_state(h=h.astype(np.float64), var=np.full((H, W), 1e-4), t_last=np.ones((H, W), np.int32), t_now=1)
    x0, y0 = m.origin()
    pose = pose12(rot(1.1, -0.08), [0.1, 0.3, 1.2])
    n = 20000
    cx, cy = rng.integers(0, W, n), rng.integers(0, H, n)
    pm = np.column_stack([x0 + (cx + rng.uniform(0.1, 0.9, n)) * r, y0 + (cy + rng.uniform(0.1, 0.9, n)) * r,
                          h[cy, cx] + rng.uniform(-1e-6, 1e-6, n)])
    pts = sensor_points(pose, pm)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.pflags & oracle_mod.PF_WALL) != 0
    o_wall = tr.status == oracle_mod.ST_WALL
    inmap = tr.status >= oracle_mod.ST_ACCEPT
    diffs = 0
    for fused in (True, False):
        _, _, (_, z32) = transform32(pose, pts, fused)
        g_wall = z32 < h[np.clip(tr.iy, 0, H - 1), np.clip(tr.ix, 0, W - 1)]
        bad = inmap & (g_wall != o_wall)
        assert not (bad & ~flagged).any()
        diffs += int(bad.sum())
    assert diffs > 20
    ze = exact_map(pose, pts)[:, 2]
    gap = np.abs(ze - h[np.clip(tr.iy, 0, H - 1), np.clip(tr.ix, 0, W - 1)])
    assert not (flagged & (gap > 1e-5)).any()
    assert flagged[inmap & (gap < AB)].all()


def test_exclusion_ramp_band(oracle_mod):
    """Exclusion ramp (Section II-C, read as a ramp): float32 decisions that
    differ are flagged PF_RANGE; none farther than 1e-5 m from the ramp."""
    b, c, th, dlim = 0.2, 1.5, 0.3, 0.9
    m = make(oracle_mod, width=80, height=80, resolution=0.1, noise_a0=0.01, excl_b=b, excl_c=c, excl_theta=th,
             excl_d=dlim)
    pose = pose12(rot(0.4, 0.0), [0.3, -0.2, 0.6])
    rng = np.random.default_rng(15)
    n = 30000
    rr = rng.uniform(0.2, 3.8, n)
    az = rng.uniform(0, 2 * math.pi, n)
    lim = np.minimum(np.where(rr <= c, b, b + (rr - c) * math.tan(float(f32(th)))), dlim)
    zr = lim + rng.uniform(-3e-6, 3e-6, n)
    P = np.asarray(pose, np.float64).reshape(3, 4)
    pm = np.column_stack([P[0, 3] + rr * np.cos(az), P[1, 3] + rr * np.sin(az), P[2, 3] + zr])
    pts = sensor_points(pose, pm)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.pflags & oracle_mod.PF_RANGE) != 0
    o_in = tr.status != oracle_mod.ST_RANGE
    tan32 = f32(math.tan(float(f32(th))))
    diffs = 0
    for fused in (True, False):
        (vx, _), (vy, _), (vz, _) = transform32(pose, pts, fused)
        rh = np.sqrt(fma32(vx, vx, mul32(vy, vy)) if fused else add32(mul32(vx, vx), mul32(vy, vy))).astype(f32)
        ramp = fma32(sub32(rh, f32(c)), tan32, f32(b)) if fused else add32(mul32(sub32(rh, f32(c)), tan32), f32(b))
        g_lim = np.minimum(np.where(rh <= f32(c), f32(b), ramp), f32(dlim))
        bad = (~(vz > g_lim)) != o_in
        assert not (bad & ~flagged).any(), f"unflagged ramp change on {(bad & ~flagged).sum()} points"
        diffs += int(bad.sum())
    assert diffs > 20
    xe = exact_map(pose, pts)
    rre = np.hypot(xe[:, 0] - P[0, 3], xe[:, 1] - P[1, 3])
    lime = np.minimum(np.where(rre <= c, b, b + (rre - c) * math.tan(float(f32(th)))), dlim)
    gap = np.minimum(np.abs(xe[:, 2] - P[2, 3] - lime), np.abs(rre - c))
    assert not (flagged & (gap > 1e-5)).any()


# -------------------------------------------------------------- ray casting

def _ray_map(oracle_mod, W, H, r, step, alpha=0.0):
    return make(oracle_mod, width=W, height=H, resolution=r, noise_a0=0.01, ray_step=step,
                cleanup_normal_thresh=alpha)


def _march32(pose, pts, x0, y0, r, step, W, H, thr, fused, guard=None):
    """Marked cells of float32 ray marches (Section II-E, Eq. 3): samples
    o + k step rhat for k step < d, the endpoint's cell skipped.  fused: the
    per-ray set-up a + k b in cell units with one FMA per coordinate; else the
    sample position in metres, then binned."""
    Pp = np.asarray(pose, f32).reshape(3, 4)
    (vx, x), (vy, y), (vz, z) = transform32(pose, pts, fused)
    d = dist32(pts, fused)
    ex, ey = cells32(x, y, x0, y0, r, fused)
    marks = np.zeros((H, W), bool)
    inv = f32(1.0 / float(f32(r)))
    for i in range(len(pts)):
        di = d[i]
        kmax = int(math.floor(float(di) / step)) + 2
        ks = np.arange(1, kmax + 1)
        kf = ks.astype(f32)
        live = mul32(kf, f32(step)) < di
        if fused:
            cstep = f32(f32(step) / di)
            ax = mul32(sub32(Pp[0, 3], f32(x0)), inv)
            ay = mul32(sub32(Pp[1, 3], f32(y0)), inv)
            bx = mul32(mul32(cstep, vx[i]), inv)
            by = mul32(mul32(cstep, vy[i]), inv)
            bz = mul32(cstep, vz[i])
            cx = np.floor(fma32(kf, bx, ax)).astype(np.int64)
            cy = np.floor(fma32(kf, by, ay)).astype(np.int64)
            zz = fma32(kf, bz, Pp[2, 3])
        else:
            f = (mul32(kf, f32(step)) / di).astype(f32)
            sx, sy = add32(Pp[0, 3], mul32(f, vx[i])), add32(Pp[1, 3], mul32(f, vy[i]))
            zz = add32(Pp[2, 3], mul32(f, vz[i]))
            cx = np.floor((sub32(sx, f32(x0)) / f32(r)).astype(f32)).astype(np.int64)
            cy = np.floor((sub32(sy, f32(y0)) / f32(r)).astype(f32)).astype(np.int64)
        ok = live & (cx >= 0) & (cy >= 0) & (cx < W) & (cy < H) & ~((cx == ex[i]) & (cy == ey[i]))
        cxo, cyo, zo = cx[ok], cy[ok], zz[ok]
        below = zo < thr[cyo, cxo]
        if guard is not None:
            below &= guard(i, cyo, cxo, fused)
        marks[cyo[below], cxo[below]] = True
    return marks


@pytest.mark.parametrize("far", [False, True])
def test_ray_threshold_band(oracle_mod, far):
    """Eq. 3 ray marks (sample below h - sqrt(var)): the cells that float32
    marches mark differently from the oracle are flagged CF_MARK, for sample
    heights within micrometres of the thresholds and positions near cell
    edges; only cells that hold an estimate are ever flagged.  Far: the map
    60 m from the origin and the ground at 50 m altitude, where float32
    rounding exceeds the 1e-6 m floor."""
    W = H = 60
    r = 0.05
    step = 0.05
    m = _ray_map(oracle_mod, W, H, r, step)
    m.shift(1193 if far else -7, -1189 if far else 11)
    x0, y0 = m.origin()
    rng = np.random.default_rng(16)
    origin = np.array([x0 + 30.37 * r, y0 + 29.81 * r, 50.8 if far else 0.8])
    pose = pose12(rot(0.2, 0.0), origin)
    n = 120                                  # 3 degrees apart: targets 1 m out lie in distinct cells
    ang = (np.arange(n) + rng.uniform(-0.1, 0.1, n)) * (2 * math.pi / n)
    dist = rng.uniform(1.2, 1.4, n)
    ends = np.column_stack([origin[0] + dist * np.cos(ang), origin[1] + dist * np.sin(ang),
                            np.full(n, origin[2] - 0.8)])
    pts = sensor_points(pose, ends)
    pe = exact_map(pose, pts)
    # target samples every 4 steps along each ray: their cells get thresholds near the sample height
    h = np.full((H, W), np.nan)
    var = np.full((H, W), np.inf)
    o = np.asarray(pose, np.float64).reshape(3, 4)[:, 3]   # the sensor origin as the pose carries it
    for i in range(n):
        v = pe[i] - o
        d = np.linalg.norm(pts[i].astype(np.float64))
        for ks in range(int(0.6 / step) + int(rng.integers(0, 3)), int(d / step) - 2, 4):
            s = o + (ks * step / d) * v
            ix, iy = int(math.floor((s[0] - x0) / r)), int(math.floor((s[1] - y0) / r))
            if np.isfinite(var[iy, ix]):
                continue
            # the ray descends: its lowest sample in this cell decides the mark
            for kk in range(ks + 1, ks + 3):
                s2 = o + (kk * step / d) * v
                if (int(math.floor((s2[0] - x0) / r)), int(math.floor((s2[1] - y0) / r))) == (ix, iy):
                    s = s2
            sd = float(np.sqrt(f32(rng.uniform(0.005, 0.02) ** 2)))
            # half the thresholds within float32 rounding of the sample, half up to
            # 3x the band away (near the origin the band is about 2e-6 m, at 50 m 5e-5 m)
            spread = (4e-6 if rng.random() < 0.5 else 1.5e-4) if far else (3e-7 if rng.random() < 0.5 else 6e-6)
            h[iy, ix] = float(f32(s[2] + sd + rng.uniform(-spread, spread)))
            var[iy, ix] = float(f32(sd * sd))
    m.set_state(h=h, var=var, t_last=np.ones((H, W), np.int32), t_now=3)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.cflags & oracle_mod.CF_MARK) != 0
    h32, v32 = h.astype(f32), var.astype(f32)
    thr = np.where(np.isfinite(v32), sub32(h32, np.sqrt(v32).astype(f32)), -np.inf).astype(f32)
    diffs = 0
    for fused in (True, False):
        g = _march32(pose, pts, x0, y0, r, step, W, H, thr, fused)
        bad = g != (tr.mark != 0)
        assert not (bad & ~flagged).any(), f"unflagged mark change on {(bad & ~flagged).sum()} cells"
        diffs += int(bad.sum())
    assert diffs > 6
    assert not (flagged & ~np.isfinite(var)).any()        # only cells a ray could mark
    assert flagged.sum() < 0.8 * np.isfinite(var).sum()   # thresholds far from the samples are not


def test_ray_guard_band(oracle_mod):
    """Eq. 4 guard |rhat . n| > alpha_n: cells whose float32 guard decides
    otherwise are flagged CF_MARK."""
    W = H = 64
    r = 0.05
    step = 0.05
    alpha = 0.35
    m = _ray_map(oracle_mod, W, H, r, step, alpha)
    x0, y0 = m.origin()
    rng = np.random.default_rng(17)
    origin = np.array([x0 + 32.4 * r, y0 + 31.7 * r, 0.6])
    pose = pose12(np.eye(3), origin)
    n = 120                                  # 3 degrees apart: targets 1 m out lie in distinct cells
    ang = (np.arange(n) + rng.uniform(-0.1, 0.1, n)) * (2 * math.pi / n)
    dist = rng.uniform(1.3, 1.5, n)
    ends = np.column_stack([origin[0] + dist * np.cos(ang), origin[1] + dist * np.sin(ang), np.zeros(n)])
    pts = sensor_points(pose, ends)
    h = np.full((H, W), np.nan)               # only the target cells hold estimates, far above the rays:
    var = np.full((H, W), np.inf)             # the guard alone decides their marks
    # per cell a normal whose |rhat . n| lies within 1.5e-7 of alpha for the ray through it
    nx = np.zeros((H, W))
    ny = np.zeros((H, W))
    nz = np.ones((H, W))
    pe = exact_map(pose, pts)
    for i in range(n):
        v = pe[i] - origin
        rh = v / np.linalg.norm(v)
        ks = int(rng.integers(int(1.0 / step), int(1.2 / step)))
        s = origin + ks * step * rh
        ix, iy = int(math.floor((s[0] - x0) / r)), int(math.floor((s[1] - y0) / r))
        # a unit normal e with rhat . e = alpha + delta
        t = alpha + rng.uniform(-1.5e-7, 1.5e-7)
        perp = np.cross(rh, [0.0, 0.0, 1.0])
        perp /= np.linalg.norm(perp)
        e = t * rh + math.sqrt(1 - t * t) * perp
        nx[iy, ix], ny[iy, ix], nz[iy, ix] = e
        h[iy, ix], var[iy, ix] = 2.0, 1e-4
    m.set_state(h=h, var=var, t_last=np.ones((H, W), np.int32), nx=nx, ny=ny, nz=nz, t_now=3)
    tr = trace(m, oracle_mod, (pts, pose))
    flagged = (tr.cflags & oracle_mod.CF_MARK) != 0
    thr = np.where(np.isfinite(var), sub32(h.astype(f32), np.sqrt(var.astype(f32)).astype(f32)), -np.inf).astype(f32)
    n32 = [a.astype(f32) for a in (nx, ny, nz)]
    (vx, _), (vy, _), (vz, _) = transform32(pose, pts, True)
    d32 = dist32(pts, True)

    def guard(i, cy, cx, fused):
        rx, ry, rz = (np.float32(v[i] / d32[i]) for v in (vx, vy, vz))
        if fused:
            dot = fma32(rx, n32[0][cy, cx], fma32(ry, n32[1][cy, cx], mul32(rz, n32[2][cy, cx])))
        else:
            dot = add32(add32(mul32(rx, n32[0][cy, cx]), mul32(ry, n32[1][cy, cx])), mul32(rz, n32[2][cy, cx]))
        return np.abs(dot) > f32(alpha)

    diffs = 0
    for fused in (True, False):
        g = _march32(pose, pts, x0, y0, r, step, W, H, thr, fused, guard)
        bad = g != (tr.mark != 0)
        assert not (bad & ~flagged).any(), f"unflagged guard change on {(bad & ~flagged).sum()} cells"
        diffs += int(bad.sum())
    assert diffs > 3


def test_ray_position_and_own_cell_bands(oracle_mod):
    """Horizontal rays of a map 60 m from the origin: (a) rays running within
    micrometres of a row edge, so float32 puts every sample in the row above
    or below (only the row above holds estimates, all above the ray); (b) rays
    whose endpoint lies within micrometres of a column edge, so float32 may
    give the endpoint the other column as its own cell and skip that column's
    samples.  Cells marked differently by float32 marches are flagged."""
    W = H = 64
    r = 0.05
    step = 0.025
    m = _ray_map(oracle_mod, W, H, r, step)
    m.shift(1201, -1213)
    x0, y0 = m.origin()
    rng = np.random.default_rng(19)
    h = np.full((H, W), np.nan)
    var = np.full((H, W), np.inf)
    z = 50.3
    ends, origins = [], []
    for j in range(30):
        row = 2 * j + 2
        edge_ray = j % 2 == 0
        dy = rng.uniform(-8e-6, 8e-6) if edge_ray else 0.021
        dx = 0.013 if edge_ray else rng.uniform(-8e-6, 8e-6)
        oy = y0 + row * r + dy
        origins.append((x0 + 3.3 * r, oy, z))
        ends.append((x0 + (40 + j % 5) * r + dx, oy, z))
        h[row, 4:50] = z + 0.06                    # thresholds 1 cm above the ray
        var[row, 4:50] = 2.5e-3
    tr_all, g_all = [], [np.zeros((H, W), bool), np.zeros((H, W), bool)]
    flagged = np.zeros((H, W), bool)
    omark = np.zeros((H, W), bool)
    m.set_state(h=h, var=var, t_last=np.ones((H, W), np.int32), t_now=3)
    clouds = []
    for o, e in zip(origins, ends):
        pose = pose12(np.eye(3), o)
        clouds.append((sensor_points(pose, np.array([e])), pose))
    tr = trace(m, oracle_mod, clouds)
    flagged = (tr.cflags & oracle_mod.CF_MARK) != 0
    h32, v32 = h.astype(f32), var.astype(f32)
    thr = np.where(np.isfinite(v32), sub32(h32, np.sqrt(v32).astype(f32)), -np.inf).astype(f32)
    diffs = 0
    for fused in (True, False):
        g = np.zeros((H, W), bool)
        for pts, pose in clouds:
            g |= _march32(pose, pts, x0, y0, r, step, W, H, thr, fused)
        bad = g != (tr.mark != 0)
        assert not (bad & ~flagged).any(), f"unflagged mark change on {(bad & ~flagged).sum()} cells"
        diffs += int(bad.sum())
    assert diffs > 10
    assert flagged.sum() < 0.8 * (tr.mark != 0).sum()


def test_ray_marks_unflagged_far_from_thresholds(oracle_mod):
    """A horizontal ray whose samples lie 1 mm from every threshold and away
    from cell edges flags nothing, and marks exactly the cells below it."""
    W, H, r, step = 60, 20, 0.1, 0.1
    m = _ray_map(oracle_mod, W, H, r, step)
    h = np.full((H, W), np.nan)
    var = np.full((H, W), np.inf)
    h[10, 32:44] = 0.2 + 0.01 + np.where(np.arange(12) % 2 == 0, 1e-3, -1e-3)  # thresholds 0.2 +- 1 mm
    var[10, 32:44] = 1e-4
    m.set_state(h=h, var=var, t_last=np.ones((H, W), np.int32), t_now=4)
    pts = np.array([[1.6, 0.0, 0.0]], f32)
    tr = trace(m, oracle_mod, (pts, pose12(np.eye(3), [0.05 + 0.013, 0.05, 0.2])))
    assert not tr.cflags.any()
    expect = np.zeros((H, W), bool)
    expect[10, 32:44] = np.arange(12) % 2 == 0
    assert np.array_equal(tr.mark != 0, expect)


# ------------------------------------------------------------- drift band

def test_drift_band_brute_force(oracle_mod):
    """Section II-D drift mean: every float32 assignment of the bin-marginal
    points to one of their candidate cells (or none) gives a mean within the
    oracle's band of its own; the band is at most three times the largest such
    deviation plus the float32 rounding terms."""
    W = H = 6
    r = 1.0
    rng = np.random.default_rng(18)
    h = rng.uniform(-0.05, 0.05, (H, W))
    nz = np.where(rng.random((H, W)) < 0.8, 1.0, 0.5)
    h[0, 5] = np.nan
    m = oracle_mod.OracleMap(oracle_mod.Params(width=W, height=H, resolution=r, noise_a0=0.01, drift_flatness=0.9))
    var = np.where(np.isnan(h), np.inf, 1e-4)
    m.set_state(h=h, var=var, t_last=np.ones((H, W), np.int32), nx=np.zeros((H, W)), ny=np.zeros((H, W)),
                nz=nz, t_now=1)
    # ordinary points at cell centres, and three at cell edges / corners (2e-7 m off)
    cen = [(ix + 0.5 - 3, iy + 0.5 - 3) for ix in range(W) for iy in range(H)]
    edge = [(1.0 + 2e-7 - 3, 2.5 - 3), (3.0 - 2e-7 - 3, 4.0 + 2e-7 - 3), (-3 + 1e-7, 1.5 - 3)]
    xy = np.array(cen + edge)
    z = rng.uniform(0.0, 0.1, len(xy))
    pts = np.column_stack([xy, z]).astype(f32)
    pose = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], f32)
    tr = m.update((pts, pose), trace=True, unit=oracle_mod.FP32_UNIT, abs_band=AB)
    mean, n, band = m.last_drift_band()
    marg = np.flatnonzero(tr.pflags & oracle_mod.PF_BIN)
    assert set(marg) == {len(cen), len(cen) + 1, len(cen) + 2}
    pe = pts.astype(np.float64)

    def contrib(i, cell):
        if cell is None:
            return None
        ix, iy = cell
        if not (0 <= ix < W and 0 <= iy < H) or np.isnan(h[iy, ix]) or not nz[iy, ix] >= 0.9:
            return None
        return pe[i, 2] - h[iy, ix]

    base = {i: contrib(i, (int(math.floor(pe[i, 0] + 3)), int(math.floor(pe[i, 1] + 3)))) for i in range(len(pe))}
    assert sum(v is not None for v in base.values()) == n
    alts = []
    for i in marg:
        qx, qy = pe[i, 0] + 3, pe[i, 1] + 3
        xs = {int(math.floor(qx)), int(math.floor(qx - 1e-5)), int(math.floor(qx + 1e-5))}
        ys = {int(math.floor(qy)), int(math.floor(qy - 1e-5)), int(math.floor(qy + 1e-5))}
        alts.append([contrib(i, (a, b)) for a in xs for b in ys])
    worst = 0.0
    for combo in itertools.product(*alts):
        vals = [v for i, v in base.items() if i not in marg and v is not None] + [v for v in combo if v is not None]
        worst = max(worst, abs(np.mean(vals) - mean))
    assert worst <= band
    assert band <= 3.0 * worst + 1e-5
