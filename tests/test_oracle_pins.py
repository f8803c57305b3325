"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand, an off-by-one in the ray samples)
fails at least one of them.  CPU only.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def pose_t(t, R=None):
    P = np.zeros((3, 4))
    P[:, :3] = np.eye(3) if R is None else R
    P[:, 3] = t
    return P.astype(np.float32).reshape(12)


def cloud(points):
    return np.asarray(points, np.float32).reshape(-1, 3)


def make(oracle_mod, **kw):
    return oracle_mod.OracleMap(oracle_mod.Params(**kw))


# ----------------------------------------------------------------- Eq. 1, Eq. 2

def test_two_point_fusion_golden(oracle_mod):
    g = load_golden("two_point_fusion.json")
    m = make(oracle_mod, **g["params"])
    pose = pose_t(g["pose_t"])
    ix, iy = g["cell"]
    tr = m.update((cloud(g["points"][:1]), pose), trace=True)
    s = m.state()
    assert (tr.ix[0], tr.iy[0]) == (ix, iy)
    assert s["h"][iy, ix] == pytest.approx(g["expected_after_first"]["h"], abs=1e-12)
    assert s["var"][iy, ix] == pytest.approx(g["expected_after_first"]["var"], rel=1e-12)
    m2 = make(oracle_mod, **g["params"])
    m2.update((cloud(g["points"]), pose))
    s2 = m2.state()
    assert s2["h"][iy, ix] == pytest.approx(g["expected_h"], abs=1e-12)
    assert s2["var"][iy, ix] == pytest.approx(g["expected_var"], rel=1e-12)
    # exactly one cell touched
    assert np.isfinite(s2["var"]).sum() == 1


def test_gate_fusion_golden(oracle_mod):
    g = load_golden("gate_fusion.json")
    m = make(oracle_mod, **g["params"])
    H, W = m.shape
    ix, iy = g["cell"]
    pr = g["prior"]
    h = np.full((H, W), np.nan)
    var = np.full((H, W), np.inf)
    h[iy, ix], var[iy, ix] = pr["h"], pr["var"]
    t_last = np.zeros((H, W), np.int32)
    t_last[iy, ix] = pr["t_last"]
    m.set_state(h=h, var=var, t_last=t_last, t_now=pr["t_now"])
    tr = m.update((cloud(g["points"]), pose_t(g["pose_t"])), trace=True)
    assert list(tr.status) == g["expected_status"]
    s = m.state()
    # the points are float32: 0.02 and -0.01 carry a rounding of <= 6e-10 relative
    assert s["h"][iy, ix] == pytest.approx(g["expected_h"], abs=2e-9)
    assert s["var"][iy, ix] == pytest.approx(g["expected_var"], rel=1e-12)
    assert s["t_last"][iy, ix] == pr["t_now"] + 1
    assert tr.counts["rejected"] == 1 and tr.counts["accepted"] == 2


def test_single_point_empty_cell_noise_model(oracle_mod):
    """Single point into an empty cell gives (p_z, sigma_p^2) with the paper's
    noise model sigma_p^2 = alpha_d d^2 (a1 = sqrt(alpha_d))."""
    alpha_d = 2.5e-3
    m = make(oracle_mod, width=50, height=40, resolution=0.1, noise_a1=math.sqrt(alpha_d))
    p = np.array([[0.3, -0.4, -1.2]], np.float32)  # d = 1.3
    t = [0.07, 0.03, 0.25]
    tr = m.update((p, pose_t(t)), trace=True)
    d = math.sqrt(sum(float(v) ** 2 for v in p[0]))
    x, y, z = (float(p[0, i]) + t[i] for i in range(3))
    # hand-computed cell: x0 = -2.5, y0 = -2.0; x = 0.37 -> 28.7, y = -0.37 -> 16.3
    assert (tr.ix[0], tr.iy[0]) == (math.floor((x + 2.5) / 0.1), math.floor((y + 2.0) / 0.1)) == (28, 16)
    s = m.state()
    assert s["h"][16, 28] == pytest.approx(float(np.float32(-1.2)) + float(np.float32(0.25)), abs=1e-12)
    assert s["var"][16, 28] == pytest.approx(alpha_d * d * d, rel=1e-12)
    assert z == pytest.approx(s["h"][16, 28], abs=1e-7)


def test_rotation_pose(oracle_mod):
    """A 90 degree yaw maps the sensor x axis onto the map y axis."""
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float)
    m = make(oracle_mod, width=100, height=100, resolution=0.04, noise_a0=0.01)
    tr = m.update((cloud([[1.0, 0.0, -0.3]]), pose_t([0.01, 0.01, 0.5], R)), trace=True)
    # p_m = (0.01, 1.01, 0.2): ix = floor(2.01/0.04) = 50, iy = floor(3.01/0.04) = 75
    assert (tr.ix[0], tr.iy[0]) == (50, 75)
    assert m.state()["h"][75, 50] == pytest.approx(0.2, abs=1e-7)


def test_weighted_least_squares_equivalence(oracle_mod):
    """With the gate and the outlier variance off, Eq. 1/2 applied point after
    point equals the inverse-variance weighted mean per cell (numpy.average)
    and the variance 1/sum(1/sigma_p^2) -- the textbook batch form."""
    pts, pose = synth.single_update(seed=11, n=3000, half=0.5)
    P = dict(width=20, height=20, resolution=0.04, noise_a0=0.004, noise_a1=0.003, noise_a2=0.002)
    m = make(oracle_mod, **P)
    tr = m.update((pts, pose), trace=True)
    s = m.state()
    p64 = pts.astype(np.float64)
    d = np.linalg.norm(p64, axis=1)
    w = 1.0 / (P["noise_a0"] + P["noise_a1"] * d + P["noise_a2"] * d * d) ** 2
    ok = tr.status == oracle_mod.ST_ACCEPT
    checked = 0
    for (ix, iy) in set(zip(tr.ix[ok], tr.iy[ok])):
        sel = ok & (tr.ix == ix) & (tr.iy == iy)
        hz = np.average(p64[sel, 2], weights=w[sel])
        assert s["h"][iy, ix] == pytest.approx(hz, abs=1e-12)
        assert s["var"][iy, ix] == pytest.approx(1.0 / w[sel].sum(), rel=1e-10)
        checked += 1
    assert checked > 200


def test_permutation_invariance(oracle_mod):
    """Every permutation of up to six points into one valid cell (gate and
    outlier variance on) gives the same result (1e-12)."""
    rng = np.random.default_rng(3)
    P = dict(width=10, height=10, resolution=0.1, noise_a0=0.01, noise_a1=0.01, mahalanobis_k=2.0,
             outlier_variance=2e-4)
    base = rng.normal(0, 0.02, (6, 3))
    base[:, :2] = rng.uniform(0.01, 0.09, (6, 2))
    base[4, 2] = 0.2  # an outlier
    results = []
    for perm in itertools.permutations(range(6)):
        m = make(oracle_mod, **P)
        h = np.full((10, 10), np.nan)
        var = np.full((10, 10), np.inf)
        h[5, 5], var[5, 5] = 0.0, 4e-4
        m.set_state(h=h, var=var, t_last=np.zeros((10, 10), np.int32), t_now=3)
        m.update((base[list(perm)].astype(np.float32), pose_t([0, 0, 0])))
        s = m.state()
        results.append((s["h"][5, 5], s["var"][5, 5]))
    hs, vs = np.array(results).T
    assert np.ptp(hs) <= 1e-12 and np.ptp(vs) <= 1e-12 * vs[0]


def test_variance_never_increases_without_rejection(oracle_mod):
    rng = np.random.default_rng(5)
    P = dict(width=30, height=30, resolution=0.05, noise_a0=0.01, noise_a2=0.01)
    m = make(oracle_mod, **P)
    pts, pose = synth.single_update(seed=5, n=4000, half=0.7)
    m.update((pts, pose))
    v1 = m.state()["var"]
    pts2, _ = synth.single_update(seed=6, n=4000, half=0.7)
    m.update((pts2, pose))
    v2 = m.state()["var"]
    fin = np.isfinite(v1)
    assert np.all(v2[fin] <= v1[fin])
    assert np.any(v2[fin] < v1[fin])
    assert rng is not None


def test_ignored_points(oracle_mod):
    P = dict(width=20, height=20, resolution=0.1, noise_a0=0.01, min_range=0.2, max_range=3.0)
    m = make(oracle_mod, **P)
    pts = cloud([[np.nan, 0, 0], [0, np.inf, 0], [0.05, 0.05, 0.05],  # non-finite, non-finite, d < min_range
                 [3.5, 0, 0],  # d > max_range
                 [1.5, 0.05, 0.0],  # out of the 2 m map (x >= 1)
                 [0.15, 0.15, -0.5]])  # the only valid in-map point
    tr = m.update((pts, pose_t([0, 0, 0])), trace=True)
    assert list(tr.status) == [0, 0, 1, 1, 2, 3]
    s = m.state()
    assert np.isfinite(s["var"]).sum() == 1
    assert tr.counts == {"in": 6, "valid": 2, "in_map": 1, "accepted": 1, "rejected": 0, "wall": 0,
                         "cells_updated": 1, "cleared": 0}


def test_wall_rule(oracle_mod):
    """More than wall_num_thresh points in a valid cell: points below the
    current height are dropped before the gate (Section II-C)."""
    P = dict(width=10, height=10, resolution=0.1, noise_a0=0.01, wall_num_thresh=3)
    zs = [-0.01, -0.02, 0.01, 0.0, 0.005]
    for n_pts, expect in ((5, [5, 5, 3, 3, 3]), (3, [3, 3, 3])):
        m = make(oracle_mod, **P)
        h = np.full((10, 10), np.nan)
        var = np.full((10, 10), np.inf)
        h[5, 5], var[5, 5] = 0.0, 1e-4
        m.set_state(h=h, var=var, t_last=np.zeros((10, 10), np.int32), t_now=0)
        pts = cloud([[0.05, 0.05, z] for z in zs[:n_pts]])
        tr = m.update((pts, pose_t([0, 0, 0])), trace=True)
        assert list(tr.status) == expect
        s = m.state()
        acc = [z for z, st in zip(zs[:n_pts], expect) if st == 3]
        # information form of the accepted points against the prior (all sp2 = 1e-4)
        lam = 1e4 + 1e4 * len(acc)
        zf = [float(np.float32(z)) for z in acc]
        assert s["h"][5, 5] == pytest.approx(1e4 * sum(zf) / lam, abs=1e-12)
        assert s["var"][5, 5] == pytest.approx(1.0 / lam, rel=1e-12)


def test_time_variance(oracle_mod):
    """sigma_t^2 is added once per update since the last write of the cell."""
    P = dict(width=10, height=10, resolution=0.1, noise_a0=0.01, time_variance=3e-5)
    m = make(oracle_mod, **P)
    pose = pose_t([0, 0, 0])
    m.update((cloud([[0.05, 0.05, 0.0]]), pose))                     # t = 1: var = 1e-4
    m.update((cloud([[0.35, 0.35, 0.0]]), pose))                     # t = 2: elsewhere
    m.update((cloud([[0.35, 0.35, 0.0]]), pose))                     # t = 3
    m.update((cloud([[0.05, 0.05, 0.1]]), pose))                     # t = 4: prior var 1e-4 + 3*3e-5
    s = m.state()
    vm = 1e-4 + 3 * 3e-5
    vp = 1e-4
    assert s["var"][5, 5] == pytest.approx(vm * vp / (vm + vp), rel=1e-12)
    assert s["h"][5, 5] == pytest.approx((vp * 0.0 + vm * float(np.float32(0.1))) / (vm + vp), abs=1e-12)
    assert s["t_last"][5, 5] == 4


# ------------------------------------------------------------------ ray casting

def _cells_state(oracle_mod, P, cells, t_last=1, t_now=5):
    m = make(oracle_mod, **P)
    H, W = m.shape
    h = np.full((H, W), np.nan)
    var = np.full((H, W), np.inf)
    for key, (hv, vv) in cells.items():
        ix, iy = map(int, key.split(","))
        h[iy, ix], var[iy, ix] = hv, vv
    m.set_state(h=h, var=var, t_last=np.full((H, W), t_last, np.int32), t_now=t_now)
    return m


def test_ray_cells_golden(oracle_mod):
    g = load_golden("ray_cells.json")
    for case in g["cases"]:
        m = _cells_state(oracle_mod, case["params"], case["cells"])
        tr = m.update((cloud([case["point"]]), pose_t(case["pose_t"])), trace=True)
        for ix, iy in case["expected_marked"]:
            assert tr.mark[iy, ix] == 1, case["name"]
            assert tr.cleared[iy, ix] == 1, case["name"]
        for ix, iy in case["expected_unmarked"]:
            assert tr.mark[iy, ix] == 0, (case["name"], ix, iy)
        assert tr.mark.sum() == len(case["expected_marked"]), case["name"]


def test_vertical_ray_clears_nothing(oracle_mod):
    P = dict(width=20, height=20, resolution=0.1, noise_a0=0.01, ray_step=0.02)
    cells = {f"{i},{j}": (0.0, 1e-4) for i in range(20) for j in range(20)}
    cells["10,10"] = (0.5, 1e-4)  # a stale obstacle right below the sensor
    m = _cells_state(oracle_mod, P, cells)
    tr = m.update((cloud([[0.0, 0.0, -1.0]]), pose_t([0.05, 0.05, 1.0])), trace=True)
    assert tr.mark.sum() == 0


def test_horizontal_ray_through_stale_box(oracle_mod):
    """A ray passing below a stale obstacle removes it; ground cells under the
    ray stay; a cell updated in the same update is kept (Section II-E)."""
    P = dict(width=60, height=20, resolution=0.1, noise_a0=0.01, ray_step=0.05)
    cells = {f"{i},10": (0.0, 1e-4) for i in range(60)}
    cells["35,10"] = (0.5, 1e-4)
    m = _cells_state(oracle_mod, P, cells)
    # sensor at x = 0.05 (ix 30), z = 0.2, point at x = 1.55 (ix 45)
    tr = m.update((cloud([[1.5, 0.0, 0.0]]), pose_t([0.05, 0.05, 0.2])), trace=True)
    assert tr.mark[10, 35] == 1 and tr.cleared[10, 35] == 1
    assert tr.mark.sum() == 1
    s = m.state()
    assert not np.isfinite(s["var"][10, 35]) and np.isnan(s["h"][10, 35])
    # same ray plus a point that lands in the obstacle cell this update: kept
    m = _cells_state(oracle_mod, P, cells)
    tr = m.update((cloud([[1.5, 0.0, 0.0], [0.5, 0.0, 0.3]]), pose_t([0.05, 0.05, 0.2])), trace=True)
    assert tr.mark[10, 35] == 1 and tr.cleared[10, 35] == 0
    assert np.isfinite(m.state()["var"][10, 35])


def test_min_age(oracle_mod):
    P = dict(width=60, height=20, resolution=0.1, noise_a0=0.01, ray_step=0.05, cleanup_min_age=3)
    cells = {"35,10": (0.5, 1e-4)}
    for t_last, cleared in ((4, 0), (3, 0), (2, 1)):  # t_now becomes 5: ages 1, 2, 3
        m = _cells_state(oracle_mod, P, cells, t_last=t_last, t_now=4)
        tr = m.update((cloud([[1.5, 0.0, 0.0]]), pose_t([0.05, 0.05, 0.2])), trace=True)
        assert tr.cleared[10, 35] == cleared, t_last


def test_normal_guard(oracle_mod):
    """|r . n| > alpha_n (Eq. 4): a horizontal ray grazing a cell whose normal
    is vertical is kept; the same ray against a wall facing it removes it."""
    P = dict(width=60, height=20, resolution=0.1, noise_a0=0.01, ray_step=0.05, cleanup_normal_thresh=0.5)
    for normal, cleared in (((0.0, 0.0, 1.0), 0), ((1.0, 0.0, 0.0), 1), ((np.nan, np.nan, np.nan), 0)):
        m = _cells_state(oracle_mod, P, {"35,10": (0.5, 1e-4)})
        H, W = m.shape
        nx = np.full((H, W), np.nan)
        ny, nz = nx.copy(), nx.copy()
        nx[10, 35], ny[10, 35], nz[10, 35] = normal
        m.set_state(nx=nx, ny=ny, nz=nz)
        tr = m.update((cloud([[1.5, 0.0, 0.0]]), pose_t([0.05, 0.05, 0.2])), trace=True)
        assert tr.cleared[10, 35] == cleared, normal


def test_threshold_uses_std_not_variance(oracle_mod):
    """Eq. 3 compares with h - sigma: with var = 0.04 (sigma = 0.2) a ray
    0.1 m below h does not penetrate, one 0.3 m below does."""
    P = dict(width=60, height=20, resolution=0.1, noise_a0=0.01, ray_step=0.05)
    for z_ray, marked in ((0.4, 0), (0.2, 1)):
        m = _cells_state(oracle_mod, P, {"35,10": (0.5, 0.04)})
        tr = m.update((cloud([[1.5, 0.0, 0.0]]), pose_t([0.05, 0.05, z_ray])), trace=True)
        assert tr.mark[10, 35] == marked


# ------------------------------------------------------------------- filters

def _field(oracle_mod, h, flags):
    H, W = h.shape
    m = make(oracle_mod, width=W, height=H, resolution=0.04, flags=flags)
    var = np.where(np.isfinite(h), 1e-4, np.inf)
    m.set_state(h=h, var=var, t_last=np.ones((H, W), np.int32), t_now=1)
    m.filters(flags)
    return m.state()


def test_normals_of_plane_exact(oracle_mod):
    a, b, c = 0.3, -0.2, 0.1
    r = 0.04
    X, Y = np.meshgrid(np.arange(8) * r, np.arange(8) * r)
    s = _field(oracle_mod, a * X + b * Y + c, oracle_mod.NORMALS)
    n = np.array([-a, -b, 1.0]) / math.sqrt(a * a + b * b + 1)
    for k, comp in enumerate(("nx", "ny", "nz")):
        assert np.allclose(s[comp], n[k], atol=1e-12, rtol=0)


def test_normals_degenerate(oracle_mod):
    h = np.full((6, 6), np.nan)
    h[2, 1:5] = 0.1          # one valid row: collinear -> NaN
    h[4, 4] = 0.0            # isolated valid cell
    s = _field(oracle_mod, h, oracle_mod.NORMALS)
    assert np.all(np.isnan(s["nz"]))
    h2 = np.full((6, 6), np.nan)
    h2[2, 2], h2[2, 3], h2[3, 2] = 0.0, 0.04, 0.0   # 3 non-collinear cells: z = x
    s2 = _field(oracle_mod, h2, oracle_mod.NORMALS)
    n = np.array([-1.0, 0.0, 1.0]) / math.sqrt(2)
    for k, comp in enumerate(("nx", "ny", "nz")):
        assert s2[comp][2, 2] == pytest.approx(n[k], abs=1e-12)


def test_smoothing(oracle_mod):
    s = _field(oracle_mod, np.full((7, 9), 0.37), oracle_mod.SMOOTH)
    assert np.allclose(s["smooth"], 0.37, atol=1e-15)
    h = np.arange(25, dtype=float).reshape(5, 5)
    s = _field(oracle_mod, h, oracle_mod.SMOOTH)
    assert s["smooth"][2, 2] == pytest.approx(12.0)
    assert s["smooth"][0, 0] == pytest.approx(np.mean([0, 1, 2, 5, 6, 7, 10, 11, 12]))
    h[1, 1] = np.nan
    s = _field(oracle_mod, h, oracle_mod.SMOOTH)
    assert np.isnan(s["smooth"][1, 1])
    assert s["smooth"][0, 0] == pytest.approx(np.mean([0, 1, 2, 5, 7, 10, 11, 12]))


def test_median_smoothing(oracle_mod):
    """5x5 lower median over the valid cells (Section II-I, median filter)."""
    s = _field(oracle_mod, np.full((7, 9), -0.21), oracle_mod.MEDIAN)
    assert np.all(s["smooth"] == -0.21)
    h = np.arange(25, dtype=float).reshape(5, 5)
    s = _field(oracle_mod, h, oracle_mod.MEDIAN)
    assert s["smooth"][2, 2] == 12.0                       # 25 values 0..24
    assert s["smooth"][0, 0] == 6.0                        # {0,1,2,5,6,7,10,11,12}
    h[1, 1] = np.nan
    s = _field(oracle_mod, h, oracle_mod.MEDIAN)
    assert np.isnan(s["smooth"][1, 1])
    assert s["smooth"][0, 0] == 5.0                        # 8 values: the lower of 5 and 7
    spike = np.full((9, 9), 0.1)
    spike[4, 4] = 3.0                                      # a lone spike is rejected
    assert _field(oracle_mod, spike, oracle_mod.MEDIAN)["smooth"][4, 4] == 0.1
    # every cell against numpy's lower median of the same window
    rng = np.random.default_rng(11)
    f = rng.normal(0.0, 0.3, (12, 13))
    f[rng.random(f.shape) < 0.2] = np.nan
    out = _field(oracle_mod, f, oracle_mod.MEDIAN)["smooth"]
    for iy in range(f.shape[0]):
        for ix in range(f.shape[1]):
            if np.isnan(f[iy, ix]):
                assert np.isnan(out[iy, ix])
                continue
            win = f[max(0, iy - 2):iy + 3, max(0, ix - 2):ix + 3]
            assert out[iy, ix] == np.quantile(win[~np.isnan(win)], 0.5, method="lower")


def test_gaussian_smoothing(oracle_mod):
    """5x5 Gaussian, sigma = 1 cell, weights renormalised over the valid cells
    (Section II-I, Gaussian filter)."""
    s = _field(oracle_mod, np.full((7, 9), 0.37), oracle_mod.GAUSS)
    assert np.allclose(s["smooth"], 0.37, atol=1e-15)
    # a symmetric kernel keeps a plane exactly where the whole window is valid
    a, b, c = 0.3, -0.2, 0.1
    X, Y = np.meshgrid(np.arange(9) * 0.04, np.arange(9) * 0.04)
    plane = a * X + b * Y + c
    s = _field(oracle_mod, plane, oracle_mod.GAUSS)
    assert np.allclose(s["smooth"][2:7, 2:7], plane[2:7, 2:7], atol=1e-12, rtol=0)
    # two valid cells: weights 1 and exp(-1/2)
    h = np.full((5, 5), np.nan)
    h[2, 2], h[2, 3] = 0.0, 1.0
    s = _field(oracle_mod, h, oracle_mod.GAUSS)
    w = math.exp(-0.5)
    assert s["smooth"][2, 2] == pytest.approx(w / (1.0 + w), abs=1e-15)
    # interior cells against scipy's separable Gaussian (same 5-tap kernel)
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(12)
    f = rng.normal(0.0, 0.3, (14, 15))
    ref = nd.gaussian_filter(f, sigma=1.0, truncate=2.0, mode="nearest")
    out = _field(oracle_mod, f, oracle_mod.GAUSS)["smooth"]
    assert np.allclose(out[2:-2, 2:-2], ref[2:-2, 2:-2], atol=1e-12, rtol=0)


def _upper_map(oracle_mod, **kw):
    P = dict(width=8, height=8, resolution=1.0, noise_a0=0.01, ray_step=1.0, flags=oracle_mod.UPPER)
    P.update(kw)
    return oracle_mod.OracleMap(oracle_mod.Params(**P))


def _pose(t):
    return np.array([1, 0, 0, t[0], 0, 1, 0, t[1], 0, 0, 1, t[2]], np.float32)


def test_upper_bound_layer_hand_worked(oracle_mod):
    """Section II-H: a ray through empty cells bounds their ground by the ray
    height.  Sensor at (-3.5, 0.5, 2), point at (1.5, 0.5, 1) on an 8 x 8 map of
    1 m cells centred on the origin, step 1 m: samples k = 1..5 at x = -3.5 + 5k/d,
    z = 2 - k/d, d = sqrt(26); sample 5 lies in the point's own cell."""
    m = _upper_map(oracle_mod)
    m.update((np.array([[5.0, 0.0, -1.0]], np.float32), _pose((-3.5, 0.5, 2.0))))
    up = m.state()["upper"]
    d = math.sqrt(26.0)
    want = np.full((8, 8), np.inf)
    for k in range(1, 5):
        want[4, k] = 2.0 - k / d
    assert np.allclose(up[np.isfinite(want)], want[np.isfinite(want)], atol=1e-6, rtol=0)
    assert np.array_equal(np.isfinite(up), np.isfinite(want))
    # a lower ray over the same cells lowers the bound (running minimum) ...
    m.update((np.array([[5.0, 0.0, -1.5]], np.float32), _pose((-3.5, 0.5, 1.8))))
    up2 = m.state()["upper"]
    assert np.all(up2[4, 1:5] <= up[4, 1:5]) and np.any(up2[4, 1:5] < up[4, 1:5])
    # ... and a cell that receives a point has no bound any more
    m.update((np.array([[0.0, 0.0, -1.5]], np.float32), _pose((-1.5, 0.5, 1.8))))
    assert np.isinf(m.state()["upper"][4, 2])
    assert np.isfinite(m.state()["var"][4, 2])


def test_upper_bound_skips_observed_cells_and_moves_with_the_map(oracle_mod):
    m = _upper_map(oracle_mod)
    h = np.full((8, 8), np.nan)
    var = np.full((8, 8), np.inf)
    h[4, 2], var[4, 2] = -5.0, 1e-4  # observed far below the ray: bounded by nothing
    m.set_state(h=h, var=var, t_last=np.zeros((8, 8), np.int32), t_now=1)
    m.update((np.array([[5.0, 0.0, -1.0]], np.float32), _pose((-3.5, 0.5, 2.0))))
    up = m.state()["upper"]
    assert np.isinf(up[4, 2]) and np.isfinite(up[4, 1]) and np.isfinite(up[4, 3])
    before = up.copy()
    m.shift(1, 0)
    after = m.state()["upper"]
    assert np.array_equal(after[:, :7], before[:, 1:]) and np.all(np.isinf(after[:, 7]))


def test_upper_bound_does_not_depend_on_point_order(oracle_mod):
    rng = np.random.default_rng(4)
    pts = np.column_stack([rng.uniform(-3.5, 3.5, 12), rng.uniform(-3.5, 3.5, 12),
                           rng.uniform(-2.5, -1.0, 12)]).astype(np.float32)  # few points: most cells stay empty
    outs = []
    for perm in (np.arange(12), rng.permutation(12)):
        m = _upper_map(oracle_mod, ray_step=0.3)
        m.update((pts[perm], _pose((0.2, -0.1, 1.5))))
        outs.append(m.state()["upper"])
    assert np.array_equal(outs[0], outs[1])
    assert np.isfinite(outs[0]).sum() > 5


def _drift_map(oracle_mod, h, nz, flat=0.9, var=1e-4):
    H, W = h.shape
    m = oracle_mod.OracleMap(oracle_mod.Params(width=W, height=H, resolution=1.0, noise_a0=0.01,
                                               drift_flatness=flat))
    v = np.where(np.isnan(h), np.inf, var)
    m.set_state(h=h, var=v, t_last=np.ones((H, W), np.int32), nx=np.zeros((H, W)), ny=np.zeros((H, W)),
                nz=nz, t_now=1)
    return m


def _cell_points(cells, z):
    """One point at the centre of each (ix, iy) cell of a 1 m grid centred on the
    origin (W = H = 6: centre at (ix - 2.5, iy - 2.5)), height z, identity pose."""
    pts = np.array([[ix - 2.5, iy - 2.5, zz] for (ix, iy), zz in zip(cells, z)], np.float32)
    return pts, np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)


def test_drift_compensation_closed_form(oracle_mod):
    """Section II-D: the mean error of points in flat cells holding an estimate
    is added to every estimate before the update."""
    h = np.zeros((6, 6))
    h[0, 5] = np.nan                                   # an empty cell
    nz = np.ones((6, 6))
    nz[3:, :] = 0.5                                    # steep rows: not flat at 0.9
    m = _drift_map(oracle_mod, h, nz)
    cells = [(1, 1), (2, 1), (4, 2), (0, 0)]           # flat cells: errors 0.05, 0.07, 0.09, 0.03
    steep = [(1, 4), (2, 5)]                           # ignored whatever their error
    pts, pose = _cell_points(cells + steep + [(5, 0)], [0.05, 0.07, 0.09, 0.03, -3.0, 4.0, 9.0])
    m.update((pts, pose))
    z = pts[:, 2].astype(np.float64)                   # the heights as the float32 points carry them
    mean = z[:4].mean()
    drift, n = m.last_drift()
    assert n == 4 and drift == pytest.approx(mean, abs=1e-15)
    s = m.state()
    assert s["h"][4, 4] == pytest.approx(mean, abs=1e-15)   # untouched cells move by the mean
    assert s["h"][3, 3] == pytest.approx(mean, abs=1e-15)
    assert s["h"][0, 5] == pytest.approx(z[6], abs=1e-15)   # the empty cell took its point as is
    # one point of the same variance as the drifted estimate: the two-point mean (Eq. 1)
    var_p = 0.01 ** 2
    assert s["h"][1, 1] == pytest.approx((var_p * mean + 1e-4 * z[0]) / (1e-4 + var_p), abs=1e-12)


def test_drift_compensation_off_and_empty(oracle_mod):
    h = np.zeros((6, 6))
    nz = np.ones((6, 6))
    for flat in (0.0, 0.9):
        m = _drift_map(oracle_mod, h, nz, flat=flat)
        pts, pose = _cell_points([(1, 1), (2, 2)], [0.2, 0.2])
        m.update((pts, pose))
        s = m.state()
        assert s["h"][4, 4] == (0.0 if flat == 0.0 else pytest.approx(float(np.float32(0.2)), abs=1e-15))
    # no flat cell with an estimate: nothing moves
    m = _drift_map(oracle_mod, h, np.full((6, 6), np.nan))
    pts, pose = _cell_points([(1, 1)], [0.3])
    m.update((pts, pose))
    assert m.last_drift() == (0.0, 0) and m.state()["h"][4, 4] == 0.0


def test_exclusion_area_ramp(oracle_mod):
    """Exclusion area (Section II-C, read as a ramp): above the sensor by more than
    b = 0.5 m within c = 1 m, then b + (r - c) tan(45 deg), at most d = 1.5 m."""
    m = oracle_mod.OracleMap(oracle_mod.Params(width=8, height=8, resolution=1.0, noise_a0=0.01, excl_b=0.5,
                                               excl_c=1.0, excl_theta=math.pi / 4, excl_d=1.5))
    # (horizontal distance along x, height above the sensor) -> kept?
    cases = [(0.5, 0.4, True), (0.5, 0.6, False), (2.0, 1.4, True), (2.0, 1.6, False),
             (3.0, 1.45, True), (3.0, 1.55, False), (1.0, 0.45, True), (1.0, 0.55, False)]
    pts = np.array([[r, 0.1, zr] for r, zr, _ in cases], np.float32)   # sensor frame = map frame - (0, 0, 1)
    pose = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 1.0], np.float32)
    tr = m.update((pts, pose), trace=True)
    kept = tr.status != oracle_mod.ST_RANGE
    assert list(kept) == [k for _, _, k in cases]


def test_overlap_clearance(oracle_mod):
    """Overlap clearance (Section II-F): estimates within 1.6 m of the sensor origin
    (0.2, 0.3) whose height is more than 0.8 m from its height 1.0 are cleared."""
    W = H = 8
    m = oracle_mod.OracleMap(oracle_mod.Params(width=W, height=H, resolution=1.0, overlap_radius=1.6,
                                               overlap_dz=0.8))
    h = np.full((H, W), 0.5)
    h[4, 4] = 2.5     # centre (0.5, 0.5): 0.36 m away, 1.5 m off -> cleared
    h[3, 5] = 1.75    # centre (1.5, -0.5): 1.53 m away, 0.75 m off -> kept
    h[3, 2] = 1.85    # centre (-1.5, -0.5): 1.86 m away -> kept (too far)
    h[5, 3] = 0.15    # centre (-0.5, 1.5): 1.38 m away, 0.85 m off -> cleared
    m.set_state(h=h, var=np.full((H, W), 1e-4), t_last=np.ones((H, W), np.int32), t_now=1)
    pose = np.array([1, 0, 0, 0.2, 0, 1, 0, 0.3, 0, 0, 1, 1.0], np.float32)
    m.update((np.zeros((0, 3), np.float32), pose))
    cleared = ~np.isfinite(m.state()["var"])
    want = np.zeros((H, W), bool)
    want[4, 4] = want[5, 3] = True
    assert np.array_equal(cleared, want)


def test_inpainting(oracle_mod):
    rng = np.random.default_rng(2)
    h = rng.uniform(0.0, 1.0, (16, 16))
    h[3, 3] = np.nan                                   # single-cell hole
    h[8:11, 8:11] = np.nan                             # 9-cell hole: too large
    h[3, 10:14] = np.nan
    h[4, 10:14] = np.nan                               # 8-cell hole: filled
    h[0, 6] = np.nan                                   # touches the border
    s = _field(oracle_mod, h, oracle_mod.INPAINT)
    ip = s["inpaint"]
    assert ip[3, 3] == pytest.approx(np.nanmin(h[2:5, 2:5]))
    assert np.all(np.isnan(ip[8:11, 8:11]))
    border = h[2:6, 9:15]
    assert np.allclose(ip[3:5, 10:14], np.nanmin(border))
    assert np.isnan(ip[0, 6])
    fin = np.isfinite(h)
    assert np.array_equal(ip[fin], h[fin])


def test_inpainting_component_shapes(oracle_mod):
    """Holes are 4-connected: lines and L shapes of 8 cells are filled, of 9
    are not, and cells touching only at a corner are separate holes."""
    rng = np.random.default_rng(3)
    h = rng.uniform(0.0, 1.0, (24, 24))
    h[2:10, 2] = np.nan                                # vertical line of 8: filled
    h[2:11, 6] = np.nan                                # vertical line of 9: too large
    h[14, 2:7] = np.nan
    h[15:18, 6] = np.nan                               # L of 8: filled
    h[14, 10:15] = np.nan
    h[15:19, 14] = np.nan                              # L of 9: too large
    h[20, 18] = np.nan
    h[21, 19] = np.nan                                 # diagonal neighbours: two holes of one cell
    s = _field(oracle_mod, h, oracle_mod.INPAINT)
    ip = s["inpaint"]
    assert np.allclose(ip[2:10, 2], np.nanmin(h[1:11, 1:4]))
    assert np.all(np.isnan(ip[2:11, 6]))
    L8 = np.isnan(h) & (np.arange(24)[:, None] >= 14) & (np.arange(24)[:, None] <= 17) & (np.arange(24)[None, :] <= 7)
    ring = np.zeros_like(L8)
    for y, x in zip(*np.nonzero(L8)):
        ring[y - 1:y + 2, x - 1:x + 2] = True
    assert np.allclose(ip[L8], np.nanmin(np.where(ring & np.isfinite(h), h, np.nan)))
    assert np.all(np.isnan(ip[14, 10:15])) and np.all(np.isnan(ip[15:19, 14]))
    assert ip[20, 18] == pytest.approx(np.nanmin(h[19:22, 17:20]))
    assert ip[21, 19] == pytest.approx(np.nanmin(h[20:23, 18:21]))


# --------------------------------------------------------------------- shift

def test_shift(oracle_mod):
    P = dict(width=30, height=20, resolution=0.05, noise_a0=0.01)
    pts, pose = synth.single_update(seed=8, n=3000, half=0.8)
    m = make(oracle_mod, **P)
    m.update((pts, pose))
    s0 = m.state()
    m.shift(3, -2)
    s1 = m.state()
    # new (ix, iy) holds old (ix + 3, iy - 2)
    assert np.array_equal(s1["h"][2:, :27], s0["h"][:18, 3:], equal_nan=True)
    assert np.all(~np.isfinite(s1["var"][:2, :])) and np.all(~np.isfinite(s1["var"][:, 27:]))
    m.shift(-3, 2)
    s2 = m.state()
    keep = np.zeros((20, 30), bool)
    keep[:18, 3:] = True
    assert np.array_equal(s2["h"][keep], s0["h"][keep], equal_nan=True)
    assert np.array_equal(s2["var"][keep], s0["var"][keep])
    assert m.shift_xy == (0, 0)
    m.shift(30, 0)
    assert np.all(~np.isfinite(m.state()["var"]))


def test_shift_moves_geometry(oracle_mod):
    """After shifting by (dx, dy) cells a point lands dx, dy cells lower in index."""
    P = dict(width=40, height=40, resolution=0.1, noise_a0=0.01)
    m = make(oracle_mod, **P)
    p = cloud([[0.33, 0.47, 0.0]])
    t1 = m.update((p, pose_t([0, 0, 0])), trace=True)
    m.shift(4, -7)
    t2 = m.update((p, pose_t([0, 0, 0])), trace=True)
    assert (t1.ix[0] - t2.ix[0], t1.iy[0] - t2.iy[0]) == (4, -7)
    assert m.origin() == pytest.approx((0.1 * (4 - 20), 0.1 * (-7 - 20)))


def test_marginal_flags(oracle_mod):
    """A point 1e-7 m from a cell edge is flagged bin-marginal; one in the middle is not."""
    m = make(oracle_mod, width=100, height=100, resolution=0.04, noise_a0=0.01)
    pts = cloud([[0.04 + 1e-7, 0.02, 0.0], [0.06, 0.02, 0.0]])
    tr = m.update((pts, pose_t([0, 0, 0])), trace=True, unit=oracle_mod.FP32_UNIT)
    assert tr.pflags[0] & oracle_mod.PF_BIN and not tr.pflags[1]
