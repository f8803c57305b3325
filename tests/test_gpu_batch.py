"""Batched form: several uneven maps updated by one kernel sequence (and by one
CUDA graph launch) give exactly the state that separate em_update calls give
(bit for bit: same kernels, order-independent exact sums), the autotuner does
not touch the maps, and capacities are enforced."""
import numpy as np
import pytest

import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BASE = dict(resolution=0.04, noise_a0=0.005, noise_a2=0.002, mahalanobis_k=2.5, outlier_variance=1e-4)
# (width, height, flags, ray step): one batch mixes ray steps of one, two and
# two and a half cells
SHAPES = [(37, 51, 0, 0.04), (100, 100, 1, 0.1), (200, 64, 0, 0.04), (120, 120, 1 | 2 | 4, 0.08)]


@pytest.fixture(scope="module")
def em():
    from paper_2204_12876_gb300 import build
    build.build()
    from paper_2204_12876_gb300 import em as mod
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_maps(em, seed):
    maps, pairs = [], []
    for j, (w, h, flags, step) in enumerate(SHAPES):
        m = em.Map(em.Params(width=w, height=h, flags=flags, ray_step=step, **BASE))
        prior = synth.random_prior(seed=seed + j, width=w, height=h, t_now=5)
        parity.prior_to_gpu(m, prior)
        m.shift(j, -j)
        maps.append(m)
        half = 0.5 * max(w, h) * 0.04
        for c in range(1 + (j == 1)):  # the second map gets two clouds
            pts, pose = synth.scattered_cloud(seed * 10 + j * 3 + c, 8000 + 3000 * j, half, nan_frac=0.03)
            pairs.append((m, dev(pts), pose))
    return maps, pairs


def states(maps):
    return [m.state() for m in maps]


def assert_same(sa, sb):
    for a, b in zip(sa, sb):
        for k in ("h", "var", "t_last", "nx", "ny", "nz", "smooth", "inpaint"):
            assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_separate_updates(em, graph):
    ref_maps, ref_pairs = make_maps(em, seed=100)
    bat_maps, bat_pairs = make_maps(em, seed=100)
    batch = em.Batch(max_maps=8, max_clouds=16, max_points=200000, max_cells=200 * 200, graph=graph)
    for rnd in range(2):  # the second round replays the captured graph
        for m in ref_maps:
            mine = [(p, q) for mm, p, q in ref_pairs if mm is m]
            m.update_multi(mine)
        batch.update(bat_pairs)
        torch.cuda.synchronize()
        assert_same(states(ref_maps), states(bat_maps))
        for a, b in zip(ref_maps, bat_maps):
            sa, sb = a.stats(), b.stats()
            for k in ("updates", "points_in", "points_valid", "points_in_map", "points_accepted",
                      "points_rejected", "cells_updated", "cells_cleared", "ray_samples"):
                assert sa[k] == sb[k], (k, rnd)
    batch.close()


def test_autotune_keeps_maps_and_picks_valid_shapes(em):
    maps, pairs = make_maps(em, seed=200)
    before = states(maps)
    info = [m.info()["t_now"] for m in maps]
    batch = em.Batch(max_maps=8, max_clouds=16, max_points=200000, max_cells=200 * 200, graph=True)
    t = batch.autotune(pairs, reps=2)
    assert t["ray_group"] in (1, 2, 4, 8, 16, 32) and t["fuse_chunk"] in (64, 128, 256, 512, 1024)
    assert 32 <= t["big_thresh"] <= 1023
    assert batch.tuning() == t
    torch.cuda.synchronize()
    assert_same(before, states(maps))
    assert [m.info()["t_now"] for m in maps] == info
    batch.update(pairs)
    assert [m.info()["t_now"] for m in maps] == [x + 1 for x in info]
    batch.close()


def test_batch_capacities(em):
    maps, pairs = make_maps(em, seed=300)
    small = em.Batch(max_maps=2, max_clouds=16, max_points=200000, max_cells=200 * 200, graph=False)
    with pytest.raises(em.EMError) as e:
        small.update(pairs)
    assert e.value.code == em.EM_ERR_CAPACITY
    few_pts = em.Batch(max_maps=8, max_clouds=16, max_points=1000, max_cells=200 * 200, graph=False)
    with pytest.raises(em.EMError) as e:
        few_pts.update(pairs)
    assert e.value.code == em.EM_ERR_CAPACITY
    tiny_cells = em.Batch(max_maps=8, max_clouds=16, max_points=200000, max_cells=100, graph=False)
    with pytest.raises(em.EMError) as e:
        tiny_cells.update(pairs)
    assert e.value.code == em.EM_ERR_CAPACITY
    # a refused batch leaves the maps untouched
    assert [m.info()["t_now"] for m in maps] == [5] * len(maps)


def dense_cloud(seed, centres, per_cell, half):
    """Clusters of per_cell points inside single cells (more than the large-cell
    threshold) plus a uniform sprinkle; sensor 0.5 m above the map origin."""
    rng = np.random.default_rng(seed)
    pts = []
    for cx, cy in centres:
        xy = np.array([cx, cy]) + rng.uniform(0.005, 0.035, (per_cell, 2))
        z = 0.1 + rng.normal(0.0, 0.01, per_cell)
        pts.append(np.column_stack([xy, z]))
    n = 4000
    pts.append(np.column_stack([rng.uniform(-half, half, (n, 2)), rng.normal(0.0, 0.02, n)]))
    pw = np.concatenate(pts).astype(np.float32)
    rng.shuffle(pw)
    t = np.array([0.0, 0.0, 0.5], np.float32)
    return (pw - t).astype(np.float32), synth.pose_matrix(np.eye(3), t)


@pytest.mark.parametrize("graph", [False, True])
def test_launch_shapes_give_identical_maps(em, graph):
    """Every tuning (records per warp chunk, large-cell threshold, lanes per ray)
    gives the same maps bit for bit, including cells with thousands of records."""
    results = []
    shapes = [dict(ray_group=4, fuse_chunk=256, big_thresh=256), dict(ray_group=1, fuse_chunk=64, big_thresh=32),
              dict(ray_group=32, fuse_chunk=1024, big_thresh=1023)]
    for tune in shapes:
        maps, pairs = make_maps(em, seed=300)
        half = 0.5 * 100 * 0.04
        pts, pose = dense_cloud(7, [(-0.52, 0.36), (0.8, -1.2), (0.0, 0.0), (1.6, 1.6)], 3000, half)
        pairs.append((maps[1], dev(pts), pose))
        batch = em.Batch(max_maps=8, max_clouds=16, max_points=400000, max_cells=200 * 200, graph=graph)
        batch.set_tuning(**tune)
        for _ in range(2):
            batch.update(pairs)
        torch.cuda.synchronize()
        results.append((states(maps), [m.stats() for m in maps]))
        batch.close()
    for st, stats in results[1:]:
        assert_same(results[0][0], st)
        for a, b in zip(results[0][1], stats):
            for k in ("points_accepted", "points_rejected", "cells_updated", "cells_cleared", "ray_samples"):
                assert a[k] == b[k], k


@pytest.mark.parametrize("persistent", [False, True])
def test_batched_config_sizes_vs_oracle(em, persistent):
    """One graph-launched batch over 8 maps drawn from the 64-map configuration
    (sides 100 to 500 cells, 10k to 400k points in random order, the ray march
    on, one map with normals, smoothing and in-painting), each over a seeded
    prior: every map agrees with the FP64 oracle fed the same prior and cloud
    (cell state, removed cells and filters; Section II-C, II-E)."""
    import oracle
    base = dict(BASE, var_min=1e-8, ray_step=0.04)
    rng = np.random.default_rng(61)
    specs = [(500, 400000, 0), (100, 10000, 0), (317, 150000, 1 | 2 | 4), (230, 400000, 0), (480, 60000, 0),
             (150, 250000, 0), (400, 320000, 0), (260, 90000, 0)]
    maps, pairs, oms, priors, clouds = [], [], [], [], []
    for j, (side, n, flags) in enumerate(specs):
        P = dict(base, width=side, height=side, flags=flags)
        prior = synth.random_prior(seed=600 + j, width=side, height=side, t_now=5)
        half = 0.5 * side * 0.04 * 1.05
        pts, pose = synth.scattered_cloud(6000 + j, n, half, yaw=float(rng.uniform(0, 6.28)))
        m = em.Map(em.Params(**P))
        parity.prior_to_gpu(m, prior)
        om = oracle.OracleMap(parity.oracle_params(P))
        parity.prior_to_oracle(om, prior)
        maps.append(m)
        oms.append(om)
        priors.append(prior)
        clouds.append((pts, pose))
        pairs.append((m, dev(pts), pose))
    batch = em.Batch(max_maps=8, max_clouds=8, max_points=sum(len(p) for p, _ in clouds), max_cells=500 * 500,
                     graph=True, persistent=persistent)
    batch.update(pairs)
    torch.cuda.synchronize()
    for j, (m, om) in enumerate(zip(maps, oms)):
        prior_valid = np.isfinite(om.state()["var"])
        tr = om.update(clouds[j], trace=True, unit=oracle.FP32_UNIT, abs_band=parity.ABS_BAND)
        stencils = ("nx", "ny", "nz", "smooth", "inpaint") if specs[j][2] else ()
        cmp = parity.compare_update(tr, om.state(), m.state(), None, prior_valid=prior_valid, check_stencils=stencils)
        assert cmp.notes["cells_compared"] > 0.9 * cmp.notes["cells_valid"], j
        st = m.stats()
        assert abs(st["points_rejected"] - tr.counts["rejected"]) <= 0.001 * tr.counts["in_map"] + 10, j
    for m in maps:
        m.close()
    batch.close()


def test_split_tiles_and_slot_overflow_give_identical_maps(em):
    """Tiles with many records are cut into pieces that several blocks fuse at
    once.  No tile cut, some tiles cut, and more tiles worth cutting than there
    are accumulator slots (the rest fused whole) all give the same map bit for
    bit, with the wall rule on (its per-cell counts span the whole tile, not
    one piece) and a few cells holding thousands of records."""
    side = 1000
    P = dict(BASE, width=side, height=side, wall_num_thresh=2)
    prior = synth.random_prior(seed=71, width=side, height=side, t_now=5, with_normals=False)
    half = 0.5 * side * 0.04
    clouds = [synth.scattered_cloud(72, 1_500_000, half, nan_frac=0.01),
              dense_cloud(73, [(0.3, -0.2), (0.34, -0.2), (-7.0, 5.0)], 3000, half)]
    dclouds = [(dev(p), q) for p, q in clouds]
    # tiles hold about 1,536 records: 16 x 1023 cuts none, 16 x 100 cuts a few
    # tens, 16 x 32 would cut all 977 (more than the 512 slots)
    shapes = [dict(ray_group=4, fuse_chunk=256, big_thresh=1023), dict(ray_group=4, fuse_chunk=256, big_thresh=100),
              dict(ray_group=4, fuse_chunk=512, big_thresh=32), dict(ray_group=4, fuse_chunk=256, big_thresh=32)]
    results = []
    for tune in shapes:
        m = em.Map(em.Params(**P))
        parity.prior_to_gpu(m, prior)
        batch = em.Batch(max_maps=1, max_clouds=2, max_points=1_600_000, max_cells=side * side, graph=False)
        batch.set_tuning(**tune)
        for _ in range(2):
            batch.update([(m, p, q) for p, q in dclouds])
        torch.cuda.synchronize()
        results.append((m.state(), m.stats()))
        batch.close()
        m.close()
    st0, stats0 = results[0]
    assert stats0["points_wall"] > 0 and stats0["points_rejected"] > 0
    for st, stats in results[1:]:
        assert_same([st0], [st])
        for k in ("points_accepted", "points_rejected", "points_wall", "cells_updated"):
            assert stats0[k] == stats[k], k


def _persistent_case(em, seed, extra_flags=0, overlap=False):
    maps, pairs = make_maps(em, seed=seed)
    half = 0.5 * 100 * 0.04
    pts, pose = dense_cloud(seed + 1, [(-0.52, 0.36), (0.8, -1.2), (0.0, 0.0)], 3000, half)
    pairs.append((maps[1], dev(pts), pose))
    if extra_flags or overlap:  # one more map: the upper-bound layer and / or the overlap clearance
        P = dict(BASE, width=90, height=70, ray_step=0.04, flags=extra_flags,
                 overlap_radius=0.6 if overlap else 0.0, overlap_dz=0.3 if overlap else 0.0)
        m = em.Map(em.Params(**P))
        parity.prior_to_gpu(m, synth.random_prior(seed=seed + 7, width=90, height=70, t_now=5))
        maps.append(m)
        c, q = synth.scattered_cloud(seed + 8, 20000, 0.5 * 90 * 0.04, nan_frac=0.02)
        pairs.append((m, dev(c), q))
    return maps, pairs


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("extra", ["plain", "upper_overlap"])
def test_persistent_launch_equals_sequence(em, graph, extra):
    """The batched update in one persistent launch (grid barriers between the
    passes) gives the maps and statistics of the kernel sequence bit for bit:
    uneven maps, two clouds for one map, cells with thousands of records, ray
    steps of one to two and a half cells, and the upper-bound layer and the
    overlap clearance."""
    flags = 32 if extra == "upper_overlap" else 0
    results = []
    for persistent in (False, True):
        maps, pairs = _persistent_case(em, 500, extra_flags=flags, overlap=extra == "upper_overlap")
        batch = em.Batch(max_maps=8, max_clouds=16, max_points=400000, max_cells=200 * 200, graph=graph,
                         persistent=persistent)
        for _ in range(3):  # the graph replays from the second round
            batch.update(pairs)
        torch.cuda.synchronize()
        for m in maps:
            m.sync()
        results.append((states(maps), [m.stats() for m in maps], [m.state().get("upper") for m in maps]))
        batch.close()
        for m in maps:
            m.close()
    (sa, ta, ua), (sb, tb, ub) = results
    assert_same(sa, sb)
    for a, b in zip(ta, tb):
        for k in ("updates", "points_valid", "points_in_map", "points_accepted", "points_rejected", "points_wall",
                  "cells_updated", "cells_cleared", "ray_samples"):
            assert a[k] == b[k], k
    for a, b in zip(ua, ub):
        if a is not None or b is not None:
            assert np.array_equal(a, b, equal_nan=True)


def test_wait_selftest_times_out_and_device_stays_usable(em):
    """The persistent launch's bounded wait, on a word that nothing sets, runs
    out with EM_ERR_TIMEOUT after its budget; the context stays usable (a
    persistent batch update afterwards gives the sequence's result)."""
    import time
    t0 = time.perf_counter()
    assert em.wait_selftest(0, 20000) == em.EM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    out = []
    for persistent in (False, True):
        maps, pairs = make_maps(em, seed=900)
        batch = em.Batch(max_maps=8, max_clouds=16, max_points=200000, max_cells=200 * 200, graph=False,
                         persistent=persistent)
        batch.update(pairs)
        for m in maps:
            m.sync()
        out.append(states(maps))
        batch.close()
    assert_same(out[0], out[1])
