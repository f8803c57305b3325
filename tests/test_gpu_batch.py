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

BASE = dict(resolution=0.04, noise_a0=0.005, noise_a2=0.002, mahalanobis_k=2.5, outlier_variance=1e-4,
            ray_step=0.04)
SHAPES = [(37, 51, 0), (100, 100, 1), (200, 64, 0), (120, 120, 1 | 2 | 4)]


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
    for j, (w, h, flags) in enumerate(SHAPES):
        m = em.Map(em.Params(width=w, height=h, flags=flags, **BASE))
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
    assert t["ray_group"] in (1, 2, 4, 8, 16, 32) and t["fuse_group"] in (4, 8, 16, 32) and t["big_thresh"] >= 1
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
