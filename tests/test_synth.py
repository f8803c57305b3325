"""The seeded input generators: the same seed gives the same inputs (every
parity case and bench line is reproducible), and the shapes and value ranges
are those the workloads state."""
import numpy as np

import synth


def test_same_seed_same_clouds():
    a, pa = synth.scattered_cloud(11, 5000, 2.0, nan_frac=0.05)
    b, pb = synth.scattered_cloud(11, 5000, 2.0, nan_frac=0.05)
    c, _ = synth.scattered_cloud(12, 5000, 2.0, nan_frac=0.05)
    assert np.array_equal(a, b, equal_nan=True) and np.array_equal(pa, pb)
    assert not np.array_equal(a, c, equal_nan=True)
    assert a.dtype == np.float32 and a.shape == (5000, 3) and pa.shape == (12,)
    frac = np.isnan(a).any(axis=1).mean()
    assert 0.03 < frac < 0.07


def test_scattered_cloud_pose_maps_back_to_the_square():
    pts, pose = synth.scattered_cloud(3, 4000, 1.5, yaw=0.7)
    P = pose.reshape(3, 4).astype(np.float64)
    world = pts.astype(np.float64) @ P[:, :3].T + P[:, 3]
    assert np.all(np.abs(world[:, :2]) <= 1.5 + 1e-5)
    assert np.allclose(P[:, :3] @ P[:, :3].T, np.eye(3), atol=1e-6)  # a rotation


def test_prior_layers():
    pr = synth.random_prior(seed=5, width=40, height=30, t_now=7, invalid_frac=0.2)
    assert pr["h"].shape == (30, 40) and pr["var"].dtype == np.float32
    empty = ~np.isfinite(pr["var"])
    assert np.array_equal(empty, np.isnan(pr["h"]))
    assert 0.1 < empty.mean() < 0.3
    ok = pr["var"][~empty]
    assert ok.min() >= 1e-5 * 0.999 and ok.max() <= 1e-3 * 1.001
    assert pr["t_last"].min() >= 0 and pr["t_last"].max() < 7
    again = synth.random_prior(seed=5, width=40, height=30, t_now=7, invalid_frac=0.2)
    assert all(np.array_equal(pr[k], again[k], equal_nan=True) for k in ("h", "var", "t_last", "nx"))


def test_batch_clouds_sizes():
    work = synth.batch_clouds(seed=4, maps=6, n_min=1000, n_max=3000)
    assert len(work) == 6
    for w in work:
        assert 100 <= w["side"] <= 500
        pts, pose = w["clouds"][0]
        assert 1000 <= len(pts) <= 3000 and pts.shape[1] == 3
