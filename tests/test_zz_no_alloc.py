"""em_update_noalloc -- the update for callers that cannot allocate device
memory at update time (a real-time loop that forbids allocation after start-up,
a framework whose allocator already holds the device memory, code preparing
work during stream capture).  Its scratch is a fixed static device array of the
library; these tests check, through the C ABI, that it produces what em_update
produces on two calls in a row, and that it refuses sizes beyond its limits.

This file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = dict(width=100, height=100, resolution=0.04, noise_a0=0.005, noise_a2=0.002, mahalanobis_k=2.5,
         outlier_variance=1e-4, ray_step=0.04)


@pytest.fixture(scope="module")
def em():
    from paper_2204_12876_gb300 import build
    build.build()
    from paper_2204_12876_gb300 import em as mod
    return mod


def test_noalloc_matches_em_update_on_two_calls(em):
    ref = em.Map(em.Params(**P))
    H, W = P["height"], P["width"]
    h = torch.full((H, W), float("nan"), device="cuda")
    var = torch.full((H, W), float("inf"), device="cuda")
    t_last = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    calls = [synth.single_update(seed=41, n=20000), synth.single_update(seed=42, n=25000)]
    for t, (pts, pose) in enumerate(calls, start=1):
        d = torch.from_numpy(pts).cuda()
        ref.update(d, pose)
        em.update_noalloc(em.Params(**P), h, var, t_last, [(d, pose)], t_now=t)
        torch.cuda.synchronize()
        s = ref.state()
        gh, gv, gt = h.cpu().numpy(), var.cpu().numpy(), t_last.cpu().numpy()
        rv, nv = np.isfinite(s["var"]), np.isfinite(gv)
        assert np.array_equal(rv, nv), t
        assert rv.sum() > 5000
        assert np.all(np.abs(gh[rv].astype(np.float64) - s["h"][rv]) <= 1e-5), t
        assert np.all(np.abs(gv[rv].astype(np.float64) / s["var"][rv] - 1.0) <= 1e-4), t
        assert np.array_equal(gt[rv], s["t_last"][rv]), t
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_limits(em):
    pts, pose = synth.single_update(seed=43, n=1000)
    d = torch.from_numpy(pts).cuda()
    big = dict(P, width=300, height=300)  # 90,000 cells > 65,536
    h = torch.zeros((300, 300), device="cuda")
    v = torch.zeros((300, 300), device="cuda")
    t = torch.zeros((300, 300), dtype=torch.int32, device="cuda")
    with pytest.raises(em.EMError) as e:
        em.update_noalloc(em.Params(**big), h, v, t, [(d, pose)], t_now=1)
    assert e.value.code == em.EM_ERR_CAPACITY
    many = torch.zeros((em.NOALLOC_MAX_POINTS + 1, 3), device="cuda")
    h = torch.zeros((100, 100), device="cuda")
    v = torch.zeros((100, 100), device="cuda")
    t = torch.zeros((100, 100), dtype=torch.int32, device="cuda")
    with pytest.raises(em.EMError) as e:
        em.update_noalloc(em.Params(**P), h, v, t, [(many, pose)], t_now=1)
    assert e.value.code == em.EM_ERR_CAPACITY
