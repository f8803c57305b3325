"""em_update_noalloc -- the update for callers that cannot allocate device
memory at update time: a real-time loop that forbids allocation after
start-up, or a framework whose allocator already holds the device memory.  Its
scratch is a fixed static device array of the library, shared by every call.
These tests check, through the C ABI, that it produces what em_update produces
on consecutive calls -- two maps of different sizes alternating through the
same scratch, several clouds, a shifted map centre and the Eq. 4 normal guard
-- and that it refuses sizes beyond its limits.

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


def _compare(ref, h, var, t_last, t):
    s = ref.state()
    gh, gv, gt = h.cpu().numpy(), var.cpu().numpy(), t_last.cpu().numpy()
    rv, nv = np.isfinite(s["var"]), np.isfinite(gv)
    assert np.array_equal(rv, nv), t
    assert np.all(np.abs(gh[rv].astype(np.float64) - s["h"][rv]) <= 1e-5), t
    assert np.all(np.abs(gv[rv].astype(np.float64) / s["var"][rv] - 1.0) <= 1e-4), t
    assert np.array_equal(gt[rv], s["t_last"][rv]), t
    return int(rv.sum())


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
        assert _compare(ref, h, var, t_last, t) > 5000
    ref.close()


def test_noalloc_alternating_maps_share_the_scratch(em):
    """A 256 x 256 map (the largest the scratch holds) and a 100 x 100 map take
    turns, each update with two clouds, a shifted map centre and the normal
    guard reading the caller's normals; every result equals em_update's."""
    rng = np.random.default_rng(44)
    cases = []
    for side, shift, seed in ((256, (9, -14), 45), (100, (-3, 5), 46)):
        Pm = dict(P, width=side, height=side, cleanup_normal_thresh=0.2)
        prior = synth.random_prior(seed=seed, width=side, height=side, t_now=4)
        ref = em.Map(em.Params(**Pm))
        ref.shift(*shift)
        ref.set_state(h=prior["h"], var=prior["var"], t_last=prior["t_last"].astype(np.float32), nx=prior["nx"],
                      ny=prior["ny"], nz=prior["nz"], t_now=prior["t_now"])
        lay = {k: torch.from_numpy(np.ascontiguousarray(prior[k])).cuda() for k in ("h", "var", "nx", "ny", "nz")}
        lay["t_last"] = torch.from_numpy(np.ascontiguousarray(prior["t_last"].astype(np.int32))).cuda()
        lay["var"][~torch.isfinite(lay["var"])] = float("inf")
        lay["h"][~torch.isfinite(lay["var"])] = float("nan")
        cases.append((Pm, shift, ref, lay))
    half = 0.038 * 256 / 2
    cleared = 0
    for t in range(5, 9):
        for Pm, shift, ref, lay in cases:
            r = Pm["resolution"]
            c = np.array([shift[0] * r, shift[1] * r])
            clouds = []
            for k in range(2):
                pts, pose = synth.single_update(seed=int(rng.integers(1 << 30)), n=15000,
                                                half=half * Pm["width"] / 256)
                pose = pose.copy()
                pose[3] += c[0]
                pose[7] += c[1]
                clouds.append((torch.from_numpy(pts).cuda(), pose))
            ref.update_multi(clouds)
            em.update_noalloc(em.Params(**Pm), lay["h"], lay["var"], lay["t_last"], clouds, t_now=t, shift=shift,
                              normals=(lay["nx"], lay["ny"], lay["nz"]))
            torch.cuda.synchronize()
            assert _compare(ref, lay["h"], lay["var"], lay["t_last"], (Pm["width"], t)) > 2000
    for _, _, ref, _ in cases:
        cleared += ref.stats()["cells_cleared"]
        ref.close()
    assert cleared > 0  # the ray march removed cells, so the guard's normals were read


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
