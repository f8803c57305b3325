"""Served form: requests from many robots through the continuous-batching
server give, for every map, exactly the state that the same requests give when
applied alone with em_update (bit for bit); admission follows the memory
budget; oversize requests are rejected; cancel / timeout / an injected
allocation failure are handled on the host (no GPU fault involved)."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BASE = dict(resolution=0.04, noise_a0=0.005, noise_a2=0.002, mahalanobis_k=2.5, outlier_variance=1e-4,
            ray_step=0.04)
SIDES = [60, 90, 120, 75, 100, 140]


@pytest.fixture(scope="module")
def em():
    from paper_2204_12876_gb300 import build
    build.build()
    from paper_2204_12876_gb300 import em as mod
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def workload(n_req=40, seed=5):
    """A seeded interleaving of requests over the maps: (map index, cloud)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        j = int(rng.integers(0, len(SIDES)))
        half = 0.5 * SIDES[j] * 0.04
        pts, pose = synth.scattered_cloud(seed * 1000 + k, int(rng.integers(2000, 20000)), half, nan_frac=0.02)
        reqs.append((j, dev(pts), pose))
    return reqs


@pytest.mark.parametrize("mode,streams", [(0, 1), (0, 3), (1, 1)])
def test_served_equals_alone(em, mode, streams):
    reqs = workload()
    # alone: each map's requests applied in order with em_update
    alone = [em.Map(em.Params(width=s, height=s, **BASE)) for s in SIDES]
    for j, p, q in reqs:
        alone[j].update(p, q)
    torch.cuda.synchronize()
    srv = em.Server(budget_bytes=1 << 30, n_streams=streams, max_batch_maps=4, max_batch_points=100_000, mode=mode)
    ids = [srv.add_map(em.Params(width=s, height=s, **BASE)) for s in SIDES]
    tickets = [srv.submit(ids[j], [(p, q)]) for j, p, q in reqs]
    results = [srv.wait(t) for t in tickets]
    assert all(r["status"] == 0 for r in results)
    assert all(r["t_submit_ns"] <= r["t_start_ns"] <= r["t_done_ns"] for r in results)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["slots_in_use"] == 0
    if mode == 0:
        assert st["max_batch_size"] > 1  # requests were batched
    for j, m in enumerate(alone):
        a = m.state()
        b = srv.map(ids[j]).state()
        for k in ("h", "var", "t_last"):
            assert np.array_equal(a[k], b[k], equal_nan=True), (j, k)
    srv.close()


def test_map_order_kept_when_a_batch_is_full(em):
    """A map's earlier request that does not fit the batch holds back its later
    ones: the map still receives its updates in arrival order."""
    half = 0.5 * 120 * 0.04
    clouds = [synth.scattered_cloud(900 + k, n, half) for k, n in enumerate((1_000, 50_000, 60_000, 1_000))]
    alone_a = em.Map(em.Params(width=120, height=120, **BASE))
    for pts, pose in clouds[2:]:
        alone_a.update(dev(pts), pose)
    torch.cuda.synchronize()
    srv = em.Server(budget_bytes=1 << 30, n_streams=1, max_batch_maps=4, max_batch_points=100_000)
    ia, ib, ic = (srv.add_map(em.Params(width=120, height=120, **BASE)) for _ in range(3))
    # a first request on map C holds the only stream (its points wait on a timed
    # kernel) while B (50k), A (60k) and A (1k) queue up behind it; the next batch
    # takes B, cannot fit A's 60k next to it, and must not take A's 1k either
    gate = torch.cuda.Event()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        torch.cuda._sleep(20_000_000)
        gate.record(side)
    tickets = [srv.submit(ic, [(dev(clouds[0][0]), clouds[0][1])], ready=gate)]
    tickets += [srv.submit(ib, [(dev(clouds[1][0]), clouds[1][1])])]
    tickets += [srv.submit(ia, [(dev(p), q)]) for p, q in clouds[2:]]
    for t in tickets:
        assert srv.wait(t)["status"] == 0
    a, b = alone_a.state(), srv.map(ia).state()
    for k in ("h", "var", "t_last"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    srv.close()


def test_admission_by_budget(em):
    reqs = workload(n_req=30, seed=6)
    probe = em.Server(budget_bytes=1 << 30, n_streams=2, max_batch_maps=4, max_batch_points=50_000)
    for s in SIDES:
        probe.add_map(em.Params(width=s, height=s, **BASE))
    base = probe.stats()["bytes_in_use"]  # batch workspaces + resident maps
    probe.close()
    budget = base + 40_000 * em.SERVE_RECORD_BYTES  # room for ~40k records in flight
    srv = em.Server(budget_bytes=budget, n_streams=2, max_batch_maps=4, max_batch_points=50_000)
    ids = [srv.add_map(em.Params(width=s, height=s, **BASE)) for s in SIDES]
    tickets = [srv.submit(ids[j], [(p, q)]) for j, p, q in reqs]
    for t in tickets:
        assert srv.wait(t)["status"] == 0
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    assert st["completed"] == len(reqs)
    # a request larger than the whole budget can never run: rejected at once
    big = dev(np.zeros((45_000, 3), np.float32))
    with pytest.raises(em.EMError) as e:
        srv.submit(ids[0], [(big, np.eye(3, 4).reshape(12))])
    assert e.value.code == em.EM_ERR_REJECTED
    # a map that does not fit the budget is refused
    with pytest.raises(em.EMError) as e:
        srv.add_map(em.Params(width=500, height=500, **BASE))
    assert e.value.code in (em.EM_ERR_REJECTED, em.EM_ERR_INVALID_ARG)
    srv.close()


def test_cancel_timeout_and_injected_allocation_failure(em):
    srv = em.Server(budget_bytes=1 << 30, n_streams=1, mode=1, fail_alloc_at=2)
    a = srv.add_map(em.Params(width=100, height=100, **BASE))
    with pytest.raises(em.EMError) as e:  # the injected failure hits the second map
        srv.add_map(em.Params(width=100, height=100, **BASE))
    assert e.value.code == em.EM_ERR_OOM
    b = srv.add_map(em.Params(width=100, height=100, **BASE))
    pts = dev(synth.scattered_cloud(1, 200_000, 2.0)[0])
    pose = np.eye(3, 4).reshape(12)
    tickets = [srv.submit(a if i % 2 else b, [(pts, pose)]) for i in range(60)]
    last = tickets[-1]
    with pytest.raises(em.EMError) as e:
        srv.wait(last, timeout_us=0)
    assert e.value.code == em.EM_ERR_TIMEOUT
    try:
        srv.cancel(last)
        r = srv.wait(last)
        assert r["status"] == em.EM_ERR_TIMEOUT and srv.stats()["cancelled"] == 1
    except em.EMError as err:  # it had already been launched
        assert err.code == em.EM_ERR_BUSY
    srv.drain()
    st = srv.stats()
    assert st["completed"] + st["cancelled"] == 60
    srv.close()


def test_submit_many_reads_back_each_update(em):
    """One call queues requests for several maps (map 0 twice); each request's
    read-back (device or pinned host buffer) holds exactly the map state its own
    update produced -- the same as em_update alone followed by em_get_layers."""
    reqs = [(j, *synth.scattered_cloud(300 + k, 5000 + 2000 * k, 0.5 * SIDES[j] * 0.04, nan_frac=0.02))
            for k, j in enumerate([0, 1, 2, 0, 3])]
    mask = em.LAYER_ELEVATION | em.LAYER_VARIANCE
    # alone: the reference read-back after each request
    alone = [em.Map(em.Params(width=s, height=s, **BASE)) for s in SIDES]
    expect = []
    for j, pts, pose in reqs:
        alone[j].update(dev(pts), pose)
        out = torch.empty(2 * SIDES[j] ** 2, dtype=torch.float32, device="cuda")
        alone[j].get_layers(mask, out=out)
        expect.append(out.cpu().numpy())
    torch.cuda.synchronize()
    for mode in (0, 1):
        srv = em.Server(budget_bytes=1 << 30, n_streams=2, max_batch_maps=4, max_batch_points=100_000, mode=mode)
        ids = [srv.add_map(em.Params(width=s, height=s, **BASE)) for s in SIDES]
        outs = []
        for q, (j, _, _) in enumerate(reqs):
            n = 2 * SIDES[j] ** 2
            outs.append(torch.full((n,), -7.0, dtype=torch.float32, device="cuda") if q % 2 else
                        torch.full((n,), -7.0, dtype=torch.float32).pin_memory())
        tickets = srv.submit_many([(ids[j], [(dev(pts), pose)], (mask, outs[q]))
                                   for q, (j, pts, pose) in enumerate(reqs)])
        res = srv.wait_many(tickets, results=True)
        assert [r["status"] for r in res] == [0] * len(reqs)
        assert [r["map_id"] for r in res] == [ids[j] for j, _, _ in reqs]
        for q in range(len(reqs)):
            got = outs[q].cpu().numpy() if outs[q].is_cuda else outs[q].numpy()
            assert np.array_equal(got, expect[q], equal_nan=True), (mode, q)
        if mode == 0:
            assert srv.stats()["max_batch_size"] > 1
        srv.close()


def test_submit_many_all_or_nothing(em):
    srv = em.Server(budget_bytes=1 << 30, n_streams=1, max_batch_maps=4, max_batch_points=100_000)
    a = srv.add_map(em.Params(width=60, height=60, **BASE))
    pts, pose = synth.scattered_cloud(7, 1000, 1.0)
    p = dev(pts)
    with pytest.raises(em.EMError) as e:  # the second request names no map: nothing is queued
        srv.submit_many([(a, [(p, pose)], None), (a + 5, [(p, pose)], None)])
    assert e.value.code == em.EM_ERR_INVALID_ARG
    assert srv.stats()["submitted"] == 0
    with pytest.raises(em.EMError) as e:  # pageable host memory cannot take a GPU-written read-back
        srv.submit_many([(a, [(p, pose)], (em.LAYER_ELEVATION, torch.empty(3600)))])
    assert e.value.code == em.EM_ERR_INVALID_ARG
    # the same through the C ABI directly: the library checks the memory kind itself
    host = np.empty(3600, np.float32)
    req = (em._Request * 1)()
    arr = (em._Cloud * 1)(em._cloud_struct(p, pose, False))
    req[0].map_id, req[0].n_clouds, req[0].clouds = a, 1, arr
    req[0].read_mask, req[0].read_to_host, req[0].read_dst = em.LAYER_ELEVATION, 1, host.ctypes.data
    tks = (ctypes.c_uint64 * 1)()
    assert em.lib.em_server_submit_many(srv._h, req, 1, None, tks) == em.EM_ERR_INVALID_ARG
    assert srv.stats()["submitted"] == 0
    t = srv.submit_many([(a, [(p, pose)], None)])
    assert srv.wait(t[0])["status"] == 0
    srv.close()


def test_requests_survive_device_synchronize_during_capture(em):
    """A fresh server captures a CUDA graph for its first batch.  A device-wide
    synchronize from another thread while that capture runs breaks it; the
    batch must then run without the graph, so every request still succeeds."""
    srv = em.Server(budget_bytes=1 << 30, n_streams=2, max_batch_maps=4, max_batch_points=100_000)
    ids = [srv.add_map(em.Params(width=s, height=s, **BASE)) for s in SIDES[:4]]
    clouds = [dev(synth.scattered_cloud(400 + j, 20000, 0.5 * SIDES[j] * 0.04)[0]) for j in range(4)]
    pose = np.eye(3, 4).reshape(12)
    tickets = srv.submit_many([(ids[j], [(clouds[j], pose)], None) for j in range(4)])
    errors = 0
    for _ in range(200):  # races the worker's capture
        try:
            torch.cuda.synchronize()
        except RuntimeError:
            errors += 1
    assert all(srv.wait(t)["status"] == 0 for t in tickets)
    torch.cuda.synchronize()
    srv.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_host_clouds_equal_device_clouds(em, mode):
    """Requests whose clouds sit in page-locked host memory (the server copies
    them to the device itself, on the batch's stream) leave every map exactly
    as the same requests with device clouds do; pageable host clouds are
    refused before anything is queued."""
    reqs = workload(n_req=24, seed=9)
    host = [(j, p.cpu().pin_memory(), q) for j, p, q in reqs]
    states = []
    for which in ("device", "host"):
        srv = em.Server(budget_bytes=1 << 30, n_streams=2, max_batch_maps=4, max_batch_points=100_000, mode=mode)
        ids = [srv.add_map(em.Params(width=s, height=s, **BASE)) for s in SIDES]
        src = reqs if which == "device" else host
        tickets = srv.submit_many([(ids[j], [(p, q)], None) for j, p, q in src])
        assert all(s == 0 for s in srv.wait_many(tickets))
        states.append([srv.map(ids[j]).state() for j in range(len(SIDES))])
        if which == "host":
            assert srv.stats()["bytes_in_use"] > 0
            pageable = torch.zeros((100, 3))
            with pytest.raises(ValueError):
                srv.submit_many([(ids[0], [(pageable, reqs[0][2])], None)])
        srv.close()
    for j in range(len(SIDES)):
        for k in ("h", "var", "t_last"):
            assert np.array_equal(states[0][j][k], states[1][j][k], equal_nan=True), (j, k)


def test_served_mix_vs_oracle(em):
    """A mix of depth-camera and LiDAR requests (one per map, maps of 200 to 500
    cells over seeded priors) served in batches on three streams: every map
    agrees with the FP64 oracle fed the same prior and cloud (Section II-C,
    II-E), within the parity tolerances."""
    import oracle
    from tests import parity
    depth_p = dict(resolution=0.04, noise_a0=0.005, noise_a2=0.002, var_min=1e-8, min_range=0.05, max_range=10.0,
                   mahalanobis_k=2.5, outlier_variance=1e-4, ray_step=0.04)
    lidar_p = dict(resolution=0.04, noise_a0=0.01, noise_a2=0.001, var_min=1e-8, min_range=0.3, max_range=40.0,
                   mahalanobis_k=2.5, outlier_variance=1e-4, ray_step=0.04)
    depth = [c for fr in synth.depth_stream(seed=8, frames=2) for c in fr["clouds"]][:6]
    lidar = [fr["clouds"][0] for fr in synth.lidar_stream(seed=9, frames=2)]
    reqs = [(dict(depth_p, width=200 + 40 * i, height=200 + 40 * i), c) for i, c in enumerate(depth)]
    reqs += [(dict(lidar_p, width=500, height=500), c) for c in lidar]
    srv = em.Server(budget_bytes=4 << 30, n_streams=3, max_batch_maps=3, max_batch_points=2_000_000)
    ids, oms = [], []
    for j, (P, _) in enumerate(reqs):
        prior = synth.random_prior(seed=700 + j, width=P["width"], height=P["height"], t_now=5)
        mid = srv.add_map(em.Params(**P))
        parity.prior_to_gpu(srv.map(mid), prior)
        om = oracle.OracleMap(parity.oracle_params(P))
        parity.prior_to_oracle(om, prior)
        ids.append(mid)
        oms.append(om)
    torch.cuda.synchronize()
    tickets = srv.submit_many([(ids[j], [(dev(p), q)], None) for j, (_, (p, q)) in enumerate(reqs)])
    assert all(s == 0 for s in srv.wait_many(tickets))
    assert srv.stats()["batches"] < len(reqs)  # requests shared batches
    for j, (_, cloud) in enumerate(reqs):
        om = oms[j]
        prior_valid = np.isfinite(om.state()["var"])
        tr = om.update(cloud, trace=True, unit=oracle.FP32_UNIT, abs_band=parity.ABS_BAND)
        cmp = parity.compare_update(tr, om.state(), srv.map(ids[j]).state(), None, prior_valid=prior_valid,
                                    check_stencils=())
        assert cmp.notes["cells_compared"] > 0.9 * cmp.notes["cells_valid"], j
    srv.close()
