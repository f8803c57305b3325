#!/usr/bin/env python
"""Benchmark of the elevation-map fusion path on one node.

Headline workload (the served stream): 32 simulated robots -- 16 with a depth
camera (76,800 points per cloud, 320x240, ~5 % invalid) and 16 with a LiDAR
(128 x 2,048 = 262,144 points, range <= 30 m) -- each with its own resident map
of 200^2 .. 500^2 cells at 0.04 m; every request fuses one cloud into its
robot's map (transform, noise model, binning, Mahalanobis gate k = 2.5, Eq. 1/2
fusion, visibility ray march and removal).  The server (em_server) admits
requests by a 40 GB budget and batches them continuously.

  value          fused points/s of the served path at saturation: K rounds of
                 one request per robot, all submitted at once, timed with
                 CUDA events recorded with the device idle on both sides
                 (barrier + synchronize).  One step = one round.
  latency_ms     p50 / p99 request latency (submit -> GPU done) at the stated
                 load, 2,000 updates/s Poisson, for the served and the plain
                 per-request path (one em_update per request).
  e2e            the served path fed from host memory through the library:
                 per round one submit_many whose 32 requests carry clouds in
                 page-locked host memory (the server copies them to the device
                 by DMA on the batch's stream) and ask for their map's
                 elevation in page-locked host memory after the update
                 (double-buffered rounds; wall clock).
  roofline       HBM roofline of the whole update step: algorithmic bytes
                 B = 12 N + 24 U per round (every point read once; every cell
                 updated or cleared read and written once) over the step time.
  ray            the ray march (k_ray), the dominant kernel: samples/s and its
                 event-timed share of a round.
  load_sweep     p50 / p99 latency and mean batch size, served vs plain, at
                 several Poisson loads.
  batched        64 maps of 100^2..500^2 cells, 10k..400k points each, with the
                 ray march, one batched update per step (graph replay,
                 autotuned shapes) vs 64 sequential em_update calls; HBM
                 roofline of the update.
  depth_stream   one robot with 4 depth cameras (4 x 76,800 points), 200x200 map,
                 one em_update_multi per frame (plain path latency).
  lidar_filters  one LiDAR robot, 500x500 map, every per-cell feature (normals,
                 box / median / Gaussian smoothing, in-painting, upper bound,
                 drift compensation): update time and kernel times.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank serves its own fleet on its own GPU (maps are
independent: weak scaling, no collective on the data path); the timing takes the
max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fused points/s & p99 map-update latency (served vs plain) at 1 GB300"
WORKLOAD = ("served stream: 32 robots (16 depth 76,800 pts, 16 LiDAR 262,144 pts), maps 200^2-500^2 @ 0.04 m, "
            "40 GB budget")
DEPTH_P = dict(resolution=0.04, noise_a0=0.005, noise_a2=0.002, var_min=1e-8, min_range=0.05, max_range=10.0,
               mahalanobis_k=2.5, outlier_variance=1e-4, ray_step=0.04)
LIDAR_P = dict(resolution=0.04, noise_a0=0.01, noise_a2=0.001, var_min=1e-8, min_range=0.3, max_range=40.0,
               mahalanobis_k=2.5, outlier_variance=1e-4, ray_step=0.04)
BATCH_P = dict(resolution=0.04, noise_a0=0.005, noise_a2=0.002, var_min=1e-8, mahalanobis_k=2.5,
               outlier_variance=1e-4, ray_step=0.04)
N_ROBOTS = 32
RATE_HZ = 2000.0
SWEEP_HZ = (2000.0, 10000.0, 40000.0)
E2E_DEPTH = 3  # rounds in flight in the end-to-end leg (each with its own read-back buffer)
CLOCK_SOAK_S = 1.0  # seconds of untimed load inside the clock sampler before the timed rounds
BUDGET = 40 << 30
L2_FLUSH_BYTES = 256 << 20


def f32params(P):
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in P.items()}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def update_bytes(points: float, cells: float) -> float:
    """Algorithmic bytes of an update: every point read once (12 B of xyz) and
    every cell the update writes (fused or cleared) read and written once (12 B
    of state each way)."""
    return 12.0 * points + 24.0 * cells


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(math.ceil(q * len(xs))) - 1)] if xs else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def file_hash(*paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


CSRC = "paper_2204_12876_gb300/csrc/"
KERNEL_SOURCES = {"ray": [CSRC + "k_ray.cu", CSRC + "ray_pass.cuh", CSRC + "em_point.cuh", CSRC + "em_internal.cuh"],
                  "count": [CSRC + "k_sort.cu", CSRC + "sort_pass.cuh", CSRC + "em_point.cuh", CSRC + "em_internal.cuh"],
                  "scatter": [CSRC + "k_sort.cu", CSRC + "sort_pass.cuh", CSRC + "em_point.cuh",
                              CSRC + "em_internal.cuh"],
                  "alloc": [CSRC + "k_sort.cu", CSRC + "sort_pass.cuh", CSRC + "em_point.cuh", CSRC + "em_internal.cuh"],
                  "fuse": [CSRC + "k_fuse.cu", CSRC + "fuse_pass.cuh", CSRC + "em_point.cuh", CSRC + "em_internal.cuh"],
                  "clear": [CSRC + "k_ray.cu", CSRC + "ray_pass.cuh", CSRC + "em_point.cuh", CSRC + "em_internal.cuh"]}


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            e = json.load(f)[workload][kernel]
        if e["source_hash"] != file_hash(*KERNEL_SOURCES[kernel]):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


def ncu_step_traffic(kernels, workload: str):
    """DRAM bytes of one step: the sum over its kernels of the committed ncu
    figures, or None unless every kernel's figure was taken on its current source."""
    tot = 0.0
    for k in kernels:
        t = ncu_traffic(k, workload)
        if t is None:
            return None
        tot += t
    return tot


# ---------------------------------------------------------------- ranks

def fleet_seed(rank: int) -> int:
    """Each rank serves its own fleet (maps are independent: no exchange)."""
    return 5 + 100 * rank


def rank_max(world: int, device: str):
    """x -> max of x over all ranks (the slowest rank sets the job's time)."""
    def f(x: float) -> float:
        if world == 1:
            return x
        import torch
        t = torch.tensor([x], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return f


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the max time."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------- workloads

def make_fleet(seed: int = 5):
    rng = np.random.default_rng(seed)
    robots = []
    for i in range(N_ROBOTS):
        kind = "depth" if i < N_ROBOTS // 2 else "lidar"
        side = int(rng.integers(200, 501))
        robots.append({"kind": kind, "params": dict(DEPTH_P if kind == "depth" else LIDAR_P, width=side, height=side)})
    return robots


_LIDAR = {}


def lidar_scans(seed: int, frames: int):
    """LiDAR scans of the seeded stream (the generator ray-casts each on the host in seconds: kept)."""
    if (seed, frames) not in _LIDAR:
        import synth
        _LIDAR[(seed, frames)] = list(synth.lidar_stream(seed=seed, frames=frames))
    return _LIDAR[(seed, frames)]


def make_pools(seed: int = 5):
    import synth
    depth = []
    for fr in synth.depth_stream(seed=seed, frames=2):
        depth.extend(fr["clouds"])  # single-camera clouds, 76,800 points each
    lidar = [fr["clouds"][0] for fr in synth.lidar_stream(seed=seed + 1, frames=2)]
    return {"depth": depth, "lidar": lidar}


def request_cloud(pools, robots, i, k):
    pool = pools[robots[i]["kind"]]
    return pool[(i + k) % len(pool)]


# ---------------------------------------------------------------- our arm

def run_ours(args, rank: int, world: int):
    import torch
    from paper_2204_12876_gb300 import build
    build.build()
    from paper_2204_12876_gb300 import em

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    hbm, sm_mhz_max, peak_kind = peaks()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    max_over_ranks = rank_max(world, "cuda")
    robots = make_fleet(seed=fleet_seed(rank))
    pools = make_pools(seed=fleet_seed(rank))
    dpools = {k: [(torch.from_numpy(p).cuda(), q) for p, q in v] for k, v in pools.items()}
    round_pts = sum(len(request_cloud(pools, robots, i, 0)[0]) for i in range(N_ROBOTS))

    def new_server(mode):
        srv = em.Server(budget_bytes=BUDGET, max_slots=4096, n_streams=args.streams, max_batch_maps=args.batch_maps,
                        max_batch_points=N_ROBOTS * 262144, max_map_cells=500 * 500, mode=mode, graph=True,
                        device=dev)
        ids = [srv.add_map(em.Params(**r["params"])) for r in robots]
        return srv, ids

    def submit_round(srv, ids, k):
        return srv.submit_many([(ids[i], [request_cloud(dpools, robots, i, k)], None) for i in range(N_ROBOTS)])

    def saturate(srv, ids, K, k0):
        """K rounds submitted at once; returns (seconds, points, batches).  The
        span is taken with CUDA events on this thread's stream, recorded with
        the device idle on both sides (the server's streams have drained before
        the closing record), so it covers every batch of the K rounds."""
        b0 = srv.stats()["batches"]
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tickets = []
        for k in range(K):
            tickets += submit_round(srv, ids, k0 + k)
        srv.wait_many(tickets)
        e1.record()
        barrier()
        sec = e0.elapsed_time(e1) / 1e3
        return max_over_ranks(sec), K * round_pts, srv.stats()["batches"] - b0

    # ---- served path: warm up (the maps fill), then autotune the batch shapes
    # on one round (scratch copies of the maps: the served maps do not advance)
    served, sids = new_server(em.SERVE_BATCHED)
    for k in range(args.warmup):
        served.wait_many(submit_round(served, sids, k))
    served.drain()
    tuner = em.Batch(max_maps=N_ROBOTS, max_clouds=N_ROBOTS, max_points=N_ROBOTS * 262144, max_cells=500 * 500,
                     graph=False, device=dev)
    pairs = [(served.map(sids[i]), *request_cloud(dpools, robots, i, args.warmup)) for i in range(N_ROBOTS)]
    tuning = tuner.autotune(pairs, reps=3)
    served.set_tuning(**tuning)
    K = args.steps
    # The sampler polls every 200 ms and the K timed rounds take milliseconds,
    # so the same rounds also run, untimed, for about a second right before the
    # timed ones inside the sampler's window: the samples see this load.
    est, _, _ = saturate(served, sids, K, args.warmup)
    soak = max(K, int(CLOCK_SOAK_S / max(est / K, 1e-6)))
    with ClockSampler(dev) as clk:
        saturate(served, sids, soak, args.warmup)
        sec, pts, timed_batches = saturate(served, sids, K, args.warmup)
    value = job_rate(pts, world, sec)
    sst = served.stats()

    # ---- plain per-request path at saturation (fresh maps)
    plain, pids = new_server(em.SERVE_PLAIN)
    for k in range(args.warmup):
        plain.wait_many(submit_round(plain, pids, k))
    psec, ppts, _ = saturate(plain, pids, K, args.warmup)
    plain_value = job_rate(ppts, world, psec)

    # ---- latency under Poisson arrivals: the stated 2,000 updates/s, then a sweep
    # of heavier loads where requests arrive while earlier batches still run
    def offered(srv, ids, rate, seconds, seed):
        rng = np.random.default_rng(seed + rank)
        n_req = max(1, int(rate * seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        who = rng.integers(0, N_ROBOTS, n_req)
        barrier()
        counters = [0] * N_ROBOTS
        tickets = []
        t0 = time.perf_counter()
        for a, i in zip(arrivals, who):
            while time.perf_counter() - t0 < a:
                pass
            tickets.append(srv.submit(ids[i], [request_cloud(dpools, robots, int(i), counters[i])]))
            counters[i] += 1
        res = srv.wait_many(tickets, results=True)
        span = time.perf_counter() - t0
        lat = [(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in res]
        bs = [r["batch_size"] for r in res]
        npts = sum(r["points"] for r in res)
        return {"p50": pct(lat, 0.50), "p99": pct(lat, 0.99), "mean": float(np.mean(lat)), "requests": n_req,
                "offered_updates_per_s": rate, "points_per_s": npts / span, "mean_batch": float(np.mean(bs))}

    lat_served = offered(served, sids, RATE_HZ, args.load_seconds, 77)
    lat_plain = offered(plain, pids, RATE_HZ, args.load_seconds, 77)
    sweep = []
    for rate in SWEEP_HZ[1:]:
        secs = max(0.25, min(args.load_seconds, 20000.0 / rate))
        sweep.append({"offered_updates_per_s": rate, "seconds": secs,
                      "served": offered(served, sids, rate, secs, 78), "plain": offered(plain, pids, rate, secs, 78)})

    # ---- per-kernel profile of one served round (event-timed, direct launches)
    pmaps = [served.map(sids[i]) for i in range(N_ROBOTS)]
    st0 = [m.stats() for m in pmaps]
    tuner.set_tuning(**tuning)
    tuner.profile(True)
    P_STEPS = 3
    for k in range(P_STEPS):
        tuner.update([(pmaps[i], *request_cloud(dpools, robots, i, k)) for i in range(N_ROBOTS)])
    prof = tuner.profile_read()
    tuner.profile(False)
    st1 = [m.stats() for m in pmaps]
    delta = lambda key: sum(b[key] - a[key] for a, b in zip(st0, st1)) / P_STEPS
    samples = delta("ray_samples")
    cells_upd = delta("cells_updated")
    cells_clr = delta("cells_cleared")
    in_map = delta("points_in_map")
    total_ms = sum(v[0] for v in prof.values() if v[1])
    kernels = {em.KERNEL_NAMES[k]: {"ms_per_launch": round(v[0] / v[1], 5), "launches": v[1],
                                    "share": round(v[0] / total_ms, 4)} for k, v in prof.items() if v[1]}
    # HBM roofline of the whole update step (every point read once, every written cell
    # read and written once) over the saturated step time
    alg = update_bytes(round_pts, cells_upd + cells_clr)
    step_s = sec / K
    roofline = {"bound": "hbm", "scope": "whole update step (one served round, all kernels)",
                "algorithmic_bytes": alg, "achieved": alg / step_s / 1e9, "peak": hbm, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": alg / step_s / 1e9 / hbm,
                "traffic": ncu_step_traffic([k for k in prof if prof[k][1]], "served_round"),
                "per_round": {"points": round_pts, "points_in_map": in_map, "cells_updated": cells_upd,
                              "cells_cleared": cells_clr}}
    ray_ms = prof["ray"][0] / prof["ray"][1] if prof.get("ray", (0, 0))[1] else None
    ray = {"kernel": "k_ray", "samples_per_launch": samples, "ms_per_launch": ray_ms,
           "samples_per_s": samples / (ray_ms / 1e3) if ray_ms else None,
           "share_of_round": kernels.get("k_ray", {}).get("share"), "traffic": ncu_traffic("ray", "served_round")}

    # ---- end to end through the library: each round's 32 clouds lie in page-locked
    # host memory (a client's ring of input buffers; the pools repeat every 8 rounds);
    # one submit_many per round hands them to the server, which copies each cloud to
    # the device by DMA on the batch's stream and writes each map's elevation into a
    # page-locked host buffer right after its update.  E2E_DEPTH rounds are in
    # flight: round k + E2E_DEPTH - 1 is queued before round k is waited for.
    P = 8
    packs = []
    for r in range(P):
        parts = [request_cloud(pools, robots, i, args.warmup + r) for i in range(N_ROBOTS)]
        packs.append([(torch.from_numpy(p).pin_memory(), q) for p, q in parts])
    cells = [r["params"]["width"] * r["params"]["height"] for r in robots]
    offs = np.concatenate([[0], np.cumsum(cells)]).astype(np.int64)
    out_bytes = int(offs[-1]) * 4
    host_out = [torch.empty(int(offs[-1]), dtype=torch.float32).pin_memory() for _ in range(E2E_DEPTH)]

    def e2e_launch(k):
        reqs = []
        for i in range(N_ROBOTS):
            reqs.append((sids[i], [packs[k % P][i]],
                         (em.LAYER_ELEVATION, host_out[k % E2E_DEPTH][int(offs[i]):int(offs[i + 1])])))
        return served.submit_many(reqs)

    e2e_rounds = max(4, K)
    e2e_launch(0)  # the first host request allocates the server's input buffers
    served.drain()
    barrier()
    t0 = time.perf_counter()
    inflight = [e2e_launch(k) for k in range(min(E2E_DEPTH - 1, e2e_rounds))]
    for k in range(E2E_DEPTH - 1, e2e_rounds + E2E_DEPTH - 1):
        if k < e2e_rounds:
            inflight.append(e2e_launch(k))
        # round k - E2E_DEPTH + 1: every map's elevation is now in its host_out buffer
        served.wait_many(inflight.pop(0))
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": e2e_rounds * round_pts * world / e2e_s, "unit": "points/s",
           "h2d_bytes_per_step": int(round_pts * 12), "d2h_bytes_per_step": int(out_bytes),
           "path": "em_server_submit_many with page-locked host clouds and host read-back (copies issued by libem.so)"}

    result = {
        "metric": METRIC,
        "value": value,
        "unit": "points/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": sec / K * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: seeded depth-camera and LiDAR clouds (pools of 8 and 2 clouds cycled), seeded terrain",
        "config": {"workload": WORKLOAD, "robots": N_ROBOTS, "points_per_step": round_pts,
                   "step": "one round = one request per robot", "streams": args.streams,
                   "batch_maps": args.batch_maps, "tuning": tuning,
                   "l2": "inputs + map state per step > L2 (about 65 MB of clouds + 200 MB of maps), no flush",
                   "parallelism": f"replicas{world}"},
        "updates_per_s": K * N_ROBOTS * world / sec,
        "plain_saturated": {"value": plain_value, "unit": "points/s", "updates_per_s": K * N_ROBOTS * world / psec},
        "latency_ms": {"load_updates_per_s": RATE_HZ, "seconds": args.load_seconds,
                       "served": lat_served, "plain": lat_plain},
        "load_sweep": sweep,
        "served_batches": {"batches": sst["batches"], "mean_batch": sst["batched_requests"] / max(1, sst["batches"]),
                           "max_batch": sst["max_batch_size"], "peak_bytes": sst["peak_bytes"]},
        "e2e": e2e,
        "gpu_launches": int(timed_batches) * len([k for k in prof if prof[k][1]]),
        "roofline": roofline,
        "ray": ray,
        "kernels": kernels,
        "clocks": dict(clk.summary(), window=f"{soak} untimed rounds of the same work (about {CLOCK_SOAK_S:g} s) "
                                              f"directly before the {K} timed rounds, and those"),
    }
    served.close()
    plain.close()
    tuner.close()
    if not args.served_only:
        result["batched"] = run_batched(args, em, torch, dev, barrier, max_over_ranks, world)
        result["depth_stream"] = run_depth(args, em, torch, dev)
        result["lidar_filters"] = run_lidar_filters(args, em, torch, dev)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(robots, pools, budget_s=args.cpu_budget)
    return result


def run_batched(args, em, torch, dev, barrier, max_over_ranks, world):
    """64 uneven maps, one batched update per step vs 64 sequential em_update."""
    import synth
    hbm, _, peak_kind = peaks()
    work = synth.batch_clouds(seed=4, maps=64)
    pts_step = sum(len(w["clouds"][0][0]) for w in work)
    clouds = [(torch.from_numpy(w["clouds"][0][0]).cuda(), w["clouds"][0][1]) for w in work]

    def fleet():
        return [em.Map(em.Params(width=w["side"], height=w["side"], **BATCH_P), device=dev) for w in work]

    maps = fleet()
    max_cells = max(w["side"] ** 2 for w in work)
    batch = em.Batch(max_maps=64, max_clouds=64, max_points=pts_step, max_cells=max_cells, graph=True, device=dev)
    pairs = [(m, p, q) for m, (p, q) in zip(maps, clouds)]
    for _ in range(args.warmup):
        batch.update(pairs)
    tuning = batch.autotune(pairs, reps=3)  # on scratch copies of the warmed-up maps
    K = args.steps
    st0 = [m.stats() for m in maps]
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        batch.update(pairs)
    e1.record()
    barrier()
    sec = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    st1 = [m.stats() for m in maps]
    cells = sum((b["cells_updated"] - a["cells_updated"]) + (b["cells_cleared"] - a["cells_cleared"])
                for a, b in zip(st0, st1)) / K
    samples = sum(b["ray_samples"] - a["ray_samples"] for a, b in zip(st0, st1)) / K
    alg = update_bytes(pts_step, cells)
    # per-kernel shares of one batch (direct launches)
    batch.profile(True)
    for _ in range(3):
        batch.update(pairs)
    prof = batch.profile_read()
    batch.profile(False)
    total_ms = sum(v[0] for v in prof.values() if v[1])
    kernels = {em.KERNEL_NAMES[k]: {"ms_per_launch": round(v[0] / v[1], 5), "share": round(v[0] / total_ms, 4)}
               for k, v in prof.items() if v[1]}
    # the same batch in one persistent launch per update (EM_BATCH_PERSISTENT), same tuning, fresh maps
    xmaps = fleet()
    xbatch = em.Batch(max_maps=64, max_clouds=64, max_points=pts_step, max_cells=max_cells, graph=True, device=dev,
                      persistent=True)
    xbatch.set_tuning(**tuning)
    xpairs = [(m, p, q) for m, (p, q) in zip(xmaps, clouds)]
    for _ in range(args.warmup):
        xbatch.update(xpairs)
    barrier()
    e0.record()
    for _ in range(K):
        xbatch.update(xpairs)
    e1.record()
    barrier()
    xsec = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    xbatch.profile(True)
    xbatch.update(xpairs)
    xprof = xbatch.profile_read()
    xbatch.profile(False)
    xbatch.close()
    # plain comparison: 64 sequential em_update on a second set of maps
    pmaps = fleet()
    for _ in range(args.warmup):
        for m, (p, q) in zip(pmaps, clouds):
            m.update(p, q)
    barrier()
    e0.record()
    for _ in range(K):
        for m, (p, q) in zip(pmaps, clouds):
            m.update(p, q)
    e1.record()
    barrier()
    psec = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    for m in maps + pmaps + xmaps:
        m.close()
    batch.close()
    return {"workload": "64 maps, side U{100..500} cells @ 0.04 m, 10k..400k points each, random point order; "
                        "fusion, outlier gate and visibility ray march (step 0.04 m)",
            "form": "one kernel sequence over every map, replayed from a captured CUDA graph (the default form)",
            "persistent": {"form": "EM_BATCH_PERSISTENT: the update's passes in one cooperative launch with grid "
                                   "barriers (stencils as kernels of their own), replayed from a captured CUDA graph",
                           "value": pts_step * K * world / xsec, "unit": "points/s", "ms_per_step": xsec / K * 1e3,
                           "kernels": {em.KERNEL_NAMES[k]: {"ms_per_launch": round(v[0] / v[1], 5)}
                                       for k, v in xprof.items() if v[1]}},
            "points_per_step": pts_step, "value": pts_step * K * world / sec, "unit": "points/s",
            "ms_per_step": sec / K * 1e3, "updates_per_s": 64 * K * world / sec, "tuning": tuning,
            "ray_samples_per_step": samples,
            "plain_sequential": {"value": pts_step * K * world / psec, "ms_per_step": psec / K * 1e3},
            "update_roofline": {"bound": "hbm", "algorithmic_bytes": alg, "achieved": alg / (sec / K) / 1e9,
                                "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                                "frac": alg / (sec / K) / 1e9 / hbm,
                                "traffic": ncu_step_traffic([k for k in prof if prof[k][1]], "batched_64maps")},
            "kernels": kernels}


def run_round(args, em, torch, which):
    """Profiler workload: one served round (the 32 robots' requests, one batch) or
    the 64-map batch, as direct launches (no graph): --warmup rounds, then
    --steps rounds with per-kernel event timing."""
    import synth
    if which == "served_round":
        robots = make_fleet(5)
        pools = make_pools(5)
        dp = {k: [(torch.from_numpy(p).cuda(), q) for p, q in v] for k, v in pools.items()}
        maps = [em.Map(em.Params(**r["params"])) for r in robots]
        batch = em.Batch(max_maps=N_ROBOTS, max_clouds=N_ROBOTS, max_points=N_ROBOTS * 262144, max_cells=500 * 500,
                         graph=False)

        def pairs(k):
            return [(maps[i], *request_cloud(dp, robots, i, k)) for i in range(N_ROBOTS)]
    else:
        work = synth.batch_clouds(seed=4, maps=64)
        maps = [em.Map(em.Params(width=w["side"], height=w["side"], **BATCH_P)) for w in work]
        cl = [(torch.from_numpy(w["clouds"][0][0]).cuda(), w["clouds"][0][1]) for w in work]
        batch = em.Batch(max_maps=64, max_clouds=64, max_points=sum(len(w["clouds"][0][0]) for w in work),
                         max_cells=max(w["side"] ** 2 for w in work), graph=False)

        def pairs(k):
            return [(m, p, q) for m, (p, q) in zip(maps, cl)]
    for k in range(args.warmup):
        batch.update(pairs(k))
    torch.cuda.synchronize()
    batch.profile(True)
    for k in range(args.steps):
        batch.update(pairs(args.warmup + k))
    prof = batch.profile_read()
    batch.profile(False)
    torch.cuda.synchronize()
    out = {"workload": which, "rounds": args.steps,
           "kernels_ms": {em.KERNEL_NAMES[k]: round(v[0] / v[1], 5) for k, v in prof.items() if v[1]}}
    batch.close()
    for m in maps:
        m.close()
    return out


def run_lidar_filters(args, em, torch, dev):
    """One LiDAR robot (128 x 2,048 points) on a 500 x 500 map with every per-cell
    feature: normals, smoothing (box, median or Gaussian), in-painting, the
    upper-bound layer and drift compensation; per-update time and kernel times."""
    import synth
    frames = lidar_scans(3, 3)
    clouds = [[(torch.from_numpy(p).cuda(), q) for p, q in fr["clouds"]] for fr in frames]
    pts = sum(len(p) for p, _ in frames[0]["clouds"])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {"workload": "128 x 2,048 LiDAR points per update, 500x500 map, normals + smoothing + in-painting + "
                       "upper bound + drift compensation", "points_per_update": pts, "smoothing": {}}
    for name, flag in (("box", em.F_SMOOTH), ("median", em.F_MEDIAN), ("gauss", em.F_GAUSS)):
        P = dict(LIDAR_P, width=500, height=500, cleanup_normal_thresh=0.1, drift_flatness=0.95,
                 flags=em.F_NORMALS | flag | em.F_INPAINT | em.F_UPPER)
        m = em.Map(em.Params(**P), device=dev)
        m.reserve(pts)
        for i in range(args.warmup):
            m.update_multi(clouds[i % len(clouds)])
        m.profile(True)
        times = []
        for i in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            m.update_multi(clouds[i % len(clouds)])
            b.record()
            times.append((a, b))
        torch.cuda.synchronize()
        prof = m.profile_read()
        m.profile(False)
        ms = [x.elapsed_time(y) for x, y in times]
        st = m.stats()
        m.close()
        out["smoothing"][name] = {
            "ms_per_update": float(np.mean(ms)), "p99_ms": pct(ms, 0.99), "points_per_s": pts / (np.mean(ms) / 1e3),
            "kernels_ms": {em.KERNEL_NAMES[k]: round(v[0] / v[1], 5) for k, v in prof.items() if v[1]},
            "drift_points": st["drift_points"], "drift_last_m": st["drift_last"]}
    out["l2"] = "flushed before every update (256 MB write, not timed); kernels_ms from per-kernel events"
    out["frames"] = (f"{args.steps} timed updates (+{args.warmup} warm-up) cycling 3 scans of the 1,000-frame "
                     "LiDAR stream; the generator ray-casts each scan on the host in seconds")
    return out


def run_depth(args, em, torch, dev):
    """Four depth cameras of one robot per frame into a 200x200 map (plain path)."""
    import synth
    pool = list(synth.depth_stream(seed=2, frames=3))
    P = dict(DEPTH_P, width=200, height=200)
    r = P["resolution"]
    dpool = [[(torch.from_numpy(p).cuda(), q) for p, q in fr["clouds"]] for fr in pool]
    pts = sum(len(p) for p, _ in pool[0]["clouds"])
    m = em.Map(em.Params(**P), device=dev)
    m.reserve(pts)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sx = sy = 0
    times = []
    for i in range(args.warmup + args.steps):
        fr = pool[i % len(pool)]
        dx, dy = int(round(fr["xy"][0] / r)) - sx, int(round(fr["xy"][1] / r)) - sy
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if dx or dy:
            m.shift(dx, dy)
            sx, sy = sx + dx, sy + dy
        m.update_multi(dpool[i % len(pool)])
        b.record()
        times.append((a, b))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in times[args.warmup:]]
    m.close()
    return {"workload": "4 x 76,800 depth points per frame, 200x200 map, shift + em_update_multi per frame",
            "frames": f"{len(ms)} timed frames (+{args.warmup} warm-up) cycling 3 frames of the 100-frame stream",
            "value": pts * len(ms) / (sum(ms) / 1e3), "unit": "points/s", "ms_per_step": float(np.mean(ms)),
            "p50_ms": pct(ms, 0.5), "p99_ms": pct(ms, 0.99),
            "l2": "flushed before every frame (256 MB write, not timed)"}


def cpu_baseline(robots, pools, budget_s: float = 12.0) -> dict:
    """The FP64 oracle, as it stands, on the host cores: (1) one thread on the
    served mix (robots in turn); (2) every host core, each thread serving its
    own robots' maps (independent maps run in parallel; ctypes releases the GIL
    during an oracle update); (3) the LiDAR configuration with every per-cell
    filter on one thread over the first 50 updates of its stream (3 scans
    cycled); (4) the 64-map batch on every host core, each thread fusing whole
    maps of it (one update each, fresh maps, in map order).  Each leg runs for a
    quarter of the budget at most."""
    import oracle
    import synth
    host_cores = os.cpu_count() or 1
    leg = budget_s / 4.0

    def serve(threads):
        per = [{"pts": 0, "n": 0} for _ in range(threads)]
        t_end = time.perf_counter() + leg

        def work(w):
            oms = {}
            n = 0
            while time.perf_counter() < t_end and n < 10000:
                i = (w + threads * n) % N_ROBOTS
                if i not in oms:
                    oms[i] = oracle.OracleMap(oracle.Params(**f32params(robots[i]["params"])))
                p, q = request_cloud(pools, robots, i, n)
                oms[i].update((p, q))
                per[w]["pts"] += len(p)
                n += 1
            per[w]["n"] = n
        t0 = time.perf_counter()
        ths = [threading.Thread(target=work, args=(w,)) for w in range(threads)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        dt = time.perf_counter() - t0
        return sum(x["pts"] for x in per) / dt, sum(x["n"] for x in per), sum(x["pts"] for x in per), dt

    v1, n1, p1, d1 = serve(1)
    vN, nN, pN, dN = serve(host_cores)
    P = dict(LIDAR_P, width=500, height=500, cleanup_normal_thresh=0.1, flags=oracle.NORMALS | oracle.SMOOTH |
             oracle.INPAINT)
    scans = [fr["clouds"] for fr in lidar_scans(3, 3)]
    om = oracle.OracleMap(oracle.Params(**f32params(P)))
    frames, lt = 0, 0.0
    t_end = time.perf_counter() + leg
    while frames < 50 and time.perf_counter() < t_end:
        t0 = time.perf_counter()
        om.update(scans[frames % 3])
        lt += time.perf_counter() - t0
        frames += 1
    # (4) the 64-map batch: threads take maps in order until the leg's time is up
    work = synth.batch_clouds(seed=4, maps=64)
    lock = threading.Lock()
    nxt = [0]
    done = {"maps": 0, "pts": 0}
    t_end = time.perf_counter() + leg

    def bwork():
        while time.perf_counter() < t_end:
            with lock:
                j = nxt[0]
                nxt[0] += 1
            if j >= len(work):
                return
            w = work[j]
            om_b = oracle.OracleMap(oracle.Params(**f32params(dict(BATCH_P, width=w["side"], height=w["side"]))))
            om_b.update(w["clouds"][0])
            with lock:
                done["maps"] += 1
                done["pts"] += len(w["clouds"][0][0])
    t0 = time.perf_counter()
    ths = [threading.Thread(target=bwork) for _ in range(host_cores)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    db = time.perf_counter() - t0
    return {"value": v1, "unit": "points/s", "cores": 1, "host_cores": host_cores, "kind": "oracle",
            "sample": f"{n1} requests of the served mix (robots in turn, {p1} points) in {d1:.1f} s, one thread",
            "all_cores": {"value": vN, "unit": "points/s", "threads": host_cores,
                          "sample": f"{nN} requests ({pN} points) in {dN:.1f} s, {host_cores} threads, "
                                    "each serving its own robots' maps"},
            "lidar_filters": {"ms_per_update": lt / max(1, frames) * 1e3, "updates": frames,
                              "sample": f"first {frames} of 50 updates of the LiDAR configuration (500x500, "
                                        "normals, box smoothing, in-painting; 3 scans cycled), one thread"},
            "batched_all_cores": {"value": done["pts"] / db, "unit": "points/s", "threads": host_cores,
                                  "sample": f"{done['maps']} of the 64 maps of the batched configuration "
                                            f"({done['pts']} points, one update each) in {db:.1f} s, "
                                            f"{host_cores} threads"}}


def run_reference(args, rank: int, world: int):
    """The oracle as the reference arm: one request of the served mix per step."""
    if rank != 0:
        return None
    robots = make_fleet(seed=5)
    pools = make_pools(seed=5)
    import oracle
    oms = {}

    def step(n):
        i = (n * 7) % N_ROBOTS  # alternates depth and LiDAR robots
        if i not in oms:
            oms[i] = oracle.OracleMap(oracle.Params(**f32params(robots[i]["params"])))
        p, q = request_cloud(pools, robots, i, n)
        oms[i].update((p, q))
        return len(p)

    for n in range(args.warmup):
        step(n)
    pts = 0
    t0 = time.perf_counter()
    for n in range(args.steps):
        pts += step(args.warmup + n)
    dt = time.perf_counter() - t0
    v = pts / dt
    return {"metric": METRIC, "impl": "reference", "value": v, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded depth-camera and LiDAR clouds",
            "config": {"workload": WORKLOAD, "step": "one request"},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": f"{args.steps} requests of the served mix, single thread"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--streams", type=int, default=3, help="batches in flight in the served path")
    ap.add_argument("--batch-maps", type=int, default=16, help="maps per batch in the served path")
    ap.add_argument("--load-seconds", type=float, default=4.0, help="duration of the Poisson-load phase")
    ap.add_argument("--cpu-budget", type=float, default=32.0, help="seconds for the four oracle legs together")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--served-only", action="store_true", help="skip the batched and depth-stream sub-results")
    ap.add_argument("--workload", default="all",
                    choices=["all", "batched", "depth", "lidar", "served_round", "batch_round"],
                    help="run only that sub-result, or one round of the served mix / the 64-map batch as a "
                         "batch of direct launches (warm-up rounds, then --steps rounds: for profiler runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        args.steps = min(args.steps, 40)  # whole requests on one host core: a few minutes at most
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload != "all":  # one sub-result alone (profiler runs)
        import torch
        from paper_2204_12876_gb300 import build
        build.build()
        from paper_2204_12876_gb300 import em
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))

        def barrier():
            torch.cuda.synchronize()

        if args.workload == "batched":
            res = run_batched(args, em, torch, 0, barrier, lambda x: x, 1)
        elif args.workload in ("served_round", "batch_round"):
            res = run_round(args, em, torch, args.workload)
        elif args.workload == "lidar":
            res = run_lidar_filters(args, em, torch, 0)
        else:
            res = run_depth(args, em, torch, 0)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    res = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
