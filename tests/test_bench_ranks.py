"""Multi-rank logic of bench.py on CPU: two gloo ranks.

Maps are independent, so ranks share no data; the only exchange is the
timing (the slowest rank sets the job's time) and the job's throughput is the
units all ranks processed over that time.  The reference arm runs on rank 0
only.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = bench.rank_max(world, "cpu")
        seconds = [0.5, 2.0][rank]  # rank 1 is the slow one
        got = mx(seconds)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.fleet_seed(rank))

        class A:
            steps, warmup = 1, 0
        ref = bench.run_reference(A(), rank, world) if rank != 0 else "skipped"
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{got} {seeds[0]} {seeds[1]} {ref is None}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(world)]
    for r in range(world):
        got, s0, s1, _ = rows[r]
        assert float(got) == 2.0  # max over ranks on every rank
        assert s0 != s1  # each rank serves its own fleet
    assert rows[1][3] == "True"  # the reference arm does no work off rank 0


def test_job_rate_and_single_rank():
    import bench
    assert bench.rank_max(1, "cpu")(3.25) == 3.25
    # 2 ranks x 1e6 points, slowest rank 0.5 s -> 4e6 points/s for the job
    assert bench.job_rate(1e6, 2, 0.5) == 4e6


def test_reference_line_keeps_the_contract():
    """The reference arm's line (the oracle on the host) carries every key of the
    bench contract, with the served metric and workload of our arm."""
    import json
    import bench

    class A:
        steps, warmup = 1, 0
    line = bench.run_reference(A(), 0, 1)
    json.dumps(line)  # one JSON line
    for k in ("metric", "impl", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "points/s"
    assert line["config"]["workload"] == bench.WORKLOAD and line["value"] > 0
    assert set(line["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
