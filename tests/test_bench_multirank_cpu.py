"""The benchmark's N > 1 host logic on CPU: two gloo ranks agree on the
slowest rank's time, the whole-job value counts every rank's work, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(dist, local_ms, "cpu")
        out[rank] = (t, bench.whole_job_gpx(4_000_000, 100, world, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 15.0
    # 2 ranks x 100 steps x 4e6 pixel-passes in 15 ms
    assert out[0][1] == pytest.approx(2 * 100 * 4e6 / 0.015 / 1e9)


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.whole_job_gpx(1e9, 1, 1, 1000.0) == pytest.approx(1.0)


def test_reference_arm_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def _rank_lat(rank):
    import numpy as np

    return np.random.default_rng(100 + rank).exponential(1e-3, size=50 + 37 * rank)


def _rank_partition(rank, world, port, n_items, out):
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.owned(n_items, world, rank)
        every = bench.gather_arrays(dist, np.asarray(mine, np.float64))
        merged = bench.gather_arrays(dist, _rank_lat(rank))
        total = bench.sum_over_ranks(dist, len(mine), "cpu")
        out[rank] = (len(mine), every.tolist(), merged.tolist(), total)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_items", [(2, 256), (3, 1000), (4, 7)])
def test_simulations_partitioned_and_latencies_merged_gloo(world, n_items):
    """The batched and serving workloads under N ranks: every simulation is
    owned by exactly one rank, shares differ by at most one, the host-side
    sums count every rank's work, and the merged latency percentiles are those
    of all ranks' latencies concatenated."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_partition, args=(world, port, n_items, out), nprocs=world, join=True)
    every = sorted(int(v) for v in out[0][1])
    assert every == list(range(n_items))
    sizes = [out[r][0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1
    want = np.concatenate([_rank_lat(r) for r in range(world)])
    for r in range(world):
        assert out[r][3] == n_items
        np.testing.assert_array_equal(np.asarray(out[r][2]), want)
    got = bench.latency_summary(np.asarray(out[0][2]))
    assert got["p50_ms"] == pytest.approx(1e3 * np.percentile(want, 50))
    assert got["p99_ms"] == pytest.approx(1e3 * np.percentile(want, 99))


def test_gpus_flag_must_match_the_launch():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "WORLD_SIZE=1" in r.stderr
