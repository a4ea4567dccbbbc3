"""The row-band decomposition of one map across ranks, on CPU (gloo).

Each rank owns a band of rows and keeps a full-size map of which only its band
and the halo rows it receives are current; every other row is overwritten
with random labels before each pass, so a missing or misplaced halo row
changes the result.  The per-band pass is the CPU oracle's pass (Table I,
Section V-B) on the rank's map, of which the band's rows are kept.  The
frames assembled from the bands (a JFA frame, then dJFA steps, Eq. 4) must
equal the oracle's unsplit frames bit for bit, for 2 and 4 ranks, steps
larger than a band (JFA's first steps on 200 rows split four ways) included.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2209_00117_gb300 import bands, inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("h,world", [(1, 1), (5, 2), (61, 4), (200, 4), (200, 3), (7, 8)])
def test_halo_plan_covers_exactly_the_rows_read(h, world):
    """For every step: a rank's halo rows are exactly the rows its band's
    pass reads outside the band (brute force), and the plan delivers each of
    them once, from the rank that owns it."""
    owners = {}
    for r in range(world):
        y0, y1 = bands.band_rows(h, world, r)
        for y in range(y0, y1):
            assert y not in owners
            owners[y] = r
    assert sorted(owners) == list(range(h))
    for k in [1, 2, 3, 4, 8, 16, 32, 64, 128, 256]:
        plan = bands.halo_plan(h, world, k)
        for dst in range(world):
            y0, y1 = bands.band_rows(h, world, dst)
            want = {y + d for y in range(y0, y1) for d in (-k, k)} & set(range(h))
            want -= set(range(y0, y1))
            got = {y for a, b in bands.halo_rows(h, world, dst, k) for y in range(a, b)}
            assert got == want, (k, dst)
            delivered = []
            for (src, d), ranges in plan.items():
                if d != dst:
                    continue
                for a, b in ranges:
                    for y in range(a, b):
                        assert owners[y] == src
                        delivered.append(y)
            assert sorted(delivered) == sorted(want), (k, dst)


def _rank_main(rank, world, port, w, h, s, steps, metric, out):
    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        g = np.random.default_rng(1000 + rank)
        xy = inputs.uniform_seeds(w, h, s, seed=5)
        disp = inputs.displacements(s, 2, steps, seed=5)
        y0, y1 = bands.band_rows(h, world, rank)
        cur = torch.from_numpy(np.full((h, w), -1, np.int32))

        def poison_outside_band(m):
            noise = g.integers(-1, s, size=(h, w), dtype=np.int32)
            keep = m.numpy()[y0:y1].copy()
            m.copy_(torch.from_numpy(noise))
            m.numpy()[y0:y1] = keep

        def exchange_rows(plan):
            poison_outside_band(cur)
            bands.exchange(dist, cur, plan, rank)

        def band_pass(nb_sched_metric):
            def run(k, nb, a, b):
                nxt = oracle.jump_pass(w, h, xy_now[0], cur.numpy(), k, nb, nb_sched_metric)
                cur.numpy()[a:b] = nxt[a:b]
            return run

        def assembled():
            parts = [None] * world
            dist.all_gather_object(parts, cur.numpy()[y0:y1].copy())
            return np.concatenate(parts, axis=0)

        xy_now = [xy]
        results = []
        # a JFA frame: emptied map, stamp, then k_1 .. 1 on the bands
        cur.copy_(torch.from_numpy(oracle.stamp(w, h, xy, np.full((h, w), -1, np.int32))))
        bands.run_passes(oracle.jfa_schedule(w, h), h, world, rank, exchange_rows, band_pass(metric))
        full = assembled()
        want = oracle.jfa(w, h, xy, metric=metric)
        results.append(bool(np.array_equal(full, want)))
        lab = want
        # dJFA steps: move, stamp on the previous map, Eq. 4's schedule
        for t in range(steps):
            xy_now[0] = oracle.move(w, h, xy_now[0], disp[t])
            cur.copy_(torch.from_numpy(oracle.stamp(w, h, xy_now[0], full)))
            bands.run_passes(oracle.djfa_schedule(w, h, s, 2, vn_waves=2), h, world, rank, exchange_rows,
                             band_pass(metric))
            full = assembled()
            lab = oracle.djfa_step(w, h, xy_now[0], lab, d_max=2, vn_waves=2, metric=metric)
            results.append(bool(np.array_equal(full, lab)))
        out[rank] = results
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("w,h,s,metric", [(64, 200, 40, 0), (97, 61, 25, 1), (150, 130, 300, 0)])
def test_band_frames_equal_unsplit_frames_gloo(world, w, h, s, metric):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, w, h, s, 3, metric, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == [True] * 4, (r, out[r])
