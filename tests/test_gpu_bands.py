"""The row-band decomposition on the GPU: R bands of one map, each in its own
context (standing in for R GPUs), halo rows staged between the contexts'
maps by device-to-device copies (standing in for NCCL send/recv) following
the same plan as the multi-rank path, and each band's rows computed by
vd_pass_rows.  The frames assembled from the bands equal the unsplit frames
of one context and the oracle, bit for bit."""
import numpy as np
import pytest

from paper_2209_00117_gb300 import bands, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00117_gb300 import build, vd

    build.build()
    return torch, vd


def _frames(torch, vd, sims, w, h, sched, djfa):
    world = len(sims)
    maps = [bands.DeviceMap(s) for s in sims]
    for k, nb in sched:
        plan = bands.halo_plan(h, world, k)
        views = [m.tensor() for m in maps]
        for (src, dst), ranges in plan.items():
            for a, b in ranges:
                views[dst][a:b].copy_(views[src][a:b])
        for r, sim in enumerate(sims):
            y0, y1 = bands.band_rows(h, world, r)
            if y0 < y1:
                sim.pass_rows(k, nb, y0, y1, djfa_frame=djfa)
    out = np.empty((h, w), np.int32)
    for r, sim in enumerate(sims):
        y0, y1 = bands.band_rows(h, world, r)
        out[y0:y1] = sim.labels()[y0:y1]
    return out


@pytest.mark.parametrize("world", [2, 3, 8])
@pytest.mark.parametrize("w,h,s,D", [(300, 211, 500, 2), (1024, 1000, 20000, 4), (96, 500, 40, 1)])
def test_band_frames_equal_unsplit(env, orc, world, w, h, s, D):
    torch, vd = env
    stream = torch.cuda.current_stream().cuda_stream
    xy = inputs.uniform_seeds(w, h, s, seed=s + world)
    disp = inputs.displacements(s, D, 3, seed=s)
    sims = []
    for _ in range(world):
        sim = vd.VoronoiSim(w, h, s)
        sim.set_stream(stream)
        sim.set_seeds(xy)
        sims.append(sim)
    ref = vd.VoronoiSim(w, h, s)
    ref.set_stream(stream)
    ref.set_seeds(xy)
    for sim in sims:
        sim.clear_labels()
        sim.stamp()
    got = _frames(torch, vd, sims, w, h, vd.jfa_schedule(w, h), djfa=False)
    ref.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(ref.labels(), lab)
    np.testing.assert_array_equal(got, lab)
    cur = xy
    for t in range(3):
        for sim in sims + [ref]:
            sim.move(disp[t])
        for sim in sims:
            sim.stamp()
        got = _frames(torch, vd, sims, w, h, vd.djfa_schedule(w, h, s, D, vn_waves=2), djfa=True)
        ref.djfa_step(d_max=D)
        cur = orc.move(w, h, cur, disp[t])
        lab = orc.djfa_step(w, h, cur, lab, d_max=D)
        np.testing.assert_array_equal(ref.labels(), lab)
        np.testing.assert_array_equal(got, lab, err_msg=f"step {t}")
    for sim in sims + [ref]:
        sim.close()


def test_pass_rows_rejects_bad_ranges(env):
    torch, vd = env
    from paper_2209_00117_gb300._native import VDError

    sim = vd.VoronoiSim(64, 40, 5)
    for y0, y1 in [(-1, 10), (10, 10), (5, 41), (30, 20)]:
        with pytest.raises(VDError):
            sim.pass_rows(4, 0, y0, y1)
    sim.close()
