"""The server: continuous batching of dJFA step requests over resident
simulations.  Each simulation's result after a mixed, bursty trace equals what
it gives alone (integer maps, tolerance 0); admission follows the HBM budget;
batches really form (fewer launches than requests)."""
import numpy as np
import pytest

from paper_2209_00117_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(512, 512, 900), (300, 211, 700), (1024, 768, 6000), (256, 256, 64), (77, 33, 9), (640, 480, 2500)]
D, RNG = 2, 4242


@pytest.fixture(scope="module")
def vd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00117_gb300 import build

    build.build()
    from paper_2209_00117_gb300 import vd as _vd

    return _vd


def _alone(vd, shape, xy, sim_id, steps):
    w, h, s = shape
    sim = vd.VoronoiSim(w, h, s)
    sim.set_seeds(xy)
    sim.jfa()
    for t in range(steps):
        sim.move(None, max_disp=D, rng_seed=RNG, stream_id=sim_id, step=t)
        sim.djfa_step(d_max=D)
    out = sim.labels()
    sim.close()
    return out


def test_mixed_trace_equals_alone(vd):
    srv = vd.VoronoiServer(max_sims=16, hbm_budget_bytes=1 << 30, d_max=D, max_disp=D, rng_seed=RNG)
    xys = [inputs.uniform_seeds(w, h, s, seed=60 + i) for i, (w, h, s) in enumerate(SHAPES)]
    ids = [srv.add_sim(w, h, xy) for (w, h, _), xy in zip(SHAPES, xys)]
    # a burst: 120 requests within a few milliseconds, several per simulation,
    # so batches form while others are in flight
    g = np.random.default_rng(3)
    targets = g.choice(ids, size=120)
    arrivals = np.sort(g.uniform(0, 0.004, size=120))
    lat = srv.run_trace(arrivals, targets)
    assert (lat > 0).all()
    st = srv.stats()
    assert st["steps_done"] >= 120 and st["pending"] == 0
    for sim_id, shape, xy in zip(ids, SHAPES, xys):
        n_steps = int((targets == sim_id).sum())
        want = _alone(vd, shape, xy, sim_id, n_steps)
        np.testing.assert_array_equal(srv.labels(sim_id), want, err_msg=f"simulation {sim_id}")
    srv.close()


def test_submit_progress_and_batching(vd):
    srv = vd.VoronoiServer(max_sims=8, hbm_budget_bytes=1 << 30, d_max=D, max_disp=D, rng_seed=RNG)
    ids = [srv.add_sim(w, h, inputs.uniform_seeds(w, h, s, seed=i)) for i, (w, h, s) in enumerate(SHAPES[:4])]
    before = srv.stats()["launches"]
    tickets = [srv.submit(i) for i in ids for _ in range(3)]
    srv.drain()
    t, lat, sims = srv.completions()
    assert sorted(t.tolist()) == sorted(tickets)
    assert (lat >= 0).all()
    # 12 requests over 4 simulations: at most 3 rounds of batches, each a few launches
    assert srv.stats()["launches"] - before < 12 * 4
    srv.close()


def test_admission_by_budget(vd):
    from paper_2209_00117_gb300._native import VD_EBUSY, VD_ENOTFOUND, VDError

    w = h = 512
    one = 2 * 512 * 512 * 4 + 2000 * 16 + 1024  # about one simulation's footprint
    srv = vd.VoronoiServer(max_sims=8, hbm_budget_bytes=int(2.5 * one), d_max=D, max_disp=D)
    a = srv.add_sim(w, h, inputs.uniform_seeds(w, h, 1000, seed=1))
    b = srv.add_sim(w, h, inputs.uniform_seeds(w, h, 1000, seed=2))
    with pytest.raises(VDError) as ei:
        srv.add_sim(w, h, inputs.uniform_seeds(w, h, 1000, seed=3))
    assert ei.value.code == VD_EBUSY
    srv.remove_sim(a)
    with pytest.raises(VDError) as ei:
        srv.submit(a)
    assert ei.value.code == VD_ENOTFOUND
    c = srv.add_sim(w, h, inputs.uniform_seeds(w, h, 1000, seed=3))  # may reuse a's slot
    assert c >= 0
    srv.submit(b)
    srv.submit(c)
    srv.drain()
    srv.close()


def test_serve1000_full_size_sample(vd):
    """The 1000-simulation serving workload at full size under an 80 GB budget:
    a 3000-request Poisson trace at 5000 req/s, then a sample of simulations
    equals the same simulations stepped alone the same number of times."""
    D = 2
    pop = inputs.batched_population(1000, sides=(512, 1024, 2048, 4096), seed=0)
    srv = vd.VoronoiServer(max_sims=1000, hbm_budget_bytes=80 * 10**9, d_max=D, max_disp=D, rng_seed=0)
    xys = {}
    for i, p in enumerate(pop):
        xy = inputs.uniform_seeds(p.w, p.h, p.s, seed=i)
        sid = srv.add_sim(p.w, p.h, xy)
        xys[sid] = (p, xy)
    assert srv.stats()["live_sims"] == 1000
    n = 3000
    arr = inputs.poisson_arrivals(5000, n, seed=5)
    tgt = np.asarray(sorted(xys), np.int32)[inputs.request_targets(n, len(xys), seed=5)]
    lat = srv.run_trace(arr, tgt)
    assert (lat > 0).all()
    for sid in sorted(set(tgt[:200].tolist()))[:6]:
        p, xy = xys[sid]
        sim = vd.VoronoiSim(p.w, p.h, p.s)
        sim.set_seeds(xy)
        sim.jfa()
        for t in range(int((tgt == sid).sum())):
            sim.move(None, max_disp=D, rng_seed=0, stream_id=sid, step=t)
            sim.djfa_step(d_max=D)
        np.testing.assert_array_equal(srv.labels(sid), sim.labels(), err_msg=f"simulation {sid}")
        sim.close()
    srv.close()
