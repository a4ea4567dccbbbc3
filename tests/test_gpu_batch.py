"""The batched engine: many ragged simulations stepped together give exactly
what each gives alone (integer maps, tolerance 0), in both execution modes,
with and without graph replay, for full and subset steps; a forced barrier
timeout is reported without hanging; the autotuner leaves the state intact."""
import numpy as np
import pytest

from paper_2209_00117_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(256, 256, 64), (37, 29, 5), (300, 211, 700), (512, 384, 2000), (64, 1, 3), (1, 1, 1),
          (1024, 512, 8192), (129, 257, 40)]


@pytest.fixture(scope="module")
def vd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00117_gb300 import build

    build.build()
    from paper_2209_00117_gb300 import vd as _vd

    return _vd


def _seeds(shapes, seed):
    return [inputs.uniform_seeds(w, h, s, seed=seed + i) for i, (w, h, s) in enumerate(shapes)]


def _alone_rng(vd, shape, xy, sim_index, steps, D, rng_seed, metric=0):
    w, h, s = shape
    sim = vd.VoronoiSim(w, h, s)
    sim.set_seeds(xy)
    sim.jfa(metric=metric)
    for t in range(steps):
        sim.move(None, max_disp=D, rng_seed=rng_seed, stream_id=sim_index, step=t)
        sim.djfa_step(d_max=D, metric=metric)
    out = sim.labels(), sim.get_seeds()
    sim.close()
    return out


@pytest.mark.parametrize("mode,graphs,rpt,bps,pbyte,minb,packed", [
    (0, 0, 1, 0, 1, 4, -1), (0, 1, 1, 0, 1, 4, -1), (0, 1, 2, 0, 1, 4, -1), (0, 1, 1, 0, 1, 4, 0),
    (1, 0, 1, 0, 1, 4, -1), (1, 0, 4, 0, 1, 4, -1), (1, 0, 1, 2, 1, 4, -1), (1, 0, 2, 3, 1, 4, -1),
    (1, 0, 1, 0, 0, 4, -1), (1, 0, 2, 0, 1, 5, -1), (0, 1, 8, 0, 1, 4, -1), (0, 1, 16, 0, 1, 4, -1)])
def test_batch_equals_alone_rng(vd, mode, graphs, rpt, bps, pbyte, minb, packed):
    """Every launch shape the batch autotuner tries (per-round or persistent,
    rows per thread, persistent blocks per SM) gives each simulation exactly
    its alone run.  Per round, the simulations with up to 32767 seeds and
    small cells run their dJFA frames' last passes on position-tagged words
    (packed = -1), here against alone runs on plain passes (maps below the
    single simulation's 2^21-pixel bound), and also with that off."""
    import torch

    D, steps, rng = 2, 3, 99
    xys = _seeds(SHAPES, 10)
    stream = torch.cuda.Stream()
    b = vd.VoronoiBatch(SHAPES, stream=stream)
    b.set_option(vd.BOPT_MODE, mode)
    b.set_option(vd.BOPT_USE_GRAPHS, graphs)
    b.set_option(vd.BOPT_ROWS_PER_THREAD, rpt)
    b.set_option(vd.BOPT_BLOCKS_PER_SM, bps)
    b.set_option(vd.BOPT_PERSISTENT_BYTE_KEYS, pbyte)
    b.set_option(vd.BOPT_PERSISTENT_MIN_BLOCKS, minb)
    b.set_option(vd.BOPT_PACKED_MAP, packed)
    assert b.get_option(vd.BOPT_PACKED_MAP) == packed
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.configure(d_max=D)
    for _ in range(steps):
        b.step(None, max_disp=D, rng_seed=rng)
    b.synchronize()
    for i, shape in enumerate(SHAPES):
        want_l, want_s = _alone_rng(vd, shape, xys[i], i, steps, D, rng)
        np.testing.assert_array_equal(b.get_seeds(i), want_s)
        np.testing.assert_array_equal(b.labels(i), want_l, err_msg=f"sim {i} {shape}")
    b.close()


def test_batch_given_moves_equal_oracle(vd, orc):
    D, steps = 2, 2
    shapes = SHAPES[:5]
    xys = _seeds(shapes, 20)
    b = vd.VoronoiBatch(shapes)
    b.set_seeds(np.concatenate(xys))
    b.jfa(metric=1)
    b.configure(d_max=D, metric=1)
    labs = [orc.jfa(w, h, xy, metric=1) for (w, h, _), xy in zip(shapes, xys)]
    for t in range(steps):
        moves = [inputs.step_displacements(s, D, t, seed=100 + i) for i, (_, _, s) in enumerate(shapes)]
        b.step(np.concatenate(moves))
        for i, (w, h, _) in enumerate(shapes):
            xys[i] = orc.move(w, h, xys[i], moves[i])
            labs[i] = orc.djfa_step(w, h, xys[i], labs[i], d_max=D, metric=1)
    for i in range(len(shapes)):
        np.testing.assert_array_equal(b.labels(i), labs[i])
    b.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_subset_steps_equal_alone(vd, mode):
    D, rng = 2, 7
    xys = _seeds(SHAPES, 30)
    b = vd.VoronoiBatch(SHAPES)
    b.set_option(vd.BOPT_MODE, mode)
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.configure(d_max=D)
    schedule = [[0, 2, 5], [1, 2, 3, 7], [2], [0, 4, 6, 7, 1]]
    count = [0] * len(SHAPES)
    for subset in schedule:
        b.step_subset(subset, max_disp=D, rng_seed=rng)
        for i in subset:
            count[i] += 1
    for i, shape in enumerate(SHAPES):
        want_l, _ = _alone_rng(vd, shape, xys[i], i, count[i], D, rng)
        np.testing.assert_array_equal(b.labels(i), want_l, err_msg=f"sim {i}")
    b.close()


def test_barrier_timeout_is_reported_and_recoverable(vd):
    from paper_2209_00117_gb300._native import VD_ETIMEOUT, VDError

    shapes = SHAPES[:4]
    xys = _seeds(shapes, 40)
    b = vd.VoronoiBatch(shapes)
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.configure(d_max=2)
    b.set_option(vd.BOPT_MODE, 1)
    b.set_option(vd.BOPT_BARRIER_TIMEOUT_US, 200_000)
    b.set_option(vd.BOPT_TEST_SKIP_ARRIVE, 1)
    b.step(None, max_disp=2, rng_seed=1)
    with pytest.raises(VDError) as ei:
        b.synchronize()
    assert ei.value.code == VD_ETIMEOUT
    # the batch stays usable: recover with a fresh frame 0 and step on
    b.set_option(vd.BOPT_TEST_SKIP_ARRIVE, 0)
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.step(None, max_disp=2, rng_seed=1)
    b.synchronize()
    fresh = vd.VoronoiBatch(shapes)
    fresh.set_seeds(np.concatenate(xys))
    fresh.jfa()
    for i in range(len(shapes)):
        np.testing.assert_array_equal(b.labels(i)[b.labels(i) < 0], fresh.labels(i)[fresh.labels(i) < 0])
        assert (b.labels(i) >= 0).all()
    fresh.close()
    b.close()


def test_autotune_keeps_state(vd):
    D, rng = 2, 5
    xys = _seeds(SHAPES, 50)
    a = vd.VoronoiBatch(SHAPES)
    c = vd.VoronoiBatch(SHAPES)
    for b in (a, c):
        b.set_seeds(np.concatenate(xys))
        b.jfa()
        b.configure(d_max=D)
        b.step(None, max_disp=D, rng_seed=rng)
    best, ms = a.autotune(steps=2, max_disp=D, rng_seed=rng)
    assert 0 <= best < len(ms) and all(m > 0 for m in ms)
    for b in (a, c):
        b.step(None, max_disp=D, rng_seed=rng)
    for i in range(len(SHAPES)):
        np.testing.assert_array_equal(a.labels(i), c.labels(i))
        np.testing.assert_array_equal(a.get_seeds(i), c.get_seeds(i))
    a.close()
    c.close()


def test_batch_rejects_bad_input(vd):
    from paper_2209_00117_gb300._native import VDError

    b = vd.VoronoiBatch([(10, 10, 2), (5, 5, 1)])
    with pytest.raises(VDError):
        b.set_seeds(np.array([[0, 0], [9, 9], [5, 0]], np.int32))  # x = 5 outside the 5-wide grid
    with pytest.raises(VDError):
        b.step(None, max_disp=1)  # not configured
    b.configure(d_max=1)
    with pytest.raises(VDError):
        b.step_subset([0, 0], max_disp=1)
    with pytest.raises(VDError):
        b.step_subset([2], max_disp=1)
    b.close()


@pytest.mark.parametrize("metric", [0, 1])
@pytest.mark.parametrize("clamp", [0, 1])
def test_batch_clamped_and_exact_keys(vd, clamp, metric):
    D, steps, rng = 2, 2, 11
    xys = _seeds(SHAPES, 70)
    b = vd.VoronoiBatch(SHAPES)
    b.set_option(vd.BOPT_CLAMPED_KEYS, clamp)
    b.set_seeds(np.concatenate(xys))
    b.jfa(metric=metric)
    b.configure(d_max=D, metric=metric)
    for _ in range(steps):
        b.step(None, max_disp=D, rng_seed=rng)
    for i, shape in enumerate(SHAPES):
        want_l, _ = _alone_rng(vd, shape, xys[i], i, steps, D, rng, metric=metric)
        np.testing.assert_array_equal(b.labels(i), want_l, err_msg=f"sim {i}")
    b.close()


def test_batched256_full_size_sample(vd):
    """The 256-simulation workload at full size in the benchmarked launch shape
    (per-round launches, graph replay, 4 rows per thread): after a few steps, a
    sample of simulations equals the same simulations run alone."""
    import torch

    D, steps, rng = 2, 3, 0
    pop = inputs.batched_population(256, seed=0)
    shapes = [(p.w, p.h, p.s) for p in pop]
    xys = [inputs.uniform_seeds(w, h, s, seed=i) for i, (w, h, s) in enumerate(shapes)]
    stream = torch.cuda.Stream()
    b = vd.VoronoiBatch(shapes, stream=stream)
    b.set_option(vd.BOPT_ROWS_PER_THREAD, 4)
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.configure(d_max=D)
    for _ in range(steps):
        b.step(None, max_disp=D, rng_seed=rng)
    b.synchronize()
    sample = sorted(set(np.random.default_rng(1).choice(len(shapes), 8, replace=False).tolist()) | {0, 255})
    for i in sample:
        want, _ = _alone_rng(vd, shapes[i], xys[i], i, steps, D, rng)
        np.testing.assert_array_equal(b.labels(i), want, err_msg=f"sim {i} {shapes[i]}")
    b.close()


@pytest.mark.parametrize("metric", [0, 1])
def test_batch_many_labels_equal_oracle(vd, orc, metric):
    """Simulations with more than 2^15 seeds (clamped 32-bit keys in both
    metrics, de-duplicated gathers at a few pixels per seed) next to small ones
    equal the oracle step by step."""
    D, steps = 3, 3
    shapes = [(600, 400, 40000), (512, 512, 70000), (300, 211, 700), (97, 61, 50)]
    xys = _seeds(shapes, 90)
    b = vd.VoronoiBatch(shapes)
    b.set_seeds(np.concatenate(xys))
    b.jfa(metric=metric)
    b.configure(d_max=D, metric=metric)
    labs = [orc.jfa(w, h, xy, metric=metric) for (w, h, _), xy in zip(shapes, xys)]
    for i in range(len(shapes)):
        np.testing.assert_array_equal(b.labels(i), labs[i], err_msg=f"frame 0 sim {i}")
    for t in range(steps):
        moves = [inputs.step_displacements(s, D, t, seed=300 + i) for i, (_, _, s) in enumerate(shapes)]
        b.step(np.concatenate(moves))
        for i, (w, h, _) in enumerate(shapes):
            xys[i] = orc.move(w, h, xys[i], moves[i])
            labs[i] = orc.djfa_step(w, h, xys[i], labs[i], d_max=D, metric=metric)
    for i in range(len(shapes)):
        np.testing.assert_array_equal(b.labels(i), labs[i], err_msg=f"sim {i} {shapes[i]}")
    b.close()


@pytest.mark.parametrize("packed", [-1, 0])
def test_batch_wide_layouts_equal_alone(vd, packed):
    """Simulations whose seed counts take each position-tagged layout in the
    per-round launches -- 8-bit (up to 32767 seeds), 7-bit with the narrow
    first pass (40000), 7-bit with the wide one (100000), 6-bit (200000 and
    2^18, where the last seed's code is also the empty code) -- batched with
    small ones, give exactly their alone runs (maps below the single
    simulation's 2^21-pixel bound, so those run plain passes), and so do
    they with the position-tagged passes off."""
    import torch

    shapes = [(1024, 1024, 40000), (1024, 768, 100000), (1024, 1024, 200000), (1000, 1000, 1 << 18),
              (512, 384, 2000), (37, 29, 5)]
    D, steps, rng = 2, 3, 7
    xys = _seeds(shapes, 40)
    stream = torch.cuda.Stream()
    b = vd.VoronoiBatch(shapes, stream=stream)
    b.set_option(vd.BOPT_PACKED_MAP, packed)
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.configure(d_max=D)
    for _ in range(steps):
        b.step(None, max_disp=D, rng_seed=rng)
    b.synchronize()
    for i, shape in enumerate(shapes):
        want_l, want_s = _alone_rng(vd, shape, xys[i], i, steps, D, rng)
        np.testing.assert_array_equal(b.get_seeds(i), want_s)
        np.testing.assert_array_equal(b.labels(i), want_l, err_msg=f"sim {i} {shape}")
    b.close()
