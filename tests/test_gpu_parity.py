"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

All arithmetic is integer (exact squared distances, lowest-index ties), so every
comparison is bit-exact: tolerance 0.  Sizes span several tiles and ragged
edges (widths not a multiple of 4 or 32, odd heights), the degenerate grids
(1 x 1, 1 x N, N x 1), coinciding seeds, and the full 2048 x 2048, 16384-seed
workload in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

from paper_2209_00117_gb300 import inputs

pytestmark = pytest.mark.gpu

E, L1 = 0, 1
M, VN = 0, 1


@pytest.fixture(scope="module")
def vd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00117_gb300 import build

    build.build()
    from paper_2209_00117_gb300 import vd as _vd

    return _vd


def _sim(vd, w, h, xy, **opts):
    sim = vd.VoronoiSim(w, h, len(xy))
    sim.set_seeds(np.ascontiguousarray(xy, np.int32))
    for k, v in opts.items():
        sim.set_option(getattr(vd, "OPT_" + k.upper()), v)
    return sim


SHAPES = [(1, 1), (1, 9), (13, 1), (5, 3), (37, 29), (64, 64), (100, 37), (257, 129), (300, 200)]


@pytest.mark.parametrize("clamp,dedup", [(-1, -1), (1, 1), (0, 1)])
@pytest.mark.parametrize("w,h", SHAPES)
def test_single_pass_matches_oracle(vd, orc, w, h, clamp, dedup):
    """One pass at every kind of step (vector, k = 1, 2, scalar), both
    neighbourhoods and metrics, in the default, forced 32-bit and forced exact
    key forms with and without de-duplicated gathers, over random maps."""
    g = np.random.default_rng(w * 1000 + h)
    s = max(1, min(40, w * h // 3))
    xy = inputs.uniform_seeds(w, h, s, seed=w + h)
    src = g.integers(-1, s, size=(h, w), dtype=np.int32)
    sim = _sim(vd, w, h, xy, clamped_keys=clamp, dedup_gathers=dedup)
    for k in [1, 2, 3, 4, 5, 6, 8, 12, 16, 64, 256, 1024]:
        for nb in [M, VN]:
            for metric in [E, L1]:
                sim.set_labels(src)
                sim.jump_pass(k, nb, metric)
                want = orc.jump_pass(w, h, xy, src, k, nb, metric)
                got = sim.labels()
                assert np.array_equal(got, want), (k, nb, metric, int((got != want).sum()))
    sim.close()


@pytest.mark.parametrize("fuse", [0, 2, 4, 8, 16])
@pytest.mark.parametrize("w,h,s", [(37, 29, 7), (257, 129, 60), (300, 200, 500), (640, 480, 100)])
def test_jfa_frame_fused_and_unfused(vd, orc, fuse, w, h, s):
    xy = inputs.uniform_seeds(w, h, s, seed=s)
    xy[s // 2] = xy[0]  # coinciding seeds
    for metric in [E, L1]:
        want = orc.jfa(w, h, xy, metric=metric)
        for tile in [(64, 32), (32, 8), (128, 16)]:
            sim = _sim(vd, w, h, xy, fuse_max_k=fuse, fuse_tile_x=tile[0], fuse_tile_y=tile[1])
            sim.jfa(metric=metric)
            got = sim.labels()
            assert np.array_equal(got, want), (fuse, tile, metric, int((got != want).sum()))
            sim.close()


@pytest.mark.parametrize("extra", [0, 1, 2])
def test_jfa_extra_passes(vd, orc, extra):
    w, h, s = 333, 222, 90
    xy = inputs.uniform_seeds(w, h, s, seed=3)
    sim = _sim(vd, w, h, xy)
    sim.jfa(extra=extra)
    np.testing.assert_array_equal(sim.labels(), orc.jfa(w, h, xy, extra=extra))
    sim.close()


@pytest.mark.parametrize("metric", [E, L1])
@pytest.mark.parametrize("w,h,s", [(333, 222, 300), (2048, 1024, 20000)])
def test_djfa_extra_passes(vd, orc, metric, w, h, s):
    """The optional extra step after Eq. 4's schedule (Section V-A) and the
    JFA+1/+2 idea of Section III on dJFA frames: vd_djfa_step, eager vd_step
    and graph-replayed vd_step with extra in {1, 2} (the graph cache must key
    on it: the extra count changes from step to step) against the oracle's
    dJFA chain, both metrics.  The larger map takes the byte-offset key."""
    D = 3
    xy = inputs.uniform_seeds(w, h, s, seed=s + 7)
    extras = [1, 2, 1, 0, 2]
    disp = inputs.displacements(s, D, len(extras), seed=s + 7)
    a = _sim(vd, w, h, xy)
    b = _sim(vd, w, h, xy, use_graphs=0)
    c = _sim(vd, w, h, xy, use_graphs=1)
    for sim in (a, b, c):
        sim.jfa(metric=metric)
    lab = orc.jfa(w, h, xy, metric=metric)
    for t, extra in enumerate(extras):
        a.move(disp[t])
        a.djfa_step(d_max=D, extra=extra, metric=metric)
        b.step(disp[t], d_max=D, extra=extra, metric=metric)
        c.step(disp[t], d_max=D, extra=extra, metric=metric)
        xy = orc.move(w, h, xy, disp[t])
        lab = orc.djfa_step(w, h, xy, lab, d_max=D, extra=extra, metric=metric)
        for name, sim in (("djfa_step", a), ("step", b), ("step+graph", c)):
            got = sim.labels()
            assert np.array_equal(got, lab), (name, t, extra, int((got != lab).sum()))
    for sim in (a, b, c):
        sim.close()


def test_degenerate_grids(vd, orc):
    for w, h, s in [(1, 1, 1), (1, 1, 5), (1, 50, 3), (70, 1, 4), (2, 2, 9), (3, 5, 15)]:
        xy = inputs.uniform_seeds(w, h, s, seed=w * 7 + h)
        sim = _sim(vd, w, h, xy)
        sim.jfa()
        np.testing.assert_array_equal(sim.labels(), orc.jfa(w, h, xy))
        prev = sim.labels()
        sim.djfa_step(d_max=1)
        np.testing.assert_array_equal(sim.labels(), orc.djfa_step(w, h, xy, prev, d_max=1))
        sim.close()


def test_all_seeds_on_one_pixel(vd, orc):
    w, h, s = 91, 47, 33
    xy = np.tile(np.array([[40, 20]], np.int32), (s, 1))
    sim = _sim(vd, w, h, xy)
    sim.jfa()
    lab = sim.labels()
    assert (lab == 0).all()
    sim.close()


def test_stamp_collisions_lowest_index(vd, orc):
    w, h = 64, 40
    g = np.random.default_rng(0)
    xy = inputs.uniform_seeds(8, 5, 300, seed=1)  # many collisions in an 8 x 5 corner
    prev = g.integers(0, 300, size=(h, w), dtype=np.int32)
    sim = _sim(vd, w, h, xy)
    sim.set_labels(prev)
    sim.stamp()
    np.testing.assert_array_equal(sim.labels(), orc.stamp(w, h, xy, prev))
    sim.close()


@pytest.mark.parametrize("case", ["one_pixel", "stale_seed_labels", "empty_and_large"])
def test_stamp_swap_and_restore(vd, orc, case):
    """The stamp on a map with stale labels takes one swap a seed and puts a
    lower index back when its seed stands on the same pixel: every seed on
    one pixel (the chain of swaps is as long as it gets), stale labels that
    name seeds now standing on the pixel (the label taken out by the first
    swap is itself a seed there), and a map of empty labels with 200000
    seeds on 64 x 64 pixels; each equal to the oracle's stamp."""
    w, h = 64, 40
    g = np.random.default_rng(7)
    if case == "one_pixel":
        n = 5000
        xy = np.tile(np.array([[3, 2]], np.int32), (n, 1))
        prev = g.integers(0, n, size=(h, w), dtype=np.int32)
    elif case == "stale_seed_labels":
        n = 2000
        xy = inputs.uniform_seeds(6, 4, n, seed=3)
        # every pixel of the corner names one of the seeds now standing on it
        prev = g.integers(0, n, size=(h, w), dtype=np.int32)
        for k in range(n - 1, -1, -1):
            prev[xy[k, 1], xy[k, 0]] = k if k % 3 else prev[xy[k, 1], xy[k, 0]]
    else:
        w, h, n = 64, 64, 200000
        xy = inputs.uniform_seeds(w, h, n, seed=5)
        prev = np.full((h, w), -1, np.int32)
    sim = _sim(vd, w, h, xy)
    for _ in range(2):
        sim.set_labels(prev)
        sim.stamp()
        np.testing.assert_array_equal(sim.labels(), orc.stamp(w, h, xy, prev))
    sim.close()


def test_move_given_and_rng(vd, orc):
    w, h, s = 500, 300, 4000
    xy = inputs.uniform_seeds(w, h, s, seed=2)
    sim = _sim(vd, w, h, xy)
    d = inputs.displacements(s, 40, 1, seed=2)[0]
    sim.move(d)
    cur = orc.move(w, h, xy, d)
    np.testing.assert_array_equal(sim.get_seeds(), cur)
    for step in range(3):
        sim.move(None, max_disp=7, rng_seed=12345, stream_id=9, step=step)
        cur = orc.move_rng(w, h, cur, 7, 12345, 9, step)
        np.testing.assert_array_equal(sim.get_seeds(), cur)
    sim.close()


@pytest.mark.parametrize("metric", [E, L1])
def test_single256_trajectory(vd, orc, metric):
    """The 256 x 256, 64-seed, 10-step workload: every frame of JFA and of the
    dJFA chain bit-exact, and the distance-correct counts equal."""
    w, h, s, steps, D = inputs.SINGLE["single256"]
    xy = inputs.uniform_seeds(w, h, s, seed=0)
    disp = inputs.displacements(s, D, steps, seed=0)
    dj = _sim(vd, w, h, xy)
    jf = _sim(vd, w, h, xy)
    dj.jfa(metric=metric)
    lab = orc.jfa(w, h, xy, metric=metric)
    np.testing.assert_array_equal(dj.labels(), lab)
    for t in range(steps):
        dj.move(disp[t])
        jf.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        dj.djfa_step(d_max=D, vn_waves=2, metric=metric)
        jf.jfa(metric=metric)
        lab = orc.djfa_step(w, h, xy, lab, d_max=D, vn_waves=2, metric=metric)
        ref = orc.jfa(w, h, xy, metric=metric)
        assert np.array_equal(dj.labels(), lab), t
        assert np.array_equal(jf.labels(), ref), t
        ed = orc.exact_dist_edt(w, h, xy, metric)
        assert dj.similarity(exact_dist=ed, ref_labels=ref, metric=metric) == \
            orc.similarity(w, h, xy, lab, exact_dist=ed, ref_label=ref, metric=metric)
        assert dj.match_count(jf) == orc.similarity(w, h, xy, lab, ref_label=ref)[1]
    dj.close()
    jf.close()


def test_graphs_and_band_order_equal_eager(vd, orc):
    import torch

    w, h, s = 1024, 768, 3000
    xy = inputs.uniform_seeds(w, h, s, seed=5)
    disp = inputs.displacements(s, 2, 4, seed=5)
    stream = torch.cuda.Stream()
    a = _sim(vd, w, h, xy)
    b = _sim(vd, w, h, xy, use_graphs=1, band_order_min_k=8)
    b.set_stream(stream)
    a.jfa()
    b.jfa()
    np.testing.assert_array_equal(a.labels(), b.labels())
    for t in range(4):
        for sim in (a, b):
            sim.move(disp[t])
            sim.djfa_step(d_max=2)
        np.testing.assert_array_equal(a.labels(), b.labels())
        b.jfa()
        a.jfa()
        np.testing.assert_array_equal(a.labels(), b.labels())
    np.testing.assert_array_equal(a.labels(), orc.jfa(w, h, orc.move(w, h, a.get_seeds(), np.zeros((s, 2), np.int32))))
    a.close()
    b.close()


@pytest.mark.parametrize("w,h,s", [(1, 1, 1), (17, 9, 3), (200, 150, 1), (256, 256, 64),
                                   (300, 211, 2000), (512, 512, 40000)])
def test_exact_diagram_matches_brute_force(vd, orc, w, h, s):
    xy = inputs.uniform_seeds(w, h, s, seed=s)
    xy[-1] = xy[0]
    sim = _sim(vd, w, h, xy)
    for metric in [E, L1]:
        lab, dist = sim.exact(metric=metric)
        want_l, want_d = orc.exact_brute(w, h, xy, metric)
        np.testing.assert_array_equal(dist, want_d)
        np.testing.assert_array_equal(lab, want_l)
    sim.close()


def test_single2048_full_size(vd, orc):
    """The 2048 x 2048, 16384-seed, [-2, 2] workload in the benchmark's launch
    configuration: frame 0 (JFA) and a chain of dJFA steps bit-exact against
    the oracle, similarity counts equal, distance-correct count vs the EDT."""
    import torch

    w, h, s, _, D = inputs.SINGLE["single2048"]
    steps = 4
    xy = inputs.uniform_seeds(w, h, s, seed=0)
    disp = inputs.displacements(s, D, steps, seed=0)
    stream = torch.cuda.Stream()
    sim = _sim(vd, w, h, xy, use_graphs=1)
    sim.set_stream(stream)
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    for t in range(steps):
        sim.move(disp[t])
        sim.djfa_step(d_max=D, vn_waves=2)
        xy = orc.move(w, h, xy, disp[t])
        lab = orc.djfa_step(w, h, xy, lab, d_max=D, vn_waves=2)
        got = sim.labels()
        assert np.array_equal(got, lab), (t, int((got != lab).sum()))
    ed = orc.exact_dist_edt(w, h, xy)
    _, gpu_d = sim.exact()
    np.testing.assert_array_equal(gpu_d, ed)
    ref = orc.jfa(w, h, xy)
    assert sim.similarity(exact_dist=ed, ref_labels=ref) == orc.similarity(w, h, xy, lab, exact_dist=ed, ref_label=ref)
    sim.close()


@pytest.mark.parametrize("s,D,metric", [(1 << 14, 4, E), (1 << 22, 16, E), (1 << 22, 16, L1)])
def test_sweep8192_first_frames(vd, orc, s, D, metric):
    """8192 x 8192 sweep points: JFA frame 0 and dJFA frame 1 bit-exact."""
    w = h = inputs.SWEEP8192["side"]
    xy = inputs.uniform_seeds(w, h, s, seed=1)
    disp = inputs.displacements(s, D, 1, seed=1)[0]
    sim = _sim(vd, w, h, xy)
    sim.jfa(metric=metric)
    lab = orc.jfa(w, h, xy, metric=metric)
    assert np.array_equal(sim.labels(), lab)
    sim.move(disp)
    sim.djfa_step(d_max=D, metric=metric)
    xy = orc.move(w, h, xy, disp)
    lab = orc.djfa_step(w, h, xy, lab, d_max=D, metric=metric)
    assert np.array_equal(sim.labels(), lab)
    sim.close()


def test_sweep8192_frame49(vd, orc):
    """8192 x 8192, 2^18 seeds, D = 4 (de-duplicated gathers, clamped keys, 6
    passes a frame): the dJFA chain stays bit-exact through frame 49, the last
    frame of a 50-step sweep run, with counter-based moves on both sides."""
    w = h = inputs.SWEEP8192["side"]
    s, D, rng = 1 << 18, 4, 2209
    xy = inputs.uniform_seeds(w, h, s, seed=49)
    sim = _sim(vd, w, h, xy, use_graphs=1)
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    for t in range(49):
        sim.move(None, max_disp=D, rng_seed=rng, stream_id=0, step=t)
        sim.djfa_step(d_max=D)
        xy = orc.move_rng(w, h, xy, D, rng, 0, t)
        lab = orc.djfa_step(w, h, xy, lab, d_max=D)
    np.testing.assert_array_equal(sim.get_seeds(), xy)
    assert np.array_equal(sim.labels(), lab)
    sim.close()


def test_invalid_arguments(vd):
    from paper_2209_00117_gb300._native import VDError

    sim = vd.VoronoiSim(10, 10, 3)
    with pytest.raises(VDError):
        sim.set_seeds(np.array([[0, 0], [10, 0], [1, 1]], np.int32))
    with pytest.raises(VDError):
        sim.set_labels(np.full((10, 10), 3, np.int32))
    with pytest.raises(VDError):
        sim.djfa_step(d_max=-1)
    with pytest.raises(VDError):
        sim.jfa(metric=7)
    with pytest.raises(VDError):
        sim.set_option(vd.OPT_FUSE_MAX_K, 99)
    with pytest.raises(VDError):
        sim.jump_pass(0)
    import torch

    bad = torch.tensor([[0, 0], [3, 30], [1, 1]], dtype=torch.int32, device="cuda")
    with pytest.raises(VDError):
        sim.set_seeds(bad)
    sim.close()


@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("metric", [E, L1])
@pytest.mark.parametrize("clamp", [0, 1])
@pytest.mark.parametrize("w,h,s", [(37, 29, 12), (300, 200, 500), (257, 129, 9), (640, 480, 5000), (64, 64, 8),
                                   (512, 256, 40000)])
def test_clamped_and_exact_keys(vd, orc, clamp, metric, dedup, w, h, s):
    """Both key forms (forced), with and without de-duplicated gathers, give
    the oracle's maps: single passes over random maps with empty labels and
    ragged edges, JFA frames and dJFA steps."""
    g = np.random.default_rng(s)
    xy = inputs.uniform_seeds(w, h, s, seed=s + 1)
    xy[-1] = xy[0]
    sim = _sim(vd, w, h, xy, clamped_keys=clamp, dedup_gathers=dedup)
    src = g.integers(-1, s, size=(h, w), dtype=np.int32)
    for k in [1, 2, 4, 16, 128]:
        for nb in [M, VN]:
            sim.set_labels(src)
            sim.jump_pass(k, nb, metric)
            np.testing.assert_array_equal(sim.labels(), orc.jump_pass(w, h, xy, src, k, nb, metric),
                                          err_msg=f"k={k}")
    sim.jfa(metric=metric)
    lab = orc.jfa(w, h, xy, metric=metric)
    np.testing.assert_array_equal(sim.labels(), lab)
    disp = inputs.displacements(s, 3, 3, seed=s)
    for t in range(3):
        sim.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        sim.djfa_step(d_max=3, metric=metric)
        lab = orc.djfa_step(w, h, xy, lab, d_max=3, metric=metric)
        np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"step {t}")
    sim.close()


def test_checkpoint_resume_is_bit_identical(vd):
    """State = (seeds, label map, RNG step): saving it mid-run and resuming in a
    fresh context continues the trajectory exactly (counter-based moves)."""
    w, h, s, D, rng = 700, 500, 3000, 3, 77
    xy = inputs.uniform_seeds(w, h, s, seed=8)
    a = _sim(vd, w, h, xy)
    a.jfa()
    for t in range(5):
        a.move(None, max_disp=D, rng_seed=rng, stream_id=0, step=t)
        a.djfa_step(d_max=D)
    seeds, labels = a.get_seeds(), a.labels()
    for t in range(5, 10):
        a.move(None, max_disp=D, rng_seed=rng, stream_id=0, step=t)
        a.djfa_step(d_max=D)
    b = _sim(vd, w, h, seeds)
    b.set_labels(labels)
    for t in range(5, 10):
        b.move(None, max_disp=D, rng_seed=rng, stream_id=0, step=t)
        b.djfa_step(d_max=D)
    np.testing.assert_array_equal(a.get_seeds(), b.get_seeds())
    np.testing.assert_array_equal(a.labels(), b.labels())
    a.close()
    b.close()


def test_async_label_readback(vd):
    """Pipelined read-back: every frame's map lands in its own host buffer while
    later frames run, equal to the synchronous read of that frame."""
    import torch

    w, h, s, D = 600, 400, 2500, 2
    xy = inputs.uniform_seeds(w, h, s, seed=12)
    disp = inputs.displacements(s, D, 6, seed=12)
    a = _sim(vd, w, h, xy)
    b = _sim(vd, w, h, xy)
    a.jfa()
    b.jfa()
    outs = [torch.empty((h, w), dtype=torch.int32).pin_memory() for _ in range(6)]
    want = []
    for t in range(6):
        for sim in (a, b):
            sim.move(disp[t])
            sim.djfa_step(d_max=D)
        a.labels_async(outs[t])  # up to two in flight; the third call waits for the oldest
        want.append(b.labels())
    a.wait_labels()
    for t in range(6):
        np.testing.assert_array_equal(outs[t].numpy(), want[t], err_msg=f"frame {t}")
    a.close()
    b.close()


@pytest.mark.parametrize("w,h,s", [(601, 403, 2500), (1000, 70, 65535), (33, 5, 9)])
def test_async_label_readback_16bit(vd, w, h, s):
    """The 16-bit read-back: every frame's dense map, interleaved with 32-bit
    read-backs through the same two slots, equals the synchronous int32 read
    (empty labels as 0xFFFF; odd widths; the largest seed count it takes)."""
    import torch

    D = 2
    xy = inputs.uniform_seeds(w, h, s, seed=13)
    disp = inputs.displacements(s, D, 5, seed=13)
    a = _sim(vd, w, h, xy)
    b = _sim(vd, w, h, xy)
    # frame 0: a map with empty labels
    src = np.random.default_rng(s).integers(-1, s, size=(h, w), dtype=np.int32)
    a.set_labels(src)
    b.set_labels(src)
    o16 = [torch.empty((h, w), dtype=torch.int16).pin_memory() for _ in range(6)]
    o32 = [torch.empty((h, w), dtype=torch.int32).pin_memory() for _ in range(6)]
    want = []
    for t in range(6):
        if t:
            for sim in (a, b):
                sim.move(disp[t - 1])
                sim.djfa_step(d_max=D)
        a.labels16_async(o16[t])
        a.labels_async(o32[t])
        want.append(b.labels())
    a.wait_labels()
    for t in range(6):
        got = o16[t].numpy().view(np.uint16).astype(np.int64)
        exp = want[t].astype(np.int64)
        exp[exp == -1] = 0xFFFF
        np.testing.assert_array_equal(got, exp, err_msg=f"frame {t}")
        np.testing.assert_array_equal(o32[t].numpy(), want[t], err_msg=f"frame {t}")
    arr = np.empty((h, w), np.uint16)
    a.labels16_async(arr)
    a.wait_labels()
    np.testing.assert_array_equal(arr.astype(np.int64), exp)
    a.close()
    b.close()


@pytest.mark.parametrize("w,h,s", [(600, 400, 2500), (601, 403, 70000), (1024, 512, 1 << 18), (33, 5, 9)])
def test_async_label_readback_24bit(vd, w, h, s):
    """The 24-bit read-back: every frame's dense map (three little-endian bytes
    a label), interleaved with 32-bit read-backs through the same two slots,
    equals the synchronous int32 read: empty labels as 0xFFFFFF, widths a
    multiple of 4 (four labels packed into three words) and not (byte
    stores), seed counts beyond 16 bits."""
    import torch

    D = 2
    xy = inputs.uniform_seeds(w, h, s, seed=17)
    disp = inputs.displacements(s, D, 5, seed=17)
    a = _sim(vd, w, h, xy)
    b = _sim(vd, w, h, xy)
    src = np.random.default_rng(s + 1).integers(-1, s, size=(h, w), dtype=np.int32)
    a.set_labels(src)
    b.set_labels(src)
    o24 = [torch.empty(3 * h * w, dtype=torch.uint8).pin_memory() for _ in range(6)]
    o32 = [torch.empty((h, w), dtype=torch.int32).pin_memory() for _ in range(6)]
    want = []
    for t in range(6):
        if t:
            for sim in (a, b):
                sim.move(disp[t - 1])
                sim.djfa_step(d_max=D)
        a.labels24_async(o24[t])
        a.labels_async(o32[t])
        want.append(b.labels())
    a.wait_labels()
    for t in range(6):
        raw = o24[t].numpy().reshape(h * w, 3).astype(np.int64)
        packed = raw[:, 0] | (raw[:, 1] << 8) | (raw[:, 2] << 16)
        exp = want[t].astype(np.int64).reshape(-1)
        exp[exp == -1] = 0xFFFFFF
        np.testing.assert_array_equal(packed, exp, err_msg=f"frame {t}")
        np.testing.assert_array_equal(vd.widen24(o24[t].numpy(), h, w), want[t], err_msg=f"frame {t}")
        np.testing.assert_array_equal(o32[t].numpy(), want[t], err_msg=f"frame {t}")
    arr = np.empty(3 * h * w, np.uint8)
    a.labels24_async(arr)
    a.wait_labels()
    np.testing.assert_array_equal(vd.widen24(arr, h, w), want[-1])
    a.close()
    b.close()


def test_async_label_readback_24bit_refuses_large_counts(vd):
    """From 2^24 seeds on a label no longer fits 24 bits: VD_EINVAL."""
    from paper_2209_00117_gb300._native import VD_EINVAL, VDError

    w, h, s = 64, 64, 1 << 24
    sim = vd.VoronoiSim(w, h, s)
    with pytest.raises(VDError) as ei:
        sim.labels24_async(np.empty(3 * h * w, np.uint8))
    assert ei.value.code == VD_EINVAL
    sim.close()


@pytest.mark.parametrize("w,h,s,extra", [(600, 400, 2500, 0), (601, 403, 70000, 0), (1024, 512, 1 << 18, 0),
                                         (33, 5, 9, 0), (64, 40, 7, 27), (96, 30, 100, 25)])
def test_async_label_readback_packed(vd, w, h, s, extra):
    """The packed read-back at the fewest bits for the seed count (plus
    `extra`, up to 32 bits a label): every frame's bit stream, interleaved
    with 32-bit read-backs through the same two slots, equals the
    synchronous int32 read, unpacked on the host and checked bit by bit
    against a plain bit-by-bit packing of that read (empty labels as all
    ones): widths a multiple of 32 (one row a thread) and not (labels of a
    thread across rows), a stream ending inside a word."""
    import torch

    bits = vd.label_bits(s) + extra
    D = 2
    xy = inputs.uniform_seeds(w, h, s, seed=19)
    disp = inputs.displacements(s, D, 4, seed=19)
    a = _sim(vd, w, h, xy)
    b = _sim(vd, w, h, xy)
    src = np.random.default_rng(s + 3).integers(-1, s, size=(h, w), dtype=np.int32)
    a.set_labels(src)
    b.set_labels(src)
    nbytes = (w * h * bits + 7) // 8
    op = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(5)]
    o32 = [torch.empty((h, w), dtype=torch.int32).pin_memory() for _ in range(5)]
    want = []
    for t in range(5):
        if t:
            for sim in (a, b):
                sim.move(disp[t - 1])
                sim.djfa_step(d_max=D)
        a.labels_packed_async(op[t], bits)
        a.labels_async(o32[t])
        want.append(b.labels())
    a.wait_labels()
    for t in range(5):
        np.testing.assert_array_equal(vd.unpack_labels(op[t].numpy(), h, w, bits, rows_per_chunk=7), want[t],
                                      err_msg=f"frame {t}")
        np.testing.assert_array_equal(o32[t].numpy(), want[t], err_msg=f"frame {t}")
    # bit-exact stream on the last frame against an independent packing
    codes = want[-1].astype(np.int64).reshape(-1) & ((1 << bits) - 1)
    bitplanes = ((codes[:, None] >> np.arange(bits)) & 1).astype(np.uint8).reshape(-1)
    ref = np.packbits(bitplanes, bitorder="little")
    np.testing.assert_array_equal(op[-1].numpy(), ref)
    a.close()
    b.close()


def test_async_label_readback_packed_refuses(vd):
    """A width that cannot hold every label apart from the empty code, or one
    outside [1, 32]: VD_EINVAL before anything is queued."""
    from paper_2209_00117_gb300._native import VD_EINVAL, VDError

    w, h, s = 64, 64, 1 << 10
    sim = vd.VoronoiSim(w, h, s)
    from paper_2209_00117_gb300 import _native as N

    for bits in (10, 0, 33):
        buf = np.empty((w * h * 32 + 7) // 8, np.uint8)
        with pytest.raises(VDError) as ei:
            N.check(sim._lib.vd_get_labels_packed_async(sim._h, buf.ctypes.data, bits))
        assert ei.value.code == VD_EINVAL
    out = np.empty((w * h * 11 + 7) // 8, np.uint8)
    sim.labels_packed_async(out, 11)
    sim.wait_labels()
    sim.close()


def test_async_label_readback_16bit_refuses_large_counts(vd):
    """From 65536 seeds on a label no longer fits 16 bits: VD_EINVAL."""
    from paper_2209_00117_gb300._native import VD_EINVAL, VDError

    w, h, s = 300, 256, 65536
    sim = _sim(vd, w, h, inputs.uniform_seeds(w, h, s, seed=1))
    with pytest.raises(VDError) as ei:
        sim.labels16_async(np.empty((h, w), np.uint16))
    assert ei.value.code == VD_EINVAL
    sim.close()


@pytest.mark.parametrize("w,h", [(32768, 8), (8, 32768), (32768, 3)])
def test_maximum_side_grids(vd, orc, w, h):
    """Grids at the maximum side (coordinates up to 32767, squared distances up
    to 2^30, steps up to 16384): JFA and a dJFA step in both key forms and both
    metrics equal the oracle."""
    s = 300
    xy = inputs.uniform_seeds(w, h, s, seed=w + h)
    disp = inputs.displacements(s, 5, 1, seed=1)[0]
    for metric in [E, L1]:
        for clamp in [0, 1]:
            sim = _sim(vd, w, h, xy, clamped_keys=clamp)
            sim.jfa(metric=metric)
            lab = orc.jfa(w, h, xy, metric=metric)
            np.testing.assert_array_equal(sim.labels(), lab)
            sim.move(disp)
            xy2 = orc.move(w, h, xy, disp)
            sim.djfa_step(d_max=5, metric=metric)
            np.testing.assert_array_equal(sim.labels(), orc.djfa_step(w, h, xy2, lab, d_max=5, metric=metric))
            sim.close()


@pytest.mark.parametrize("graphs", [0, 1])
def test_dependent_launch_chain_matches_oracle(vd, orc, graphs):
    """Frames whose stamp and pass kernels are chained with programmatic
    dependent launch (the default) equal plain stream order and the oracle,
    eagerly and from graphs, on a side stream, for both metrics."""
    import torch

    w, h, s, D = 2048, 1536, 9000, 3
    xy = inputs.uniform_seeds(w, h, s, seed=77)
    disp = inputs.displacements(s, D, 3, seed=77)
    stream = torch.cuda.Stream()
    on = _sim(vd, w, h, xy, use_graphs=graphs, pdl=1)
    off = _sim(vd, w, h, xy, use_graphs=graphs, pdl=0)
    on.set_stream(stream)
    assert on.get_option(vd.OPT_PDL) == 1 and off.get_option(vd.OPT_PDL) == 0
    for metric in [E, L1]:
        on.set_seeds(xy)
        off.set_seeds(xy)
        on.jfa(metric=metric)
        off.jfa(metric=metric)
        lab = orc.jfa(w, h, xy, metric=metric)
        np.testing.assert_array_equal(on.labels(), lab)
        np.testing.assert_array_equal(off.labels(), lab)
        cur = xy
        for t in range(3):
            cur = orc.move(w, h, cur, disp[t])
            lab = orc.djfa_step(w, h, cur, lab, d_max=D, metric=metric)
            for sim in (on, off):
                sim.move(disp[t])
                sim.djfa_step(d_max=D, metric=metric)
            np.testing.assert_array_equal(on.labels(), lab)
            np.testing.assert_array_equal(off.labels(), lab)
    on.close()
    off.close()


@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("moves", ["host", "device", "rng"])
def test_step_equals_move_then_frame(vd, orc, graphs, moves):
    """vd_step (the move with the stamp's first half folded in, one graph per
    step) equals vd_move_seeds + vd_djfa_step and the oracle, across buffer
    parities, a seed update (repair frame) and both metrics."""
    import torch

    w, h, s, D = 700, 500, 3000, 3
    xy = inputs.uniform_seeds(w, h, s, seed=31)
    a = _sim(vd, w, h, xy, use_graphs=graphs)
    b = _sim(vd, w, h, xy, use_graphs=graphs)
    a.jfa()
    b.jfa()
    lab = orc.jfa(w, h, xy)
    g = np.random.default_rng(4)
    for t in range(8):
        metric = E if t < 5 else L1
        if t == 3:  # a seed update: the next frame is the repair frame
            remove = g.choice(len(xy), 40, replace=False).astype(np.int32)
            add = np.stack([g.integers(0, w, 25), g.integers(0, h, 25)], axis=1).astype(np.int32)
            for sim in (a, b):
                sim.update_seeds(remove, add)
            xy, lab = orc.update_seeds(w, h, xy, lab, remove, add)
        n = len(xy)
        if moves == "rng":
            a.step(None, max_disp=D, rng_seed=9, stream_id=0, step=t, d_max=D, metric=metric)
            b.move(None, max_disp=D, rng_seed=9, stream_id=0, step=t)
            xy = orc.move_rng(w, h, xy, D, 9, 0, t)
        else:
            d = inputs.step_displacements(n, D, t, seed=5)
            dd = torch.from_numpy(d).cuda() if moves == "device" else d
            a.step(dd, d_max=D, metric=metric)
            b.move(dd)
            xy = orc.move(w, h, xy, d)
        b.djfa_step(d_max=D, metric=metric)
        lab = orc.repair_step(w, h, xy, lab, metric=metric) if t == 3 else \
            orc.djfa_step(w, h, xy, lab, d_max=D, metric=metric)
        np.testing.assert_array_equal(a.labels(), lab, err_msg=f"step {t}")
        np.testing.assert_array_equal(b.labels(), lab, err_msg=f"step {t}")
        np.testing.assert_array_equal(a.get_seeds(), xy)
    a.close()
    b.close()


@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("w,h,s", [(37, 29, 12), (100, 37, 16), (64, 64, 16), (257, 129, 9), (300, 200, 500),
                                   (512, 512, 16384), (512, 256, 65535), (512, 256, 65536),
                                   (2048, 1024, 1 << 20)])
def test_byte_offset_keys(vd, orc, dedup, w, h, s):
    """The byte-offset key form, forced on every Euclidean pass, gives the
    oracle's maps.  Random maps with empty labels put the far position and
    seeds far outside the key window among the candidates (winners there are
    recomputed); maps of real labels only, JFA frames and dJFA steps exercise
    the unchecked path.  65535 seeds fill the 16-bit label field up to the
    empty-label code; 65536 and 2^20 seeds run the wide form (17- and 21-bit
    label fields, windows of half-width 64 and 16).  Widths not a multiple of
    32 read the row padding."""
    g = np.random.default_rng(s + w)
    xy = inputs.uniform_seeds(w, h, s, seed=s + 3)
    sim = _sim(vd, w, h, xy, byte_keys=1, dedup_gathers=dedup)
    for lo in (-1, 0):
        src = g.integers(lo, s, size=(h, w), dtype=np.int32)
        for k in [1, 2, 3, 4, 8, 16, 128]:
            for nb in [M, VN]:
                sim.set_labels(src)
                sim.jump_pass(k, nb, E)
                np.testing.assert_array_equal(sim.labels(), orc.jump_pass(w, h, xy, src, k, nb, E),
                                              err_msg=f"k={k} nb={nb} lo={lo}")
    # a smooth map (the previous JFA frame) with every candidate near its seed
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    for k in [16, 4, 1]:
        sim.set_labels(lab)
        sim.jump_pass(k, M, E)
        np.testing.assert_array_equal(sim.labels(), orc.jump_pass(w, h, xy, lab, k, M, E), err_msg=f"k={k}")
    sim.set_labels(lab)  # the dJFA chain starts from the JFA frame, like the oracle's
    disp = inputs.displacements(s, 2, 2, seed=s)
    for t in range(2):
        sim.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        sim.djfa_step(d_max=2)
        lab = orc.djfa_step(w, h, xy, lab, d_max=2)
        np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"step {t}")
    # the flag leaves Manhattan passes on their own key forms
    sim.set_labels(src)
    sim.jump_pass(4, M, L1)
    np.testing.assert_array_equal(sim.labels(), orc.jump_pass(w, h, xy, src, 4, M, L1))
    sim.close()


@pytest.mark.parametrize("pack,minb", [(0, 8), (1, 6), (2, 8)])
@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("w,h,s", [(37, 29, 12), (300, 211, 500), (517, 263, 65535), (640, 480, 65536),
                                   (1000, 700, 1 << 18)])
def test_blocked_byte_pass(vd, orc, pack, minb, dedup, w, h, s):
    """The register-blocked byte-key pass (each thread owns the quads at
    (x, y), (x + k, y), (x, y + k), (x + k, y + k)) against the oracle: steps
    that are multiples of 4 (including ones not a power of two, ones wider
    than half the grid and ones that leave a quad block's far quads off the
    map), both neighbourhoods, every key packing and register budget, maps of
    random labels with and without empty ones, and dJFA steps in the
    narrow (below 2^16 seeds) and wide (17-, 19-bit label) forms."""
    g = np.random.default_rng(s + w + pack)
    xy = inputs.uniform_seeds(w, h, s, seed=s + 5)
    sim = _sim(vd, w, h, xy, byte_keys=1, dedup_gathers=dedup, blocked_pass=1, key_pack=pack,
               blocked_min_blocks=minb)
    for lo in (-1, 0):
        src = g.integers(lo, s, size=(h, w), dtype=np.int32)
        for k in [4, 8, 12, 16, 20, 64, 256]:
            for nb in [M, VN]:
                sim.set_labels(src)
                sim.jump_pass(k, nb, E)
                got = sim.labels()
                want = orc.jump_pass(w, h, xy, src, k, nb, E)
                assert np.array_equal(got, want), (k, nb, lo, int((got != want).sum()))
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    disp = inputs.displacements(s, 3, 2, seed=s)
    for t in range(2):
        sim.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        sim.djfa_step(d_max=3)
        lab = orc.djfa_step(w, h, xy, lab, d_max=3)
        np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"step {t}")
    sim.close()


def test_blocked_pass_matches_plain_at_full_size(vd, orc):
    """8192 x 8192 with 2^18 seeds, moves in [-4, 4] (the benchmark's default
    point): three dJFA steps with the blocked pass forced on and off give the
    same maps, and the first equals the oracle."""
    w = h = 8192
    s, D = 1 << 18, 4
    xy = inputs.uniform_seeds(w, h, s, seed=7)
    disp = inputs.displacements(s, D, 3, seed=7)
    a = _sim(vd, w, h, xy, use_graphs=1, blocked_pass=1)
    b = _sim(vd, w, h, xy, use_graphs=1, blocked_pass=0)
    a.jfa()
    b.jfa()
    lab = orc.jfa(w, h, xy)
    for t in range(3):
        for sim in (a, b):
            sim.step(disp[t], d_max=D)
        la = a.labels()
        np.testing.assert_array_equal(la, b.labels(), err_msg=f"step {t}")
        if t == 0:
            xy = orc.move(w, h, xy, disp[t])
            lab = orc.djfa_step(w, h, xy, lab, d_max=D)
            np.testing.assert_array_equal(la, lab)
    a.close()
    b.close()


@pytest.mark.parametrize("key", ["exact", "clamped", "byte"])
@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("w,h,s", [(37, 29, 3), (300, 211, 40), (517, 263, 500), (1000, 700, 70000)])
def test_sparse_pass(vd, orc, key, dedup, w, h, s):
    """The sparse pass (unchanged quads copied through, the rest scored after
    a per-block compaction), forced on every step it applies to (k % 4 == 0,
    k = 1, k = 2), against the oracle: smooth maps (a JFA frame: most quads
    unchanged), the same with scattered wrong and empty labels, and nearly
    empty maps (the stamps of a JFA frame's first pass), both neighbourhoods
    and metrics, each key form, with and without de-duplicated gathers; then
    a JFA frame and two dJFA steps."""
    g = np.random.default_rng(s + w)
    xy = inputs.uniform_seeds(w, h, s, seed=s + 9)
    xy[-1] = xy[0]
    forms = {"exact": dict(clamped_keys=0, byte_keys=0), "clamped": dict(clamped_keys=1, byte_keys=0),
             "byte": dict(byte_keys=1)}[key]
    sim = _sim(vd, w, h, xy, sparse_pass=1, dedup_gathers=dedup, **forms)
    smooth = orc.jfa(w, h, xy)
    noisy = smooth.copy()
    pick = g.random((h, w)) < 0.01
    noisy[pick] = g.integers(-1, s, size=int(pick.sum()), dtype=np.int32)
    stamped = orc.stamp(w, h, xy, np.full((h, w), -1, np.int32))
    for name, src in (("smooth", smooth), ("noisy", noisy), ("stamped", stamped)):
        for k in [1, 2, 4, 8, 16, 64]:
            for nb in [M, VN]:
                for metric in [E, L1]:
                    sim.set_labels(src)
                    sim.jump_pass(k, nb, metric)
                    got = sim.labels()
                    want = orc.jump_pass(w, h, xy, src, k, nb, metric)
                    assert np.array_equal(got, want), (name, k, nb, metric, int((got != want).sum()))
    for metric in [E, L1]:
        sim.jfa(metric=metric)
        lab = orc.jfa(w, h, xy, metric=metric)
        np.testing.assert_array_equal(sim.labels(), lab)
        cur = xy
        disp = inputs.displacements(s, 3, 2, seed=s + metric)
        for t in range(2):
            sim.move(disp[t])
            cur = orc.move(w, h, cur, disp[t])
            sim.djfa_step(d_max=3, metric=metric)
            lab = orc.djfa_step(w, h, cur, lab, d_max=3, metric=metric)
            np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"metric {metric} step {t}")
        sim.set_seeds(xy)
    sim.close()


@pytest.mark.parametrize("s,D", [(1 << 14, 4), (1 << 10, 1)])
def test_sparse_auto_matches_plain_at_full_size(vd, orc, s, D):
    """8192 x 8192 sweep points where the auto rule runs the sparse pass for
    the small steps of every frame: JFA frame 0 and three graph-replayed dJFA
    steps equal the same frames with the sparse pass off, and frame 0 and the
    first step equal the oracle."""
    w = h = 8192
    xy = inputs.uniform_seeds(w, h, s, seed=11)
    disp = inputs.displacements(s, D, 3, seed=11)
    a = _sim(vd, w, h, xy, use_graphs=1)
    b = _sim(vd, w, h, xy, use_graphs=1, sparse_pass=0)
    a.jfa()
    b.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(a.labels(), lab)
    np.testing.assert_array_equal(b.labels(), lab)
    for t in range(3):
        for sim in (a, b):
            sim.step(disp[t], d_max=D)
        la = a.labels()
        np.testing.assert_array_equal(la, b.labels(), err_msg=f"step {t}")
        if t == 0:
            xy = orc.move(w, h, xy, disp[t])
            lab = orc.djfa_step(w, h, xy, lab, d_max=D)
            np.testing.assert_array_equal(la, lab)
    a.close()
    b.close()


@pytest.mark.parametrize("band", [0, 16])
@pytest.mark.parametrize("w,h,s", [(5, 3, 2), (37, 29, 7), (300, 211, 500), (1000, 700, 70000), (2048, 1024, 1000)])
def test_jfa_position_map(vd, orc, band, w, h, s):
    """JFA frames whose k % 4 == 0 passes run on the (label, position) map,
    forced on (with and without k-strided band order), against the oracle:
    both metrics, JFA+2, coinciding seeds, a grid whose only such pass is
    also its last (5 x 3), eager and graph-replayed frames around a move."""
    xy = inputs.uniform_seeds(w, h, s, seed=s + w)
    xy[-1] = xy[0]
    for metric in [E, L1]:
        for extra in [0, 2]:
            sim = _sim(vd, w, h, xy, jfa_position_map=1, band_order_min_k=band)
            sim.jfa(extra=extra, metric=metric)
            got = sim.labels()
            want = orc.jfa(w, h, xy, extra=extra, metric=metric)
            assert np.array_equal(got, want), (metric, extra, int((got != want).sum()))
            sim.close()
    sim = _sim(vd, w, h, xy, jfa_position_map=1, use_graphs=1)
    d = inputs.displacements(s, 5, 1, seed=s)[0]
    sim.jfa()
    np.testing.assert_array_equal(sim.labels(), orc.jfa(w, h, xy))
    sim.move(d)
    sim.jfa()
    np.testing.assert_array_equal(sim.labels(), orc.jfa(w, h, orc.move(w, h, xy, d)))
    sim.close()


@pytest.mark.parametrize("w,h,s,D", [(1024, 768, 4000, 2), (2048, 2048, 1 << 14, 4)])
def test_autotune_keeps_state_and_results(vd, orc, w, h, s, D):
    """vd_autotune times the pass launch shapes on the context's own dJFA
    steps and keeps the fastest: the state after tuning equals the state
    before it, and the tuned context's next steps equal an untuned twin's
    (and the oracle's) bit for bit."""
    import torch

    xy = inputs.uniform_seeds(w, h, s, seed=13)
    disp = inputs.displacements(s, D, 3, seed=13)
    a = _sim(vd, w, h, xy, use_graphs=1)
    b = _sim(vd, w, h, xy, use_graphs=1)
    a.jfa()
    b.jfa()
    before = a.labels()
    chosen, times = a.autotune(d_max=D, max_disp=D, steps=3)
    assert len(times) >= 8 and all(t > 0 for t in times)
    assert chosen["pass_tile"] in (32, 64, 128) and chosen["fuse_max_k"] in (0, 2, 4)
    assert chosen["packed_map"] in (-1, 0)
    np.testing.assert_array_equal(a.labels(), before)
    np.testing.assert_array_equal(a.get_seeds(), xy)
    assert a.get_option(vd.OPT_PASS_TILE) == chosen["pass_tile"]
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(before, lab)
    for t in range(3):
        for sim in (a, b):
            sim.step(disp[t], d_max=D)
        xy = orc.move(w, h, xy, disp[t])
        lab = orc.djfa_step(w, h, xy, lab, d_max=D)
        np.testing.assert_array_equal(a.labels(), b.labels(), err_msg=f"step {t}")
        np.testing.assert_array_equal(a.labels(), lab, err_msg=f"step {t}")
    torch.cuda.synchronize()
    a.close()
    b.close()


@pytest.mark.parametrize("tile", [32, 128])
def test_pass_tiles(vd, orc, tile):
    """The 32 x 4 and 128 x 1 block tiles of the pass give the oracle's maps
    (ragged widths: fewer quads per row than the tile)."""
    for w, h, s in [(37, 29, 12), (300, 211, 500), (1000, 700, 70000)]:
        xy = inputs.uniform_seeds(w, h, s, seed=w)
        sim = _sim(vd, w, h, xy, pass_tile=tile)
        g = np.random.default_rng(w)
        src = g.integers(-1, s, size=(h, w), dtype=np.int32)
        for k in [1, 2, 3, 4, 16]:
            for nb in [M, VN]:
                sim.set_labels(src)
                sim.jump_pass(k, nb)
                np.testing.assert_array_equal(sim.labels(), orc.jump_pass(w, h, xy, src, k, nb, E))
        sim.jfa()
        lab = orc.jfa(w, h, xy)
        np.testing.assert_array_equal(sim.labels(), lab)
        d = inputs.displacements(s, 2, 1, seed=w)[0]
        sim.move(d)
        sim.djfa_step(d_max=2)
        np.testing.assert_array_equal(sim.labels(), orc.djfa_step(w, h, orc.move(w, h, xy, d), lab, d_max=2))
        sim.close()


@pytest.mark.parametrize("max_k,rows", [(8, 16), (16, 16), (16, 8)])
@pytest.mark.parametrize("w,h,s", [(37, 29, 12), (300, 211, 500), (517, 263, 65535), (640, 480, 65536),
                                   (1000, 700, 1 << 18)])
def test_smem_tile_pass(vd, orc, max_k, rows, w, h, s):
    """The byte-key pass over a shared-memory tile (256 x 16 or 256 x 8 pixels staged
    with a k-pixel halo as (label, seed position) pairs) against the oracle:
    k = 1, 2 and multiples of 4 up to 16 (12 included), both neighbourhoods,
    maps of random labels with and without empty ones (the far position
    staged outside the map and the empty label make winners fail the check:
    the recomputation path), ragged widths and heights, the narrow and wide
    byte forms, then a JFA frame and dJFA steps."""
    g = np.random.default_rng(s + w + max_k)
    xy = inputs.uniform_seeds(w, h, s, seed=s + 17)
    sim = _sim(vd, w, h, xy, byte_keys=1, smem_tile_max_k=max_k, smem_tile_rows=rows)
    for lo in (-1, 0):
        src = g.integers(lo, s, size=(h, w), dtype=np.int32)
        for k in [1, 2, 4, 8, 12, 16]:
            for nb in [M, VN]:
                sim.set_labels(src)
                sim.jump_pass(k, nb, E)
                got = sim.labels()
                want = orc.jump_pass(w, h, xy, src, k, nb, E)
                assert np.array_equal(got, want), (k, nb, lo, int((got != want).sum()))
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    for k in [8, 4, 2, 1]:
        sim.set_labels(lab)
        sim.jump_pass(k, M, E)
        np.testing.assert_array_equal(sim.labels(), orc.jump_pass(w, h, xy, lab, k, M, E), err_msg=f"k={k}")
    sim.set_labels(lab)  # the dJFA chain starts from the JFA frame, like the oracle's
    disp = inputs.displacements(s, 3, 2, seed=s)
    for t in range(2):
        sim.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        sim.djfa_step(d_max=3)
        lab = orc.djfa_step(w, h, xy, lab, d_max=3)
        np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"step {t}")
    sim.close()


@pytest.mark.parametrize("s,D", [(1 << 18, 4), (1 << 14, 4)])
def test_smem_tile_auto_matches_plain_at_full_size(vd, orc, s, D):
    """8192 x 8192 sweep points with the tiled pass on (steps up to 8) and
    off: three graph-replayed dJFA steps give the same maps, the first equal
    to the oracle."""
    w = h = 8192
    xy = inputs.uniform_seeds(w, h, s, seed=19)
    disp = inputs.displacements(s, D, 3, seed=19)
    a = _sim(vd, w, h, xy, use_graphs=1, smem_tile_max_k=8)
    b = _sim(vd, w, h, xy, use_graphs=1, smem_tile_max_k=0)
    a.jfa()
    b.jfa()
    lab = orc.jfa(w, h, xy)
    for t in range(3):
        for sim in (a, b):
            sim.step(disp[t], d_max=D)
        la = a.labels()
        np.testing.assert_array_equal(la, b.labels(), err_msg=f"step {t}")
        if t == 0:
            xy = orc.move(w, h, xy, disp[t])
            lab = orc.djfa_step(w, h, xy, lab, d_max=D)
            np.testing.assert_array_equal(la, lab)
    a.close()
    b.close()


@pytest.mark.parametrize("w,h,s", [(37, 29, 12), (300, 211, 500), (517, 263, 32767), (1000, 70, 40000),
                                   (640, 480, 65536), (700, 500, 131071), (1000, 700, 131072),
                                   (1024, 700, 1 << 18), (701, 499, (1 << 18) + 1), (1500, 900, 400000)])
def test_packed_map_frames(vd, orc, w, h, s):
    """dJFA frames whose byte-key passes run on position-tagged words (forced
    on) against the oracle, for each word layout: up to 32767 seeds (8-bit
    position fields), 32768 .. 2^17 - 1 (7-bit; below 2^16 seeds, as 40000,
    the frame's first pass folds with the narrow byte-offset key), 2^17 ..
    2^18 (6-bit, where the last seed's label code is also the empty code),
    above 2^18 (4-bit, the label split around the x field, distances
    saturated, the frame's first pass on the clamped key).  Frames after the JFA frame with moves, extra
    passes and no Von Neumann waves, then frames stamped onto random maps with
    and without empty labels: nearly every quad there fails the winner check
    and is recomputed, and empty pixels cross the packed passes.  Ragged
    widths and heights put the map border inside blocks."""
    g = np.random.default_rng(s + w)
    xy = inputs.uniform_seeds(w, h, s, seed=s + 29)
    sim = _sim(vd, w, h, xy, byte_keys=1, packed_map=1)
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    disp = inputs.displacements(s, 5, 3, seed=s + 1)
    for t, (D, vn, extra) in enumerate([(5, 2, 0), (2, 0, 1), (1, 2, 2)]):
        sim.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        sim.djfa_step(d_max=D, vn_waves=vn, extra=extra)
        lab = orc.djfa_step(w, h, xy, lab, d_max=D, vn_waves=vn, extra=extra)
        got = sim.labels()
        assert np.array_equal(got, lab), (t, int((got != lab).sum()))
    for lo in (-1, 0):
        src = g.integers(lo, s, size=(h, w), dtype=np.int32)
        for D in (1, 4):
            sim.set_labels(src)
            sim.djfa_step(d_max=D)
            got = sim.labels()
            want = orc.djfa_step(w, h, xy, src, d_max=D)
            assert np.array_equal(got, want), (lo, D, int((got != want).sum()))
    sim.close()


@pytest.mark.parametrize("s,D", [(1 << 18, 4), (1 << 16, 4), (1 << 14, 4), (1 << 22, 4), (1 << 22, 16)])
def test_packed_auto_matches_plain_at_full_size(vd, orc, s, D):
    """8192 x 8192 sweep points with the position-tagged passes (auto) and
    without: three graph-replayed dJFA steps give the same maps, the first
    equal to the oracle (2^22 seeds: the 4-bit layout, from the first pass
    with moves of 4, from the third with moves of 16)."""
    w = h = 8192
    xy = inputs.uniform_seeds(w, h, s, seed=23)
    disp = inputs.displacements(s, D, 3, seed=23)
    a = _sim(vd, w, h, xy, use_graphs=1)
    b = _sim(vd, w, h, xy, use_graphs=1, packed_map=0)
    a.jfa()
    b.jfa()
    lab = orc.jfa(w, h, xy)
    for t in range(3):
        for sim in (a, b):
            sim.step(disp[t], d_max=D)
        la = a.labels()
        np.testing.assert_array_equal(la, b.labels(), err_msg=f"step {t}")
        if t == 0:
            xy = orc.move(w, h, xy, disp[t])
            lab = orc.djfa_step(w, h, xy, lab, d_max=D)
            np.testing.assert_array_equal(la, lab)
    a.close()
    b.close()


@pytest.mark.parametrize("w,h,s", [(32768, 8, 300), (8, 32768, 300), (32768, 40, 20000), (40, 32768, 140000),
                                   (32768, 24, 300000)])
def test_packed_map_maximum_sides(vd, orc, w, h, s):
    """Position-tagged passes (forced on) on grids at the maximum side: x or y
    up to 32767 taken modulo 2^M in the words, element indices up to 2^30,
    the 8-, 7-, 6- and 4-bit layouts; dJFA steps after the JFA frame equal
    the oracle."""
    xy = inputs.uniform_seeds(w, h, s, seed=w + 3 * h)
    disp = inputs.displacements(s, 4, 2, seed=2)
    sim = _sim(vd, w, h, xy, byte_keys=1, packed_map=1)
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    for t in range(2):
        sim.move(disp[t])
        xy = orc.move(w, h, xy, disp[t])
        sim.djfa_step(d_max=4)
        lab = orc.djfa_step(w, h, xy, lab, d_max=4)
        got = sim.labels()
        assert np.array_equal(got, lab), (t, int((got != lab).sum()))
    sim.close()
