"""Seed removal and insertion between frames (the paper leaves both to future
work, Section VII; the rule is the library's own and the oracle's): the update
and the frames after it equal the oracle bit for bit (integer maps,
tolerance 0)."""
import numpy as np
import pytest

from paper_2209_00117_gb300 import inputs

pytestmark = pytest.mark.gpu

E, L1 = 0, 1


@pytest.fixture(scope="module")
def vd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00117_gb300 import build

    build.build()
    from paper_2209_00117_gb300 import vd as _vd

    return _vd


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _update(g, w, h, s, n_remove, n_add):
    remove = g.choice(s, size=n_remove, replace=False).astype(np.int32)
    add = np.stack([g.integers(0, w, n_add), g.integers(0, h, n_add)], axis=1).astype(np.int32)
    return remove, add


@pytest.mark.parametrize("metric", [E, L1])
@pytest.mark.parametrize("w,h,s,n_remove,n_add", [(97, 61, 40, 10, 5), (300, 211, 2000, 700, 300),
                                                   (512, 512, 5000, 4999, 0), (640, 480, 900, 0, 400),
                                                   (257, 129, 60, 59, 100)])
@pytest.mark.parametrize("graphs", [0, 1])
def test_update_and_following_frames_match_oracle(vd, orc, metric, w, h, s, n_remove, n_add, graphs):
    g = np.random.default_rng(w + s + n_remove)
    D = 2
    xy = inputs.uniform_seeds(w, h, s, seed=s)
    sim = vd.VoronoiSim(w, h, s)
    sim.set_option(vd.OPT_USE_GRAPHS, graphs)
    sim.set_seeds(xy)
    sim.jfa(metric=metric)
    lab = orc.jfa(w, h, xy, metric=metric)
    for t in range(2):
        d = inputs.step_displacements(len(xy), D, t, seed=1)
        sim.move(d)
        sim.djfa_step(d_max=D, metric=metric)
        xy = orc.move(w, h, xy, d)
        lab = orc.djfa_step(w, h, xy, lab, d_max=D, metric=metric)
    remove, add = _update(g, w, h, len(xy), n_remove, n_add)
    sim.update_seeds(remove, add)
    xy, lab = orc.update_seeds(w, h, xy, lab, remove, add)
    assert sim.n_seeds == len(xy)
    np.testing.assert_array_equal(sim.get_seeds(), xy)
    np.testing.assert_array_equal(sim.labels(), lab)
    # the next frame: the repair schedule after a removal, the dJFA one otherwise
    for t in range(3):
        d = inputs.step_displacements(len(xy), D, 10 + t, seed=2)
        sim.move(d)
        sim.djfa_step(d_max=D, metric=metric)
        xy = orc.move(w, h, xy, d)
        if t == 0 and n_remove > 0:
            lab = orc.repair_step(w, h, xy, lab, metric=metric)
        else:
            lab = orc.djfa_step(w, h, xy, lab, d_max=D, metric=metric)
        np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"frame {t} after the update")
    assert (lab >= 0).all()
    sim.close()


def test_growth_past_capacity_and_exact_diagram(vd, orc):
    """The seed count grows far past the one given at creation; every buffer
    sized by it follows (the exact diagram's bucket ids included)."""
    w, h, s = 400, 300, 50
    g = np.random.default_rng(5)
    xy = inputs.uniform_seeds(w, h, s, seed=5)
    sim = vd.VoronoiSim(w, h, s)
    sim.set_seeds(xy)
    sim.jfa()
    lab0, _ = sim.exact()  # sizes the bucket scratch at 50 seeds
    lab = orc.jfa(w, h, xy)
    for n_remove, n_add in [(10, 500), (0, 2000), (100, 3)]:
        remove, add = _update(g, w, h, len(xy), n_remove, n_add)
        sim.update_seeds(remove, add)
        xy, lab = orc.update_seeds(w, h, xy, lab, remove, add)
        sim.djfa_step(d_max=1)
        lab = orc.repair_step(w, h, xy, lab) if n_remove else orc.djfa_step(w, h, xy, lab, d_max=1)
        np.testing.assert_array_equal(sim.labels(), lab)
        ex_l, ex_d = sim.exact()
        want_l, want_d = orc.exact_brute(w, h, xy, E)
        np.testing.assert_array_equal(ex_l, want_l)
        np.testing.assert_array_equal(ex_d, want_d)
    assert sim.n_seeds == len(xy) == 50 - 10 + 500 + 2000 - 100 + 3
    sim.close()


def test_invalid_updates_change_nothing(vd):
    from paper_2209_00117_gb300._native import VD_EINVAL, VDError

    w, h, s = 64, 48, 20
    xy = inputs.uniform_seeds(w, h, s, seed=9)
    sim = vd.VoronoiSim(w, h, s)
    sim.set_seeds(xy)
    sim.jfa()
    before_l, before_s = sim.labels(), sim.get_seeds()
    for remove, add in [([1, 1], None), ([20], None), ([-1], None), (list(range(20)), None),
                        (None, [[64, 0]]), (None, [[0, -3]]), ([0], [[5, 48]])]:
        with pytest.raises(VDError) as ei:
            sim.update_seeds(remove, add)
        assert ei.value.code == VD_EINVAL
        assert sim.n_seeds == s
        np.testing.assert_array_equal(sim.labels(), before_l)
        np.testing.assert_array_equal(sim.get_seeds(), before_s)
    sim.update_seeds(list(range(20)), [[3, 4]])  # all replaced: one seed owns the map
    assert sim.n_seeds == 1
    sim.djfa_step(d_max=1)
    assert (sim.labels() == 0).all()
    sim.close()


def test_device_inputs_and_full_size(vd, orc):
    """2048 x 2048 with 16384 seeds: 1000 removed and 1500 added from CUDA
    tensors, then the repair frame and dJFA frames, against the oracle."""
    import torch

    w = h = 2048
    s, D = 16384, 2
    g = np.random.default_rng(2048)
    xy = inputs.uniform_seeds(w, h, s, seed=1)
    sim = vd.VoronoiSim(w, h, s)
    sim.set_option(vd.OPT_USE_GRAPHS, 1)
    sim.set_seeds(xy)
    sim.jfa()
    lab = orc.jfa(w, h, xy)
    remove, add = _update(g, w, h, s, 1000, 1500)
    sim.update_seeds(torch.from_numpy(remove).cuda(), torch.from_numpy(add).cuda())
    xy, lab = orc.update_seeds(w, h, xy, lab, remove, add)
    np.testing.assert_array_equal(sim.labels(), lab)
    for t in range(3):
        sim.move(None, max_disp=D, rng_seed=3, stream_id=0, step=t)
        sim.djfa_step(d_max=D)
        xy = orc.move_rng(w, h, xy, D, 3, 0, t)
        lab = orc.repair_step(w, h, xy, lab) if t == 0 else orc.djfa_step(w, h, xy, lab, d_max=D)
        np.testing.assert_array_equal(sim.labels(), lab, err_msg=f"frame {t}")
    sim.close()
