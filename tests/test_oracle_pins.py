"""Pins the CPU oracle to facts fixed outside it (no GPU needed).

Each test checks the oracle against something it does not itself compute: the
worked example and hand-evaluated equations of the paper (golden files), a
library routine that solves a special case (scipy distance matrices and
distance transforms), closed forms (the perpendicular bisector, the set of
pixels one jump pass reaches), invariants (the exact diagram is a fixed point
of every pass; a pass never makes a pixel worse) and published test vectors.
The cases are chosen so that a dropped neighbour, a transposed axis, a wrong
sign, a wrong tie-break or an in-place (non-Jacobi) pass fails at least one.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage
from scipy.spatial.distance import cdist

from paper_2209_00117_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

M, VN = 0, 1  # Moore, Von Neumann
E, L1 = 0, 1  # Euclidean, Manhattan


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


# --------------------------------------------------------------------------
# Schedules: Eq. 2 and Eq. 3-4
# --------------------------------------------------------------------------

def test_jfa_schedule_worked_example(orc):
    ks = [r[0] for r in _golden("jfa_schedule_8x8.txt")]
    assert [k for k, _ in orc.jfa_schedule(8, 8)] == ks
    assert all(nb == M for _, nb in orc.jfa_schedule(8, 8))


def test_jfa_first_step_table(orc):
    for n, k1, passes in _golden("jfa_first_step.txt"):
        assert orc.jfa_first_step(n, n) == k1, n
        assert len(orc.jfa_schedule(n, n)) == passes, n
        # a rectangle uses its longer side
        assert orc.jfa_first_step(n, 1) == k1 and orc.jfa_first_step(1, n) == k1


def test_djfa_first_step_table(orc):
    for w, h, s, d, d1, passes in _golden("djfa_first_step.txt"):
        assert orc.djfa_first_step(w, h, s, d) == d1, (w, h, s, d)
        assert len(orc.djfa_schedule(w, h, s, d, vn_waves=2)) == passes, (w, h, s, d)


def test_djfa_first_step_matches_floating_formula(orc):
    """The exact integer form of Eq. 4 agrees with a floating evaluation of the
    printed formula wherever the float is not within rounding of a power of 2."""
    g = np.random.default_rng(5)
    checked = 0
    for _ in range(3000):
        w = int(g.integers(1, 5000))
        h = int(g.integers(1, 5000))
        s = int(g.integers(1, 200000))
        d = int(g.integers(0, 300))
        l_avg = math.sqrt(w * h / s)
        arg = max(2.0 * l_avg, float(d))
        e = math.log2(arg) if arg > 0 else -math.inf
        if abs(e - round(e)) < 1e-9:
            continue
        ce = math.ceil(e)
        want = 2 ** ce if ce >= 0 else 0
        assert orc.djfa_first_step(w, h, s, d, capped=False) == want, (w, h, s, d)
        cap = orc.jfa_first_step(w, h)
        assert orc.djfa_first_step(w, h, s, d) == min(want, cap)
        checked += 1
    assert checked > 2500


def test_djfa_behaviour_claims(orc):
    """Section V-A: more seeds never lengthen the schedule; few seeds give
    JFA's schedule; a large d_max takes over."""
    w = h = 1024
    prev = None
    for s in [1, 2, 5, 17, 100, 1000, 10 ** 4, 10 ** 5, 10 ** 6]:
        d1 = orc.djfa_first_step(w, h, s, 1)
        if prev is not None:
            assert d1 <= prev
        prev = d1
    assert orc.djfa_first_step(w, h, 1, 1) == orc.jfa_first_step(w, h)
    assert orc.djfa_first_step(w, h, 10 ** 6, 100) == 128
    assert orc.djfa_first_step(w, h, 10 ** 6, 1) == 4


def test_schedule_neighbourhoods_and_extra(orc):
    sch = orc.djfa_schedule(2048, 2048, 16384, 2, vn_waves=2)
    assert [nb for _, nb in sch] == [VN, VN, M, M, M, M]
    sch1 = orc.djfa_schedule(2048, 2048, 16384, 2, vn_waves=1, extra=1)
    assert sch1 == [(32, VN), (16, M), (8, M), (4, M), (2, M), (1, M), (1, M)]
    assert orc.jfa_schedule(8, 8, extra=1) == [(4, M), (2, M), (1, M), (1, M)]
    assert orc.jfa_schedule(8, 8, extra=2) == [(4, M), (2, M), (1, M), (2, M), (1, M)]
    assert orc.jfa_schedule(1, 1) == []


# --------------------------------------------------------------------------
# The exact diagram, Eq. 1
# --------------------------------------------------------------------------

def _pixels(w, h):
    yy, xx = np.mgrid[0:h, 0:w]
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


@pytest.mark.parametrize("metric,name", [(E, "sqeuclidean"), (L1, "cityblock")])
def test_brute_force_matches_library_argmin(orc, metric, name):
    g = np.random.default_rng(1)
    for trial in range(12):
        w = int(g.integers(1, 23))
        h = int(g.integers(1, 19))
        s = int(g.integers(1, 9))
        xy = inputs.uniform_seeds(w, h, s, seed=trial)
        if trial % 3 == 0 and s > 1:
            xy[1] = xy[0]  # duplicate position
        dm = cdist(_pixels(w, h), xy.astype(np.float64), name)
        want_label = np.argmin(dm, axis=1).reshape(h, w)  # first minimum = lowest index
        want_dist = np.rint(dm.min(axis=1)).astype(np.int64).reshape(h, w)
        label, dist = orc.exact_brute(w, h, xy, metric)
        np.testing.assert_array_equal(label, want_label)
        np.testing.assert_array_equal(dist, want_dist)


def test_two_seeds_split_on_bisector(orc):
    w, h = 37, 23
    a = np.array([5, 7])
    b = np.array([28, 15])
    label, _ = orc.exact_brute(w, h, np.stack([a, b]))
    p = _pixels(w, h)
    # closer to a  <=>  2 p.(b - a) < |b|^2 - |a|^2 ; equality -> lower index (a)
    lhs = 2 * (p @ (b - a))
    rhs = b @ b - a @ a
    want = np.where(lhs <= rhs, 0, 1).reshape(h, w)
    np.testing.assert_array_equal(label, want)
    # swap the indices: ties go to the new lower index
    label2, _ = orc.exact_brute(w, h, np.stack([b, a]))
    want2 = np.where(lhs < rhs, 1, 0).reshape(h, w)
    np.testing.assert_array_equal(label2, want2)


def test_seed_pixels_own_themselves(orc):
    w, h = 31, 17
    xy = inputs.uniform_seeds(w, h, 40, seed=3)
    label, dist = orc.exact_brute(w, h, xy)
    for k, (x, y) in enumerate(xy):
        lowest = min(j for j in range(len(xy)) if tuple(xy[j]) == (x, y))
        assert label[y, x] == lowest
        assert dist[y, x] == 0


@pytest.mark.parametrize("w,h,s", [(1, 1, 1), (1, 40, 3), (53, 1, 2), (64, 48, 30),
                                   (97, 61, 5), (128, 128, 400)])
def test_edt_matches_scipy_and_brute(orc, w, h, s):
    xy = inputs.uniform_seeds(w, h, s, seed=w * h + s)
    mask = np.ones((h, w), bool)
    mask[xy[:, 1], xy[:, 0]] = False
    want_e = np.rint(ndimage.distance_transform_edt(mask) ** 2).astype(np.int64)
    want_l1 = ndimage.distance_transform_cdt(mask, metric="taxicab").astype(np.int64)
    np.testing.assert_array_equal(orc.exact_dist_edt(w, h, xy, E), want_e)
    np.testing.assert_array_equal(orc.exact_dist_edt(w, h, xy, L1), want_l1)
    if w * h * s <= 2_000_000:
        np.testing.assert_array_equal(orc.exact_brute(w, h, xy, E)[1], want_e)
        np.testing.assert_array_equal(orc.exact_brute(w, h, xy, L1)[1], want_l1)


def test_edt_no_seeds(orc):
    d = orc.exact_dist_edt(5, 4, np.zeros((0, 2), np.int32))
    assert (d == np.iinfo(np.int32).max).all()


# --------------------------------------------------------------------------
# One jump pass: Table I, Section V-B
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nb", [M, VN])
def test_single_label_reach(orc, nb):
    """After one pass from a map holding one label at q0, exactly the pixels
    that have q0 among their neighbours (offset k, Table I) hold it."""
    w, h = 41, 29
    offs = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    if nb == VN:
        offs = [o for o in offs if o[0] == 0 or o[1] == 0]
    for (qx, qy) in [(3, 2), (20, 14), (39, 27), (0, 28)]:
        for k in [1, 2, 3, 4, 8, 16]:
            src = np.full((h, w), -1, np.int32)
            src[qy, qx] = 0
            dst = orc.jump_pass(w, h, np.array([[qx, qy]]), src, k, nb)
            want = np.full((h, w), -1, np.int32)
            want[qy, qx] = 0
            for ox, oy in offs:
                px, py = qx - ox * k, qy - oy * k
                if 0 <= px < w and 0 <= py < h:
                    want[py, px] = 0
            np.testing.assert_array_equal(dst, want, err_msg=f"q0={(qx, qy)} k={k}")


@pytest.mark.parametrize("metric", [E, L1])
@pytest.mark.parametrize("nb", [M, VN])
def test_exact_diagram_is_fixed_point(orc, metric, nb):
    g = np.random.default_rng(2)
    for trial in range(6):
        w, h = int(g.integers(8, 40)), int(g.integers(8, 40))
        xy = inputs.uniform_seeds(w, h, int(g.integers(2, 25)), seed=100 + trial)
        xy[-1] = xy[0]
        label, _ = orc.exact_brute(w, h, xy, metric)
        for k in [1, 2, 4, 8, 16, 64]:
            np.testing.assert_array_equal(orc.jump_pass(w, h, xy, label, k, nb, metric), label)


def _key(orc, w, h, xy, label, metric):
    """Per pixel (distance, label) of a map, distance = inf for empty."""
    ys, xs = np.mgrid[0:h, 0:w]
    lab = label.astype(np.int64)
    sx = np.where(lab >= 0, xy[np.maximum(lab, 0), 0], 0).astype(np.int64)
    sy = np.where(lab >= 0, xy[np.maximum(lab, 0), 1], 0).astype(np.int64)
    if metric == E:
        d = (sx - xs) ** 2 + (sy - ys) ** 2
    else:
        d = np.abs(sx - xs) + np.abs(sy - ys)
    d = np.where(lab >= 0, d, np.iinfo(np.int64).max)
    return d, lab


def test_pass_never_worsens_a_pixel(orc):
    g = np.random.default_rng(3)
    w, h = 57, 33
    xy = inputs.uniform_seeds(w, h, 30, seed=7)
    src = g.integers(-1, 30, size=(h, w), dtype=np.int32)
    for k in [1, 2, 4, 16]:
        for nb in [M, VN]:
            dst = orc.jump_pass(w, h, xy, src, k, nb)
            d0, l0 = _key(orc, w, h, xy, src, E)
            d1, l1 = _key(orc, w, h, xy, dst, E)
            assert ((d1 < d0) | ((d1 == d0) & (l1 <= l0))).all()


def test_pass_tie_break_lowest_index(orc):
    # seeds 1 and 3 are both at squared distance 25 from pixel (5, 5)
    xy = np.array([[0, 0], [5, 0], [0, 10], [10, 5]], np.int32)
    w = h = 11
    for own, nbr in [(3, 1), (1, 3)]:
        src = np.full((h, w), -1, np.int32)
        src[5, 5] = own
        src[5, 6] = nbr  # neighbour at (+1, 0) with k = 1
        dst = orc.jump_pass(w, h, xy, src, 1)
        assert dst[5, 5] == 1


def test_pass_is_jacobi_not_in_place(orc):
    """A label travels exactly k per pass: an in-place sweep would carry it further."""
    w, h = 16, 1
    src = np.full((h, w), -1, np.int32)
    src[0, 0] = 0
    dst = orc.jump_pass(w, h, np.array([[0, 0]]), src, 1)
    assert list(dst[0, :3]) == [0, 0, -1]
    dst = orc.jump_pass(w, h, np.array([[15, 0]]), np.flip(src, 1).copy(), 1)
    assert list(dst[0, -3:]) == [-1, 0, 0]


def test_pass_large_k_is_identity(orc):
    w, h = 19, 13
    xy = inputs.uniform_seeds(w, h, 5, seed=1)
    src = np.random.default_rng(0).integers(-1, 5, size=(h, w), dtype=np.int32)
    np.testing.assert_array_equal(orc.jump_pass(w, h, xy, src, 19), src)


# --------------------------------------------------------------------------
# JFA and dJFA
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w,h", [(1, 1), (2, 1), (1, 7), (8, 8), (13, 5), (64, 64), (100, 37)])
def test_jfa_single_seed_owns_all(orc, w, h):
    for (x, y) in [(0, 0), (w - 1, h - 1), (w // 2, h // 3)]:
        lab = orc.jfa(w, h, np.array([[x, y]]))
        assert (lab == 0).all()


def test_jfa_invariants(orc):
    for trial in range(5):
        w, h = 70 + 9 * trial, 45 + 4 * trial
        xy = inputs.uniform_seeds(w, h, 20 + 30 * trial, seed=trial)
        xy[3] = xy[7]
        lab = orc.jfa(w, h, xy)
        assert (lab >= 0).all() and (lab < len(xy)).all()
        for k, (x, y) in enumerate(xy):
            lowest = min(j for j in range(len(xy)) if tuple(xy[j]) == (x, y))
            assert lab[y, x] == lowest
        d_exact = orc.exact_dist_edt(w, h, xy)
        ne, _ = orc.similarity(w, h, xy, lab, exact_dist=d_exact)
        assert ne >= 0.99 * w * h  # JFA's errors are rare (Section III)
        # extra passes never reduce the distance-correct count
        ne1, _ = orc.similarity(w, h, xy, orc.jfa(w, h, xy, extra=1), exact_dist=d_exact)
        ne2, _ = orc.similarity(w, h, xy, orc.jfa(w, h, xy, extra=2), exact_dist=d_exact)
        assert ne1 >= ne and ne2 >= ne


def test_djfa_on_empty_map_with_cap_equals_jfa(orc):
    """With delta_1 capped to k_1 and no Von Neumann waves, a dJFA step on an
    empty map runs JFA's passes: the two code paths agree."""
    w, h = 96, 80
    xy = inputs.uniform_seeds(w, h, 3, seed=9)
    assert orc.djfa_first_step(w, h, 3, 1) == orc.jfa_first_step(w, h)
    empty = np.full((h, w), -1, np.int32)
    for metric in [E, L1]:
        np.testing.assert_array_equal(
            orc.djfa_step(w, h, xy, empty, d_max=1, vn_waves=0, metric=metric),
            orc.jfa(w, h, xy, metric=metric))


def test_djfa_without_motion_keeps_exact_map(orc):
    w, h = 64, 50
    xy = inputs.uniform_seeds(w, h, 40, seed=4)
    exact, _ = orc.exact_brute(w, h, xy)
    for vn in [0, 1, 2]:
        np.testing.assert_array_equal(orc.djfa_step(w, h, xy, exact, d_max=2, vn_waves=vn), exact)


def test_move_clamps(orc):
    w, h = 10, 6
    xy = np.array([[0, 0], [9, 5], [4, 3], [1, 4]], np.int32)
    dxy = np.array([[-2, -1], [1, 2], [3, -3], [-1, 1]], np.int32)
    np.testing.assert_array_equal(orc.move(w, h, xy, dxy), [[0, 0], [9, 5], [7, 0], [0, 5]])


def test_splitmix64_vectors(orc):
    for state, n, out in _golden("splitmix64.txt"):
        assert orc.splitmix64(state, n) == out


def test_rng_displacement_range_and_uniformity(orc):
    for D in [0, 1, 2, 16]:
        vals = np.array([orc.rng_displacement(7, 3, 11, k, a, D)
                         for k in range(3000) for a in (0, 1)])
        assert vals.min() >= -D and vals.max() <= D
        if D > 0:
            counts = np.bincount(vals + D, minlength=2 * D + 1)
            expected = len(vals) / (2 * D + 1)
            chi2 = ((counts - expected) ** 2 / expected).sum()
            assert chi2 < 3 * (2 * D + 1) + 30
    # distinct counters give distinct streams
    a = [orc.rng_displacement(0, 0, 0, k, 0, 1000) for k in range(50)]
    b = [orc.rng_displacement(0, 0, 1, k, 0, 1000) for k in range(50)]
    c = [orc.rng_displacement(0, 1, 0, k, 0, 1000) for k in range(50)]
    assert a != b and a != c


def test_similarity_counts(orc):
    w, h = 33, 21
    xy = inputs.uniform_seeds(w, h, 12, seed=2)
    exact, dist = orc.exact_brute(w, h, xy)
    assert orc.similarity(w, h, xy, exact, exact_dist=dist, ref_label=exact) == (w * h, w * h)
    worse = exact.copy()
    # relabel one pixel with a seed strictly farther away
    y, x = 10, 10
    d = [(orc.distance(*xy[k], x, y), k) for k in range(len(xy))]
    far = max(d)[1]
    worse[y, x] = far
    assert orc.similarity(w, h, xy, worse, exact_dist=dist, ref_label=exact) == (w * h - 1, w * h - 1)


def test_djfa_similarity_level_single256(orc):
    """Section VI-B: Euclidean dJFA stays close to JFA on the 256^2, 64-seed,
    [-1, 1]-move workload (reported near 100%)."""
    w, h, s, steps, D = inputs.SINGLE["single256"]
    xy = inputs.uniform_seeds(w, h, s, seed=0)
    disp = inputs.displacements(s, D, steps, seed=0)
    lab = orc.jfa(w, h, xy)
    for t in range(steps):
        xy = orc.move(w, h, xy, disp[t])
        lab = orc.djfa_step(w, h, xy, lab, d_max=D, vn_waves=2)
        ref = orc.jfa(w, h, xy)
        _, nm = orc.similarity(w, h, xy, lab, ref_label=ref)
        assert nm >= 0.99 * w * h, (t, nm / (w * h))


# --------------------------------------------------------------------------
# Seed insertion and removal (future work in Section VII; the library's rule)
# --------------------------------------------------------------------------

def _random_update(g, w, h, s, n_remove, n_add):
    remove = g.choice(s, size=n_remove, replace=False).astype(np.int32)
    add = np.stack([g.integers(0, w, n_add), g.integers(0, h, n_add)], axis=1).astype(np.int32)
    return remove, add


def test_update_without_changes_is_identity(orc):
    w, h, s = 41, 29, 30
    xy = inputs.uniform_seeds(w, h, s, seed=21)
    lab = orc.jfa(w, h, xy)
    new_xy, new_lab = orc.update_seeds(w, h, xy, lab)
    np.testing.assert_array_equal(new_xy, xy)
    np.testing.assert_array_equal(new_lab, lab)


@pytest.mark.parametrize("trial", range(6))
def test_update_relabels_by_position_and_order(orc, trial):
    """Every labelled pixel keeps the same seed position (its seed survived) or
    becomes empty (its seed left); survivors keep their relative order; new
    seeds follow them in the order given."""
    g = np.random.default_rng(40 + trial)
    w, h, s = int(g.integers(5, 60)), int(g.integers(5, 60)), int(g.integers(2, 80))
    xy = inputs.uniform_seeds(w, h, s, seed=trial)
    lab = orc.jfa(w, h, xy)
    remove, add = _random_update(g, w, h, s, int(g.integers(0, s)), int(g.integers(0, 20)))
    new_xy, new_lab = orc.update_seeds(w, h, xy, lab, remove, add)
    gone = np.zeros(s, bool)
    gone[remove] = True
    survivors = np.flatnonzero(~gone)
    assert len(new_xy) == len(survivors) + len(add)
    np.testing.assert_array_equal(new_xy[:len(survivors)], xy[survivors])
    np.testing.assert_array_equal(new_xy[len(survivors):], add.reshape(-1, 2))
    emptied = gone[np.maximum(lab, 0)] & (lab >= 0)
    assert (new_lab[emptied] == -1).all()
    kept = (lab >= 0) & ~emptied
    np.testing.assert_array_equal(new_xy[new_lab[kept]], xy[lab[kept]])
    # order: a survivor's new index is the number of survivors before it
    assert (np.searchsorted(survivors, lab[kept]) == new_lab[kept]).all()


@pytest.mark.parametrize("metric", [E, L1])
def test_single_survivor_repair_is_brute_force(orc, metric):
    """Remove every seed but one: the repair frame gives the one-seed diagram
    of Eq. 1 (the survivor owns every pixel)."""
    g = np.random.default_rng(7)
    for w, h, s in [(1, 1, 3), (33, 17, 20), (64, 64, 90), (100, 3, 12)]:
        xy = inputs.uniform_seeds(w, h, s, seed=w)
        lab = orc.jfa(w, h, xy, metric=metric)
        keep = int(g.integers(0, s))
        remove = np.array([k for k in range(s) if k != keep], np.int32)
        new_xy, new_lab = orc.update_seeds(w, h, xy, lab, remove)
        assert len(new_xy) == 1
        out = orc.repair_step(w, h, new_xy, new_lab, metric=metric)
        want, _ = orc.exact_brute(w, h, new_xy, metric)
        np.testing.assert_array_equal(out, want)


@pytest.mark.parametrize("metric", [E, L1])
def test_repair_keeps_an_exact_map(orc, metric):
    """On a map that already is the exact diagram (Eq. 1, lowest-index ties) the
    repair frame changes nothing: no candidate is closer than a nearest seed."""
    for trial in range(4):
        w, h = 30 + 7 * trial, 25 + 3 * trial
        xy = inputs.uniform_seeds(w, h, 15 + 10 * trial, seed=trial)
        xy[-1] = xy[0]
        lab, _ = orc.exact_brute(w, h, xy, metric)
        np.testing.assert_array_equal(orc.repair_step(w, h, xy, lab, metric=metric), lab)


def test_repair_covers_every_pixel_and_seed_pixels_own_themselves(orc):
    """After removals (up to all but one) and insertions, the repair frame leaves
    no empty pixel and every seed pixel holds the lowest index standing on it
    (the seed is at distance 0 from itself, Eq. 1)."""
    g = np.random.default_rng(11)
    for trial in range(8):
        w, h, s = int(g.integers(10, 90)), int(g.integers(10, 90)), int(g.integers(3, 200))
        xy = inputs.uniform_seeds(w, h, s, seed=300 + trial)
        lab = orc.jfa(w, h, xy)
        remove, add = _random_update(g, w, h, s, int(g.integers(1, s)), int(g.integers(0, 30)))
        new_xy, new_lab = orc.update_seeds(w, h, xy, lab, remove, add)
        out = orc.repair_step(w, h, new_xy, new_lab)
        assert (out >= 0).all()
        for k in range(len(new_xy) - 1, -1, -1):
            x, y = new_xy[k]
            same = np.flatnonzero((new_xy[:, 0] == x) & (new_xy[:, 1] == y))
            assert out[y, x] == same[0]


def test_invalid_updates_change_nothing(orc):
    w, h, s = 20, 10, 5
    xy = inputs.uniform_seeds(w, h, s, seed=2)
    lab = orc.jfa(w, h, xy)
    assert orc.update_seeds(w, h, xy, lab, remove=[1, 1]) is None
    assert orc.update_seeds(w, h, xy, lab, remove=[5]) is None
    assert orc.update_seeds(w, h, xy, lab, remove=[-1]) is None
    assert orc.update_seeds(w, h, xy, lab, remove=[0, 1, 2, 3, 4]) is None
    assert orc.update_seeds(w, h, xy, lab, add=[[20, 0]]) is None
    assert orc.update_seeds(w, h, xy, lab, add=[[0, -1]]) is None
    new_xy, _ = orc.update_seeds(w, h, xy, lab, remove=[0, 1, 2, 3, 4], add=[[3, 3]])
    np.testing.assert_array_equal(new_xy, [[3, 3]])
