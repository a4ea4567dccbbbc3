"""Host model of the swap-and-restore stamp (k_stamp_xchg in vd_kernels.cuh):
every seed k standing on a pixel swaps its index in, and when the label r
it took out is a lower index whose seed stands on the same pixel, puts r back
with an atomic minimum.  The claim is that the pixel ends at the lowest index
standing on it, whatever the order the swaps and minima take (reading R4 of
the stamp: the lowest index wins, stale labels are replaced).  Here every
schedule of those operations is drawn at random for small sets of seeds,
with stale starting labels that do or do not name a seed now on the pixel,
and the empty label, and the end value is checked.  (The GPU tests check
the kernel itself against the oracle's stamp.)"""
import numpy as np
import pytest


def _run(order, seeds_here, pos_of, pixel, start):
    """Executes the per-seed programs (swap; then maybe an atomic minimum)
    in the interleaving `order` (a sequence of seed indices, each appearing
    twice: its swap, then its second step)."""
    value = start
    taken = {}
    for k in order:
        if k not in taken:
            taken[k] = value
            value = k
        else:
            r = taken[k]
            if 0 <= r < k and pos_of[r] == pixel:
                value = min(value, r)
    return value


@pytest.mark.parametrize("trial", range(40))
def test_any_schedule_ends_at_the_lowest_index(trial):
    rng = np.random.default_rng(trial)
    n = int(rng.integers(8, 40))
    pixel = 0
    # seeds on the pixel and elsewhere (positions 0 .. 3)
    pos_of = rng.integers(0, 4, n)
    pos_of[rng.integers(0, n)] = pixel
    here = [k for k in range(n) if pos_of[k] == pixel]
    starts = [-1, int(rng.integers(0, n))] + [k for k in here[:2]]
    for start in starts:
        for _ in range(200):
            ops = np.array(here + here)
            rng.shuffle(ops)
            # each seed's swap precedes its second step: the first occurrence
            # of k in the shuffled sequence is its swap
            assert _run(list(ops), here, pos_of, pixel, start) == min(here)


def test_single_seed_and_stale_labels():
    pos_of = np.array([5, 0, 5, 0])
    # one seed (1) on pixel 0, the stale label 2 names a seed elsewhere
    assert _run([1, 1], [1], pos_of, 0, 2) == 1
    # a stale lower label whose seed is not on the pixel is dropped
    assert _run([3, 3], [3], np.array([9, 9, 9, 0]), 0, 0) == 3
    # the empty label is dropped
    assert _run([3, 3], [3], np.array([9, 9, 9, 0]), 0, -1) == 3
