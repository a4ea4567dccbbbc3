"""The allocation-free exact-diagram entry point, called through the C ABI.

vd_exact_noalloc serves callers that must not allocate device memory (code
under another framework's memory manager, allocation-free real-time loops,
plugin hosts); it uses a scratch array compiled into the library instead of
cudaMalloc.  This file runs last so that a failure here leaves every other
test already run.  It checks, on two calls in a row with different sizes (so
the second call reuses scratch the first one filled), that the new entry
point returns exactly what the context-based vd_exact returns and what the
CPU oracle's brute force of Eq. 1 returns (integer maps, tolerance 0), that a
request at the documented bound (200000 seeds on the grid that needs the most
buckets) fits, and that oversized requests and out-of-grid seeds are rejected.
"""
import numpy as np
import pytest

from paper_2209_00117_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00117_gb300 import _native, build, vd

    build.build()
    return torch, _native, vd


def _call(torch, native, xy_dev, w, h, metric, lab, dist):
    lib = native.lib()
    stream = torch.cuda.current_stream().cuda_stream
    return lib.vd_exact_noalloc(xy_dev.data_ptr(), xy_dev.shape[0], w, h, metric,
                                None if lab is None else lab.data_ptr(),
                                None if dist is None else dist.data_ptr(), stream)


def test_exact_noalloc_matches_vd_exact_twice(env, orc):
    torch, native, vd = env
    cases = [(300, 211, 2000, 7, vd.EUCLID), (512, 384, 700, 8, vd.MANHATTAN)]
    for w, h, s, seed, metric in cases:
        xy = inputs.uniform_seeds(w, h, s, seed=seed)
        xy[-1] = xy[0]  # coinciding seeds: lowest index must win
        sim = vd.VoronoiSim(w, h, s)
        sim.set_seeds(xy)
        want_l, want_d = sim.exact(metric=metric)
        sim.close()
        xy_dev = torch.from_numpy(xy).cuda()
        lab = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        rc = _call(torch, native, xy_dev, w, h, metric, lab, dist)
        torch.cuda.synchronize()
        assert rc == native.VD_OK, native.last_error()
        np.testing.assert_array_equal(lab.cpu().numpy(), want_l)
        np.testing.assert_array_equal(dist.cpu().numpy(), want_d)
        brute_l, brute_d = orc.exact_brute(w, h, xy, metric)
        np.testing.assert_array_equal(lab.cpu().numpy(), brute_l)
        np.testing.assert_array_equal(dist.cpu().numpy(), brute_d)


def test_exact_noalloc_at_the_bound(env):
    """200000 seeds on 632 x 632 (just under 2 pixels a seed: one bucket a
    pixel, the most buckets per seed the bucket rule keeps, so the largest
    scratch need at this seed count): the request fits and equals vd_exact,
    twice in a row."""
    torch, native, vd = env
    w = h = 632
    s = 200000
    xy = inputs.uniform_seeds(w, h, s, seed=11)
    sim = vd.VoronoiSim(w, h, s)
    sim.set_seeds(xy)
    want_l, want_d = sim.exact()
    sim.close()
    xy_dev = torch.from_numpy(xy).cuda()
    for _ in range(2):
        lab = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        rc = _call(torch, native, xy_dev, w, h, vd.EUCLID, lab, dist)
        torch.cuda.synchronize()
        assert rc == native.VD_OK, native.last_error()
        np.testing.assert_array_equal(lab.cpu().numpy(), want_l)
        np.testing.assert_array_equal(dist.cpu().numpy(), want_d)


def test_exact_noalloc_rejects_bad_requests(env):
    torch, native, vd = env
    w = h = 2048
    big = torch.from_numpy(inputs.uniform_seeds(w, h, 400000, seed=1)).cuda()
    out = torch.empty((h, w), dtype=torch.int32, device="cuda")
    assert _call(torch, native, big, w, h, vd.EUCLID, out, None) == native.VD_EINVAL
    assert "static maximum" in native.last_error()
    xy = inputs.uniform_seeds(64, 64, 10, seed=2)
    xy[3] = (64, 5)  # x outside the 64-wide grid
    bad = torch.from_numpy(xy).cuda()
    out = torch.empty((64, 64), dtype=torch.int32, device="cuda")
    assert _call(torch, native, bad, 64, 64, vd.EUCLID, out, None) == native.VD_EINVAL
    assert "outside" in native.last_error()
    # the rejected calls leave the entry point usable
    good = torch.from_numpy(inputs.uniform_seeds(64, 64, 10, seed=3)).cuda()
    assert _call(torch, native, good, 64, 64, vd.EUCLID, out, None) == native.VD_OK
    torch.cuda.synchronize()
