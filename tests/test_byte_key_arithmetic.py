"""Host-side check of the byte-offset key's arithmetic (the exactness argument
of the Euclidean byte-offset pass), written out with numpy integer operations:

* v = e - (x_p | y_p << 16) + 2^15 carries dx and dy, modulo 256, in its bytes
  0 and 2, so the dot product of those two signed bytes with themselves is
  dx^2 + dy^2 whenever both lie in [-128, 127];
* the winner test, (e + h * 0x10001 - (x_p | y_p << 16)) & mask == 0 with
  mask = (0xFFFF & ~(2h - 1)) * 0x10001, holds exactly when dx and dy lie in
  [-h, h);
* the far entry (49151, 0) of the position table fails that test from every
  pixel of a grid up to 32768 wide;
* inside the window no key d * 2^lb + label wraps, for the window the host
  picks for lb.

Everything here is plain modular integer arithmetic; the GPU parity tests
check the kernels themselves against the oracle.
"""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def _pack(x, y):
    return (np.asarray(x, np.uint64) | (np.asarray(y, np.uint64) << np.uint64(16))) & M32


def _signed_byte(b):
    b = b.astype(np.int64)
    return np.where(b >= 128, b - 256, b)


def _dp4a_bytes02(v):
    b0 = _signed_byte(v & np.uint64(0xFF))
    b2 = _signed_byte((v >> np.uint64(16)) & np.uint64(0xFF))
    return b0 * b0 + b2 * b2


def _window(lb):
    """The host's choice: 128 for the 16-bit field, else the largest power of
    two h with (2h^2 + 1) * 2^lb <= 2^32."""
    if lb == 16:
        return 128
    for h in (64, 32, 16, 8, 4, 2):
        if (2 * h * h + 1) << lb <= 1 << 32:
            return h
    return 0


def _cases(rng, n):
    px = rng.integers(0, 32768, n)
    py = rng.integers(0, 32768, n)
    near = rng.random(n) < 0.7
    dx = np.where(near, rng.integers(-200, 200, n), rng.integers(-32767, 32768, n))
    dy = np.where(near, rng.integers(-200, 200, n), rng.integers(-32767, 32768, n))
    sx = np.clip(px + dx, 0, 32767)
    sy = np.clip(py + dy, 0, 32767)
    return px, py, sx, sy


def test_distance_bytes_exact_in_signed_byte_range():
    rng = np.random.default_rng(0)
    px, py, sx, sy = _cases(rng, 400_000)
    e = _pack(sx, sy)
    v = (e + np.uint64(0x8000) - _pack(px, py)) & M32
    d = _dp4a_bytes02(v)
    dx, dy = sx - px, sy - py
    inside = (dx >= -128) & (dx <= 127) & (dy >= -128) & (dy <= 127)
    assert inside.sum() > 100_000
    np.testing.assert_array_equal(d[inside], dx[inside] ** 2 + dy[inside] ** 2)


def test_window_test_iff_inside_window():
    rng = np.random.default_rng(1)
    px, py, sx, sy = _cases(rng, 400_000)
    e = _pack(sx, sy)
    dx, dy = sx - px, sy - py
    for h in (128, 64, 32, 16, 8):
        mask = np.uint64(((0xFFFF & ~(2 * h - 1)) * 0x10001) & 0xFFFFFFFF)
        t = (e + np.uint64(h * 0x10001) - _pack(px, py)) & M32
        ok = (t & mask) == 0
        inside = (dx >= -h) & (dx < h) & (dy >= -h) & (dy < h)
        assert inside.sum() > 100, h
        np.testing.assert_array_equal(ok, inside, err_msg=f"h={h}")


def test_window_edges_exhaustive():
    # every offset in [-2h - 3, 2h + 3]^2 around pixels at the grid's corners and middle
    for h in (128, 16, 8):
        r = np.arange(-2 * h - 3, 2 * h + 4)
        dx, dy = [a.ravel() for a in np.meshgrid(r, r)]
        mask = np.uint64(((0xFFFF & ~(2 * h - 1)) * 0x10001) & 0xFFFFFFFF)
        for px, py in [(300, 300), (16000, 9), (32767 - 300, 32767 - 300)]:
            sx, sy = px + dx, py + dy
            t = (_pack(sx, sy) + np.uint64(h * 0x10001) - _pack(px, py)) & M32
            ok = (t & mask) == 0
            inside = (dx >= -h) & (dx < h) & (dy >= -h) & (dy < h)
            np.testing.assert_array_equal(ok, inside, err_msg=f"h={h} pixel={(px, py)}")
            if h == 128:
                v = (_pack(sx, sy) + np.uint64(0x8000) - _pack(px, py)) & M32
                np.testing.assert_array_equal(_dp4a_bytes02(v)[inside], (dx ** 2 + dy ** 2)[inside])


def test_far_entry_fails_from_every_pixel():
    px, py = [a.ravel() for a in np.meshgrid(np.arange(0, 32768, 7), np.arange(0, 32768, 511))]
    far = _pack(49151, 0)
    for h in (128, 64, 32, 16, 8):
        mask = np.uint64(((0xFFFF & ~(2 * h - 1)) * 0x10001) & 0xFFFFFFFF)
        t = (far + np.uint64(h * 0x10001) - _pack(px, py)) & M32
        assert np.all((t & mask) != 0), h


def test_no_key_wraps_inside_the_window():
    for lb in range(16, 31):
        h = _window(lb)
        if h == 0:
            continue
        # the largest distance inside the window and the largest label field
        d_max = 2 * h * h
        assert d_max * (1 << lb) + (1 << lb) - 1 < 1 << 32, lb
        # and the winner bound d < h^2 leaves room below every outside seed (d >= h^2)
        assert (h * h) * (1 << lb) <= 1 << 32
    assert _window(16) == 128 and _window(17) == 64 and _window(19) == 32 and _window(23) == 8


def test_empty_label_field_indexes_the_far_entry():
    # key = d * 2^lb + (-1) mod 2^32 leaves all ones in the label field; plus
    # one, masked, is 0: entry 0 of the position table, the far position
    for lb in (16, 17, 19, 23):
        for d in (0, 1, 5, 12345, 32768):
            key = (d * (1 << lb) + 0xFFFFFFFF) & 0xFFFFFFFF
            assert key & ((1 << lb) - 1) == (1 << lb) - 1
            assert (key + 1) & ((1 << lb) - 1) == 0
        # a real label c < n < 2^lb indexes entry c + 1
        for c in (0, 7, (1 << lb) - 2):
            key = (3 * (1 << lb) + c) & 0xFFFFFFFF
            assert (key + 1) & ((1 << lb) - 1) == c + 1
