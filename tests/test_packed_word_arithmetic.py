"""Host-side check of the position-tagged words' arithmetic (the dJFA passes
of vd_pass_pk.cuh), written out with numpy integer operations for each word
layout M (8: up to 32767 seeds; 7: to 2^17 - 1; 6: to 2^18; 4: to 2^22, the
label split around the x field and distances saturated at 63):

* a pixel's key of a candidate word is exactly d * 2^ks (+ 2^15 for M = 8)
  + label code whenever the candidate's seed lies in the window [-h, h)^2
  around the pixel (h = 2^(M-1)) (M = 4: min(d, 63)): the guard bit absorbs
  the borrow out of the x field, the label bits below it see no borrow, and
  the masked field bytes read as signed numbers are 2^(8-M) dx and
  2^(8-M) dy;
* for any seed, in the window or not, the key's low bits are the label code
  and the distance part does not wrap (wide keys stay below 2^31; narrow
  ones hold d <= 2^15 in their upper 16 bits, compared as unsigned; M = 4
  keys stay below 63 * 2^26 + 2^26);
* keys order in-window candidates as (d, label) does (the tie rule; with
  M = 4 for d < 63, the distances the winner check accepts);
* a word decodes to its label, the empty word to -1 (with M = 6 and 2^18
  seeds the last seed's code is also the empty code, told apart by the flag
  bit), and the winner check's table index (code + 1) mod 2^lb lands on the
  far entry for the empty code only;
* the word rebuilt from a winning key and the seed position is the
  candidate's own word.

The GPU parity tests check the kernels themselves against the oracle.
"""
import numpy as np
import pytest

U = np.uint64
M32 = U(0xFFFFFFFF)


class Layout:
    def __init__(self, m):
        self.m = m
        self.narrow = m == 8
        self.split = m == 4
        self.lb = 15 if self.narrow else 26 if self.split else 24 - m
        self.ks = 16 if self.narrow else self.lb
        # the key's label code: all the label bits where the word holds them
        self.lm = 0x030FFFFF if self.split else (1 << self.lb) - 1
        self.h = 1 << (m - 1)
        self.xm = (1 << m) - 1
        self.xs = 8 if self.narrow else 20 if self.split else self.lb
        self.ys = 32 - m
        self.fm = (self.xm << self.xs) | (self.xm << self.ys)
        self.g = 0x00800000 if self.narrow else 0x04000000 if self.split else 0x01000000
        self.ef = 0x02000000 if m == 6 else 0x08000000 if self.split else 0
        self.empty = (0xFF | (0x7F << 16) | self.g) if self.narrow else (self.lm | self.g | self.ef)

    def neg_pix(self, x, y):
        p = ((U(x) & U(self.xm)) << U(self.xs)) | ((U(y) & U(self.xm)) << U(self.ys))
        return (U(0) - p) & M32

    def word(self, l, x, y):
        l, x, y = U(l), U(x), U(y)
        if self.narrow:
            return ((l & U(0xFF)) | ((x & U(0xFF)) << U(8)) | ((l & U(0x7F00)) << U(8)) | U(self.g) |
                    ((y & U(0xFF)) << U(24)))
        if self.split:
            l = (l & U(0xFFFFF)) | ((l & U(0x300000)) << U(4))
        return l | U(self.g) | ((x & U(self.xm)) << U(self.xs)) | ((y & U(self.xm)) << U(self.ys))

    def code_label(self, c):
        """The label a key's (or word's) code names (M = 4: the split bits joined)."""
        c = U(c)
        if self.split:
            return ((c & U(0xFFFFF)) | ((c >> U(4)) & U(0x300000))).astype(np.int64)
        return (c & U(self.lm)).astype(np.int64)

    def label(self, w):
        w = U(w)
        if self.ef:
            return np.where((w & U(self.ef)) != 0, -1, self.code_label(w))
        c = ((w & U(0xFF)) | ((w >> U(8)) & U(0x7F00))) if self.narrow else (w & U(self.lm))
        return np.where(c == U(self.lm), -1, c.astype(np.int64))

    @staticmethod
    def _dp4a_self(b):
        s = np.zeros(np.shape(b), np.int64)
        for j in range(4):
            byte = ((b >> U(8 * j)) & U(0xFF)).astype(np.int64)
            byte = np.where(byte >= 128, byte - 256, byte)
            s += byte * byte
        return s.astype(np.uint64)

    def key(self, w, pn):
        b = ((U(w) + U(pn)) & M32) & U(self.fm)
        d = self._dp4a_self(b)
        if self.narrow:
            # byte permute 0x5420: bytes (w.b0, w.b2, d.b0, d.b1)
            return (U(w) & U(0xFF)) | (((U(w) >> U(16)) & U(0xFF)) << U(8)) | ((d & U(0xFFFF)) << U(16))
        if self.split:
            # 256 d, saturated at 63 * 256, times 2^18
            return (np.minimum(d, U(63 * 256)) * U(1 << 18) + (U(w) & U(self.lm))) & M32
        return (d * U(1 << (8 + self.m)) + (U(w) & U(self.lm))) & M32

    def word_of_key(self, key, x, y):
        e = U(x) | (U(y) << U(16))
        if self.narrow:
            # byte permute 0x6140: bytes (key.b0, e.b0, key.b1, e.b2)
            return ((key & U(0xFF)) | ((e & U(0xFF)) << U(8)) | (((key >> U(8)) & U(0xFF)) << U(16)) |
                    (((e >> U(16)) & U(0xFF)) << U(24)))
        f = (U(self.g) | ((e << U(self.xs)) & U(self.xm << self.xs)) |
             ((e << U(16 - self.m)) & U(self.xm << self.ys))) & M32
        return (key & U(self.lm)) | f

    def index(self, key):
        """The winner check's position-table index: (label + 1) mod 2^22 for
        M = 4, (code + 1) mod 2^lb otherwise."""
        if self.split:
            return (U(self.code_label(key)) + U(1)) & U(0x3FFFFF)
        return (U(key) + U(1)) & U(self.lm)


LAYOUTS = [Layout(8), Layout(7), Layout(6), Layout(4)]
# largest seed count each layout takes
N_MAX = {8: 32767, 7: 131071, 6: 262144, 4: 1 << 22}


def _cases(rng, lay, n, near):
    x0 = 4 * rng.integers(0, 8192, n)  # a quad's first pixel (x0 % 4 == 0)
    i = rng.integers(0, 4, n)
    px = x0 + i
    py = rng.integers(0, 32768, n)
    if near:
        dx = rng.integers(-lay.h, lay.h, n)
        dy = rng.integers(-lay.h, lay.h, n)
    else:
        dx = rng.integers(-32767, 32768, n)
        dy = rng.integers(-32767, 32768, n)
    sx = np.clip(px + dx, 0, 32767)
    sy = np.clip(py + dy, 0, 32767)
    labels = rng.integers(0, N_MAX[lay.m], n)
    return x0, i, px, py, sx, sy, labels


def _pixel_pn(lay, x0, y, i):
    return (lay.neg_pix(x0, y) - (U(i) << U(lay.xs))) & M32


@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda l: f"M{l.m}")
def test_keys_exact_inside_the_window(lay):
    rng = np.random.default_rng(lay.m)
    x0, i, px, py, sx, sy, lab = _cases(rng, lay, 400000, near=True)
    inside = (sx - px >= -lay.h) & (sx - px < lay.h) & (sy - py >= -lay.h) & (sy - py < lay.h)
    w = lay.word(lab, sx, sy)
    k = lay.key(w, _pixel_pn(lay, x0, py, i))
    d = ((sx - px) ** 2 + (sy - py) ** 2).astype(np.uint64)
    if lay.split:
        want = np.minimum(d, U(63)) * U(1 << lay.ks) + (w & U(lay.lm))
        assert (lay.code_label(w & U(lay.lm)) == lab).all()
    else:
        want = d * U(1 << lay.ks) + U(lab) + (U(1 << 15) if lay.narrow else U(0))
    assert inside.mean() > 0.9
    np.testing.assert_array_equal(k[inside], want[inside])


@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda l: f"M{l.m}")
def test_key_low_bits_and_range_for_any_seed(lay):
    rng = np.random.default_rng(10 + lay.m)
    x0, i, px, py, sx, sy, lab = _cases(rng, lay, 400000, near=False)
    k = lay.key(lay.word(lab, sx, sy), _pixel_pn(lay, x0, py, i))
    if lay.narrow:
        assert (k < U(1 << 32)).all() and ((k >> U(16)) <= U(1 << 15)).all()
    elif lay.split:
        assert (k < U(1 << 32)).all() and ((k >> U(26)) <= U(63)).all()
    else:
        assert (k < U(1 << 31)).all()
    np.testing.assert_array_equal(lay.code_label(k & U(lay.lm)), lab)
    # the empty word's key also names the empty code
    ke = lay.key(np.full(1000, lay.empty, np.uint64), _pixel_pn(lay, x0[:1000], py[:1000], i[:1000]))
    assert ((ke & U(lay.lm)) == U(lay.lm)).all() and (ke < U(1 << 32)).all()


@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda l: f"M{l.m}")
def test_key_order_is_distance_then_label(lay):
    rng = np.random.default_rng(20 + lay.m)
    n = 200000
    x0, i, px, py, sx, sy, lab = _cases(rng, lay, n, near=True)
    _, _, _, _, sx2, sy2, lab2 = _cases(rng, lay, n, near=True)
    sx2 = np.clip(px + rng.integers(-lay.h, lay.h, n), 0, 32767)
    sy2 = np.clip(py + rng.integers(-lay.h, lay.h, n), 0, 32767)
    ins = lambda sx_, sy_: (sx_ - px >= -lay.h) & (sx_ - px < lay.h) & (sy_ - py >= -lay.h) & (sy_ - py < lay.h)
    ok = ins(sx, sy) & ins(sx2, sy2)
    pn = _pixel_pn(lay, x0, py, i)
    k1 = lay.key(lay.word(lab, sx, sy), pn)
    k2 = lay.key(lay.word(lab2, sx2, sy2), pn)
    d1 = (sx - px) ** 2 + (sy - py) ** 2
    d2 = (sx2 - px) ** 2 + (sy2 - py) ** 2
    if lay.split:
        # saturated distances tie at 63 (the check rejects such winners)
        d1, d2 = np.minimum(d1, 63), np.minimum(d2, 63)
        assert ((d1 < 63) & (d2 < 63) & ok).mean() > 0.5
    less = (d1 < d2) | ((d1 == d2) & (lab < lab2))
    np.testing.assert_array_equal((k1 < k2)[ok], less[ok])


@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda l: f"M{l.m}")
def test_labels_empty_word_and_check_index(lay):
    rng = np.random.default_rng(30 + lay.m)
    lab = rng.integers(0, N_MAX[lay.m], 100000)
    x = rng.integers(0, 32768, 100000)
    y = rng.integers(0, 32768, 100000)
    np.testing.assert_array_equal(lay.label(lay.word(lab, x, y)), lab)
    assert int(lay.label(np.array([lay.empty], np.uint64))[0]) == -1
    if lay.m == 6:
        # 2^18 seeds: the last seed's code is the all-ones code, a real label
        assert int(lay.label(lay.word(np.array([N_MAX[6] - 1]), np.array([5]), np.array([9])))[0]) == N_MAX[6] - 1
    if lay.split:
        # 2^22 seeds: the last seed's code is the all-ones code, a real label
        top = N_MAX[4] - 1
        assert int(lay.label(lay.word(np.array([top]), np.array([5]), np.array([9])))[0]) == top
        assert int(lay.code_label(U(lay.lm))) == top
    # the winner check indexes the position table (far entry first) with
    # (label + 1) mod 2^lb (M = 4: mod 2^22, the label joined from its split
    # code): seeds land on their entry, the empty code on the far one
    if lay.split:
        live = lab[lab < N_MAX[4] - 1]
        codes = np.concatenate([lay.word(live, 0, 0) & U(lay.lm), [U(lay.lm)]]).astype(np.uint64)
        want = live + 1
    else:
        live = lab[lab < lay.lm]
        codes = np.concatenate([live, [lay.lm]]).astype(np.uint64)
        want = live + 1
    idx = lay.index(codes)
    np.testing.assert_array_equal(idx[:-1].astype(np.int64), want)
    assert int(idx[-1]) == 0


@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda l: f"M{l.m}")
def test_winner_word_is_the_candidate_word(lay):
    rng = np.random.default_rng(40 + lay.m)
    x0, i, px, py, sx, sy, lab = _cases(rng, lay, 200000, near=True)
    w = lay.word(lab, sx, sy)
    k = lay.key(w, _pixel_pn(lay, x0, py, i))
    np.testing.assert_array_equal(lay.word_of_key(k, sx, sy), w)
