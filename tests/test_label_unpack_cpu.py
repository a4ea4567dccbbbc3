"""Host side of the packed label read-back (vd_get_labels_packed_async): the
unpacking helper against a plain bit-by-bit packing (numpy packbits, least
significant bit first), for every width from 1 to 32 bits, ragged sizes,
streams ending inside a byte, and the empty code."""
import numpy as np
import pytest

from paper_2209_00117_gb300 import vd


def _pack(labels, bits):
    codes = np.asarray(labels, np.int64).reshape(-1) & ((1 << bits) - 1)
    planes = ((codes[:, None] >> np.arange(bits)) & 1).astype(np.uint8).reshape(-1)
    return np.packbits(planes, bitorder="little")


@pytest.mark.parametrize("bits", list(range(1, 33)))
def test_unpack_round_trip(bits):
    rng = np.random.default_rng(bits)
    for h, w in ((1, 1), (3, 7), (17, 33), (64, 40)):
        hi = (1 << bits) - 1  # labels 0 .. 2^bits - 2, and -1
        lab = rng.integers(-1, hi, size=(h, w), dtype=np.int64).astype(np.int32) if bits < 32 else \
            rng.integers(-1, 1 << 31, size=(h, w), dtype=np.int64).astype(np.int32)
        packed = _pack(lab, bits)
        assert packed.size == (h * w * bits + 7) // 8
        np.testing.assert_array_equal(vd.unpack_labels(packed, h, w, bits, rows_per_chunk=2), lab)


def test_label_bits_and_size_check():
    assert [vd.label_bits(n) for n in (1, 2, 3, 255, 256, 262143, 262144)] == [1, 2, 2, 8, 9, 18, 19]
    with pytest.raises(ValueError):
        vd.unpack_labels(np.zeros(3, np.uint8), 2, 2, 7)
