"""The oracle's bit-packed storage (Sect. 6.4.3, Table 5) against what the paper and plain
integer arithmetic fix: the paper's storage percentages, a bit stream built as one big integer
(independent of the numpy bit matrices), round trips over the whole field ranges, saturation
of 8-bit storage, and losslessness of 11-bit storage on the hardest blocks."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import fds as ofds, pack
from paper_1512_02951_gb300 import synth


def _bigint_stream(codes, widths):
    """Fields LSB-first as one integer, then little-endian bytes."""
    acc, pos = 0, 0
    for c, w in zip(codes, widths):
        assert 0 <= c < (1 << w)
        acc |= c << pos
        pos += w
    return acc.to_bytes((pos + 7) // 8, "little")


def test_paper_storage_percentages():
    for line in read_golden("paper_storage.txt"):
        f = line.split()
        form, bits, pct = int(f[0]), int(f[1]), float(f[2])
        _, priv = pack.sizes(8, 8, 5, form)          # one block: 3 channel-blocks
        assert priv * 8 >= 3 * bits > priv * 8 - 8    # whole bytes of 3 x bits
        _, widths = pack.fields_of(np.zeros((1, 6), dtype=np.int64), True, form)
        assert int(widths.sum()) == bits
        assert round(100 * bits / (64 * 8), 2) == pct


def test_hand_built_fields():
    # DC 2040, AC -1, AC 1023, AC -1023, AC 0 in 11-bit storage
    vals = np.array([[2040, -1, 1023, -1023, 0]])
    codes, widths = pack.fields_of(vals, True, 11)
    assert codes.tolist() == [2040, 1024 | 1, 1023, 1024 | 1023, 0]
    assert pack.pack_bits(codes, widths) == _bigint_stream(codes.tolist(), widths.tolist())
    assert pack.pack_bits(codes, widths)[:2] == bytes([0b11111000, 0b00001111])


@pytest.mark.parametrize("form", [11, 8])
def test_round_trip_over_the_ranges(form):
    rng = np.random.default_rng(form)
    lim = 1023 if form == 11 else 127
    vals = rng.integers(-lim, lim + 1, (500, 7))
    vals[:, 0] = rng.integers(0, 2041, 500)
    vals[:3, 1:] = [[lim] * 6, [-lim] * 6, [0] * 6]
    codes, widths = pack.fields_of(vals, True, form)
    data = pack.pack_bits(codes, widths)
    assert data == _bigint_stream(codes.tolist(), widths.tolist())
    assert np.array_equal(pack.decode(pack.unpack_bits(data, widths), widths, True, 7), vals)


def test_eight_bit_storage_saturates_and_eleven_bit_rejects():
    vals = np.array([[2040, 200, -300, 127, -128]])
    codes, widths = pack.fields_of(vals, True, 8)
    back = pack.decode(pack.unpack_bits(pack.pack_bits(codes, widths), widths), widths, True, 5)
    assert back.tolist() == [[2040, 127, -127, 127, -127]]
    with pytest.raises(OverflowError):
        pack.fields_of(np.array([[0, 1024]]), True, 11)
    with pytest.raises(OverflowError):
        pack.fields_of(np.array([[2048, 0]]), True, 11)


def _edges(w, h):
    yy, xx = np.mgrid[0:h, 0:w]
    img = np.stack([((yy // 2 + xx // 2) % 2) * 255, (xx % 8 < 4) * 255, ((yy + xx) % 3) * 120], axis=-1)
    return img.astype(np.uint8)


@pytest.mark.parametrize("k", [0, 5, 63])
def test_eleven_bit_storage_is_lossless_eight_bit_is_not(k):
    img = _edges(64, 48)
    key, iv = synth.make_key(3), synth.make_iv(4)
    ref = ofds.restore(*ofds.protect(img, key, iv, k), key, iv, k, 64, 48)
    pub, priv = pack.protect_packed(img, key, iv, k, 11)
    assert (len(pub), len(priv)) == pack.sizes(64, 48, k, 11)
    assert np.array_equal(pack.restore_packed(pub, priv, key, iv, k, 11, 64, 48), ref)
    pub8, priv8 = pack.protect_packed(img, key, iv, k, 8)
    back8 = pack.restore_packed(pub8, priv8, key, iv, k, 8, 64, 48)
    assert not np.array_equal(back8, ref)             # saturated AC: lossy, as Table 5 says
