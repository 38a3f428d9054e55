"""Pins of oracle/strong.py (strong level of protection, Sect. 6.3.2, Fig. 8)."""
import hashlib

import numpy as np
import pytest

from oracle import aes, fds, public, strong
from paper_1512_02951_gb300 import synth

KEY, IV = bytes(range(16)), bytes(range(16, 32))


def test_hash_primitive_is_sha512():
    # FIPS 180-4 example: SHA-512("abc")
    want = ("ddaf35a193617abacc417349ae20413112e6fa4e89a97ea20a9eeee64b55d39a"
            "2192992a274fc1a836ba3c23a3feebbd454d4423643ce80e2a9ac94fa54ca49f")
    assert hashlib.sha512(b"abc").hexdigest() == want


@pytest.mark.parametrize("k", [0, 5])
def test_flat_image_mask_layout(k):
    # a flat block: Part 1 = (8 c, 0, .., 0), public image 128; the strong image is
    # 128 XOR the digest of those k + 1 little-endian int16, digest byte 8 y + x at (y, x)
    c = (37, 200, 3)
    img = np.empty((8, 16, 3), dtype=np.uint8)
    img[...] = c
    got, _ = strong.protect_strong(img, KEY, IV, k)
    for ch in range(3):
        msg = (8 * c[ch]).to_bytes(2, "little") + bytes(2 * k)
        d = np.frombuffer(hashlib.sha512(msg).digest(), dtype=np.uint8).reshape(8, 8)
        for bx in range(2):
            assert np.array_equal(got[:, 8 * bx: 8 * bx + 8, ch], 128 ^ d)


def test_mask_is_an_involution_and_depends_on_every_coefficient():
    rng = np.random.default_rng(2)
    part1 = rng.integers(-50, 50, size=(2, 3, 3, 6))
    m = strong.masks(part1)
    assert m.shape == (2, 3, 3, 8, 8)
    img = rng.integers(0, 256, size=(16, 24, 3)).astype(np.uint8)
    assert np.array_equal(strong._apply_mask(strong._apply_mask(img, part1), part1), img)
    for j in range(6):          # one coefficient changed by one: a different mask
        p2 = part1.copy()
        p2[1, 2, 0, j] += 1
        m2 = strong.masks(p2)
        assert not np.array_equal(m2[1, 2, 0], m[1, 2, 0])
        assert np.array_equal(np.delete(m2.reshape(-1, 64), 15, 0), np.delete(m.reshape(-1, 64), 15, 0))


@pytest.mark.parametrize("k", [0, 5])
def test_round_trip_quality_and_hiding(k):
    img = synth.make_image(64, 48, 3 + k)
    s_img, cipher = strong.protect_strong(img, KEY, IV, k)
    assert cipher == fds.protect(img, KEY, IV, k)[1]                  # Part 1 as in the first level
    back = strong.restore_strong(s_img, cipher, KEY, IV, k)
    assert fds.psnr(back, img) > 40.0                                  # public image bytes are rounded
    # without Part 1 the public image is hidden: the strong image is close to uniform noise
    r = public.correlation(public.pair_sums(s_img))
    assert np.all(np.abs(r) < 0.15)
    plain = public.correlation(public.pair_sums(img))
    assert np.all(plain > 0.8)


def test_restore_matches_first_level_when_the_public_image_is_exact():
    # if the public image round trip loses nothing (no clamping, integral pixels), the strong
    # level restores exactly what the first level restores
    pub = np.zeros((1, 2, 3, 58), dtype=np.int16)
    pub[..., fds.ZIGZAG.index((0, 4)) - 6] = 16
    part1 = np.zeros((1, 2, 3, 6), dtype=np.int64)
    part1[..., 0] = 800
    part1[..., 2] = 3
    cipher = aes.ctr_xcrypt(KEY, IV, part1.astype("<i2").tobytes())
    s_img = strong._apply_mask(public.public_image(pub, 5, 16, 8), part1)
    assert np.array_equal(strong.restore_strong(s_img, cipher, KEY, IV, 5),
                          fds.restore(pub, cipher, KEY, IV, 5, 16, 8))
