"""Pins of the oracle's fragmentation, layouts and protect/restore pipeline (Sect. 6.3.1)."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import dct, fds
from paper_1512_02951_gb300 import synth


def _lib_ctr(key, iv, data):
    c = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    e = c.Cipher(c.algorithms.AES(key), c.modes.CTR(iv)).encryptor()
    return e.update(data) + e.finalize()


def test_zigzag_starts_with_the_papers_default_selection():
    want = [tuple(int(t) for t in ln.split()) for ln in read_golden("paper_selection.txt")]
    assert fds.ZIGZAG[:6] == want


def test_zigzag_is_a_diagonal_snake():
    zz = fds.ZIGZAG
    assert sorted(zz) == [(u, v) for u in range(8) for v in range(8)]
    s = [u + v for u, v in zz]
    assert s == sorted(s)
    for (u0, v0), (u1, v1) in zip(zz, zz[1:]):
        assert max(abs(u1 - u0), abs(v1 - v0)) == 1            # neighbours in the grid
    assert zz[-1] == (7, 7)


def test_sizes():
    assert fds.sizes(512, 512, 0) == (64 * 64 * 3 * 126, 64 * 64 * 3 * 2)
    assert fds.sizes(4096, 4096, 5) == (91226112, 9437184)
    with pytest.raises(ValueError):
        fds.sizes(100, 64, 0)
    with pytest.raises(ValueError):
        fds.sizes(64, 64, 64)


@pytest.mark.parametrize("k", [0, 5])
def test_private_layout_with_constant_blocks(k):
    # constant blocks: DC = 8 * value, every AC = 0; the decrypted private stream must hold
    # 8 * value at ((by * BX + bx) * 3 + c) * (k + 1), zeros elsewhere
    by, bx = 2, 3
    vals = np.arange(by * bx * 3).reshape(by, bx, 3) * 7 % 256
    blocks = np.broadcast_to(vals[..., None, None], (by, bx, 3, 8, 8))
    img = dct.blocks_to_image(np.ascontiguousarray(blocks)).astype(np.uint8)
    key, iv = synth.make_key(1), synth.make_iv(2)
    public, private = fds.protect(img, key, iv, k)
    assert not public.any()
    plain = np.frombuffer(_lib_ctr(key, iv, private), dtype="<i2").reshape(by, bx, 3, k + 1)
    assert np.array_equal(plain[..., 0], 8 * vals)
    assert not plain[..., 1:].any()
    back = fds.restore(public, private, key, iv, k, bx * 8, by * 8)
    assert np.array_equal(back, img)                            # constant blocks are lossless


@pytest.mark.parametrize("k", [0, 5, 63])
def test_split_merge_round_trip(k):
    rng = np.random.default_rng(k)
    q = rng.integers(-500, 500, (3, 4, 8, 8))
    p1, p2 = fds.split(q, k)
    assert p1.shape[-1] == k + 1 and p2.shape[-1] == 63 - k
    assert np.array_equal(fds.merge(p1, p2), q)


@pytest.mark.parametrize("k", [0, 5])
def test_protect_restore_quality(k):
    img = synth.make_image(256, 192, 1)
    key, iv = synth.make_key(3), synth.make_iv(4)
    public, private = fds.protect(img, key, iv, k)
    assert public.shape == (24, 32, 3, 63 - k) and public.dtype == np.int16
    assert len(private) == fds.sizes(256, 192, k)[1]
    back = fds.restore(public, private, key, iv, k, 256, 192)
    diff = np.abs(back.astype(int) - img)
    assert diff.max() <= 3
    frac = float(np.mean(diff == 0))
    assert 0.88 < frac < 0.97                  # int16 rounding is not lossless (Table 5 reading)
    assert fds.psnr(back, img) > 55.0
    # the same fragments under another key do not restore the image
    wrong = fds.restore(public, private, synth.make_key(5), iv, k, 256, 192)
    assert fds.psnr(wrong, img) < 20.0


def test_private_fragment_is_the_encrypted_low_frequencies():
    img = synth.make_image(64, 64, 9)
    key, iv = synth.make_key(6), synth.make_iv(7)
    public, private, f = fds.protect(img, key, iv, 5, return_f64=True)
    plain = np.frombuffer(_lib_ctr(key, iv, private), dtype="<i2").reshape(8, 8, 3, 6)
    for i, (u, v) in enumerate(fds.ZIGZAG[:6]):
        assert np.abs(plain[..., i] - f[..., u, v]).max() <= 0.5 + 1e-9
    for i, (u, v) in enumerate(fds.ZIGZAG[6:]):
        assert np.abs(public[..., i] - f[..., u, v]).max() <= 0.5 + 1e-9
