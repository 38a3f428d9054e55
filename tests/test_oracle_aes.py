"""Pins of the oracle's AES-128 and CTR mode against FIPS-197 and an independent library."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import aes


def _crypto():
    return pytest.importorskip("cryptography.hazmat.primitives.ciphers")


def _lib_ecb(key, block):
    c = _crypto()
    e = c.Cipher(c.algorithms.AES(key), c.modes.ECB()).encryptor()
    return e.update(block) + e.finalize()


def _lib_ctr(key, iv, data):
    c = _crypto()
    e = c.Cipher(c.algorithms.AES(key), c.modes.CTR(iv)).encryptor()
    return e.update(data) + e.finalize()


def test_gf_inverse_is_field_inverse():
    for a in range(1, 256):
        assert aes.gf_mul(a, aes.gf_inv(a)) == 1
    assert aes.gf_inv(0) == 0


def test_sbox_is_a_permutation():
    assert sorted(aes.SBOX.tolist()) == list(range(256))


def test_fips197_golden_vectors():
    lines = read_golden("fips197_aes128.txt")
    kinds = set()
    for ln in lines:
        f = ln.split()
        kinds.add(f[0])
        if f[0] == "cipher":
            key, pt, ct = (bytes.fromhex(x) for x in f[1:4])
            got = aes.encrypt_blocks(aes.expand_key(key), np.frombuffer(pt, np.uint8)[None])
            assert got.tobytes() == ct
            assert _lib_ecb(key, pt) == ct          # the fixture itself is checked too
        elif f[0] == "keyexp":
            key, first, words = bytes.fromhex(f[1]), int(f[2]), bytes.fromhex(f[3])
            w = aes.expand_key(key)
            assert w[first: first + 4].tobytes() == words
        elif f[0] == "gfmul":
            a, b, r = (int(x, 16) for x in f[1:4])
            assert aes.gf_mul(a, b) == r
    assert kinds == {"cipher", "keyexp", "gfmul"}


def test_cipher_matches_library_on_random_keys():
    rng = np.random.default_rng(7)
    for _ in range(64):
        key = rng.bytes(16)
        pts = rng.integers(0, 256, (8, 16), dtype=np.uint8)
        got = aes.encrypt_blocks(aes.expand_key(key), pts)
        for i in range(8):
            assert got[i].tobytes() == _lib_ecb(key, pts[i].tobytes())


@pytest.mark.parametrize("iv_hex", [
    "00000000000000000000000000000000",
    "ffffffffffffffffffffffffffffffff",   # wraps modulo 2^128
    "0123456789abcdefffffffffffffffff",   # carry across the 64-bit boundary
    "000000000000000000000000fffffffe",   # carry across the 32-bit boundary
    "f0e1d2c3b4a5968778695a4b3c2d1e0f",
])
@pytest.mark.parametrize("nbytes", [1, 15, 16, 17, 94, 256])
def test_ctr_matches_library(iv_hex, nbytes):
    rng = np.random.default_rng(nbytes)
    key = rng.bytes(16)
    iv = bytes.fromhex(iv_hex)
    data = rng.bytes(nbytes)
    assert aes.ctr_xcrypt(key, iv, data) == _lib_ctr(key, iv, data)


def test_ctr_offset_is_a_suffix_of_the_message():
    rng = np.random.default_rng(3)
    key, iv = rng.bytes(16), bytes.fromhex("00000000000000000000000000fffffe")
    data = rng.bytes(160)
    whole = aes.ctr_xcrypt(key, iv, data)
    assert aes.ctr_xcrypt(key, iv, data[48:], offset=48) == whole[48:]


def test_ctr_is_an_involution():
    rng = np.random.default_rng(4)
    key, iv, data = rng.bytes(16), rng.bytes(16), rng.bytes(1000)
    ct = aes.ctr_xcrypt(key, iv, data)
    assert ct != data
    assert aes.ctr_xcrypt(key, iv, ct) == data
