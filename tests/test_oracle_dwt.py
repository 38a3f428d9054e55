"""Pins of oracle/dwt.py (selective encryption with the DWT, Sect. 6.8-6.12, Figs. 16-18)."""
import hashlib

import numpy as np
import pytest

from conftest import read_golden
from oracle import aes, dwt

KEY, IV = bytes(range(16)), bytes(range(100, 116))


def test_lifting_worked_examples():
    # by hand from the lifting equations: a ramp (the 5/3 predict step cancels linear
    # signals; the symmetric extension x[8] = x[6] leaves one detail at the edge) ...
    assert dwt._lift_forward_1d(np.array([10, 20, 30, 40, 50, 60, 70, 80])).tolist() == \
        [10, 30, 50, 73, 0, 0, 0, 10]
    # ... and an impulse where floor differs from truncation: d0 = 0 - floor(-1/2) = 1
    assert dwt._lift_forward_1d(np.array([0, 0, -1, 0, 0, 0, 0, 0])).tolist() == [1, 0, 0, 0, 1, 1, 0, 0]
    assert dwt._lift_inverse_1d(np.array([1, 0, 0, 0, 1, 1, 0, 0])).tolist() == [0, 0, -1, 0, 0, 0, 0, 0]


def test_constant_and_orientation():
    c = dwt.forward(np.full((8, 8), 200))
    want = np.zeros((8, 8), dtype=np.int64)
    want[:2, :2] = 72                          # constant 200 - 128 in the second-level LL only
    assert np.array_equal(c, want)
    # a horizontal ramp: rows transform to [10, 30, 50, 73 | 0, 0, 0, 10] (shifted by -128),
    # columns are constant, so only the first-level HL (top-right) holds the edge detail
    ramp = np.tile(np.array([10, 20, 30, 40, 50, 60, 70, 80]) + 128, (8, 1))
    c = dwt.forward(ramp)
    assert np.array_equal(c[:4, 4:], np.tile([0, 0, 0, 10], (4, 1)))
    assert not c[4:, :].any()
    assert np.array_equal(dwt.forward(ramp.T), c.T)


def test_integer_to_integer_and_lossless():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 256, size=(5000, 8, 8))
    x[:100] = rng.integers(0, 2, size=(100, 8, 8)) * 255          # extremes
    assert np.array_equal(dwt.inverse(dwt.forward(x)), x)
    lv = dwt.levels(dwt.forward(x))
    assert np.array_equal(dwt.from_levels(*lv), dwt.forward(x))


def _error_bounds():
    """Guaranteed bound on |coefficient| for inputs in [-128, 127]: the lifting without floors
    is a linear map M; each floor adds an error in [-1/2, 1/2] (floor((a + b) / 2) of an
    integer sum is off by 0 or -1/2; floor((a + b + 2) / 4) = (a + b) / 4 + 1/2 + [-1, 0]),
    which later steps carry linearly.  |c| <= max |M x| + 1/2 sum |J_k|."""
    def lin(x, eps):
        it = iter(eps)

        def lift(v):                           # along the last axis, with error terms
            e, o = v[..., 0::2], v[..., 1::2]
            r = np.concatenate([e[..., 1:], e[..., -1:]], -1)
            d = o - (e + r) / 2 - np.array([[next(it) for _ in range(d_.shape[-1])] for d_ in [o]]).reshape(-1)
            left = np.concatenate([d[..., :1], d[..., :-1]], -1)
            s = e + (left + d) / 4 + np.array([next(it) for _ in range(e.shape[-1])])
            return np.concatenate([s, d], -1)

        def d2(b):
            rows = np.stack([lift(b[i]) for i in range(b.shape[0])])
            cols = np.stack([lift(rows[:, j]) for j in range(rows.shape[1])], axis=1)
            return cols

        c = d2(x)
        c[:4, :4] = d2(c[:4, :4].copy())
        return c

    n_eps = 8 * 8 * 2 + 4 * 4 * 2
    zero = np.zeros(n_eps)
    M = np.stack([lin(np.eye(64)[i].reshape(8, 8), zero) for i in range(64)], axis=-1)       # [8, 8, 64]
    J = np.stack([lin(np.zeros((8, 8)), np.eye(n_eps)[k]) for k in range(n_eps)], axis=-1)  # [8, 8, n_eps]
    lin_max = np.maximum(np.where(M > 0, 127 * M, -128 * M).sum(-1), np.where(M > 0, 128 * M, -127 * M).sum(-1))
    return lin_max + 0.5 * np.abs(J).sum(-1)


def test_field_widths_hold_for_every_input():
    # Sect. 6.9.4: 10 bits for every first-level detail and the second-level LL, HL, LH;
    # 11 bits for the second-level HH; the bound is guaranteed, and 11 bits are needed
    bound = _error_bounds()
    widths = np.full((8, 8), 10)
    widths[2:4, 2:4] = 11
    assert np.all(np.floor(bound) <= (1 << (widths - 1)) - 1), bound   # coefficients are integers
    rng = np.random.default_rng(7)
    hh2 = np.abs(dwt.forward(rng.integers(0, 2, size=(20000, 8, 8)) * 255)[:, 2:4, 2:4]).max()
    assert hh2 > 511


def test_paper_storage_arithmetic():
    # Sect. 6.9.4: level 1 = 40 bits, level 2 = 124 bits, level 3 = 480 bits, 644 in total,
    # "about 26 % more than original" (512 bits)
    g = {k: int(v) for k, v in (ln.split() for ln in read_golden("paper_dwt_storage.txt"))}
    assert sum(dwt.L1_BITS) == g["level1_bits"] and sum(dwt.L2_BITS) == g["level2_bits"]
    assert sum(dwt.L3_BITS) == g["level3_bits"]
    assert round(100 * (g["level1_bits"] + g["level2_bits"] + g["level3_bits"] - 512) / 512) == g["extra_percent"]


def test_field_packing_by_hand():
    # two's complement, least significant bit first: -1 in 10 bits = ten ones, then 5 = 101
    assert dwt.pack_fields([-1, 5], (10, 10), 3) == bytes([0xFF, 0x17, 0x00])
    assert dwt.unpack_fields(bytes([0xFF, 0x17, 0x00]), (10, 10)) == [-1, 5]
    with pytest.raises(OverflowError):
        dwt.pack_fields([512], (10,), 2)


def test_hash_primitives():
    # FIPS 180-4 examples: SHA-256("abc"), SHA-512("abc")
    assert hashlib.sha256(b"abc").hexdigest() == \
        "ba7816bf8f01cfea414140de5dae2223b00361a396177a9cb410ff61f20015ad"
    assert hashlib.sha512(b"abc").hexdigest().startswith("ddaf35a193617aba")


def test_protect_layout_on_a_constant_matrix():
    # one constant block: level 1 = four times 72 (200 - 128) in 10-bit fields, levels 2, 3 zero
    m = np.full((8, 8), 200, dtype=np.uint8)
    l1, l2, l3 = dwt.protect(m, KEY, IV)
    l1_plain = dwt.pack_fields([72] * 4, dwt.L1_BITS, 5)
    assert l1 == aes.ctr_xcrypt(KEY, IV, l1_plain)
    m2 = hashlib.sha256(KEY + IV + (0).to_bytes(8, "big") + l1_plain).digest()
    assert l2 == m2[:16]                       # zero coefficients: the mask itself
    m3 = hashlib.sha512(KEY + IV + (0).to_bytes(8, "big") + bytes(16)).digest()
    assert l3 == m3[:60]


def test_round_trip_chunking_and_sensitivity():
    rng = np.random.default_rng(3)
    data = rng.integers(0, 256, size=5000, dtype=np.uint8).tobytes()    # arbitrary bytes
    m = dwt.to_matrix(data, 64)
    assert m.shape == (80, 64) and m.reshape(-1)[:5000].tobytes() == data and not m.reshape(-1)[5000:].any()
    l1, l2, l3 = dwt.protect(m, KEY, IV)
    assert (len(l1), len(l2), len(l3)) == (80 * 5, 80 * 16, 80 * 60)
    assert np.array_equal(dwt.restore(l1, l2, l3, KEY, IV, 64, 80), m)
    # a different key changes every level; a changed pixel changes its block's masks only
    k2 = bytes([KEY[0] ^ 1]) + KEY[1:]
    o1, o2, o3 = dwt.protect(m, k2, IV)
    assert o1 != l1 and o2 != l2 and o3 != l3
    m2 = m.copy()
    m2[9, 9] ^= 1                               # block (1, 1) = block index 9
    p1, p2, p3 = dwt.protect(m2, KEY, IV)
    diff = [b for b in range(80) if p3[60 * b: 60 * b + 60] != l3[60 * b: 60 * b + 60]]
    assert diff == [9]
