"""Pins of oracle/public.py (paper-form public image, Sect. 6.5.1 Fig. 10; statistics,
Sect. 6.6) against closed forms, brute force and high-precision direct evaluation."""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import fds, public
from paper_1512_02951_gb300 import synth


def _decimal_cos(x: Decimal) -> Decimal:
    """cos by its Taylor series in the current decimal precision (|x| < 8 here)."""
    term, total, n = Decimal(1), Decimal(1), 0
    while True:
        n += 2
        term = -term * x * x / (n * (n - 1))
        if abs(term) < Decimal(10) ** -(getcontext().prec + 2):
            return total
        total += term


def _decimal_pi() -> Decimal:
    """pi by Machin's formula, 16 arctan(1/5) - 4 arctan(1/239)."""
    def arctan_inv(m: int) -> Decimal:
        x, total, k = Decimal(1) / m, Decimal(0), 0
        term = x
        while abs(term) > Decimal(10) ** -(getcontext().prec + 2):
            total += term / (2 * k + 1) * (-1) ** k
            k += 1
            term = x ** (2 * k + 1)
        return total
    return 16 * arctan_inv(5) - 4 * arctan_inv(239)


def _direct_public_block(coefs: np.ndarray) -> np.ndarray:
    """8x8 bytes: round-half-away(sum_uv b_u(y) b_v(x) F[u, v]) clamped, in 60-digit decimal
    arithmetic straight from the definition of the orthonormal DCT-II basis."""
    getcontext().prec = 60
    pi = _decimal_pi()
    half_sqrt2 = Decimal(2).sqrt() / 2

    def b(u, y):
        c = half_sqrt2 if u == 0 else Decimal(1)
        return c / 2 * _decimal_cos(Decimal((2 * y + 1) * u) * pi / 16)

    out = np.zeros((8, 8), dtype=np.int64)
    for y in range(8):
        for x in range(8):
            s = sum(b(u, y) * b(v, x) * int(coefs[u, v]) for u in range(8) for v in range(8)
                    if coefs[u, v])
            r = int((abs(s) + Decimal("0.5")).to_integral_value(rounding="ROUND_FLOOR"))
            out[y, x] = min(max(r if s >= 0 else -r, 0), 255)
    return out


def _fragment_with(k, entries, by=1, bx=1):
    """A public fragment [by, bx, 3, 63 - k] of zeros with (u, v) -> value set in every
    channel-block."""
    pub = np.zeros((by, bx, 3, 63 - k), dtype=np.int16)
    zz = fds.ZIGZAG
    for (u, v), val in entries.items():
        z = zz.index((u, v))
        assert z > k
        pub[..., z - k - 1] = val
    return pub


@pytest.mark.parametrize("k", [0, 5, 63])
def test_flat_and_empty_fragments_give_mid_grey(k):
    img = np.full((16, 24, 3), 77, dtype=np.uint8)
    pub, _ = fds.protect(img, bytes(16), bytes(16), k)
    assert np.all(public.public_image(pub, k, 24, 16) == 128)
    if k == 63:   # no public coefficients at all, whatever the image
        pub, _ = fds.protect(synth.make_image(24, 16, 3), bytes(16), bytes(16), 63)
        assert np.all(public.public_image(pub, 63, 24, 16) == 128)


def test_half_integer_pixels_round_away_from_zero():
    # F[0, 4] = 4 alone: b_0(y) b_4(x) F = +-4/8 = +-0.5 (cos((2x+1) pi / 4) = +-1/sqrt(2)),
    # so pixels are exactly 128.5 or 127.5 -> 129 or 128 (half away from zero)
    pub = _fragment_with(5, {(0, 4): 4})
    got = public.public_image(pub, 5, 8, 8)[..., 0]
    sign = np.sign(np.cos((2 * np.arange(8) + 1) * np.pi / 4))
    want = np.where(sign > 0, 129, 128)[None, :].repeat(8, axis=0)
    assert np.array_equal(got, want)
    # F[4, 0] = -4: rows instead of columns, 127.5 -> 128 and 128.5 -> 129
    pub = _fragment_with(5, {(4, 0): -4})
    got = public.public_image(pub, 5, 8, 8)[..., 1]
    want = np.where(sign > 0, 128, 129)[:, None].repeat(8, axis=1)
    assert np.array_equal(got, want)


def test_matches_direct_decimal_evaluation():
    rng = np.random.default_rng(5)
    for k in (0, 5, 20):
        pub = rng.integers(-300, 301, size=(1, 2, 3, 63 - k)).astype(np.int16)
        pub[..., ::3] //= 16                       # a mix of small and large values
        got = public.public_image(pub, k, 16, 8)
        part1 = np.zeros((1, 2, 3, k + 1), dtype=np.int64)
        part1[..., 0] = 1024
        coefs = fds.merge(part1, pub.astype(np.int64))
        for bx in range(2):
            for c in range(3):
                want = _direct_public_block(coefs[0, bx, c])
                assert np.array_equal(got[:, 8 * bx: 8 * bx + 8, c], want), (k, bx, c)


def test_public_fragment_back_from_an_exact_public_image():
    # coefficients whose public image is integral and unclamped come back exactly
    pub = _fragment_with(5, {(0, 4): 16, (4, 4): -24, (4, 0): 8}, by=2, bx=1)
    img = public.public_image(pub, 5, 8, 16)
    assert np.array_equal(public.public_from_image(img, 5), pub)


def test_histogram_and_pair_sums_by_brute_force():
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(5, 7, 3)).astype(np.uint8)
    hist = public.histogram(img)
    for c in range(3):
        for level in range(256):
            assert hist[c, level] == sum(1 for y in range(5) for x in range(7) if img[y, x, c] == level)
    sums = public.pair_sums(img)
    for d, (dy, dx) in enumerate([(0, 1), (1, 0), (1, 1)]):
        for c in range(3):
            pairs = [(int(img[y, x, c]), int(img[y + dy, x + dx, c]))
                     for y in range(5 - dy) for x in range(7 - dx)]
            want = (len(pairs), sum(a for a, _ in pairs), sum(b for _, b in pairs),
                    sum(a * a for a, _ in pairs), sum(b * b for _, b in pairs), sum(a * b for a, b in pairs))
            assert tuple(int(v) for v in sums[d, c]) == want


def test_correlation_closed_forms():
    yy, xx = np.mgrid[0:16, 0:16]
    ramp = np.stack([xx * 8, yy * 8, (xx + yy) * 4], axis=-1).astype(np.uint8)
    r = public.correlation(public.pair_sums(ramp))
    assert np.allclose(r, 1.0)            # every neighbour is an increasing affine function
    board = np.repeat((((xx + yy) % 2) * 255)[..., None], 3, axis=-1).astype(np.uint8)
    r = public.correlation(public.pair_sums(board))
    assert np.allclose(r[0], -1.0) and np.allclose(r[1], -1.0)   # y = 255 - x
    assert np.allclose(r[2], 1.0)                                  # diagonal neighbours equal
    flat = np.full((8, 8, 3), 9, dtype=np.uint8)
    assert np.all(np.isnan(public.correlation(public.pair_sums(flat))))   # zero variance
    noise = np.random.default_rng(3).integers(0, 256, size=(256, 256, 3)).astype(np.uint8)
    assert np.all(np.abs(public.correlation(public.pair_sums(noise))) < 0.02)
