"""Exact rounding of DCT / inverse-DCT values of integer blocks.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sect. 6.4.3 turns the float coefficients "back to integer" and warns that the conversion can
lose information.  The reading used here: round half away from zero, decided on the EXACT
real value.  Exact .5 ties are common (every block whose pixel sum S is 4 mod 8 has a DC
coefficient S/8 that is one), so the decision cannot be left to float64.

Why the decision can be made exactly.  With c(m) = cos(m pi / 16),

    b_u(y) b_v(x) = (1/4) c(a) c(b) = (1/8) [c(a - b) + c(a + b)],
    a = 4 if u == 0 else (2y + 1) u,   b = 4 if v == 0 else (2x + 1) v

(for u = 0 the basis value 1/(2 sqrt 2) is (1/2) c(4)).  Each c(m) folds to +-c(j) with
j in 0..8, c(0) = 1 and c(8) = 0, so for an integer block

    8 F[u, v] = N_0 + sum_{j=1..7} N_j c(j)           with integers N_j,

and likewise 8 p[y, x] = M_0 + sum_j M_j c(j) for the inverse transform of integer
coefficients.  {1, c(1), ..., c(7)} is a basis of Q(cos pi/16) over Q (degree phi(32)/2 = 8,
and c(j) = T_j(c(1)) with T_j the Chebyshev polynomial of degree j), so:

  * F is a half-integer  <=>  N_1..N_7 = 0 and N_0 = 4 (mod 8);
  * otherwise the side of the half-integer h on which F lies is the sign of the algebraic
    number (N_0 - 8h) + sum_j N_j c(j).  2 c(j) are algebraic integers, so twice that number is
    a nonzero algebraic integer whenever some N_j (j >= 1) is nonzero; its norm is then a
    nonzero integer and every conjugate has modulus <= 2|a_0| + 2 sum|N_j|.  Hence
    |value| >= 1 / (2 (2|a_0| + 2 sum|N_j|)^7).  Evaluating in fixed point with an error
    below that bound gives the exact sign; `exact_sign` checks the bound on every call.

The fixed-point cosines come from the closed forms c(4) = sqrt2/2, c(2), c(6) =
sqrt(2 +- sqrt2)/2, c(1), c(7) = sqrt(2 +- sqrt(2 + sqrt2))/2, c(3), c(5) =
sqrt(2 +- sqrt(2 - sqrt2))/2 (half-angle formula), evaluated with integer square roots.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

FRAC_BITS = 384          # fixed-point scale of the cosine constants
_GUARD = 32              # extra bits carried while taking nested square roots


def fold_cos(m: int) -> tuple[int, int]:
    """cos(m pi/16) = sign * cos(j pi/16) with j in 0..8; returns (j, sign)."""
    m %= 32
    if m > 16:
        m = 32 - m                      # cos(2 pi - t) = cos t
    if m > 8:
        return 16 - m, -1               # cos(pi - t) = -cos t
    return m, 1


def _fixed_cosines() -> list[int]:
    """c(j) * 2^FRAC_BITS rounded down, j = 0..8, each within 1 + 2^-32 units of the true value
    (every nested integer square root is off by less than one unit at the guarded scale)."""
    s = FRAC_BITS + _GUARD
    one = 1 << s

    def fsqrt(a: int) -> int:           # sqrt of a fixed-point number at scale 2^s
        return math.isqrt(a << s)

    r2 = fsqrt(2 * one)                 # sqrt 2
    p2 = fsqrt(2 * one + r2)            # sqrt(2 + sqrt 2)
    m2 = fsqrt(2 * one - r2)            # sqrt(2 - sqrt 2)
    vals = {
        0: 2 * one,                     # values here are 2 c(j)
        4: r2,
        2: p2,
        6: m2,
        1: fsqrt(2 * one + p2),
        7: fsqrt(2 * one - p2),
        3: fsqrt(2 * one + m2),
        5: fsqrt(2 * one - m2),
        8: 0,
    }
    return [vals[j] >> (_GUARD + 1) for j in range(9)]


COS_FIXED = _fixed_cosines()


def basis_coords() -> np.ndarray:
    """K[u, v, y, x, j]: integer coordinates of 8 b_u(y) b_v(x) = c(a-b) + c(a+b) in the
    basis {1, c(1), ..., c(7)} (j = 0 is the rational part)."""
    k = np.zeros((8, 8, 8, 8, 8), dtype=np.int64)
    for u in range(8):
        for y in range(8):
            a = 4 if u == 0 else (2 * y + 1) * u
            for v in range(8):
                for x in range(8):
                    b = 4 if v == 0 else (2 * x + 1) * v
                    for m in (a - b, a + b):
                        j, sgn = fold_cos(m)
                        if j < 8:
                            k[u, v, y, x, j] += sgn
    return k


K = basis_coords()


def exact_sign(a0: int, n: Sequence[int]) -> int:
    """Sign of a0 + sum_{j=1..7} n[j-1] c(j), exactly (see the module docstring)."""
    n = [int(t) for t in n]
    a0 = int(a0)
    if not any(n):
        return (a0 > 0) - (a0 < 0)
    err = 2 * sum(abs(t) for t in n)             # each constant is within 1 + 2^-32 units
    # the norm bound 1/(2 (2|a0| + 2 sum|n|)^7) must sit above the evaluation error
    # 2 err 2^-FRAC_BITS (err already counts 2 sum|n|)
    if 4 * err * (2 * abs(a0) + err) ** 7 >= (1 << FRAC_BITS):
        raise ArithmeticError("fixed-point precision too small for these magnitudes")
    d = a0 * (1 << FRAC_BITS) + sum(t * COS_FIXED[j + 1] for j, t in enumerate(n))
    if d > err:
        return 1
    if d < -err:
        return -1
    raise AssertionError("unreachable: a nonzero element of Z[cos(pi/16)] below its norm bound")


def round_half_away(approx: float, coords: Sequence[int], band: float) -> int:
    """round-half-away-from-zero of the value V with 8 V = coords[0] + sum_j coords[j] c(j).

    `approx` is a float64 value of V accurate to far better than `band`; it only picks the
    half-integer to compare with.  Outside the band around m + 1/2 the float decides;
    inside it the decision is exact."""
    m = math.floor(approx)
    if abs(approx - (m + 0.5)) >= band:
        return int(math.copysign(math.floor(abs(approx) + 0.5), approx))
    n0 = int(coords[0])
    rest = [int(t) for t in coords[1:8]]
    s = exact_sign(n0 - 8 * m - 4, rest)       # sign of 8V - 8(m + 1/2)
    if s > 0:
        return m + 1
    if s < 0:
        return m
    return m + 1 if m >= 0 else m              # exact tie: away from zero


def forward_coords(block: np.ndarray, u: int, v: int) -> np.ndarray:
    """Coordinates (N_0..N_7) of 8 F[u, v] for one integer 8x8 block p[y, x]."""
    return np.einsum("yx,yxj->j", np.asarray(block, dtype=np.int64), K[u, v])


def inverse_coords(coefs: np.ndarray, y: int, x: int) -> np.ndarray:
    """Coordinates (M_0..M_7) of 8 p[y, x] for one integer 8x8 coefficient block F[u, v]."""
    return np.einsum("uv,uvj->j", np.asarray(coefs, dtype=np.int64), K[:, :, y, x])
