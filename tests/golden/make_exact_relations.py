"""Write tests/golden/exact_near_relations.txt: integer vectors (N_0, ..., N_7) for which

    s = N_0 + sum_{j=1..7} N_j cos(j pi / 16)

is nonzero but tiny (|s| far below 2^-40).  Added to an odd multiple of 4 (N_0 + 4 + 8m), such
a vector puts 8V within |s| of a rounding boundary of V = m + 1/2, closer than any 64-bit
fixed-point evaluation can resolve, so the exact rounding step of Sect. 6.4.3 (as read here:
round half away from zero of the exact value) must fall back to its wide evaluation.

The vectors are found by lattice reduction (Lenstra-Lenstra-Lovasz, written out below with
exact rational arithmetic) of the lattice spanned by the rows (e_i, round(C v_i)), v = (1,
cos(pi/16), ..., cos(7 pi/16)) taken from the oracle's 384-bit fixed-point cosines: a short
vector of that lattice has small integer coordinates and a small value of s.  {1, c(1), ..,
c(7)} is a basis of Q(cos pi/16) over Q, so s is never exactly zero unless every N_j is.

Only inputs are produced here; the expected rounding results come from oracle/exact.py at
test time.  Run:  python tests/golden/make_exact_relations.py
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402

OUT = os.path.join(HERE, "exact_near_relations.txt")


def lll(basis: list[list[int]], delta: Fraction = Fraction(99, 100)) -> list[list[int]]:
    """LLL-reduce the rows of `basis` (integer vectors); textbook form with exact
    Gram-Schmidt coefficients, recomputed after every change (the dimension is 8)."""
    b = [list(r) for r in basis]
    n = len(b)

    def dot(x, y):
        return sum(p * q for p, q in zip(x, y))

    def gram_schmidt():
        bs, mu = [], [[Fraction(0)] * n for _ in range(n)]
        for i in range(n):
            v = [Fraction(x) for x in b[i]]
            for j in range(i):
                mu[i][j] = Fraction(dot(b[i], bs[j])) / dot(bs[j], bs[j])
                v = [p - mu[i][j] * q for p, q in zip(v, bs[j])]
            bs.append(v)
        return bs, mu

    bs, mu = gram_schmidt()
    k = 1
    while k < n:
        for j in range(k - 1, -1, -1):
            q = round(mu[k][j])
            if q:
                b[k] = [p - q * r for p, r in zip(b[k], b[j])]
                bs, mu = gram_schmidt()
        if dot(bs[k], bs[k]) >= (delta - mu[k][k - 1] ** 2) * dot(bs[k - 1], bs[k - 1]):
            k += 1
        else:
            b[k], b[k - 1] = b[k - 1], b[k]
            bs, mu = gram_schmidt()
            k = max(k - 1, 1)
    return b


def value_fixed(n: list[int]) -> int:
    """s * 2^FRAC_BITS from the oracle's fixed-point cosines (n = N_0..N_7)."""
    return n[0] * (1 << exact.FRAC_BITS) + sum(n[j] * exact.COS_FIXED[j] for j in range(1, 8))


def ambiguous_at_64_bits(n: list[int], m: int) -> bool:
    """True if a 64-bit fixed-point evaluation (cosines rounded to 2^-62, error bound
    sum_j |N_j| units) of 8V = N_0 + 4 + 8m + sum N_j c(j) cannot tell on which side of the
    half-integer boundary V lies."""
    q62 = [0] + [(exact.COS_FIXED[j] + (1 << (exact.FRAC_BITS - 63))) >> (exact.FRAC_BITS - 62)
                 for j in range(1, 8)]
    n0 = n[0] + 4 + 8 * m
    d = (n0 << 62) + sum(n[j] * q62[j] for j in range(1, 8))
    err = sum(abs(t) for t in n[1:])
    rem = (d + (4 << 62)) % (1 << 65)
    return rem <= err or rem >= (1 << 65) - err


def relations() -> list[list[int]]:
    found = []
    subsets = [list(range(8)), [0, 1, 3, 5, 7], [0, 2, 4, 6], [0, 1, 2, 3, 4], [0, 4, 5, 6, 7]]
    for scale in (72, 80, 88):
        for sub in subsets:
            c = 1 << scale
            rows = []
            for i, j in enumerate(sub):
                e = [0] * len(sub)
                e[i] = 1
                vj = (1 << exact.FRAC_BITS) if j == 0 else exact.COS_FIXED[j]
                rows.append(e + [(vj * c) >> exact.FRAC_BITS])
            for r in lll(rows):
                n = [0] * 8
                for i, j in enumerate(sub):
                    n[j] = r[i]
                if not any(n[1:]):
                    continue
                if n[0] < 0 or (n[0] == 0 and next(t for t in n[1:] if t) < 0):
                    n = [-t for t in n]
                if max(abs(t) for t in n) >= 1 << 14 or n in found:
                    continue
                if ambiguous_at_64_bits(n, 0) and ambiguous_at_64_bits([-t for t in n], 0):
                    found.append(n)
    return found


def main() -> None:
    rel = relations()
    with open(OUT, "w") as fh:
        fh.write("# Integer vectors N_0 .. N_7 with s = N_0 + sum_j N_j cos(j pi/16) nonzero and tiny.\n")
        fh.write("# Written by tests/golden/make_exact_relations.py (lattice reduction over the oracle's\n")
        fh.write("# 384-bit cosines).  Each line: the eight integers, then log2 |s| for reference.\n")
        fh.write("# Used as 8V = N_0 + 4 + 8m + ... : V within |s|/8 of the half-integer m + 1/2.\n")
        for n in rel:
            v = value_fixed(n)
            lg = (abs(v).bit_length() - exact.FRAC_BITS)
            fh.write(" ".join(str(t) for t in n) + f"  # log2|s| ~ {lg}\n")
    print(f"{len(rel)} relations -> {OUT}")


if __name__ == "__main__":
    main()
