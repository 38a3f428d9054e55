"""Write fds_cos_limbs.h: cos(j pi / 16), j = 1..7, as 256-bit fixed-point numbers.

The exact-rounding fallback of the CUDA kernels decides the sign of
a0 + sum_j N_j cos(j pi / 16) with integer a0, N_j.  It needs the cosines to about 2^-256.
They are computed here from the Taylor series of cos, with pi from Machin's formula
pi = 16 atan(1/5) - 4 atan(1/239), all in integer fixed point with 64 guard bits, then
truncated to 256 fractional bits (each value within one unit of 2^-256).

It also writes round(cos(j pi / 16) * 2^62), j = 1..7, for the 128-bit first try of the
same decision.

Run:  python gen_cos_limbs.py > fds_cos_limbs.h
"""
FRAC = 256
GUARD = 64
S = FRAC + GUARD
ONE = 1 << S


def atan_inv(n):
    """atan(1/n) * 2^S by its alternating series."""
    total, term, k, sign = 0, ONE // n, 1, 1
    n2 = n * n
    while term:
        total += sign * (term // k)
        term //= n2
        k += 2
        sign = -sign
    return total


PI = 16 * atan_inv(5) - 4 * atan_inv(239)


def cos_fixed(j):
    """cos(j pi / 16) * 2^S by its Taylor series (argument < pi/2)."""
    x = PI * j // 16
    x2 = x * x >> S
    total, term, n = 0, ONE, 0
    while term:
        total += term if n % 4 == 0 else -term
        term = term * x2 >> S
        term //= (n + 1) * (n + 2)
        n += 2
    return total


def main():
    print("/* Generated by gen_cos_limbs.py: floor(cos(j pi/16) * 2^256), j = 1..7, as eight")
    print(" * 32-bit limbs, least significant first (an initializer for uint32_t[7][8]). */")
    print("#pragma once")
    print("#define FDS_COS_LIMBS_INIT \\")
    print("  { \\")
    for j in range(1, 8):
        v = cos_fixed(j) >> GUARD
        limbs = [(v >> (32 * i)) & 0xFFFFFFFF for i in range(8)]
        print("    {" + ", ".join("0x%08xu" % t for t in limbs) + "}, /* j = %d */ \\" % j)
    print("  }")
    print("/* round(cos(j pi/16) * 2^62), j = 1..7 */")
    q62 = [(cos_fixed(j) + (1 << (S - 63))) >> (S - 62) for j in range(1, 8)]
    print("#define FDS_COS_Q62_INIT \\")
    print("  {" + ", ".join("%dll" % v for v in q62) + "}")


if __name__ == "__main__":
    main()
