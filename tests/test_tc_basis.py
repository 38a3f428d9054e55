"""The tensor-core form's B operand, checked on the host: decoded from its swizzled byte image
independently of the library, its limbs are integers exact in the operand type, their sum is
the orthonormal DCT-II basis (Sect. 6.4.2) to within the split's remainder, the rational
coefficients sit in limb 0 alone, and the library's error bound covers the remainder and
stays below the kernel's rounding guard."""
import ctypes

import numpy as np
import pytest

from oracle import dct as odct

# form -> (limb shifts, rounding guard, largest limb exact in the operand type)
FORMS = {"bf16": ((9, 8, 8), 2.0 ** -11, 256), "tf32": ((12, 11), 2.0 ** -10, 2048),
         "f16": ((13, 11, 11), 2.0 ** -12, 2048)}
# the f16 form holds its rows in zigzag order and its A operand is p - 128 (|.| <= 128)
PIXEL_BOUND = {"bf16": 255, "tf32": 255, "f16": 128}


def _zigzag():
    from oracle import fds as ofds
    return [8 * u + v for (u, v) in ofds.ZIGZAG]


@pytest.fixture(scope="module")
def api():
    from paper_1512_02951_gb300 import api, build

    build.build()
    return api


def _decode(form, img):
    """limbs[l, pos, kk] from the 128-byte swizzled K-major image (layout of fds.h)."""
    shifts = FORMS[form][0]
    nl = len(shifts)
    raw = np.frombuffer(img, dtype=np.uint8)
    limbs = np.zeros((nl, 64, 64))
    zz = _zigzag()
    for l in range(nl):
        for pos in range(64):
            n = 64 * l + pos
            for kk in range(64):
                if form == "f16":                       # row n = 64 l + zigzag index
                    off = n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2
                    limbs[l, zz[pos], kk] = float(raw[off:off + 2].view(np.float16)[0])
                    continue
                if form == "bf16":
                    off = n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2
                    bits = int(raw[off]) | int(raw[off + 1]) << 8
                    val = np.array([bits << 16], dtype=np.uint32).view(np.float32)[0]
                else:
                    atom, k2 = kk >> 5, kk & 31
                    off = atom * 128 * 128 + n * 128 + (((k2 >> 2) ^ (n & 7)) << 4) + (k2 & 3) * 4
                    val = raw[off:off + 4].view(np.float32)[0]
                limbs[l, pos, kk] = float(val)
    return limbs


@pytest.mark.parametrize("form", sorted(FORMS))
def test_limbs_reconstruct_the_basis(api, form):
    shifts, guard, lmax = FORMS[form]
    img, bound = api.tc_basis(form)
    limbs = _decode(form, img)
    assert np.all(limbs == np.round(limbs)) and np.abs(limbs).max() <= lmax
    b = odct.basis_matrix()
    basis = np.einsum("uy,vx->uvyx", b, b).reshape(64, 64)      # [8u+v, 8y+x]
    approx = np.zeros_like(basis)
    e = 0
    for l, s in enumerate(shifts):
        e += s
        approx += limbs[l] * 2.0 ** -e
    rem = np.abs(basis - approx)
    # each limb rounds to nearest: the remainder is at most half a unit of the last limb
    assert rem.max() <= 2.0 ** -(e + 1) * (1 + 1e-9)
    pb = PIXEL_BOUND[form]
    worst = (pb * rem.sum(axis=1)).max()
    assert worst <= bound < guard
    # 8-bit pixels keep every partial sum of every limb an integer below 2^24
    assert (pb * np.abs(limbs).sum(axis=2)).max() < 2 ** 24


@pytest.mark.parametrize("form", sorted(FORMS))
def test_rational_coefficients_are_limb_zero_only(api, form):
    shifts = FORMS[form][0]
    limbs = _decode(form, api.tc_basis(form)[0])
    for u in (0, 4):
        for v in (0, 4):
            pos = 8 * u + v
            assert np.all(np.abs(limbs[0, pos]) == 2.0 ** (shifts[0] - 3))   # B = +-1/8
            assert not limbs[1:, pos].any()


def test_swizzle_is_a_permutation_of_the_rows(api):
    # every 16-byte chunk of every row lands inside that row, each exactly once
    for n in range(192):
        offs = sorted((((c ^ (n & 7)) << 4) for c in range(8)))
        assert offs == [16 * c for c in range(8)]


def test_tc_host_argument_checks(api):
    from paper_1512_02951_gb300 import _lib
    lib = _lib.load()
    key = bytes(16)
    assert lib.fds_protect_image_tc(3, 8, 64, 64, 0, key, key, 16, 16, None) == -1   # unknown form
    assert b"form" in lib.fds_last_error()
    assert lib.fds_protect_image_tc(0, 8, 100, 64, 0, key, key, 16, 16, None) == -1  # width
    assert lib.fds_protect_image_tc(0, 8, 64, 64, 64, key, key, 16, 16, None) == -1  # k
    assert lib.fds_protect_image_tc(1, 8, 64, 64, 0, key, key, 24, 16, None) == -1   # alignment
    assert lib.fds_debug_dct_tc(0, None, 64, 64, 16, None) == -1
    assert lib.fds_tc_basis(5, None, 0, None) == -1
    assert lib.fds_protect_image_tc(2, 8, 64, 64, 17, key, key, 16, 16, None) == -1  # k not instantiated
    small = (ctypes.c_uint8 * 16)()
    assert lib.fds_tc_basis(0, small, 16, None) == -1
    with pytest.raises(ValueError):
        api.tc_basis("fp8")


def _decode_inverse(img):
    """limbs[l, p, z] of the inverse table: row n = 64 l + p (p = 8y + x), K index z (zigzag)."""
    raw = np.frombuffer(img, dtype=np.uint8)
    limbs = np.zeros((3, 64, 64))
    for l in range(3):
        for p in range(64):
            n = 64 * l + p
            for z in range(64):
                off = n * 128 + (((z >> 3) ^ (n & 7)) << 4) + (z & 7) * 2
                limbs[l, p, z] = float(raw[off:off + 2].view(np.float16)[0])
    return limbs


def test_inverse_limbs_reconstruct_the_transposed_basis(api):
    img, bound = api.tc_basis("f16_inverse")
    limbs = _decode_inverse(img)
    assert np.all(limbs == np.round(limbs)) and np.abs(limbs).max() <= 128
    b = odct.basis_matrix()
    basis = np.einsum("uy,vx->uvyx", b, b).reshape(64, 64)      # [8u+v, 8y+x]
    zz = _zigzag()
    inv = basis[zz, :].T                                         # [8y+x, zigzag z]
    approx = limbs[0] * 2.0 ** -9 + limbs[1] * 2.0 ** -17 + limbs[2] * 2.0 ** -25
    rem = np.abs(inv - approx)
    assert rem.max() <= 2.0 ** -26 * (1 + 1e-9)                 # half a unit of the last limb
    # the bound per unit of sum |q| covers the remainder and stays below the kernel's 2^-24
    assert rem.max() <= bound < 2.0 ** -24
    # coefficients below 2048 keep every partial sum of every limb an integer below 2^24
    assert (2047 * np.abs(limbs).sum(axis=2)).max() < 2 ** 24
    # the rational basis functions ((u, v) in {0, 4}^2: +-1/8) sit in limb 0 alone
    for u in (0, 4):
        for v in (0, 4):
            z = zz.index(8 * u + v)
            assert np.all(np.abs(limbs[0, :, z]) == 64) and not limbs[1:, :, z].any()


def test_tc_restore_host_argument_checks(api):
    from paper_1512_02951_gb300 import _lib
    lib = _lib.load()
    key = bytes(16)
    assert lib.fds_restore_image_tc(0, 16, 16, 64, 64, 5, key, key, 8, None) == -1   # not the f16 form
    assert b"FDS_TC_F16" in lib.fds_last_error()
    assert lib.fds_restore_image_tc(2, 16, 16, 100, 64, 5, key, key, 8, None) == -1  # width
    assert lib.fds_restore_image_tc(2, 16, 16, 64, 64, 64, key, key, 8, None) == -1  # k
    assert lib.fds_restore_image_tc(2, 24, 16, 64, 64, 5, key, key, 8, None) == -1   # alignment
    assert lib.fds_restore_image_tc(2, 16, None, 64, 64, 5, key, key, 8, None) == -1  # null
