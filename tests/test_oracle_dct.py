"""Pins of the oracle's float64 8x8 DCT (Sect. 6.4.2, 6.4.3) against closed forms, a library
transform and the paper's printed bound."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import dct, fds
from paper_1512_02951_gb300 import synth


def test_basis_is_orthonormal():
    b = dct.basis_matrix()
    assert np.abs(b @ b.T - np.eye(8)).max() < 1e-15


def test_matches_library_dct_ii_orthonormal():
    fft = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(0)
    p = rng.integers(0, 256, (50, 8, 8))
    want = fft.dctn(p.astype(np.float64), type=2, norm="ortho", axes=(-2, -1))
    assert np.abs(dct.dct2(p) - want).max() < 1e-10
    back = fft.idctn(want, type=2, norm="ortho", axes=(-2, -1))
    assert np.abs(dct.idct2(want) - back).max() < 1e-10


def test_round_trip_without_rounding():
    rng = np.random.default_rng(1)
    p = rng.integers(0, 256, (20, 8, 8)).astype(np.float64)
    assert np.abs(dct.idct2(dct.dct2(p)) - p).max() < 1e-12


@pytest.mark.parametrize("c", [0, 1, 17, 128, 255])
def test_constant_block_has_only_dc_equal_8c(c):
    f = dct.dct2(np.full((8, 8), c))
    assert abs(f[0, 0] - 8 * c) < 1e-12
    f[0, 0] = 0
    assert np.abs(f).max() < 1e-12


def test_dc_bound_printed_in_paper():
    bound = int(read_golden("paper_dc_bound.txt")[0])
    f = dct.dct2(np.full((8, 8), 255))
    assert abs(f[0, 0] - bound) < 1e-12
    rng = np.random.default_rng(2)
    assert dct.dct2(rng.integers(0, 256, (200, 8, 8)))[:, 0, 0].max() <= bound


def test_u_is_vertical_v_is_horizontal():
    # a pattern varying along x only (horizontal frequency 3) lands on row u = 0, column v = 3
    x = np.arange(8)
    p = np.tile(np.cos((2 * x + 1) * 3 * math.pi / 16), (8, 1))
    f = dct.dct2(p)
    f[0, 3] = 0
    assert np.abs(f).max() < 1e-12


def test_block_tiling_indexing():
    img = synth.make_image(24, 16, 5)
    b = dct.image_to_blocks(img)
    assert b.shape == (2, 3, 3, 8, 8)
    assert b[1, 2, 1, 3, 4] == img[8 + 3, 16 + 4, 1]
    assert np.array_equal(dct.blocks_to_image(b), img)


def test_energy_of_default_selection():
    # Sect. 6.3.1: the DC coefficient and the next 5 AC coefficients hold over 95% of the energy
    img = synth.make_image(256, 256, 1)
    f = dct.dct2(dct.image_to_blocks(img))
    zz = fds.ZIGZAG[:6]
    sel = sum(f[..., u, v] ** 2 for u, v in zz).sum()
    assert sel / (f ** 2).sum() > 0.95
