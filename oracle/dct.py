"""8x8 DCT-II / inverse in float64, and 8x8 block tiling of an RGB bitmap.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sect. 6.4.2: the 2-D transform is separable -- a product of the vertical 1-D basis with its
horizontal counterpart.  Sect. 6.4.3 fixes the scaling: the DC coefficient of an 8-bit block
is bounded by 2040 = 8 * 255, which is the orthonormal DCT-II with no level shift:

    F[u, v] = sum_y sum_x p[y, x] * b_u(y) * b_v(x),
    b_u(y)  = (C(u) / 2) * cos((2y + 1) u pi / 16),   C(0) = 1/sqrt(2), C(u > 0) = 1,

u the vertical (row) frequency, v the horizontal (column) frequency.  The basis matrix is
orthogonal, so the inverse is the transpose.
"""
from __future__ import annotations

import math

import numpy as np


def basis_matrix() -> np.ndarray:
    """B[u, y] = b_u(y), the orthonormal 8-point DCT-II basis in float64."""
    b = np.empty((8, 8), dtype=np.float64)
    for u in range(8):
        cu = math.sqrt(0.5) if u == 0 else 1.0
        for y in range(8):
            b[u, y] = 0.5 * cu * math.cos((2 * y + 1) * u * math.pi / 16.0)
    return b


_B = basis_matrix()


def dct2(blocks: np.ndarray) -> np.ndarray:
    """Forward 2-D DCT of (..., 8, 8) blocks indexed [y, x]: F = B P B^T (float64)."""
    return _B @ np.asarray(blocks, dtype=np.float64) @ _B.T


def idct2(coefs: np.ndarray) -> np.ndarray:
    """Inverse 2-D DCT of (..., 8, 8) coefficients indexed [u, v]: P = B^T F B (float64)."""
    return _B.T @ np.asarray(coefs, dtype=np.float64) @ _B


def image_to_blocks(img: np.ndarray) -> np.ndarray:
    """H x W x 3 uint8 image -> (BY, BX, 3, 8, 8) blocks, block (by, bx) channel c holding
    pixels img[8 by + y, 8 bx + x, c] at [y, x] (Sect. 6.3.1: DCT 8x8 per block)."""
    h, w, ch = img.shape
    if ch != 3 or h % 8 or w % 8:
        raise ValueError("expected H x W x 3 with H, W multiples of 8")
    return img.reshape(h // 8, 8, w // 8, 8, 3).transpose(0, 2, 4, 1, 3)


def blocks_to_image(blocks: np.ndarray) -> np.ndarray:
    """Inverse of image_to_blocks."""
    by, bx, ch, _, _ = blocks.shape
    return blocks.transpose(0, 3, 1, 4, 2).reshape(by * 8, bx * 8, ch)
