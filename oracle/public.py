"""The paper's own form of the public fragment and the statistics used to assess it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Public image (Sect. 6.5.1, Fig. 10; Fig. 7 (b)): the public fragment as an image -- each
channel-block's coefficients with the selected (private) zigzag positions 0..k "padded with
zeros", inverse-transformed, stored one byte per pixel.

Readings where the paper is silent:
  - the inverse transform of the zero-padded block has zero mean; a byte needs an offset, so
    the block is shifted to mid-grey: the DC coefficient (always private) is set to 1024 =
    8 x 128 instead of 0, i.e. every pixel of the block gets + 128;
  - the stored byte is round-half-away-from-zero of that exact pixel value, clamped to
    [0, 255] -- the same rounding and clamp as restore (the decision is exact);
  - the public coefficients come back from a public image by the forward transform and the
    same exact rounding (a constant offset changes the DC coefficient only, which is private).

Statistics (Sect. 6.6): the per-channel histogram (Sect. 6.6.1) and the correlation
coefficient of adjacent pixels, r = cov(x, y) / (sqrt(D(x)) sqrt(D(y))), horizontally,
vertically and diagonally (Sect. 6.6.2).  Reading: the paper samples 10,000 random pairs; here
every adjacent pair of the image is used (the sample estimates this value), and the sums are
kept as exact integers.
"""
from __future__ import annotations

import math

import numpy as np

from . import dct, fds

MID_GREY_DC = 1024          # 8 * 128: + 128 on every pixel of the block
DIRECTIONS = ("horizontal", "vertical", "diagonal")
_OFFSETS = {"horizontal": (0, 1), "vertical": (1, 0), "diagonal": (1, 1)}


def public_image(public: np.ndarray, k: int, width: int, height: int) -> np.ndarray:
    """H x W x 3 uint8 image of the public fragment (int16 [BY, BX, 3, 63 - k]): zigzag
    positions 1..k zero, DC 1024, positions k+1..63 from the fragment; exact inverse
    transform, round half away from zero, clamp to [0, 255]."""
    by, bx = height // 8, width // 8
    part2 = np.asarray(public, dtype=np.int64).reshape(by, bx, 3, 63 - k)
    part1 = np.zeros((by, bx, 3, k + 1), dtype=np.int64)
    part1[..., 0] = MID_GREY_DC
    p = fds.quantised_idct(fds.merge(part1, part2))
    return dct.blocks_to_image(np.clip(p, 0, 255).astype(np.uint8))


def public_from_image(image: np.ndarray, k: int) -> np.ndarray:
    """The public fragment (int16 [BY, BX, 3, 63 - k]) recovered from a public image: exact
    rounded forward transform, positions k+1..63."""
    q, _ = fds.quantised_dct(dct.image_to_blocks(np.asarray(image, dtype=np.uint8)))
    _, part2 = fds.split(q, k)
    return part2.astype(np.int16)


def histogram(image: np.ndarray) -> np.ndarray:
    """[3, 256] int64: pixel counts per channel and level (Sect. 6.6.1)."""
    img = np.asarray(image, dtype=np.uint8)
    return np.stack([np.bincount(img[..., c].reshape(-1), minlength=256) for c in range(3)]).astype(np.int64)


def pair_sums(image: np.ndarray) -> np.ndarray:
    """[3 directions, 3 channels, 6] int64: (n, sum x, sum y, sum x^2, sum y^2, sum x y) over
    every pair (x, y) of a pixel and its right / lower / lower-right neighbour."""
    img = np.asarray(image, dtype=np.int64)
    h, w, _ = img.shape
    out = np.zeros((3, 3, 6), dtype=np.int64)
    for d, name in enumerate(DIRECTIONS):
        dy, dx = _OFFSETS[name]
        x = img[: h - dy, : w - dx]
        y = img[dy:, dx:]
        for c in range(3):
            xc, yc = x[..., c], y[..., c]
            out[d, c] = (xc.size, xc.sum(), yc.sum(), (xc * xc).sum(), (yc * yc).sum(), (xc * yc).sum())
    return out


def correlation(sums: np.ndarray) -> np.ndarray:
    """r_xy from pair sums (..., 6); nan where a variance is zero (Sect. 6.6.2)."""
    s = np.asarray(sums, dtype=np.int64)
    out = np.full(s.shape[:-1], math.nan)
    for idx in np.ndindex(*s.shape[:-1]):
        n, sx, sy, sxx, syy, sxy = (int(v) for v in s[idx])
        cov = n * sxy - sx * sy                       # n^2 cov, exact
        dx, dy = n * sxx - sx * sx, n * syy - sy * sy  # n^2 D(x), n^2 D(y), exact
        if dx > 0 and dy > 0:
            out[idx] = cov / math.sqrt(dx * dy)
    return out
