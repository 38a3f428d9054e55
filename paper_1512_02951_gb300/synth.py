"""Seeded synthetic inputs: RGB bitmaps, AES keys, initial counter blocks, request mixes.

This module holds no arithmetic of the protection method itself (no transform, no rounding,
no cipher). It only draws pseudo-random inputs, so that the CUDA library, its tests, the
benchmark and the CPU oracle can all be fed the same seeded data.

The paper's test images ('Barbara', 'baboon', the La Poste bitmaps; Sect. 6.3 and 6.6) are
not available, so the images are smooth synthetic scenes: a sum of 20 random isotropic
2-D Gaussians per image with independent per-channel amplitudes on a mid-grey base, plus
uniform noise of +-8 grey levels, rounded and clipped to uint8.  The recipe:

  rng      = numpy.random.default_rng(seed)
  centres  = U[0, W) x U[0, H)                 (20 of them)
  sigma    = U[0.05, 0.3] * max(W, H)          (isotropic)
  amp[c]   = U[-120, 120] per channel
  image    = 128 + sum_g amp[g, c] * exp(-((x-cx)^2 + (y-cy)^2) / (2 sigma^2))
           + U[-8, 8] noise, then rint and clip to [0, 255]

Images are H x W x 3 (row-major, channels interleaved), W and H multiples of 8.
"""
from __future__ import annotations

import math

import numpy as np

N_GAUSSIANS = 20


def make_image(width: int, height: int, seed: int) -> np.ndarray:
    """One seeded H x W x 3 uint8 image (see the module docstring for the recipe)."""
    if width % 8 or height % 8 or width <= 0 or height <= 0:
        raise ValueError("width and height must be positive multiples of 8")
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, width, N_GAUSSIANS)
    cy = rng.uniform(0.0, height, N_GAUSSIANS)
    sigma = rng.uniform(0.05, 0.3, N_GAUSSIANS) * max(width, height)
    amp = rng.uniform(-120.0, 120.0, (N_GAUSSIANS, 3))
    xs = np.arange(width, dtype=np.float64)
    ys = np.arange(height, dtype=np.float64)
    gx = np.exp(-((xs[None, :] - cx[:, None]) ** 2) / (2.0 * sigma[:, None] ** 2))  # (n, W)
    gy = np.exp(-((ys[None, :] - cy[:, None]) ** 2) / (2.0 * sigma[:, None] ** 2))  # (n, H)
    img = np.empty((height, width, 3), dtype=np.float32)
    for c in range(3):
        img[:, :, c] = (gy.T @ (amp[:, c, None] * gx)).astype(np.float32)
    img += 128.0
    img += rng.uniform(-8.0, 8.0, (height, width, 3)).astype(np.float32)
    np.rint(img, out=img)
    np.clip(img, 0.0, 255.0, out=img)
    return img.astype(np.uint8)


def make_key(seed: int) -> bytes:
    """A seeded 16-byte AES-128 key."""
    return np.random.default_rng(seed).bytes(16)


def make_iv(seed: int) -> bytes:
    """A seeded 16-byte initial counter block."""
    return np.random.default_rng(seed).bytes(16)


def round8(x: float) -> int:
    """Nearest multiple of 8, at least 64."""
    return max(64, int(round(x / 8.0)) * 8)


def batch_sizes(n: int, seed: int, lo: int = 64, hi: int = 2048) -> list[tuple[int, int]]:
    """n (width, height) pairs, each log-uniform in [lo, hi] and rounded to a multiple of 8."""
    rng = np.random.default_rng(seed)
    lw = rng.uniform(math.log(lo), math.log(hi), n)
    lh = rng.uniform(math.log(lo), math.log(hi), n)
    return [(min(hi, round8(math.exp(a))), min(hi, round8(math.exp(b)))) for a, b in zip(lw, lh)]


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of n requests of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
