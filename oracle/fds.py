"""Selective encryption of an RGB bitmap, first level of protection (Sect. 6.3.1, Fig. 6),
and its inverse (defragmentation, Sect. 3.2 / Sect. 5.2 Fig. 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

protect(image, key, iv, k):
  1. cut each channel into 8x8 blocks (Sect. 6.3.1);
  2. 2-D DCT-II of every block (Sect. 6.4.2), float64;
  3. every coefficient to int16 by round-half-away-from-zero of its exact value
     (Sect. 6.4.3; the decision is exact, see exact.py);
  4. fragmentation by the selection ratio: zigzag positions 0..k form Part 1 (confidential),
     k+1..63 form Part 2 (public).  The default selection of Sect. 6.3.1 -- [0,0], [0,1],
     [1,0], [2,0], [1,1], [0,2] -- is zigzag 0..5, i.e. k = 5; k = 0 keeps the DC coefficient
     alone (the DC-only scheme cited in Sect. 6.2.1);
  5. Part 1 is encrypted with AES-128 in counter mode (Sect. 6.12, Sect. 6.5.2).

Layouts (the paper leaves them open):
  public   int16 [BY][BX][3][63 - k], zigzag positions k+1..63 in order
  private  the int16 little-endian byte stream of [BY][BX][3][k + 1] (zigzag 0..k),
           AES-128-CTR encrypted as one message per image with a 16-byte initial counter
           block, incremented as a 128-bit big-endian integer per 16-byte keystream block.

restore(public, private, key, iv, k, width, height): decrypt Part 1, merge with Part 2 by the
inverse zigzag, inverse DCT, round half away from zero (exact), clamp to [0, 255].
"""
from __future__ import annotations

import math

import numpy as np

from . import aes, dct, exact

# float64 evaluation error of the 8x8 transforms here is below 1e-9 for any int16 input
# (|terms| sum to < 6e5, 16 rounded operations, unit roundoff 1.1e-16); values within this
# band of a half-integer are re-decided exactly.
BAND = 1e-6


def zigzag_order() -> list[tuple[int, int]]:
    """JPEG zigzag scan of an 8x8 block as (u, v) = (row, column) pairs.

    Anti-diagonals s = u + v in increasing order; on odd s the scan walks u upward from its
    smallest value, on even s downward from its largest.  Its first six entries are the
    default selection of Sect. 6.3.1: [0,0], [0,1], [1,0], [2,0], [1,1], [0,2]."""
    order = []
    for s in range(15):
        us = list(range(max(0, s - 7), min(s, 7) + 1))
        if s % 2 == 0:
            us.reverse()
        order.extend((u, s - u) for u in us)
    return order


ZIGZAG = zigzag_order()


def sizes(width: int, height: int, k: int) -> tuple[int, int]:
    """(public bytes, private bytes) of one image: 2 (63 - k) and 2 (k + 1) bytes per
    channel-block."""
    if width % 8 or height % 8 or width <= 0 or height <= 0 or not 0 <= k <= 63:
        raise ValueError("bad image size or selection ratio")
    ncb = (width // 8) * (height // 8) * 3
    return ncb * 2 * (63 - k), ncb * 2 * (k + 1)


def _round_array(approx: np.ndarray, coords_of) -> np.ndarray:
    """Round every entry of `approx` half away from zero, exactly.

    coords_of(idx) returns the exact integer coordinates (len(idx), 8) of 8x the values at the
    flat indices idx.  Only entries within BAND of a half-integer need them."""
    flat = approx.reshape(-1)
    q = np.copysign(np.floor(np.abs(flat) + 0.5), flat).astype(np.int64)
    near = np.nonzero(np.abs(flat - np.floor(flat) - 0.5) < BAND)[0]
    for start in range(0, near.size, 8192):
        idx = near[start: start + 8192]
        coords = coords_of(idx)
        for t, i in enumerate(idx):
            q[i] = exact.round_half_away(float(flat[i]), coords[t], BAND)
    return q.reshape(approx.shape)


def quantised_dct(blocks: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(q, F): exact-rounded int64 coefficients and float64 coefficients of (..., 8, 8)
    integer blocks."""
    f = dct.dct2(blocks)
    flat_blocks = np.asarray(blocks, dtype=np.int64).reshape(-1, 8, 8)

    def coords_of(idx):
        b, uv = np.divmod(idx, 64)
        u, v = np.divmod(uv, 8)
        return np.einsum("myx,myxj->mj", flat_blocks[b], exact.K[u, v])

    return _round_array(f, coords_of), f


def quantised_idct(coefs: np.ndarray) -> np.ndarray:
    """Exact-rounded (not clamped) inverse DCT of (..., 8, 8) integer coefficient blocks."""
    p = dct.idct2(coefs)
    flat = np.asarray(coefs, dtype=np.int64).reshape(-1, 8, 8)
    kt = exact.K.transpose(2, 3, 0, 1, 4)          # [y, x, u, v, j]

    def coords_of(idx):
        b, yx = np.divmod(idx, 64)
        y, x = np.divmod(yx, 8)
        return np.einsum("muv,muvj->mj", flat[b], kt[y, x])

    return _round_array(p, coords_of)


def split(q: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Fragment (..., 8, 8) integer coefficients by zigzag position: (Part 1, Part 2)."""
    zz_u = np.array([u for u, _ in ZIGZAG])
    zz_v = np.array([v for _, v in ZIGZAG])
    scan = q[..., zz_u, zz_v]                       # (..., 64) in zigzag order
    return scan[..., : k + 1], scan[..., k + 1:]


def merge(part1: np.ndarray, part2: np.ndarray) -> np.ndarray:
    """Inverse of split: (..., k+1) and (..., 63-k) zigzag-ordered values -> (..., 8, 8)."""
    scan = np.concatenate([part1, part2], axis=-1)
    out = np.zeros(scan.shape[:-1] + (8, 8), dtype=scan.dtype)
    for i, (u, v) in enumerate(ZIGZAG):
        out[..., u, v] = scan[..., i]
    return out


def _check_int16(x: np.ndarray) -> np.ndarray:
    if x.size and (x.min() < -32768 or x.max() > 32767):
        raise OverflowError("coefficient outside int16")
    return x.astype(np.int16)


def protect(img: np.ndarray, key: bytes, iv: bytes, k: int, return_f64: bool = False):
    """First level of protection of one H x W x 3 uint8 image.

    Returns (public int16 [BY, BX, 3, 63-k], private ciphertext bytes) and, with
    return_f64, the float64 coefficients [BY, BX, 3, 8, 8] before rounding."""
    if not 0 <= k <= 63:
        raise ValueError("k must be in 0..63")
    blocks = dct.image_to_blocks(np.asarray(img, dtype=np.uint8))
    q, f = quantised_dct(blocks)
    part1, part2 = split(_check_int16(q), k)
    plain = np.ascontiguousarray(part1).astype("<i2").tobytes()
    cipher = aes.ctr_xcrypt(key, iv, plain)
    out = (np.ascontiguousarray(part2), cipher)
    return out + (f,) if return_f64 else out


def restore(public: np.ndarray, private: bytes, key: bytes, iv: bytes, k: int,
            width: int, height: int) -> np.ndarray:
    """Inverse of protect: H x W x 3 uint8 image."""
    by, bx = height // 8, width // 8
    plain = aes.ctr_xcrypt(key, iv, bytes(private))
    part1 = np.frombuffer(plain, dtype="<i2").astype(np.int64).reshape(by, bx, 3, k + 1)
    part2 = np.asarray(public, dtype=np.int64).reshape(by, bx, 3, 63 - k)
    p = quantised_idct(merge(part1, part2))
    return dct.blocks_to_image(np.clip(p, 0, 255).astype(np.uint8))


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    """Peak signal-to-noise ratio in dB for 8-bit data (Sect. 6.4.3, Table 5); inf if equal."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0.0 else 10.0 * math.log10(255.0 ** 2 / mse)
