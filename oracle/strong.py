"""Strong level of protection (Sect. 6.3.2, Fig. 8; Fig. 7 (d)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The first level leaves the high frequencies readable.  The strong level hides them as well,
cheaply: per channel-block, the selected coefficients (Part 1) are hashed with SHA-512 into a
512-bit string, and the public image of the block (the inverse transform of the remaining
coefficients padded with zeros: 64 pixels, 512 bits) is XORed with it, pixel by pixel.  Part 1
itself is AES-128-CTR encrypted as in the first level.

Readings where the paper is silent:
  - the hashed message is the channel-block's Part 1 as stored: k + 1 int16 little-endian
    values in zigzag order (the plaintext, before encryption); the key does not enter the
    hash (Fig. 8 hashes Part 1 alone);
  - digest byte j (SHA-512 output order) is XORed onto pixel (y, x) = (j // 8, j % 8) of the
    block, in its channel;
  - the public image is the one of oracle/public.py (DC 1024, exact rounding, clamp);
  - restore: Part 1 decrypted, the mask removed, the public coefficients recovered from the
    public image by the forward transform (exact rounding), merged with Part 1 and inverse
    transformed as in the first level.  The public image holds rounded, clamped bytes, so
    this path is not exact; its PSNR is the measure (Sect. 6.4.3, Table 5).

SHA-512 is taken from the Python standard library (hashlib, FIPS 180-4), a library primitive.
"""
from __future__ import annotations

import hashlib

import numpy as np

from . import aes, dct, fds, public


def masks(part1: np.ndarray) -> np.ndarray:
    """[..., 8, 8] uint8: SHA-512 of each channel-block's Part 1 (int16 LE bytes of [..., k+1]),
    digest byte 8 y + x at (y, x)."""
    p = np.ascontiguousarray(np.asarray(part1, dtype=np.int64).astype("<i2"))
    flat = p.reshape(-1, p.shape[-1])
    out = np.empty((flat.shape[0], 64), dtype=np.uint8)
    for i in range(flat.shape[0]):
        out[i] = np.frombuffer(hashlib.sha512(flat[i].tobytes()).digest(), dtype=np.uint8)
    return out.reshape(p.shape[:-1] + (8, 8))


def _apply_mask(image: np.ndarray, part1: np.ndarray) -> np.ndarray:
    """image (H x W x 3 uint8) XOR the per-block masks of part1 [BY, BX, 3, k+1]."""
    blocks = dct.image_to_blocks(np.asarray(image, dtype=np.uint8))      # [BY, BX, 3, 8, 8]
    return dct.blocks_to_image(blocks ^ masks(part1))


def protect_strong(img: np.ndarray, key: bytes, iv: bytes, k: int) -> tuple[np.ndarray, bytes]:
    """(strong public image H x W x 3 uint8, Part 1 ciphertext bytes)."""
    h, w, _ = np.asarray(img).shape
    pub, cipher = fds.protect(img, key, iv, k)
    part1 = np.frombuffer(aes.ctr_xcrypt(key, iv, cipher), dtype="<i2").reshape(h // 8, w // 8, 3, k + 1)
    return _apply_mask(public.public_image(pub, k, w, h), part1), cipher


def restore_strong(strong: np.ndarray, cipher: bytes, key: bytes, iv: bytes, k: int) -> np.ndarray:
    """The H x W x 3 uint8 image back from the strong public image and Part 1's ciphertext."""
    h, w, _ = np.asarray(strong).shape
    part1 = np.frombuffer(aes.ctr_xcrypt(key, iv, bytes(cipher)), dtype="<i2").reshape(h // 8, w // 8, 3, k + 1)
    pimg = _apply_mask(strong, part1)
    return fds.restore(public.public_from_image(pimg, k), cipher, key, iv, k, w, h)
