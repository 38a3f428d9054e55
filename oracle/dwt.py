"""Selective encryption with the DWT (Sect. 6.8-6.12, Figs. 16-18): agnostic, lossless.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Any data is read as a grey-level matrix of bytes (Sect. 6.9.3) and cut into 8x8 blocks.  Per
block (Fig. 18):
  1. a two-level 2-D Le Gall 5/3 DWT by integer lifting (Sect. 6.9.1, Eqs. 1-2): the 8x8 block
     gives the first-level HL, LH, HH (4x4 each) and LL (4x4), which the second level splits
     into 2x2 LL, HL, LH, HH;
  2. level 1 coefficients = the second-level LL (4 values), level 2 = the second-level HL, LH,
     HH (12), level 3 = the first-level HL, LH, HH (48);
  3. level 1 is encrypted with AES-128 in counter mode; level 1 hashed with SHA-256 (with the
     key and IV, Sect. 6.9.3) gives 256 bits that mask level 2 by XOR; level 2 hashed with
     SHA-512 gives 512 bits that mask level 3 (Sect. 6.9.3);
  4. levels 1 and 2 form the private fragment, level 3 the public one.
The transform maps integers to integers and is inverted exactly, so restore is lossless.

Storage (Sect. 6.9.4): the input bytes are taken as -128..127; the first-level HL, LH, HH
and the second-level LL, HL, LH fit 10 bits, the second-level HH 11 bits: level 1 = 40 bits,
level 2 = 124 bits, level 3 = 480 bits per block.

Readings where the paper is silent, ambiguous or garbled:
  - lifting (Eqs. 1-2 as printed subtract a term of the input odd samples in the update step,
    which is not invertible): the reversible 5/3 lifting of JPEG 2000,
        d[n] = x[2n+1] - floor((x[2n] + x[2n+2]) / 2)
        s[n] = x[2n]   + floor((d[n-1] + d[n] + 2) / 4)
    with whole-sample symmetric extension at the block edges (x[8] = x[6], d[-1] = d[0]);
  - 2-D order: rows first (horizontal), then columns (Sect. 6.9.4); low-pass outputs first,
    so LL is the top-left quadrant, HL top-right (horizontal high), LH bottom-left, HH
    bottom-right; the input is shifted by -128 first (Sect. 6.9.4's -128..127);
  - the 11-bit coefficients: the text names the "lower left corner four", its bound matrix
    puts the 648 maxima (which need 11 bits) at the second-level HH, which is used;
  - fields: two's complement, w bits, least significant bit first in a byte stream (stream bit
    b = bit b mod 8 of byte b / 8); per block, level 1 takes 5 bytes, level 2 16 bytes (124
    bits and 4 zero bits), level 3 60 bytes; fields in quadrant order (HL, LH, HH), row-major;
  - the hashed messages: key (16 bytes) || IV (16) || the block index (8 bytes, big-endian,
    the "counter" of Sect. 6.12) || the packed plaintext of the previous level (level 1: 5
    bytes, level 2: 16 bytes); the level 2 bytes are XORed with digest bytes 0..15, the level 3
    bytes with digest bytes 0..59;
  - level 1 of every block, 5 bytes each in block order, is one AES-128-CTR message from the
    IV, as in the first level of protection;
  - blocks in raster order; the matrix is H x W bytes, W and H multiples of 8.  Chunking of
    arbitrary data (Sect. 6.9.3): the bytes fill W-byte rows, zero-padded to whole blocks.
"""
from __future__ import annotations

import hashlib

import numpy as np

from . import aes

L1_BITS = (10,) * 4
L2_BITS = (10,) * 8 + (11,) * 4
L3_BITS = (10,) * 48
L1_BYTES, L2_BYTES, L3_BYTES = 5, 16, 60


def _lift_forward_1d(x: np.ndarray) -> np.ndarray:
    """One level of the reversible 5/3 lifting along the last axis (length 2m): [s | d]."""
    x = np.asarray(x, dtype=np.int64)
    n = x.shape[-1]
    even, odd = x[..., 0::2], x[..., 1::2]
    right = np.concatenate([even[..., 1:], even[..., -1:]], axis=-1)      # x[2n+2], x[n] = x[n-2]
    d = odd - np.floor_divide(even + right, 2)
    left = np.concatenate([d[..., :1], d[..., :-1]], axis=-1)             # d[n-1], d[-1] = d[0]
    s = even + np.floor_divide(left + d + 2, 4)
    assert n % 2 == 0
    return np.concatenate([s, d], axis=-1)


def _lift_inverse_1d(y: np.ndarray) -> np.ndarray:
    y = np.asarray(y, dtype=np.int64)
    m = y.shape[-1] // 2
    s, d = y[..., :m], y[..., m:]
    left = np.concatenate([d[..., :1], d[..., :-1]], axis=-1)
    even = s - np.floor_divide(left + d + 2, 4)
    right = np.concatenate([even[..., 1:], even[..., -1:]], axis=-1)
    odd = d + np.floor_divide(even + right, 2)
    out = np.empty(y.shape, dtype=np.int64)
    out[..., 0::2], out[..., 1::2] = even, odd
    return out


def dwt2(block: np.ndarray) -> np.ndarray:
    """One 2-D level on (..., n, n): rows then columns, quadrants [[LL, HL], [LH, HH]]."""
    rows = _lift_forward_1d(block)
    return np.swapaxes(_lift_forward_1d(np.swapaxes(rows, -1, -2)), -1, -2)


def idwt2(coefs: np.ndarray) -> np.ndarray:
    cols = np.swapaxes(_lift_inverse_1d(np.swapaxes(coefs, -1, -2)), -1, -2)
    return _lift_inverse_1d(cols)


def forward(blocks: np.ndarray) -> np.ndarray:
    """Two-level DWT of (..., 8, 8) byte blocks (shifted by -128): (..., 8, 8) int64."""
    c = dwt2(np.asarray(blocks, dtype=np.int64) - 128)
    c[..., :4, :4] = dwt2(c[..., :4, :4])
    return c


def inverse(coefs: np.ndarray) -> np.ndarray:
    c = np.array(coefs, dtype=np.int64)
    c[..., :4, :4] = idwt2(c[..., :4, :4])
    return idwt2(c) + 128


def levels(c: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(level 1 [..., 4], level 2 [..., 12], level 3 [..., 48]) of two-level coefficients."""
    lv1 = c[..., 0:2, 0:2].reshape(c.shape[:-2] + (4,))
    lv2 = np.concatenate([c[..., 0:2, 2:4].reshape(c.shape[:-2] + (4,)),      # 2nd HL
                          c[..., 2:4, 0:2].reshape(c.shape[:-2] + (4,)),      # 2nd LH
                          c[..., 2:4, 2:4].reshape(c.shape[:-2] + (4,))], -1)  # 2nd HH
    lv3 = np.concatenate([c[..., 0:4, 4:8].reshape(c.shape[:-2] + (16,)),     # 1st HL
                          c[..., 4:8, 0:4].reshape(c.shape[:-2] + (16,)),     # 1st LH
                          c[..., 4:8, 4:8].reshape(c.shape[:-2] + (16,))], -1)  # 1st HH
    return lv1, lv2, lv3


def from_levels(lv1, lv2, lv3) -> np.ndarray:
    lv1, lv2, lv3 = (np.asarray(v, dtype=np.int64) for v in (lv1, lv2, lv3))
    c = np.zeros(lv1.shape[:-1] + (8, 8), dtype=np.int64)
    c[..., 0:2, 0:2] = lv1.reshape(lv1.shape[:-1] + (2, 2))
    c[..., 0:2, 2:4] = lv2[..., 0:4].reshape(lv2.shape[:-1] + (2, 2))
    c[..., 2:4, 0:2] = lv2[..., 4:8].reshape(lv2.shape[:-1] + (2, 2))
    c[..., 2:4, 2:4] = lv2[..., 8:12].reshape(lv2.shape[:-1] + (2, 2))
    c[..., 0:4, 4:8] = lv3[..., 0:16].reshape(lv3.shape[:-1] + (4, 4))
    c[..., 4:8, 0:4] = lv3[..., 16:32].reshape(lv3.shape[:-1] + (4, 4))
    c[..., 4:8, 4:8] = lv3[..., 32:48].reshape(lv3.shape[:-1] + (4, 4))
    return c


def pack_fields(values, widths, nbytes: int) -> bytes:
    """Two's complement fields, LSB first, zero-padded to nbytes."""
    bits = []
    for v, w in zip(values, widths):
        v = int(v)
        if not -(1 << (w - 1)) <= v < (1 << (w - 1)):
            raise OverflowError(f"{v} does not fit {w} bits")
        u = v & ((1 << w) - 1)
        bits.extend((u >> j) & 1 for j in range(w))
    bits.extend([0] * (8 * nbytes - len(bits)))
    return np.packbits(np.array(bits, dtype=np.uint8), bitorder="little").tobytes()


def unpack_fields(data: bytes, widths) -> list[int]:
    bits = np.unpackbits(np.frombuffer(data, dtype=np.uint8), bitorder="little")
    out, pos = [], 0
    for w in widths:
        u = sum(int(bits[pos + j]) << j for j in range(w))
        out.append(u - (1 << w) if u >> (w - 1) else u)
        pos += w
    return out


def _mask(hash_fn, key: bytes, iv: bytes, index: int, prev: bytes, n: int) -> bytes:
    return hash_fn(key + iv + index.to_bytes(8, "big") + prev).digest()[:n]


def _xor(a: bytes, b: bytes) -> bytes:
    return bytes(x ^ y for x, y in zip(a, b))


def to_matrix(data: bytes, width: int) -> np.ndarray:
    """Agnostic chunking (Sect. 6.9.3): bytes as rows of `width`, zero-padded to 8-row blocks."""
    if width <= 0 or width % 8:
        raise ValueError("width must be a positive multiple of 8")
    rows = -(-len(data) // width)
    rows = max(8, -(-rows // 8) * 8)
    buf = np.zeros(rows * width, dtype=np.uint8)
    buf[: len(data)] = np.frombuffer(data, dtype=np.uint8)
    return buf.reshape(rows, width)


def _blocks(matrix: np.ndarray) -> np.ndarray:
    h, w = matrix.shape
    if h % 8 or w % 8:
        raise ValueError("H and W must be multiples of 8")
    return np.asarray(matrix, dtype=np.uint8).reshape(h // 8, 8, w // 8, 8).transpose(0, 2, 1, 3).reshape(-1, 8, 8)


def protect(matrix: np.ndarray, key: bytes, iv: bytes) -> tuple[bytes, bytes, bytes]:
    """(level 1 ciphertext: 5 B/block, level 2 masked: 16 B/block, level 3 masked: 60 B/block)."""
    lv1, lv2, lv3 = levels(forward(_blocks(matrix)))
    p1, p2, p3 = [], [], []
    for b in range(lv1.shape[0]):
        l1 = pack_fields(lv1[b], L1_BITS, L1_BYTES)
        l2 = pack_fields(lv2[b], L2_BITS, L2_BYTES)
        l3 = pack_fields(lv3[b], L3_BITS, L3_BYTES)
        p1.append(l1)
        p2.append(_xor(l2, _mask(hashlib.sha256, key, iv, b, l1, L2_BYTES)))
        p3.append(_xor(l3, _mask(hashlib.sha512, key, iv, b, l2, L3_BYTES)))
    return aes.ctr_xcrypt(key, iv, b"".join(p1)), b"".join(p2), b"".join(p3)


def restore(level1: bytes, level2: bytes, level3: bytes, key: bytes, iv: bytes, width: int,
            height: int) -> np.ndarray:
    """The H x W byte matrix back, exactly."""
    nb = (width // 8) * (height // 8)
    l1s = aes.ctr_xcrypt(key, iv, bytes(level1))
    lv1 = np.zeros((nb, 4), dtype=np.int64)
    lv2 = np.zeros((nb, 12), dtype=np.int64)
    lv3 = np.zeros((nb, 48), dtype=np.int64)
    for b in range(nb):
        l1 = l1s[L1_BYTES * b: L1_BYTES * (b + 1)]
        l2 = _xor(level2[L2_BYTES * b: L2_BYTES * (b + 1)], _mask(hashlib.sha256, key, iv, b, l1, L2_BYTES))
        l3 = _xor(level3[L3_BYTES * b: L3_BYTES * (b + 1)], _mask(hashlib.sha512, key, iv, b, l2, L3_BYTES))
        lv1[b], lv2[b], lv3[b] = unpack_fields(l1, L1_BITS), unpack_fields(l2, L2_BITS), unpack_fields(l3, L3_BITS)
    px = inverse(from_levels(lv1, lv2, lv3))
    by, bx = height // 8, width // 8
    return px.reshape(by, bx, 8, 8).transpose(0, 2, 1, 3).reshape(height, width).astype(np.uint8)
