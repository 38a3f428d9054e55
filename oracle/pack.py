"""Bit-packed coefficient storage (Sect. 6.4.3, Table 5): the paper's 11-bit and 8-bit
storage of DCT coefficients instead of 16-bit words.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What the paper fixes: the DC coefficient (at most 2040) takes 11 bits; an AC coefficient takes
11 bits, a sign bit and a 10-bit magnitude (0..1023) ("11-bit storage"), or 8 bits, a sign bit
and a 7-bit magnitude ("8-bit storage", lossy).  Its storage arithmetic: 11 x 6 / 64 / 8 =
12.9 % of the image for the six selected coefficients with 11-bit storage, 5 / 64 +
11 / 8 / 64 = 9.96 % with 8-bit storage.

Readings where the paper is silent:
  - the DC field is unsigned; an AC field is sign-magnitude with the sign in its top bit
    (set for negative values; -0 never occurs);
  - 8-bit storage saturates an AC magnitude above 127 to 127 (the paper's bound is garbled);
  - both fragments are packed (the public fragment is int16 coefficients here, not the
    paper's IDCT image), each channel-block's fields in fragment order (zigzag k+1..63,
    resp. 0..k), channel-blocks in [by][bx][c] order;
  - a field of width w occupies the next w bits of the stream, least significant bit first;
    stream bit b is bit b % 8 of byte b // 8; the last byte is padded with zero bits;
  - the packed private stream is AES-128-CTR encrypted like the int16 one (one message per
    image, 128-bit big-endian counter from the IV).
"""
from __future__ import annotations

import numpy as np

from . import aes, fds

FORMS = (11, 8)          # AC field width: 11-bit or 8-bit storage
DC_BITS = 11


def ac_bits(form: int) -> int:
    if form not in FORMS:
        raise ValueError("form must be 11 or 8")
    return form


def fields_of(values: np.ndarray, first_is_dc: bool, form: int) -> tuple[np.ndarray, np.ndarray]:
    """Field codes and widths of one fragment [n_cb, m] in stream order (row-major).

    DC (column 0 when first_is_dc): unsigned, must be in 0..2047.  AC: sign-magnitude; 11-bit
    storage needs |value| <= 1023, 8-bit storage saturates |value| to 127."""
    v = np.asarray(values, dtype=np.int64)
    w = ac_bits(form)
    mag_max = (1 << (w - 1)) - 1
    widths = np.full(v.shape, w, dtype=np.int64)
    mag = np.abs(v)
    ac = mag[..., 1:] if first_is_dc else mag
    if w == 8:
        mag = np.minimum(mag, mag_max)
    elif ac.size and ac.max() > mag_max:
        raise OverflowError("AC coefficient outside the 11-bit storage range")
    codes = np.where(v < 0, (1 << (w - 1)) | mag, mag)
    if first_is_dc and v.shape[-1] > 0:
        dc = v[..., 0]
        if dc.size and (dc.min() < 0 or dc.max() >= (1 << DC_BITS)):
            raise OverflowError("DC coefficient outside 11 bits")
        codes[..., 0] = dc
        widths[..., 0] = DC_BITS
    return codes.reshape(-1), widths.reshape(-1)


def pack_bits(codes: np.ndarray, widths: np.ndarray) -> bytes:
    """Concatenate fields LSB-first into bytes (zero-padded to a whole byte)."""
    codes = np.asarray(codes, dtype=np.int64)
    widths = np.asarray(widths, dtype=np.int64)
    j = np.arange(DC_BITS)
    bitmat = (codes[:, None] >> j[None, :]) & 1              # bit j of every field
    bits = bitmat[j[None, :] < widths[:, None]]               # each field's w bits, in order
    bits = np.concatenate([bits, np.zeros(-bits.size % 8, dtype=np.int64)])
    return np.packbits(bits.astype(np.uint8), bitorder="little").tobytes()


def unpack_bits(data: bytes, widths: np.ndarray) -> np.ndarray:
    """The field codes of `widths` from the start of `data`."""
    widths = np.asarray(widths, dtype=np.int64)
    bits = np.unpackbits(np.frombuffer(data, dtype=np.uint8), bitorder="little").astype(np.int64)
    start = np.concatenate([[0], np.cumsum(widths)[:-1]]) if widths.size else widths
    j = np.arange(DC_BITS)
    inside = j[None, :] < widths[:, None]
    idx = np.where(inside, start[:, None] + j[None, :], 0)
    return (np.where(inside, bits[idx], 0) << j[None, :]).sum(axis=1)


def decode(codes: np.ndarray, widths: np.ndarray, first_is_dc: bool, m: int) -> np.ndarray:
    """Signed values [n_cb, m] from field codes (inverse of fields_of, up to saturation)."""
    n = codes.size // m if m else 0
    c = codes.reshape(n, m)
    w = widths.reshape(n, m)
    sign = (c >> (w - 1)) & 1
    mag = c & ((1 << (w - 1)) - 1)
    v = np.where(sign == 1, -mag, mag)
    if first_is_dc and m > 0:
        v[:, 0] = c[:, 0]
    return v


def sizes(width: int, height: int, k: int, form: int) -> tuple[int, int]:
    """Bytes of the packed public and private fragments."""
    ncb = (width // 8) * (height // 8) * 3
    w = ac_bits(form)
    pub_bits = ncb * (63 - k) * w
    priv_bits = ncb * (DC_BITS + k * w)
    return (pub_bits + 7) // 8, (priv_bits + 7) // 8


def protect_packed(img: np.ndarray, key: bytes, iv: bytes, k: int, form: int) -> tuple[bytes, bytes]:
    """The first level of protection with packed storage: (public bytes, private ciphertext)."""
    pub, priv = fds.protect(img, key, iv, k)
    ncb = (img.shape[0] // 8) * (img.shape[1] // 8) * 3
    plain = np.frombuffer(aes.ctr_xcrypt(key, iv, priv), dtype="<i2").astype(np.int64)
    part1 = plain.reshape(ncb, k + 1)
    part2 = np.asarray(pub, dtype=np.int64).reshape(ncb, 63 - k)
    pub_codes, pub_w = fields_of(part2, False, form)
    priv_codes, priv_w = fields_of(part1, True, form)
    return pack_bits(pub_codes, pub_w), aes.ctr_xcrypt(key, iv, pack_bits(priv_codes, priv_w))


def restore_packed(public: bytes, private: bytes, key: bytes, iv: bytes, k: int, form: int,
                   width: int, height: int) -> np.ndarray:
    """Inverse of protect_packed (exact for 11-bit storage)."""
    ncb = (width // 8) * (height // 8) * 3
    w = ac_bits(form)
    pub_w = np.full(ncb * (63 - k), w, dtype=np.int64)
    priv_w = np.tile(np.array([DC_BITS] + [w] * k, dtype=np.int64), ncb)
    part2 = decode(unpack_bits(public, pub_w), pub_w, False, 63 - k).reshape(ncb, 63 - k)
    plain = aes.ctr_xcrypt(key, iv, bytes(private))
    part1 = decode(unpack_bits(plain, priv_w), priv_w, True, k + 1)
    pub16 = part2.astype("<i2").reshape(height // 8, width // 8, 3, 63 - k)
    priv16 = aes.ctr_xcrypt(key, iv, part1.astype("<i2").tobytes())
    return fds.restore(pub16, priv16, key, iv, k, width, height)
