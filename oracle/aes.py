"""AES-128 (FIPS-197) and CTR mode (NIST SP 800-38A, Sect. 6.5), plain numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper encrypts the confidential fragment (Part 1) with AES-128 (Sect. 6.3.1, Fig. 6;
Sect. 6.5.2) and names counter mode for it (Sect. 6.12).  Nothing below is transcribed
from a table: the S-box is generated from its definition in FIPS-197 Sect. 5.1.1
(multiplicative inverse in GF(2^8) followed by the affine map), the round constants from
powers of x in GF(2^8) (FIPS-197 Sect. 5.2).

State layout follows FIPS-197 Sect. 3.4: input byte in[r + 4c] is state s[r, c].
Blocks are handled as (n, 16) uint8 arrays so that many counter blocks are enciphered at once.
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------- GF(2^8)
# FIPS-197 Sect. 4.2: bytes are polynomials over GF(2) modulo m(x) = x^8 + x^4 + x^3 + x + 1.
_M_POLY = 0x11B


def gf_mul(a: int, b: int) -> int:
    """Product in GF(2^8) (FIPS-197 Sect. 4.2): shift-and-add with reduction by m(x)."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & 0x100:
            a ^= _M_POLY
    return r


def gf_inv(a: int) -> int:
    """Multiplicative inverse in GF(2^8), 0 -> 0 (FIPS-197 Sect. 5.1.1): a^254 = a^-1."""
    if a == 0:
        return 0
    r, base, e = 1, a, 254
    while e:
        if e & 1:
            r = gf_mul(r, base)
        base = gf_mul(base, base)
        e >>= 1
    return r


def _affine(b: int) -> int:
    """FIPS-197 Sect. 5.1.1 eq. (5.1): b'_i = b_i ^ b_(i+4) ^ b_(i+5) ^ b_(i+6) ^ b_(i+7) ^ c_i,
    c = 0x63, indices mod 8."""
    out = 0
    for i in range(8):
        bit = ((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8))
               ^ (b >> ((i + 6) % 8)) ^ (b >> ((i + 7) % 8)) ^ (0x63 >> i)) & 1
        out |= bit << i
    return out


SBOX = np.array([_affine(gf_inv(x)) for x in range(256)], dtype=np.uint8)
_MUL2 = np.array([gf_mul(x, 2) for x in range(256)], dtype=np.uint8)
_MUL3 = np.array([gf_mul(x, 3) for x in range(256)], dtype=np.uint8)

# ShiftRows (FIPS-197 Sect. 5.1.2): s'[r, c] = s[r, (c + r) mod 4], byte index r + 4c.
# _SHIFT_ROWS[out] = index of the input byte that lands at output byte `out`.
_SHIFT_ROWS = np.zeros(16, dtype=np.int64)
for _c in range(4):
    for _r in range(4):
        _SHIFT_ROWS[_r + 4 * _c] = _r + 4 * ((_c + _r) % 4)


# --------------------------------------------------------------------------- key schedule
def expand_key(key: bytes) -> np.ndarray:
    """KeyExpansion for Nk = 4, Nr = 10 (FIPS-197 Sect. 5.2).

    Returns the 44 words w[0..43] as a (44, 4) uint8 array (word i = bytes w[i][0..3])."""
    if len(key) != 16:
        raise ValueError("AES-128 key must be 16 bytes")
    w = [list(key[4 * i: 4 * i + 4]) for i in range(4)]
    rcon = 1
    for i in range(4, 44):
        temp = list(w[i - 1])
        if i % 4 == 0:
            temp = temp[1:] + temp[:1]                      # RotWord
            temp = [int(SBOX[t]) for t in temp]              # SubWord
            temp[0] ^= rcon                                  # Rcon[i/4] = (x^(i/4 - 1), 0, 0, 0)
            rcon = gf_mul(rcon, 2)
        w.append([a ^ b for a, b in zip(w[i - 4], temp)])
    return np.array(w, dtype=np.uint8)


# --------------------------------------------------------------------------- cipher
def _mix_columns(s: np.ndarray) -> np.ndarray:
    """MixColumns (FIPS-197 Sect. 5.1.3, eq. 5.6) on every column of every block."""
    out = np.empty_like(s)
    for c in range(4):
        s0, s1, s2, s3 = (s[:, 4 * c + r] for r in range(4))
        out[:, 4 * c + 0] = _MUL2[s0] ^ _MUL3[s1] ^ s2 ^ s3
        out[:, 4 * c + 1] = s0 ^ _MUL2[s1] ^ _MUL3[s2] ^ s3
        out[:, 4 * c + 2] = s0 ^ s1 ^ _MUL2[s2] ^ _MUL3[s3]
        out[:, 4 * c + 3] = _MUL3[s0] ^ s1 ^ s2 ^ _MUL2[s3]
    return out


def encrypt_blocks(round_keys: np.ndarray, blocks: np.ndarray) -> np.ndarray:
    """Cipher() of FIPS-197 Sect. 5.1 on an (n, 16) uint8 array of input blocks."""
    rk = round_keys.reshape(11, 16)        # round r uses words w[4r .. 4r+3]
    s = np.asarray(blocks, dtype=np.uint8) ^ rk[0]
    for rnd in range(1, 10):
        s = SBOX[s][:, _SHIFT_ROWS]        # SubBytes then ShiftRows
        s = _mix_columns(s)
        s ^= rk[rnd]                       # AddRoundKey
    s = SBOX[s][:, _SHIFT_ROWS]
    return s ^ rk[10]


# --------------------------------------------------------------------------- CTR
def ctr_counter_blocks(iv: bytes, first_block: int, n: int) -> np.ndarray:
    """Counter blocks T_i = IV + i mod 2^128, i = first_block .. first_block + n - 1.

    NIST SP 800-38A Sect. 6.5 with the standard incrementing function applied to the whole
    16-byte block, read as a big-endian integer (the convention of OpenSSL's aes-128-ctr)."""
    base = int.from_bytes(iv, "big")
    raw = b"".join(((base + first_block + i) % (1 << 128)).to_bytes(16, "big") for i in range(n))
    return np.frombuffer(raw, dtype=np.uint8).reshape(n, 16)


def ctr_xcrypt(key: bytes, iv: bytes, data: bytes, offset: int = 0) -> bytes:
    """CTR encryption = decryption (NIST SP 800-38A Sect. 6.5): C_j = P_j xor CIPH_K(T_j).

    `offset` is the position of data[0] in the message; it must be a multiple of 16."""
    if offset % 16:
        raise ValueError("offset must be a multiple of 16")
    n = len(data)
    if n == 0:
        return b""
    nblk = (n + 15) // 16
    ks = encrypt_blocks(expand_key(key), ctr_counter_blocks(iv, offset // 16, nblk))
    ks = ks.reshape(-1)[:n]
    return (np.frombuffer(data, dtype=np.uint8) ^ ks).tobytes()
