// Device building blocks of the selective-protection kernels (sm_103a).
//
//  * 8-point DCT-II / inverse butterflies in float32 (Sect. 6.4.2: separable 8x8 transform)
//  * AES-128 with T-tables in shared memory and CTR counter blocks (FIPS-197; Sect. 6.12)
//  * the exact-rounding fallback (Sect. 6.4.3 reading: round half away from zero of the exact
//    value): exact integer coordinates in Z[cos(pi/16)], a 128-bit fixed-point decision and,
//    at a rounding boundary, a 256-bit one that is exact by a norm bound
#pragma once

#include <stdint.h>

#include "fds_cos_limbs.h"

namespace fds {

// ------------------------------------------------------------------------------------------
// constants
// cos(j pi / 16)
constexpr double kC1 = 0.98078528040323044912618223613424;
constexpr double kC2 = 0.92387953251128675612818318939679;
constexpr double kC3 = 0.83146961230254523707878837761791;
constexpr double kC5 = 0.55557023301960222474283081394853;
constexpr double kC6 = 0.38268343236508977172845998403040;
constexpr double kC7 = 0.19509032201612826784828486847702;
constexpr double kLambda = 0.35355339059327376220042218105242;  // 1 / (2 sqrt 2) = b_0

// 2^23 + 2^22: adding it to a float of magnitude < 2^22 rounds to an integer (to nearest,
// ties to even) that sits in the low mantissa bits.
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

// zigzag scan position of (u, v): anti-diagonals s = u + v; odd s walks u upward from its
// smallest value, even s downward from its largest.
__host__ __device__ constexpr int zigzag_of(int u, int v) {
  int z = 0;
  for (int s = 0; s < 15; ++s) {
    int lo = s > 7 ? s - 7 : 0, hi = s < 7 ? s : 7;
    if (s != u + v) {
      z += hi - lo + 1;
      continue;
    }
    return (s & 1) ? z + (u - lo) : z + (hi - u);
  }
  return -1;
}

// ------------------------------------------------------------------------------------------
// 8-point butterflies.  All constants are products computed in double and rounded once.
//
// Forward: x -> X with X_k = sum_n b_k(n) x_n for k in {1, 2, 3, 5, 6, 7} (times `irr`), and
// X_0 = sum_n x_n, X_4 = sum_n w_n x_n (w = +1 -1 -1 +1 +1 -1 -1 +1) left unscaled when
// RAT_UNSCALED, else multiplied by b_0 = 1/(2 sqrt 2).  Unscaled rational outputs of integer
// inputs are exact, which keeps F[0][0], F[0][4], F[4][0], F[4][4] exact (each is an
// integer / 8).
template <bool RAT_UNSCALED, bool IRR_LAMBDA>
__device__ __forceinline__ void dct8_sd(const float (&s)[4], const float (&d)[4], float (&x)[8]) {
  constexpr double m = IRR_LAMBDA ? kLambda : 1.0;
  constexpr float a2 = (float)(0.5 * m * kC2), a6 = (float)(0.5 * m * kC6);
  constexpr float h1 = (float)(0.5 * m * kC1), h3 = (float)(0.5 * m * kC3);
  constexpr float h5 = (float)(0.5 * m * kC5), h7 = (float)(0.5 * m * kC7);
  constexpr float lam = (float)kLambda;
  const float e0 = s[0] + s[3], e1 = s[1] + s[2], f0 = s[0] - s[3], f1 = s[1] - s[2];
  if (RAT_UNSCALED) {
    x[0] = e0 + e1;
    x[4] = e0 - e1;
  } else {
    x[0] = fmaf(e0, lam, e1 * lam);
    x[4] = fmaf(e0, lam, e1 * -lam);
  }
  x[2] = fmaf(f0, a2, f1 * a6);
  x[6] = fmaf(f0, a6, f1 * -a2);
  // odd rows of the basis on d_n = x_n - x_(7-n), n = 0..3
  x[1] = fmaf(d[3], h7, fmaf(d[2], h5, fmaf(d[1], h3, d[0] * h1)));
  x[3] = fmaf(d[3], -h5, fmaf(d[2], -h1, fmaf(d[1], -h7, d[0] * h3)));
  x[5] = fmaf(d[3], h3, fmaf(d[2], h7, fmaf(d[1], -h1, d[0] * h5)));
  x[7] = fmaf(d[3], -h1, fmaf(d[2], h3, fmaf(d[1], -h5, d[0] * h7)));
}

template <bool RAT_UNSCALED, bool IRR_LAMBDA>
__device__ __forceinline__ void dct8(float (&x)[8]) {
  const float s[4] = {x[0] + x[7], x[1] + x[6], x[2] + x[5], x[3] + x[4]};
  const float d[4] = {x[0] - x[7], x[1] - x[6], x[2] - x[5], x[3] - x[4]};
  dct8_sd<RAT_UNSCALED, IRR_LAMBDA>(s, d, x);
}

// Row pass straight from pixel bytes.  X_i = 2^23 + p_i (a float built from the byte), so
// d_i = X_i - X_(7-i) = p_i - p_(7-i) and s_i = (X_i - (2^24 + 256)) + X_(7-i) =
// (p_i - 128) + (p_(7-i) - 128) are exact: the level shift by 128 costs nothing.
__device__ __forceinline__ void dct8_row_bytes(const float (&X)[8], float (&x)[8]) {
  constexpr float c2 = 16777472.0f;  // 2^24 + 256
  const float s[4] = {(X[0] - c2) + X[7], (X[1] - c2) + X[6], (X[2] - c2) + X[5], (X[3] - c2) + X[4]};
  const float d[4] = {X[0] - X[7], X[1] - X[6], X[2] - X[5], X[3] - X[4]};
  dct8_sd<true, false>(s, d, x);
}

// Error weight of one 8-point pass over exact inputs: |d_0| + .. + |d_3| + |f_0| + |f_1| with
// f_0 = s_0 - s_3, f_1 = s_1 - s_2 (small integers, so the sum is exact).  The rounding error
// of every irrational output of the pass is at most 2.46 u times this weight (u = 2^-24).
__device__ __forceinline__ float pass_weight(const float (&s)[4], const float (&d)[4]) {
  return ((fabsf(d[0]) + fabsf(d[1])) + (fabsf(d[2]) + fabsf(d[3]))) + (fabsf(s[0] - s[3]) + fabsf(s[1] - s[2]));
}

// dct8_row_bytes that also returns the row's error weight
__device__ __forceinline__ float dct8_row_bytes_w(const float (&X)[8], float (&x)[8]) {
  constexpr float c2 = 16777472.0f;  // 2^24 + 256
  const float s[4] = {(X[0] - c2) + X[7], (X[1] - c2) + X[6], (X[2] - c2) + X[5], (X[3] - c2) + X[4]};
  const float d[4] = {X[0] - X[7], X[1] - X[6], X[2] - X[5], X[3] - X[4]};
  dct8_sd<true, false>(s, d, x);
  return pass_weight(s, d);
}

// dct8<true, true> of an exact-integer column that also returns its error weight
__device__ __forceinline__ float dct8_rat_w(float (&x)[8]) {
  const float s[4] = {x[0] + x[7], x[1] + x[6], x[2] + x[5], x[3] + x[4]};
  const float d[4] = {x[0] - x[7], x[1] - x[6], x[2] - x[5], x[3] - x[4]};
  dct8_sd<true, true>(s, d, x);
  return pass_weight(s, d);
}

// ---- the same butterflies on pairs of independent columns (packed f32x2 arithmetic); every
// lane performs exactly the scalar operations, so the results are bit-identical
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float k) { return __fmul2_rn(a, make_float2(k, k)); }
__device__ __forceinline__ float2 fma2(float2 a, float k, float2 c) { return __ffma2_rn(a, make_float2(k, k), c); }

template <bool RAT_UNSCALED, bool IRR_LAMBDA>
__device__ __forceinline__ void dct8_sd2(const float2 (&s)[4], const float2 (&d)[4], float2 (&x)[8]) {
  constexpr double m = IRR_LAMBDA ? kLambda : 1.0;
  constexpr float a2 = (float)(0.5 * m * kC2), a6 = (float)(0.5 * m * kC6);
  constexpr float h1 = (float)(0.5 * m * kC1), h3 = (float)(0.5 * m * kC3);
  constexpr float h5 = (float)(0.5 * m * kC5), h7 = (float)(0.5 * m * kC7);
  constexpr float lam = (float)kLambda;
  const float2 e0 = add2(s[0], s[3]), e1 = add2(s[1], s[2]), f0 = sub2(s[0], s[3]), f1 = sub2(s[1], s[2]);
  if (RAT_UNSCALED) {
    x[0] = add2(e0, e1);
    x[4] = sub2(e0, e1);
  } else {
    x[0] = fma2(e0, lam, mul2(e1, lam));
    x[4] = fma2(e0, lam, mul2(e1, -lam));
  }
  x[2] = fma2(f0, a2, mul2(f1, a6));
  x[6] = fma2(f0, a6, mul2(f1, -a2));
  x[1] = fma2(d[3], h7, fma2(d[2], h5, fma2(d[1], h3, mul2(d[0], h1))));
  x[3] = fma2(d[3], -h5, fma2(d[2], -h1, fma2(d[1], -h7, mul2(d[0], h3))));
  x[5] = fma2(d[3], h3, fma2(d[2], h7, fma2(d[1], -h1, mul2(d[0], h5))));
  x[7] = fma2(d[3], -h1, fma2(d[2], h3, fma2(d[1], -h5, mul2(d[0], h7))));
}

template <bool RAT_UNSCALED, bool IRR_LAMBDA>
__device__ __forceinline__ void dct8_2(float2 (&x)[8]) {
  const float2 s[4] = {add2(x[0], x[7]), add2(x[1], x[6]), add2(x[2], x[5]), add2(x[3], x[4])};
  const float2 d[4] = {sub2(x[0], x[7]), sub2(x[1], x[6]), sub2(x[2], x[5]), sub2(x[3], x[4])};
  dct8_sd2<RAT_UNSCALED, IRR_LAMBDA>(s, d, x);
}

// dct8_rat_w on two exact-integer columns at once; returns the sum of both error weights
__device__ __forceinline__ float dct8_rat_w2(float2 (&x)[8]) {
  const float2 s[4] = {add2(x[0], x[7]), add2(x[1], x[6]), add2(x[2], x[5]), add2(x[3], x[4])};
  const float2 d[4] = {sub2(x[0], x[7]), sub2(x[1], x[6]), sub2(x[2], x[5]), sub2(x[3], x[4])};
  dct8_sd2<true, true>(s, d, x);
  const float wx = ((fabsf(d[0].x) + fabsf(d[1].x)) + (fabsf(d[2].x) + fabsf(d[3].x))) +
                   (fabsf(s[0].x - s[3].x) + fabsf(s[1].x - s[2].x));
  const float wy = ((fabsf(d[0].y) + fabsf(d[1].y)) + (fabsf(d[2].y) + fabsf(d[3].y))) +
                   (fabsf(s[0].y - s[3].y) + fabsf(s[1].y - s[2].y));
  return wx + wy;
}

// idct8 on two independent columns at once (bit-identical per lane)
__device__ __forceinline__ void idct8_2(float2 (&x)[8]) {
  constexpr float lam = (float)kLambda;
  constexpr float c2 = (float)(0.5 * kC2), c6 = (float)(0.5 * kC6);
  constexpr float h1 = (float)(0.5 * kC1), h3 = (float)(0.5 * kC3);
  constexpr float h5 = (float)(0.5 * kC5), h7 = (float)(0.5 * kC7);
  const float2 a = fma2(x[0], lam, mul2(x[4], lam)), b = fma2(x[0], lam, mul2(x[4], -lam));
  const float2 t1 = fma2(x[2], c2, mul2(x[6], c6)), t2 = fma2(x[2], c6, mul2(x[6], -c2));
  const float2 e0 = add2(a, t1), e1 = add2(b, t2), e2 = sub2(b, t2), e3 = sub2(a, t1);
  const float2 o0 = fma2(x[7], h7, fma2(x[5], h5, fma2(x[3], h3, mul2(x[1], h1))));
  const float2 o1 = fma2(x[7], -h5, fma2(x[5], -h1, fma2(x[3], -h7, mul2(x[1], h3))));
  const float2 o2 = fma2(x[7], h3, fma2(x[5], h7, fma2(x[3], -h1, mul2(x[1], h5))));
  const float2 o3 = fma2(x[7], -h1, fma2(x[5], h3, fma2(x[3], -h5, mul2(x[1], h7))));
  x[0] = add2(e0, o0);
  x[7] = sub2(e0, o0);
  x[1] = add2(e1, o1);
  x[6] = sub2(e1, o1);
  x[2] = add2(e2, o2);
  x[5] = sub2(e2, o2);
  x[3] = add2(e3, o3);
  x[4] = sub2(e3, o3);
}

// Inverse: X (orthonormal coefficients) -> x_n = sum_k b_k(n) X_k.
__device__ __forceinline__ void idct8(float (&x)[8]) {
  constexpr float lam = (float)kLambda;
  constexpr float c2 = (float)(0.5 * kC2), c6 = (float)(0.5 * kC6);
  constexpr float h1 = (float)(0.5 * kC1), h3 = (float)(0.5 * kC3);
  constexpr float h5 = (float)(0.5 * kC5), h7 = (float)(0.5 * kC7);
  const float a = fmaf(x[0], lam, x[4] * lam), b = fmaf(x[0], lam, x[4] * -lam);
  const float t1 = fmaf(x[2], c2, x[6] * c6), t2 = fmaf(x[2], c6, x[6] * -c2);
  const float e0 = a + t1, e1 = b + t2, e2 = b - t2, e3 = a - t1;
  const float o0 = fmaf(x[7], h7, fmaf(x[5], h5, fmaf(x[3], h3, x[1] * h1)));
  const float o1 = fmaf(x[7], -h5, fmaf(x[5], -h1, fmaf(x[3], -h7, x[1] * h3)));
  const float o2 = fmaf(x[7], h3, fmaf(x[5], h7, fmaf(x[3], -h1, x[1] * h5)));
  const float o3 = fmaf(x[7], -h1, fmaf(x[5], h3, fmaf(x[3], -h5, x[1] * h7)));
  x[0] = e0 + o0;
  x[7] = e0 - o0;
  x[1] = e1 + o1;
  x[6] = e1 - o1;
  x[2] = e2 + o2;
  x[5] = e2 - o2;
  x[3] = e3 + o3;
  x[4] = e3 - o3;
}

// ------------------------------------------------------------------------------------------
// AES-128 (FIPS-197).  A state column is a 32-bit word holding bytes 4c .. 4c+3 of the block
// little-endian (byte r of the column at bits 8r); round keys use the same word convention.

__host__ __device__ inline uint8_t gf_xtime(uint8_t a) {
  return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1B : 0x00));
}

__host__ __device__ inline uint8_t gf_mul(uint8_t a, uint8_t b) {
  uint8_t r = 0;
  for (int i = 0; i < 8; ++i) {
    if (b & 1) r ^= a;
    a = gf_xtime(a);
    b >>= 1;
  }
  return r;
}

// S-box entry from its definition: inverse in GF(2^8) (x^254, 0 -> 0), then the affine map
// b ^ rotl(b,1) ^ rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ 0x63.
__host__ __device__ inline uint8_t aes_sbox(uint8_t x) {
  uint8_t inv = 1, p = gf_mul(x, x);
  for (int i = 0; i < 7; ++i) {
    inv = gf_mul(inv, p);
    p = gf_mul(p, p);
  }
  if (x == 0) inv = 0;
  uint8_t r = 0x63;
  for (int k = 0; k < 5; ++k) r ^= (uint8_t)((inv << k) | (inv >> ((8 - k) & 7)));
  return r;
}

// T0[x] = (2S, S, S, 3S) as bytes 0..3: the MixColumns column of S[x] in row 0.
__host__ __device__ inline uint32_t aes_t0(uint8_t x) {
  uint8_t s = aes_sbox(x), s2 = gf_xtime(s), s3 = (uint8_t)(s2 ^ s);
  return (uint32_t)s2 | ((uint32_t)s << 8) | ((uint32_t)s << 16) | ((uint32_t)s3 << 24);
}

// Encrypt one block in place.  rk: 44 round-key words; T: four shared-memory tables,
// T[r][x] = rotl(T0[x], 8r) (the MixColumns column of S[x] entering from row r).  The last
// round takes S[x] from byte 1 of T[0][x].
__device__ __forceinline__ void aes128_encrypt(uint32_t (&s)[4], const uint32_t* rk,
                                               const uint32_t* T) {
  // table entry by byte offset: byte b of a word, times 4, is (w >> (8b - 2)) & 0x3fc
  const char* Tc = reinterpret_cast<const char*>(T);
  auto t0 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + ((w << 2) & 0x3fcu)); };
  auto t1 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + 1024 + ((w >> 6) & 0x3fcu)); };
  auto t2 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + 2048 + ((w >> 14) & 0x3fcu)); };
  auto t3 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + 3072 + ((w >> 22) & 0x3fcu)); };
  uint32_t s0 = s[0] ^ rk[0], s1 = s[1] ^ rk[1], s2 = s[2] ^ rk[2], s3 = s[3] ^ rk[3];
  // the nine middle rounds stay a loop: a compact body keeps the kernels' hot code in the
  // instruction cache (the unrolled form was measurably slower)
#pragma unroll 1
  for (int r = 1; r < 10; ++r) {
    const uint32_t n0 = t0(s0) ^ t1(s1) ^ t2(s2) ^ t3(s3) ^ rk[4 * r];
    const uint32_t n1 = t0(s1) ^ t1(s2) ^ t2(s3) ^ t3(s0) ^ rk[4 * r + 1];
    const uint32_t n2 = t0(s2) ^ t1(s3) ^ t2(s0) ^ t3(s1) ^ rk[4 * r + 2];
    const uint32_t n3 = t0(s3) ^ t1(s0) ^ t2(s1) ^ t3(s2) ^ rk[4 * r + 3];
    s0 = n0;
    s1 = n1;
    s2 = n2;
    s3 = n3;
  }
  // last round: SubBytes + ShiftRows + AddRoundKey; byte r of column c = S[row r of column c+r];
  // S[x] is byte 1 of T0[x] (__byte_perm selector 0x4441 etc. moves it to byte r)
  s[0] = (__byte_perm(t0(s0), 0u, 0x4441u) | __byte_perm(t0(s1 >> 8), 0u, 0x4414u) |
          __byte_perm(t0(s2 >> 16), 0u, 0x4144u) | __byte_perm(t0(s3 >> 24), 0u, 0x1444u)) ^ rk[40];
  s[1] = (__byte_perm(t0(s1), 0u, 0x4441u) | __byte_perm(t0(s2 >> 8), 0u, 0x4414u) |
          __byte_perm(t0(s3 >> 16), 0u, 0x4144u) | __byte_perm(t0(s0 >> 24), 0u, 0x1444u)) ^ rk[41];
  s[2] = (__byte_perm(t0(s2), 0u, 0x4441u) | __byte_perm(t0(s3 >> 8), 0u, 0x4414u) |
          __byte_perm(t0(s0 >> 16), 0u, 0x4144u) | __byte_perm(t0(s1 >> 24), 0u, 0x1444u)) ^ rk[42];
  s[3] = (__byte_perm(t0(s3), 0u, 0x4441u) | __byte_perm(t0(s0 >> 8), 0u, 0x4414u) |
          __byte_perm(t0(s1 >> 16), 0u, 0x4144u) | __byte_perm(t0(s2 >> 24), 0u, 0x1444u)) ^ rk[43];
}

constexpr int kTrepWords = 256 * 32;   // T0 replicated: entry x of copy L at word 32 x + L

// 32-bit load from a shared-memory window address
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// AES-128 with one T-table, T0, replicated in shared memory: 2^(SH-2) copies, entry x of copy
// c at word 2^(SH-2) x + c, lane L reading copy L mod 2^(SH-2).  SH = 7 (32 copies, 32 KB):
// lane L always reads bank L, so a warp's 32 lookups never conflict; SH = 6 (16 copies,
// 16 KB): lanes L and L + 16 share a copy and meet in a bank at most pairwise.  Tl = the
// shared-window address of the table plus 4 * (its copy for this lane).  The table index is
// taken out of the state word by one byte permute and scaled by a shift-add into the address
// (measured alone, 32 copies: 805 instead of 956 instructions and 8.2 instead of 10.1 SM
// cycles per block against masking shifted words; 16 copies: 9.8; four separate 1 KB tables,
// bank conflicts: 14.9).  T_r[x] = rotl(T0[x], 8 r) by byte permutes; S[x] is byte 1 of T0[x]
// (last round).
template <int SH>
__device__ __forceinline__ uint32_t trep_at(uint32_t Tl, uint32_t w, uint32_t sel) {
  return lds_u32(Tl + (__byte_perm(w, 0u, sel) << SH));
}
template <int SH = 7>
__device__ __forceinline__ void aes128_encrypt_rep(uint32_t (&s)[4], const uint32_t* rk, uint32_t Tl) {
  auto l0 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4440u); };
  auto l1 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4441u); };
  auto l2 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4442u); };
  auto l3 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4443u); };
  auto r8 = [](uint32_t x) { return __byte_perm(x, x, 0x2103u); };
  auto r16 = [](uint32_t x) { return __byte_perm(x, x, 0x1032u); };
  auto r24 = [](uint32_t x) { return __byte_perm(x, x, 0x0321u); };
  uint32_t s0 = s[0] ^ rk[0], s1 = s[1] ^ rk[1], s2 = s[2] ^ rk[2], s3 = s[3] ^ rk[3];
#pragma unroll 1
  for (int r = 1; r < 10; ++r) {
    const uint32_t n0 = l0(s0) ^ r8(l1(s1)) ^ r16(l2(s2)) ^ r24(l3(s3)) ^ rk[4 * r];
    const uint32_t n1 = l0(s1) ^ r8(l1(s2)) ^ r16(l2(s3)) ^ r24(l3(s0)) ^ rk[4 * r + 1];
    const uint32_t n2 = l0(s2) ^ r8(l1(s3)) ^ r16(l2(s0)) ^ r24(l3(s1)) ^ rk[4 * r + 2];
    const uint32_t n3 = l0(s3) ^ r8(l1(s0)) ^ r16(l2(s1)) ^ r24(l3(s2)) ^ rk[4 * r + 3];
    s0 = n0;
    s1 = n1;
    s2 = n2;
    s3 = n3;
  }
  s[0] = (__byte_perm(l0(s0), 0u, 0x4441u) | __byte_perm(l1(s1), 0u, 0x4414u) |
          __byte_perm(l2(s2), 0u, 0x4144u) | __byte_perm(l3(s3), 0u, 0x1444u)) ^ rk[40];
  s[1] = (__byte_perm(l0(s1), 0u, 0x4441u) | __byte_perm(l1(s2), 0u, 0x4414u) |
          __byte_perm(l2(s3), 0u, 0x4144u) | __byte_perm(l3(s0), 0u, 0x1444u)) ^ rk[41];
  s[2] = (__byte_perm(l0(s2), 0u, 0x4441u) | __byte_perm(l1(s3), 0u, 0x4414u) |
          __byte_perm(l2(s0), 0u, 0x4144u) | __byte_perm(l3(s1), 0u, 0x1444u)) ^ rk[42];
  s[3] = (__byte_perm(l0(s3), 0u, 0x4441u) | __byte_perm(l1(s0), 0u, 0x4414u) |
          __byte_perm(l2(s1), 0u, 0x4144u) | __byte_perm(l3(s2), 0u, 0x1444u)) ^ rk[43];
}

// The same on M independent blocks at once, their rounds interleaved: the M lookups chains
// overlap, so one warp keeps the table pipe busy where a single block per thread would wait
// out each round's load latency.
template <int M, int SH = 7>
__device__ __forceinline__ void aes128_encrypt_rep_n(uint32_t (&s)[M][4], const uint32_t* rk, uint32_t Tl) {
  auto l0 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4440u); };
  auto l1 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4441u); };
  auto l2 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4442u); };
  auto l3 = [&](uint32_t w) { return trep_at<SH>(Tl, w, 0x4443u); };
  auto r8 = [](uint32_t x) { return __byte_perm(x, x, 0x2103u); };
  auto r16 = [](uint32_t x) { return __byte_perm(x, x, 0x1032u); };
  auto r24 = [](uint32_t x) { return __byte_perm(x, x, 0x0321u); };
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int c = 0; c < 4; ++c) s[m][c] ^= rk[c];
#pragma unroll 1
  for (int r = 1; r < 10; ++r) {
    const uint32_t k0 = rk[4 * r], k1 = rk[4 * r + 1], k2 = rk[4 * r + 2], k3 = rk[4 * r + 3];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const uint32_t s0 = s[m][0], s1 = s[m][1], s2 = s[m][2], s3 = s[m][3];
      s[m][0] = l0(s0) ^ r8(l1(s1)) ^ r16(l2(s2)) ^ r24(l3(s3)) ^ k0;
      s[m][1] = l0(s1) ^ r8(l1(s2)) ^ r16(l2(s3)) ^ r24(l3(s0)) ^ k1;
      s[m][2] = l0(s2) ^ r8(l1(s3)) ^ r16(l2(s0)) ^ r24(l3(s1)) ^ k2;
      s[m][3] = l0(s3) ^ r8(l1(s0)) ^ r16(l2(s1)) ^ r24(l3(s2)) ^ k3;
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint32_t s0 = s[m][0], s1 = s[m][1], s2 = s[m][2], s3 = s[m][3];
    s[m][0] = (__byte_perm(l0(s0), 0u, 0x4441u) | __byte_perm(l1(s1), 0u, 0x4414u) |
               __byte_perm(l2(s2), 0u, 0x4144u) | __byte_perm(l3(s3), 0u, 0x1444u)) ^ rk[40];
    s[m][1] = (__byte_perm(l0(s1), 0u, 0x4441u) | __byte_perm(l1(s2), 0u, 0x4414u) |
               __byte_perm(l2(s3), 0u, 0x4144u) | __byte_perm(l3(s0), 0u, 0x1444u)) ^ rk[41];
    s[m][2] = (__byte_perm(l0(s2), 0u, 0x4441u) | __byte_perm(l1(s3), 0u, 0x4414u) |
               __byte_perm(l2(s0), 0u, 0x4144u) | __byte_perm(l3(s1), 0u, 0x1444u)) ^ rk[42];
    s[m][3] = (__byte_perm(l0(s3), 0u, 0x4441u) | __byte_perm(l1(s0), 0u, 0x4414u) |
               __byte_perm(l2(s1), 0u, 0x4144u) | __byte_perm(l3(s2), 0u, 0x1444u)) ^ rk[43];
  }
}

// AES-128 with the pair table: T0 and T2 = rotl(T0, 16), each replicated per lane, in one
// 64 KB table that starts at shared-window address kTpairWin (a multiple of 64 KB).  Entry x
// of table j (0: T0, 1: T2), copy L, is the word at window address kTpairWin + 256 x + 128 j +
// 4 L; lane L reads copy L, so a warp's 32 lookups fall in 32 distinct banks.  One byte
// permute forms the whole address of a lookup: the state byte goes to bits 8..15 and the
// lane's constant supplies bits 0..7 (128 j + 4 L) and 16..31 (kTpairWin >> 16), so a lookup
// is a permute and a load, with no address arithmetic.  The two other tables are rotations:
// T1 = rotl(T0, 8) and T3 = rotl(T2, 8), so column c of a middle round is
//   T0[s_c.0] ^ T2[s_{c+2}.2] ^ rk_c ^ rotl8(T0[s_{c+1}.1] ^ T2[s_{c+3}.3]),
// one rotation per column.  In the last round S[x] is byte 1 and byte 2 of T0[x] and byte 0
// and byte 3 of T2[x], so each output byte is taken where it already sits.  Measured alone
// (GB300, one CTA of 1024 threads per SM): 596 instructions and 6.3 SM cycles per keystream
// block against 800 and 8.15 with T0 replicated in a 32 KB table (the same table placed at
// an arbitrary address costs an add per lookup: 750 and 8.0).
constexpr uint32_t kTpairWin = 0x10000u;
constexpr int kTpairBytes = 65536;

// the lane's constants for T0 and T2 lookups.  The lane index is read from %laneid where the
// constants are needed (a volatile read the compiler does not hoist), so that they are not
// kept live through a kernel's other phases.
struct PairLanes {
  uint32_t c0, c2;
};
__device__ __forceinline__ PairLanes pair_lanes() {
  uint32_t lane;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(lane));
  const uint32_t hi = kTpairWin & 0xffff0000u, l4 = 4u * lane;
  return PairLanes{hi | l4, hi | (128u + l4)};
}
// byte X of w looked up in the table whose lane constant is lc
template <int X>
__device__ __forceinline__ uint32_t tpair(uint32_t w, uint32_t lc) {
  return lds_u32(__byte_perm(w, lc, 0x7604u | ((uint32_t)X << 4)));
}
// Fill the pair table at `tab` (shared memory, window address kTpairWin) from T0 in global
// memory (256 words): threads t = 0 .. nthreads - 1 of the CTA; a barrier must follow
__device__ __forceinline__ void fill_pair_table(uint8_t* tab, const uint32_t* T0, int t, int nthreads) {
  for (int i = t; i < 2048; i += nthreads) {
    const int x = i >> 3, m = i & 7;
    const uint32_t t0 = __ldg(T0 + x), t2 = __byte_perm(t0, t0, 0x1032u);
    reinterpret_cast<uint4*>(tab + 256 * x)[m] = make_uint4(t0, t0, t0, t0);
    reinterpret_cast<uint4*>(tab + 256 * x + 128)[m] = make_uint4(t2, t2, t2, t2);
  }
}
__device__ __forceinline__ void aes128_encrypt_pair(uint32_t (&s)[4], const uint32_t* rk, PairLanes lc) {
  auto r8 = [](uint32_t x) { return __byte_perm(x, x, 0x2103u); };
  uint32_t s0 = s[0] ^ rk[0], s1 = s[1] ^ rk[1], s2 = s[2] ^ rk[2], s3 = s[3] ^ rk[3];
#pragma unroll 1
  for (int r = 1; r < 10; ++r) {
    const uint32_t n0 = tpair<0>(s0, lc.c0) ^ tpair<2>(s2, lc.c2) ^ rk[4 * r] ^ r8(tpair<1>(s1, lc.c0) ^ tpair<3>(s3, lc.c2));
    const uint32_t n1 = tpair<0>(s1, lc.c0) ^ tpair<2>(s3, lc.c2) ^ rk[4 * r + 1] ^ r8(tpair<1>(s2, lc.c0) ^ tpair<3>(s0, lc.c2));
    const uint32_t n2 = tpair<0>(s2, lc.c0) ^ tpair<2>(s0, lc.c2) ^ rk[4 * r + 2] ^ r8(tpair<1>(s3, lc.c0) ^ tpair<3>(s1, lc.c2));
    const uint32_t n3 = tpair<0>(s3, lc.c0) ^ tpair<2>(s1, lc.c2) ^ rk[4 * r + 3] ^ r8(tpair<1>(s0, lc.c0) ^ tpair<3>(s2, lc.c2));
    s0 = n0;
    s1 = n1;
    s2 = n2;
    s3 = n3;
  }
  // output byte r of column c = S[byte r of column c + r]: bytes 0 and 3 from T2, 1 and 2 from T0
  auto last = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    const uint32_t lo = __byte_perm(tpair<0>(a, lc.c2), tpair<1>(b, lc.c0), 0x3250u);
    const uint32_t hi = __byte_perm(tpair<2>(c, lc.c0), tpair<3>(d, lc.c2), 0x7210u);
    return __byte_perm(lo, hi, 0x7610u);
  };
  s[0] = last(s0, s1, s2, s3) ^ rk[40];
  s[1] = last(s1, s2, s3, s0) ^ rk[41];
  s[2] = last(s2, s3, s0, s1) ^ rk[42];
  s[3] = last(s3, s0, s1, s2) ^ rk[43];
}

// aes128_encrypt on M independent blocks, their rounds interleaved (the same four shared
// T-tables): a thread with M blocks overlaps their table-lookup latencies.
template <int M>
__device__ __forceinline__ void aes128_encrypt_n(uint32_t (&s)[M][4], const uint32_t* rk, const uint32_t* T) {
  const char* Tc = reinterpret_cast<const char*>(T);
  auto t0 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + ((w << 2) & 0x3fcu)); };
  auto t1 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + 1024 + ((w >> 6) & 0x3fcu)); };
  auto t2 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + 2048 + ((w >> 14) & 0x3fcu)); };
  auto t3 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tc + 3072 + ((w >> 22) & 0x3fcu)); };
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int c = 0; c < 4; ++c) s[m][c] ^= rk[c];
#pragma unroll 1
  for (int r = 1; r < 10; ++r) {
    const uint32_t k0 = rk[4 * r], k1 = rk[4 * r + 1], k2 = rk[4 * r + 2], k3 = rk[4 * r + 3];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const uint32_t s0 = s[m][0], s1 = s[m][1], s2 = s[m][2], s3 = s[m][3];
      s[m][0] = t0(s0) ^ t1(s1) ^ t2(s2) ^ t3(s3) ^ k0;
      s[m][1] = t0(s1) ^ t1(s2) ^ t2(s3) ^ t3(s0) ^ k1;
      s[m][2] = t0(s2) ^ t1(s3) ^ t2(s0) ^ t3(s1) ^ k2;
      s[m][3] = t0(s3) ^ t1(s0) ^ t2(s1) ^ t3(s2) ^ k3;
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint32_t s0 = s[m][0], s1 = s[m][1], s2 = s[m][2], s3 = s[m][3];
    s[m][0] = (__byte_perm(t0(s0), 0u, 0x4441u) | __byte_perm(t0(s1 >> 8), 0u, 0x4414u) |
               __byte_perm(t0(s2 >> 16), 0u, 0x4144u) | __byte_perm(t0(s3 >> 24), 0u, 0x1444u)) ^ rk[40];
    s[m][1] = (__byte_perm(t0(s1), 0u, 0x4441u) | __byte_perm(t0(s2 >> 8), 0u, 0x4414u) |
               __byte_perm(t0(s3 >> 16), 0u, 0x4144u) | __byte_perm(t0(s0 >> 24), 0u, 0x1444u)) ^ rk[41];
    s[m][2] = (__byte_perm(t0(s2), 0u, 0x4441u) | __byte_perm(t0(s3 >> 8), 0u, 0x4414u) |
               __byte_perm(t0(s0 >> 16), 0u, 0x4144u) | __byte_perm(t0(s1 >> 24), 0u, 0x1444u)) ^ rk[42];
    s[m][3] = (__byte_perm(t0(s3), 0u, 0x4441u) | __byte_perm(t0(s0 >> 8), 0u, 0x4414u) |
               __byte_perm(t0(s1 >> 16), 0u, 0x4144u) | __byte_perm(t0(s2 >> 24), 0u, 0x1444u)) ^ rk[43];
  }
}

// Counter block IV + n (128-bit big-endian addition) as four state columns.
// iv_hi / iv_lo: the IV's bytes 0..7 / 8..15 read as big-endian integers.
__device__ __forceinline__ void ctr_block(uint64_t iv_hi, uint64_t iv_lo, uint64_t n,
                                          uint32_t (&s)[4]) {
  const uint64_t lo = iv_lo + n;
  const uint64_t hi = iv_hi + (lo < n ? 1ull : 0ull);
  s[0] = __byte_perm((uint32_t)(hi >> 32), 0u, 0x0123);
  s[1] = __byte_perm((uint32_t)hi, 0u, 0x0123);
  s[2] = __byte_perm((uint32_t)(lo >> 32), 0u, 0x0123);
  s[3] = __byte_perm((uint32_t)lo, 0u, 0x0123);
}

// ------------------------------------------------------------------------------------------
// Exact decision for values near a rounding boundary.
//
// With c(m) = cos(m pi/16): 8 b_u(y) b_v(x) = c(a-b) + c(a+b), a = 4 if u == 0 else
// (2y+1)u, b = 4 if v == 0 else (2x+1)v.  So 8 F[u][v] of an integer block, and 8 p[y][x] of
// an integer coefficient block, are N_0 + sum_{j=1..7} N_j c(j) with integers N_j, and the
// side of a half-integer h is the sign of (N_0 - 8h) + sum N_j c(j).

// cos(j pi/16), j = 1..7, to 256 fractional bits (each translation unit holds its own copy)
static __constant__ uint32_t c_cos_limbs[7][8] = FDS_COS_LIMBS_INIT;

// fold c(m) to +-c(j): accumulate `val` into coordinate j of acc (c(8) = 0 is dropped)
__device__ __forceinline__ void add_cos_term(int (&acc)[9], int m, int val) {
  m &= 31;
  if (m > 16) m = 32 - m;
  if (m > 8)
    acc[16 - m] -= val;
  else
    acc[m] += val;
}

// Sign of a0 + sum_{j=1..7} n[j] c(j), evaluated with c(j) to 256 fractional bits.
// A nonzero value of this form has modulus >= 1 / (2 (2|a0| + 2 sum|n|)^7) (2 c(j) are
// algebraic integers, the field has degree 8, every conjugate is at most 2|a0| + 2 sum|n|),
// far above the evaluation error for |a0|, sum|n| < 2^26.  Returns +1 / -1, 0 for an exact
// zero; *fail is set if the fixed-point value lands inside its error bound although the
// irrational part is nonzero (impossible by the bound above).
__device__ inline int exact_sign(int a0, const int (&n)[9], bool* fail) {
  int any = 0;
  long long err = 0;
#pragma unroll
  for (int j = 1; j < 8; ++j) {
    any |= n[j];
    err += 2ll * (n[j] < 0 ? -(long long)n[j] : (long long)n[j]);
  }
  if (!any) return (a0 > 0) - (a0 < 0);
  uint32_t L[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) L[i] = 0;
  long long top = a0;
  for (int j = 1; j < 8; ++j) {
    const long long nj = n[j];
    long long carry = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const long long t = (long long)L[i] + nj * (long long)c_cos_limbs[j - 1][i] + carry;
      L[i] = (uint32_t)t;
      carry = t >> 32;
    }
    top += carry;
  }
  // D = top * 2^256 + sum L[i] 2^(32 i), |D - value * 2^256| <= err (< 2^32)
  if (top > 0) return 1;
  if (top < -1) return -1;
  uint32_t mid = 0;
  if (top == 0) {
#pragma unroll
    for (int i = 1; i < 8; ++i) mid |= L[i];
    if (mid || (long long)L[0] > err) return 1;
  } else {  // top == -1: D = L - 2^256
    uint32_t all = 0xffffffffu;
#pragma unroll
    for (int i = 1; i < 8; ++i) all &= L[i];
    if (all != 0xffffffffu || (long long)(0xffffffffu - L[0]) + 1 > err) return -1;
  }
  *fail = true;
  return 1;
}

// round(c(j) 2^62), j = 1..7
static __constant__ long long c_cos_q62[7] = FDS_COS_Q62_INIT;

// Round half away from zero, exactly, of the value V with 8V = n[0] + sum_{j=1..7} n[j] c(j).
// First in 64-bit fixed point (error <= sum|n[j]| units of 2^-62 of 8V), which decides unless
// 8V is that close to an odd multiple of 4 (a rounding boundary); then exact_sign decides.
// *escalated counts the exact_sign calls with a nonzero irrational part.
__device__ inline int exact_round(const int (&n)[9], int* escalated, bool* fail) {
  __int128 d = (__int128)n[0] << 62;
  long long err = 0;
#pragma unroll
  for (int j = 1; j < 8; ++j) {
    d += (__int128)n[j] * (__int128)c_cos_q62[j - 1];
    err += n[j] < 0 ? -(long long)n[j] : (long long)n[j];
  }
  // X / 2^65 = V + 1/2; floor of it is the answer away from the boundaries
  const __int128 X = d + ((__int128)4 << 62);
  const long long q = (long long)(X >> 65);
  const __int128 rem = X - ((__int128)q << 65);                 // in [0, 2^65)
  if (rem > (__int128)err && rem < ((__int128)1 << 65) - (__int128)err) return (int)q;
  const int upper = rem <= (__int128)err ? (int)q : (int)q + 1;  // boundary at V = upper - 1/2
  if (err) ++*escalated;
  const int sgn = exact_sign(n[0] - 8 * upper + 4, n, fail);
  return sgn > 0 ? upper : (sgn < 0 ? upper - 1 : (upper >= 1 ? upper : upper - 1));
}

// d = c + sum of the four products of unsigned bytes of a with signed bytes of b
__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// d = c + a.lo16 * b.byte0 + a.hi16 * b.byte1 (lo) or ... b.byte2, b.byte3 (hi), all signed
__device__ __forceinline__ int dp2a_lo(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_hi(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.hi.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

}  // namespace fds
