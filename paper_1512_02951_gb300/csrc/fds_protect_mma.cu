// Warp-specialised tensor-core protect kernel (Sect. 6.3.1, Fig. 6): 8x8 DCT-II of every
// channel-block as tcgen05 MMAs, exact int16 rounding, zigzag fragmentation and
// AES-128-CTR of the confidential fragment, one persistent CTA per SM.
//
// The transform as a matrix product.  For channel c of the 128 pixel blocks of a tile,
// D[128 x 192] = A[128 x 64] B[192 x 64]^T with
//   A[b][8y + x] = p - 128 of pixel (y, x) of block b (f16, exact),
//   B[64 l + z][8y + x] = limb l of s = 2^13 b_u(y) b_v(x), (u, v) the zigzag position z,
//     split as s ~ L0 + L1 2^-11 + L2 2^-22 with integer limbs |L0| <= 1970, |L1|, |L2| <= 1024
//     (exact in f16),
// so accumulator column 64 l + z of lane b is the exact integer sum over the block's 64
// pixels of (p - 128) L_l: every product and partial sum is an integer below 2^24, whatever
// order the tensor core adds them in.  The coefficient is F = D0 2^-13 + (D1 + D2 2^-11) 2^-24.
// The major part D0 2^-13 is exact and is the one rounded to an integer; the residual
// r = F - round(D0 2^-13) is formed in two roundings from the minor limbs, so that |computed
// r - exact r| is a few 2^-25 plus the limb remainder (about 2e-7 in all; the host proves the
// bound when it builds B).  A value with |r| within that guard of 1/2 is re-decided exactly
// from integer coordinates in Z[cos(pi/16)] (Sect. 6.4.3 reading: round half away from zero
// of the exact value); with a guard this small that almost never happens outside true ties.
// The four rational coefficients ((u, v) in {0, 4}^2, B = +-1/8) come out of limb 0 as exact
// integers 8F and are rounded in integer arithmetic.  The columns are in zigzag order, so the
// rounded values leave in fragment order without any permutation.
//
// Warps (one CTA per SM, tiles of 128 consecutive pixel blocks, tile g of the image at
// blockIdx.x + i * gridDim.x):
//   0       control: the tiles' 8 pixel rows into a two-slot ring (bulk copies when the tile
//           lies in one block row and is 16-byte aligned, else cp.async pieces), and, from one
//           elected thread, 4 MMAs (K = 64) per channel into a 2-slot TMEM ring (192 columns
//           each), committed to mbarriers
//   1..8    epilogue, two warps per TMEM lane quadrant, one thread per pixel block (TMEM lane =
//           block): the first rounds zigzag coefficients 0-31 of each channel, the second
//           32-63; both write int16 pairs to the quadrant's staging area in fragment layout
//           (private words XORed with the keystream), and the quadrant's 32 blocks of public
//           and private fragment leave by bulk store
//   9..12   work, one per SM sub-partition, one thread per pixel block: the block's three
//           channels de-interleaved into A (one 16 KB operand per channel) as soon as the
//           previous tile's MMA of the channel has read it, then a quarter of the tile's CTR
//           keystream (AES-128, one thread per 16-byte block, T0 replicated per shared-memory
//           bank so that a warp's table lookups never conflict) into a two-slot ring; a
//           tile's operands and keystream are ready while the epilogue rounds the previous tile
// Near ties are recorded (tile, block, channel, zigzag position, stored value) and decided
// after the CTA's last tile from the image in global memory; a changed value is patched by
// XOR (old ^ new) into the public int16 or, CTR being a stream cipher, the ciphertext.
#include <utility>

#include "fds_aux.h"
#include "fds_mma.cuh"

namespace fds {

constexpr int kPmBlocks = 128;                       // pixel blocks per tile (MMA M)
constexpr int kPmRowBytes = kPmBlocks * 24;          // one pixel row of the tile
constexpr int kPmPixBytes = 8 * kPmRowBytes;         // 24 KB
constexpr int kPmEpiWarps = 8;                       // accumulators -> fragments, two per TMEM quadrant
constexpr int kPmWorkWarps = 4;                      // pixels -> A operands, and the keystream
constexpr int kPmWarps = 1 + kPmEpiWarps + kPmWorkWarps;
constexpr int kPmPixSlots = 2;                       // pixel tiles in flight
constexpr int kPmThreads = 32 * kPmWarps;
constexpr int kPmStageWarp = 32 * 3 * 128;           // one quadrant's staging: 12 KB
constexpr int kPmListCap = 512;                      // recorded near ties per CTA
constexpr int kPmMaxK = 7;                           // largest selection this kernel takes
constexpr int kPmN = 64 * kMmaFwdLimbs;              // accumulator columns per channel
constexpr int kPmTmemCols = 512;
constexpr int kPmAccSlots = kPmTmemCols / kPmN >= 4 ? 4 : 2;   // accumulator slots (a ring)

template <int K>
struct PmSmem {
  static constexpr int kKsTile = 768 * (K + 1);      // keystream bytes of one tile
  static constexpr int kB = 0;                       // B operand, 24 KB
  static constexpr int kA = kB + kMmaFwdBytes;       // A operands, 3 x 16 KB
  static constexpr int kPix = kA + 3 * 16384;        // pixel ring, 2 x 24 KB
  static constexpr int kStage = kPix + kPmPixSlots * kPmPixBytes;
  static constexpr int kKs = kStage + 4 * kPmStageWarp;
  static constexpr int kT = kKs + 2 * kKsTile;      // AES T0 replicated per bank, 32 KB
  static constexpr int kList = kT + 4 * kTrepWords;
  static constexpr int kBar = kList + 8 * kPmListCap;
  static constexpr int kMisc = kBar + 256;
  static constexpr int kBytes = kMisc + 64 + 1024;   // + slack for the 1024-byte alignment
};
static_assert(PmSmem<kPmMaxK>::kBytes <= 227 * 1024, "shared memory");

// mbarriers (index into the barrier array)
enum : int {
  kBarPixFull = 0,     // [3] producer -> work warps (32 arrivals + bytes)
  kBarPixEmpty = 3,    // [3] work warps -> producer (kPmWorkWarps)
  kBarAFull = 6,       // [3] work warps -> MMA (kPmWorkWarps)
  kBarAEmpty = 9,      // [3] MMA commit -> work warps (1)
  kBarAccFull = 12,    // [kPmAccSlots] MMA commit -> epilogue (1)
  kBarAccEmpty = 16,   // [kPmAccSlots] epilogue -> MMA (kPmEpiWarps)
  kBarKsFull = 20,     // [2] work warps -> epilogue (kPmWorkWarps)
  kBarKsEmpty = 22,    // [2] epilogue warps of coefficients 0-31 -> work warps (4)
  kBarStageFree = 24,  // [4] per quadrant: the previous tile's bulk stores have read the staging (1)
  kBarStageFull = 28,  // [4] per quadrant: coefficients 32-63 are in the staging (1)
  kBarCount = 32
};
// misc ints
enum : int { kMiscList = 0, kMiscEsc = 1, kMiscFail = 2, kMiscAbort = 3, kMiscTmem = 8 };   // [0..7] zeroed at start

// zigzag index -> (u, v)
__host__ __device__ constexpr int zz_u(int z) {
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v)
      if (zigzag_of(u, v) == z) return u;
  return -1;
}
__host__ __device__ constexpr int zz_v(int z) {
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v)
      if (zigzag_of(u, v) == z) return v;
  return -1;
}
__host__ __device__ constexpr bool zz_rational(int z) {
  return (zz_u(z) == 0 || zz_u(z) == 4) && (zz_v(z) == 0 || zz_v(z) == 4);
}

// Bytes c, c+3, c+6, c+9 of the 12 bytes w0..w2 (pixels x = 0..3 of channel c) as one word.
template <int C>
__device__ __forceinline__ uint32_t gather4(uint32_t w0, uint32_t w1, uint32_t w2) {
  constexpr int p0 = C, p1 = C + 3, p2 = C + 6, p3 = C + 9;
  // first permute: the bytes below 8 from (w0, w1), at their final places
  constexpr uint32_t s1 = (uint32_t)(p0 < 8 ? p0 : 0) | ((uint32_t)(p1 < 8 ? p1 : 0) << 4) |
                          ((uint32_t)(p2 < 8 ? p2 : 0) << 8) | ((uint32_t)(p3 < 8 ? p3 : 0) << 12);
  // second permute: keep them, take the others from w2 (index 4 + byte)
  constexpr uint32_t s2 = (uint32_t)(p0 < 8 ? 0 : 4 + p0 - 8) | ((uint32_t)(p1 < 8 ? 1 : 4 + p1 - 8) << 4) |
                          ((uint32_t)(p2 < 8 ? 2 : 4 + p2 - 8) << 8) | ((uint32_t)(p3 < 8 ? 3 : 4 + p3 - 8) << 12);
  return __byte_perm(__byte_perm(w0, w1, s1), w2, s2);
}

// four pixel bytes -> two words of f16 pairs (p - 128), exact
__device__ __forceinline__ void bytes_to_f16x2(uint32_t g, uint32_t& h0, uint32_t& h1) {
  const uint32_t a = __byte_perm(g, 0x64646464u, 0x4140u);   // (1024 + p0, 1024 + p1) as f16
  const uint32_t b = __byte_perm(g, 0x64646464u, 0x4342u);
  const __half2 off = __halves2half2(__ushort_as_half(0x6480u), __ushort_as_half(0x6480u));   // 1152
  const __half2 ra = __hsub2(*reinterpret_cast<const __half2*>(&a), off);
  const __half2 rb = __hsub2(*reinterpret_cast<const __half2*>(&b), off);
  h0 = *reinterpret_cast<const uint32_t*>(&ra);
  h1 = *reinterpret_cast<const uint32_t*>(&rb);
}

struct PmArgs {
  const uint8_t* pixels;
  int16_t* pub_out;
  uint8_t* priv_out;
  float* dbg;                    // DEBUG: pre-rounding coefficients [cb][8][8]
  const uint32_t* T;             // AES T-tables (device)
  const uint32_t* cfwd;          // exact-coordinate tables (device)
  const uint4* bop;              // B operand image, 16 KB (device)
  unsigned long long* counters;  // 3 counters (device)
  int32_t width, nblocks, ntiles;
  float guard;                   // proven bound on |computed F - exact F| (any value)
  float guard_rem;               // the part of it that does not scale with |F|
  uint64_t iv_hi, iv_lo;
  uint32_t rk[44];
};

// One coefficient Z from its limb accumulators d0, d1, d2: the bits of F + 1.5 2^23 (their
// low 16 bits are the int16 result), the residual r = F - round(F) (0 for the rational
// positions, rounded exactly in integer arithmetic) and S = 2^13 F as computed (for the
// per-value guard and the DEBUG export).
template <int Z>
__device__ __forceinline__ uint32_t coef_bits(float d0, float d1, float d2, float& r, float& S) {
  if constexpr (zz_rational(Z)) {
    const int T8 = __float2int_rn(d0 * (1.0f / 1024.0f));   // 8F (level-shifted for the DC), exact
    int q;
    if constexpr (Z == 0) {
      q = (T8 + 8192 + 4) >> 3;
      S = (float)(T8 + 8192) * 1024.0f;
    } else {
      q = (T8 + 4 - (T8 < 0 ? 1 : 0)) >> 3;
      S = (float)T8 * 1024.0f;
    }
    r = 0.0f;
    return (uint32_t)q;
  } else {
    const float t = kMmaFwdLimbs == 3 ? fmaf(d2, 1.0f / 2048.0f, d1) : d1;   // D1 + D2 2^-11
    S = fmaf(t, 1.0f / 2048.0f, d0);                          // 2^13 F
    const float y = fmaf(S, 1.0f / 8192.0f, kMagic);          // round(F)
    r = fmaf(S, 1.0f / 8192.0f, -(y - kMagic));               // F - round(F), exact
    return __float_as_uint(y);
  }
}

// the pair (Z, Z + 1), on packed f32x2 instructions when both are irrational
template <int Z>
__device__ __forceinline__ void coef_pair(float a0, float a1, float a2, float b0, float b1, float b2, uint32_t& qa,
                                          uint32_t& qb, float& ra, float& rb, float& Sa, float& Sb) {
  if constexpr (!zz_rational(Z) && !zz_rational(Z + 1)) {
    const float2 t = kMmaFwdLimbs == 3
                         ? __ffma2_rn(make_float2(a2, b2), make_float2(1.0f / 2048.0f, 1.0f / 2048.0f), make_float2(a1, b1))
                         : make_float2(a1, b1);
    const float2 S = __ffma2_rn(t, make_float2(1.0f / 2048.0f, 1.0f / 2048.0f), make_float2(a0, b0));
    const float2 y = __ffma2_rn(S, make_float2(1.0f / 8192.0f, 1.0f / 8192.0f), make_float2(kMagic, kMagic));
    const float2 ym = __fadd2_rn(y, make_float2(-kMagic, -kMagic));
    const float2 r = __ffma2_rn(S, make_float2(1.0f / 8192.0f, 1.0f / 8192.0f), make_float2(-ym.x, -ym.y));
    qa = __float_as_uint(y.x);
    qb = __float_as_uint(y.y);
    ra = r.x;
    rb = r.y;
    Sa = S.x;
    Sb = S.y;
  } else {
    qa = coef_bits<Z>(a0, a1, a2, ra, Sa);
    qb = coef_bits<Z + 1>(b0, b1, b2, rb, Sb);
  }
}

// The 16 coefficients z = 16 P .. 16 P + 15 of one channel-block from their limb accumulators.
template <int P, int... I>
__device__ __forceinline__ void round_part_seq(const uint32_t (&d)[3][16], uint32_t (&q)[16], float (&r)[16],
                                               float (&F)[16], std::integer_sequence<int, I...>) {
  (coef_pair<16 * P + 2 * I>(__uint_as_float(d[0][2 * I]), __uint_as_float(d[1][2 * I]), __uint_as_float(d[2][2 * I]),
                             __uint_as_float(d[0][2 * I + 1]), __uint_as_float(d[1][2 * I + 1]),
                             __uint_as_float(d[2][2 * I + 1]), q[2 * I], q[2 * I + 1], r[2 * I], r[2 * I + 1],
                             F[2 * I], F[2 * I + 1]),
   ...);
}

// Decide coefficient z of channel c of image block gb exactly, from the image in global memory.
__device__ __forceinline__ int decide_exact(const PmArgs& a, long long gb, int c, int z, int* esc, bool* fail) {
  int n[9];
  const int pos = 8 * zz_u(z) + zz_v(z);
  coords_fwd_global(a.pixels + block_offset(a.width, (int)gb), 3ull * (uint64_t)a.width, c, pos, a.cfwd, n);
  return exact_round(n, esc, fail);
}

// Work warp w (one thread per pixel block 32w + lane of the tile): per tile, the block's 8
// pixel rows from the ring into registers; per channel, as soon as the previous tile's MMA of
// that channel has read its A slot, the block's 64 pixels of the channel as f16 (p - 128) into
// A; then this warp's share of the tile's CTR keystream (16-byte blocks j = 32 ((w + i) mod 4)
// + lane + 128 r, so that the warp with one round more rotates from tile to tile).
template <int K>
__device__ __forceinline__ void pm_work(const PmArgs& a, uint8_t* smem, uint64_t* bar, volatile int* abort, int nt,
                                        const uint32_t* Ts) {
  using Sm = PmSmem<K>;
  constexpr int NB = 48 * (K + 1);            // keystream blocks of a full tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = warp - 1 - kPmEpiWarps;
  const int bl = 32 * w + lane;
  const int G = (int)gridDim.x;
  const uint32_t Tl = smem_u32(Ts) + 4u * lane;   // this lane's copy of T0 (shared-window address)
  for (int i = 0; i < nt; ++i) {
    const int s = i % kPmPixSlots;
    if (!mbar_wait_abort(bar + kBarPixFull + s, (i / kPmPixSlots) & 1, abort)) break;
    const uint8_t* pix = smem + Sm::kPix + s * kPmPixBytes + bl * 24;
    uint32_t px[8][6];
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const uint2* rp = reinterpret_cast<const uint2*>(pix + y * kPmRowBytes);
      const uint2 p01 = rp[0], p23 = rp[1], p45 = rp[2];
      px[y][0] = p01.x, px[y][1] = p01.y, px[y][2] = p23.x, px[y][3] = p23.y, px[y][4] = p45.x, px[y][5] = p45.y;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar + kBarPixEmpty + s);       // the ring slot may be refilled
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (i >= 1 && !mbar_wait_abort(bar + kBarAEmpty + c, (i - 1) & 1, abort)) { ok = false; break; }
      uint8_t* A = smem + Sm::kA + c * 16384;
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        uint32_t lo, hi;
        if (c == 0) {
          lo = gather4<0>(px[y][0], px[y][1], px[y][2]);
          hi = gather4<0>(px[y][3], px[y][4], px[y][5]);
        } else if (c == 1) {
          lo = gather4<1>(px[y][0], px[y][1], px[y][2]);
          hi = gather4<1>(px[y][3], px[y][4], px[y][5]);
        } else {
          lo = gather4<2>(px[y][0], px[y][1], px[y][2]);
          hi = gather4<2>(px[y][3], px[y][4], px[y][5]);
        }
        uint4 v;
        bytes_to_f16x2(lo, v.x, v.y);
        bytes_to_f16x2(hi, v.z, v.w);
        *reinterpret_cast<uint4*>(A + sw128_offset(bl, y)) = v;
      }
      fence_proxy_async();                     // the A rows, for the tensor core
      __syncwarp();
      if (lane == 0) mbar_arrive(bar + kBarAFull + c);
    }
    if (!ok) break;
    if (a.dbg) continue;                       // DEBUG: no keystream
    // ---- keystream of tile i into slot i & 1 (free once the epilogue has used tile i - 2's)
    const int ks = i & 1;
    if (i >= 2 && !mbar_wait_abort(bar + kBarKsEmpty + ks, ((i >> 1) - 1) & 1, abort)) break;
    const uint64_t first = (uint64_t)((int)blockIdx.x + i * G) * (uint64_t)NB;
    uint8_t* kdst = smem + Sm::kKs + ks * Sm::kKsTile;
#pragma unroll 1
    for (int j = 32 * ((w + i) & 3) + lane; j < NB; j += 128) {
      uint32_t st[4];
      ctr_block(a.iv_hi, a.iv_lo, first + (uint64_t)j, st);
      aes128_encrypt_rep(st, a.rk, Tl);
      *reinterpret_cast<uint4*>(kdst + 16 * j) = make_uint4(st[0], st[1], st[2], st[3]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar + kBarKsFull + ks);
  }
}

// Epilogue warp (TMEM lane quadrant q, half H; one thread per pixel block): per tile and
// channel, zigzag coefficients 32H .. 32H + 31 from the accumulators (two passes of 16) to the
// quadrant's staging area, then (half 0) the quadrant's fragments out by bulk store.
template <int K, bool DEBUG, int H>
__device__ __forceinline__ void pm_epilogue(const PmArgs& a, uint8_t* smem, uint64_t* bar, int* misc,
                                            volatile int* abort, uint2* list, uint32_t tmem, int nt) {
  using Sm = PmSmem<K>;
  constexpr int kPubCb = 2 * (63 - K), kPrivCb = 2 * (K + 1);
  static_assert(K < 32, "only half 0 reads the keystream");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;                     // TMEM lane quadrant (the warp's SM sub-partition)
  const int bl = 32 * q + lane;               // block inside the tile
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
  uint8_t* stage = smem + Sm::kStage + q * kPmStageWarp;
  uint8_t* st_pub = stage;                    // 32 blocks x 3 x kPubCb
  uint8_t* st_priv = stage + 32 * 3 * kPubCb; // 32 blocks x 3 x kPrivCb
  const float thr = 0.5f - a.guard;          // fixed worst-case guard
  const float thr_rel = 0.5f - a.guard_rem;  // per-value guard: plus |S| 2^-37
  const int G = (int)gridDim.x;
  int esc = 0;
  bool fail = false;
  int n = 0;
  for (int i = 0; i < nt; ++i) {
    const int s = i & 1;
    const int g = (int)blockIdx.x + i * G;
    const int b0 = g * kPmBlocks, nb = min(kPmBlocks, a.nblocks - b0);
    if (!DEBUG) {
      if (H == 0) {
        if (!mbar_wait_abort(bar + kBarKsFull + s, (i >> 1) & 1, abort)) break;
        if (lane == 0) {
          bulk_wait_read_n<0>();                          // the previous tile's stores have read the staging
          mbar_arrive(bar + kBarStageFree + q);
        }
        __syncwarp();
      } else if (!mbar_wait_abort(bar + kBarStageFree + q, i & 1, abort)) {
        break;
      }
    }
    const uint16_t* ks16 = reinterpret_cast<const uint16_t*>(smem + Sm::kKs + s * Sm::kKsTile);
    bool ok = true;
#pragma unroll 1
    for (int c = 0; c < 3; ++c, ++n) {
      const int slot = n % kPmAccSlots;
      if (!mbar_wait_abort(bar + kBarAccFull + slot, (n / kPmAccSlots) & 1, abort)) { ok = false; break; }
      tc_fence_after_sync();
      const long long gb = (long long)b0 + bl;               // block of the image
      const int cbw = 3 * lane + c;                          // channel-block inside the quadrant
      const int cbt = 3 * bl + c;                            // channel-block inside the tile
      uint16_t* pub16 = reinterpret_cast<uint16_t*>(st_pub + cbw * kPubCb);
      uint16_t* priv16 = reinterpret_cast<uint16_t*>(st_priv + cbw * kPrivCb);
      const uint16_t* kc16 = ks16 + cbt * (K + 1);
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        constexpr int dummy = 0;
        (void)dummy;
        uint32_t d[3][16];
#pragma unroll
        for (int l = 0; l < kMmaFwdLimbs; ++l) tmem_ld16(tl + (uint32_t)(slot * kPmN + 64 * l + 32 * H + 16 * pass), d[l]);
#pragma unroll
        for (int l = kMmaFwdLimbs; l < 3; ++l)
#pragma unroll
          for (int j = 0; j < 16; ++j) d[l][j] = 0u;
        tmem_ld_wait();
        if (pass == 1) {
          tc_fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar + kBarAccEmpty + slot);   // the registers hold the slot now
        }
        uint32_t qv[16];
        float r[16], S[16];
        if (pass == 0)
          round_part_seq<2 * H>(d, qv, r, S, std::make_integer_sequence<int, 8>{});
        else
          round_part_seq<2 * H + 1>(d, qv, r, S, std::make_integer_sequence<int, 8>{});
        if (bl >= nb) continue;
        const int zb = 32 * H + 16 * pass;
        if (DEBUG) {
          float* out = a.dbg + (uint64_t)(3 * gb + c) * 64ull;
#pragma unroll
          for (int i2 = 0; i2 < 16; ++i2) {
            const int z = zb + i2;
            out[8 * zz_u(z) + zz_v(z)] = S[i2] * (1.0f / 8192.0f);
          }
          continue;
        }
#pragma unroll
        for (int i2 = 0; i2 < 16; i2 += 2) {
          const int z = zb + i2;
          if constexpr ((K & 1) == 1) {   // both fragments hold whole words per channel-block
            const uint32_t wv = __byte_perm(qv[i2], qv[i2 + 1], 0x5410u);
            if (z <= K)
              *reinterpret_cast<uint32_t*>(priv16 + z) = wv ^ *reinterpret_cast<const uint32_t*>(kc16 + z);
            else
              *reinterpret_cast<uint32_t*>(pub16 + (z - K - 1)) = wv;
          } else {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int ze = z + e;
              const uint16_t v = (uint16_t)qv[i2 + e];
              if (ze <= K)
                priv16[ze] = v ^ kc16[ze];
              else
                pub16[ze - K - 1] = v;
            }
          }
        }
        // near ties: |r| within the fixed worst-case guard of 1/2 first (cheap, rarely true),
        // then with the value's own bound g_rem + |2^13 F| 2^-37 (the rounding of S is relative)
        bool near = false;
#pragma unroll
        for (int i2 = 0; i2 < 16; ++i2) near |= fabsf(r[i2]) > thr;
        if (near) {   // rare: record the positions (or decide them now if the list is full)
          uint32_t m = 0;
#pragma unroll
          for (int i2 = 0; i2 < 16; ++i2) {
            // S = 2^13 F again (the same operations as in round_part_seq)
            const float t = kMmaFwdLimbs == 3 ? fmaf(__uint_as_float(d[2][i2]), 1.0f / 2048.0f, __uint_as_float(d[1][i2]))
                                              : __uint_as_float(d[1][i2]);
            const float Sv = fmaf(t, 1.0f / 2048.0f, __uint_as_float(d[0][i2]));
            m |= (fmaf(fabsf(Sv), 1.0f / 137438953472.0f, fabsf(r[i2])) > thr_rel ? 1u : 0u) << i2;
          }
          while (m) {
            const int i2 = __ffs(m) - 1;
            m &= m - 1;
            const int z = zb + i2;
            uint16_t* dst = z <= K ? priv16 + z : pub16 + (z - K - 1);
            const uint32_t q0 = (uint32_t)(uint16_t)(*dst ^ (z <= K ? kc16[z] : (uint16_t)0));
            const int idx = atomicAdd(&misc[kMiscList], 1);
            if (idx < kPmListCap) {
              list[idx] = make_uint2((uint32_t)g, (uint32_t)bl | ((uint32_t)c << 7) | ((uint32_t)z << 9) | (q0 << 16));
            } else {
              const int qx = decide_exact(a, gb, c, z, &esc, &fail);
              *dst ^= (uint16_t)(q0 ^ (uint32_t)qx);
            }
          }
        }
      }
    }
    if (!ok) break;
    if (DEBUG) continue;
    if (H == 0) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar + kBarKsEmpty + s);
    }
    fence_proxy_async();
    __syncwarp();
    if (H != 0) {
      if (lane == 0) mbar_arrive(bar + kBarStageFull + q);   // this half is in place
      continue;
    }
    if (!mbar_wait_abort(bar + kBarStageFull + q, i & 1, abort)) break;
    if (lane == 0) {   // the quadrant's 32 blocks of both fragments, one bulk store each
      const int nbw = min(32, max(0, nb - 32 * q));
      const uint64_t cb0 = 3ull * (uint64_t)(b0 + 32 * q);
      const int pb = nbw * 3 * kPubCb, vb = nbw * 3 * kPrivCb;
      uint8_t* pdst = reinterpret_cast<uint8_t*>(a.pub_out) + cb0 * kPubCb;
      uint8_t* vdst = a.priv_out + cb0 * kPrivCb;
      if (pb >> 4) bulk_store(pdst, st_pub, (uint32_t)(pb & ~15));
      if (vb >> 4) bulk_store(vdst, st_priv, (uint32_t)(vb & ~15));
      bulk_commit();
      for (int j = pb & ~15; j < pb; j += 2)
        *reinterpret_cast<uint16_t*>(pdst + j) = *reinterpret_cast<const uint16_t*>(st_pub + j);
      for (int j = vb & ~15; j < vb; j += 2)
        *reinterpret_cast<uint16_t*>(vdst + j) = *reinterpret_cast<const uint16_t*>(st_priv + j);
    }
  }
  if (H == 0 && lane == 0) {
    bulk_wait_all();
    asm volatile("fence.proxy.async.global;\n" ::: "memory");   // bulk writes, then the patches
  }
  if (esc) atomicAdd(&misc[kMiscEsc], esc);
  if (fail) atomicAdd(&misc[kMiscFail], 1);
}

template <int K, bool DEBUG>
__global__ void __launch_bounds__(kPmThreads, 1) protect_mma_kernel(const __grid_constant__ PmArgs a) {
  using Sm = PmSmem<K>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sm::kBar);
  int* misc = reinterpret_cast<int*>(smem + Sm::kMisc);
  volatile int* abort = misc + kMiscAbort;
  uint2* list = reinterpret_cast<uint2*>(smem + Sm::kList);
  uint32_t* Ts = reinterpret_cast<uint32_t*>(smem + Sm::kT);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int G = (int)gridDim.x;
  const int nt = a.ntiles > (int)blockIdx.x ? (a.ntiles - (int)blockIdx.x + G - 1) / G : 0;   // this CTA's tiles
  if (nt == 0) return;
  const uint64_t w3 = 3ull * (uint64_t)a.width;
  const int bxc = a.width >> 3;

  // ---- set-up
  for (int i = t; i < kTrepWords; i += kPmThreads) Ts[i] = __ldg(a.T + (i >> 5));
  for (int i = t; i < kMmaFwdBytes / 16; i += kPmThreads) reinterpret_cast<uint4*>(smem + Sm::kB)[i] = a.bop[i];
  if (t < 8) misc[t] = 0;
  if (t == 0) {
    constexpr uint32_t W = kPmWorkWarps, E = kPmEpiWarps;
    const uint32_t counts[kBarCount] = {32, 32, 32, W, W, W, W, W, W, 1, 1, 1, 1, 1, 1, 1, E, E, E, E,
                                        W, W, 4, 4, 1, 1, 1, 1, 1, 1, 1, 1};
    for (int i = 0; i < kBarCount; ++i) mbar_init_n(bar + i, counts[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc<kPmTmemCols>(reinterpret_cast<uint32_t*>(misc + kMiscTmem));
  fence_proxy_async();                                 // the B operand, for the tensor core
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = static_cast<uint32_t>(misc[kMiscTmem]);
  auto tile_of = [&](int i) { return (int)blockIdx.x + i * G; };

  if (warp == 0) {
    // ================= control: pixel tiles into the ring, MMAs =================
    auto load_tile = [&](int i) {            // issue tile i's pixel rows into its ring slot
      const int s = i % kPmPixSlots;
      const int g = tile_of(i);
      const int b0 = g * kPmBlocks, nb = min(kPmBlocks, a.nblocks - b0);
      uint8_t* pix = smem + Sm::kPix + s * kPmPixBytes;
      const uint8_t* row0 = a.pixels + block_offset(a.width, b0);
      const bool bulk = (b0 % bxc) + nb <= bxc && (w3 & 15) == 0 && ((nb * 24) & 15) == 0 &&
                        (reinterpret_cast<uintptr_t>(row0) & 15) == 0;
      if (bulk) {
        if (lane == 0) {
          mbar_expect_tx(bar + kBarPixFull + s, (uint32_t)(8 * nb * 24));
          for (int y = 0; y < 8; ++y)
            bulk_load(pix + y * kPmRowBytes, row0 + (uint64_t)y * w3, (uint32_t)(nb * 24), bar + kBarPixFull + s);
        } else {
          mbar_arrive(bar + kBarPixFull + s);
        }
      } else {
        for (int p = lane; p < 8 * 3 * nb; p += 32) {
          const int y = p / (3 * nb), r = p - y * 3 * nb, bb = r / 3, q8 = r - 3 * bb;
          cp_async8(pix + y * kPmRowBytes + bb * 24 + 8 * q8,
                    a.pixels + block_offset(a.width, b0 + bb) + (uint64_t)y * w3 + 8 * q8);
        }
        cp_async_arrive(bar + kBarPixFull + s);
      }
    };
    int loaded = 0;
    for (; loaded < nt && loaded < kPmPixSlots; ++loaded) load_tile(loaded);
    const uint32_t idesc = idesc_f16(kPmN, false);
    const uint64_t db = sw128_kmajor_desc(smem_u32(smem + Sm::kB));
    int n = 0;
    bool ok = true;
    for (int i = 0; i < nt && ok; ++i) {
      for (int c = 0; c < 3; ++c, ++n) {
        const int slot = n % kPmAccSlots;
        if (!mbar_wait_abort(bar + kBarAFull + c, i & 1, abort)) { ok = false; break; }
        if (n >= kPmAccSlots && !mbar_wait_abort(bar + kBarAccEmpty + slot, ((n / kPmAccSlots) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        tc_fence_after_sync();
        if (lane == 0) {
          const uint64_t da = sw128_kmajor_desc(smem_u32(smem + Sm::kA + c * 16384));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_f16(tmem + (uint32_t)(slot * kPmN), da + 2 * ks, db + 2 * ks, idesc, ks > 0 ? 1u : 0u);
          mma_commit(bar + kBarAccFull + slot);
          mma_commit(bar + kBarAEmpty + c);
        }
        __syncwarp();
      }
      // tile i's pixels have been read by now (its A operands are complete): refill the slot
      if (ok && loaded < nt) {
        if (!mbar_wait_abort(bar + kBarPixEmpty + (i % kPmPixSlots), (i / kPmPixSlots) & 1, abort)) break;
        load_tile(loaded++);
      }
    }
    // copies still in flight into the ring must land, and the last MMA must have completed,
    // before the CTA can exit
    for (int j = max(0, loaded - kPmPixSlots); j < loaded; ++j)
      mbar_wait_abort(bar + kBarPixFull + (j % kPmPixSlots), (j / kPmPixSlots) & 1, abort);
    if (n > 0) mbar_wait_abort(bar + kBarAccFull + ((n - 1) % kPmAccSlots), ((n - 1) / kPmAccSlots) & 1, abort);
  } else if (warp <= kPmEpiWarps) {
    // ================= epilogue =================
    if (warp <= 4)
      pm_epilogue<K, DEBUG, 0>(a, smem, bar, misc, abort, list, tmem, nt);
    else
      pm_epilogue<K, DEBUG, 1>(a, smem, bar, misc, abort, list, tmem, nt);
  } else {
    // ================= work: A operands and keystream =================
    pm_work<K>(a, smem, bar, abort, nt, Ts);
  }

  // ================= after the tiles: near ties, counters, TMEM =================
  __syncthreads();
  if (!DEBUG) {
    const int nl = min(misc[kMiscList], kPmListCap);
    int esc = 0;
    bool fail = false;
    for (int e = t; e < nl && !*abort; e += kPmThreads) {
      const uint2 en = list[e];
      const int g = (int)en.x, bl = (int)(en.y & 127u), c = (int)((en.y >> 7) & 3u), z = (int)((en.y >> 9) & 63u);
      const uint32_t q0 = en.y >> 16;
      const long long gb = (long long)g * kPmBlocks + bl;
      const int qx = decide_exact(a, gb, c, z, &esc, &fail);
      if ((uint32_t)(qx & 0xffff) != q0) {
        const uint64_t cbg = 3ull * (uint64_t)gb + (uint64_t)c;
        uint16_t* p = z <= K ? reinterpret_cast<uint16_t*>(a.priv_out) + cbg * (uint64_t)(K + 1) + z
                             : reinterpret_cast<uint16_t*>(a.pub_out) + cbg * (uint64_t)(63 - K) + (z - K - 1);
        *p ^= (uint16_t)(q0 ^ (uint32_t)qx);
      }
    }
    if (esc) atomicAdd(&misc[kMiscEsc], esc);
    if (fail) atomicAdd(&misc[kMiscFail], 1);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (t == 0 && a.counters) {
    const int queued = misc[kMiscList];
    if (queued) atomicAdd(&a.counters[0], (unsigned long long)queued);
    if (misc[kMiscEsc]) atomicAdd(&a.counters[1], (unsigned long long)misc[kMiscEsc]);
    if (misc[kMiscFail] || *abort) atomicAdd(&a.counters[2], (unsigned long long)(misc[kMiscFail] + (*abort ? 1 : 0)));
  }
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc<kPmTmemCols>(tmem);
  }
}

template <int K, bool DEBUG>
static cudaError_t pm_launch_k(const PmArgs& a, cudaStream_t s, int sms) {
  static bool attr[kMaxAttrDevices];
  cudaError_t e = smem_attr_once(protect_mma_kernel<K, DEBUG>, PmSmem<K>::kBytes, attr);
  if (e != cudaSuccess) return e;
  const int grid = a.ntiles < sms ? a.ntiles : sms;
  if (grid > 0) protect_mma_kernel<K, DEBUG><<<grid, kPmThreads, PmSmem<K>::kBytes, s>>>(a);
  return cudaGetLastError();
}

// TileArgs of one image -> the tensor-core protect; k must be 0 .. kPmMaxK
cudaError_t launch_protect_mma(const TileArgs& t, const uint4* bop, float guard, float guard_rem, cudaStream_t s,
                               bool debug, int sms) {
  PmArgs a{};
  a.pixels = t.pixels_in;
  a.pub_out = t.pub_out;
  a.priv_out = t.priv_out;
  a.dbg = t.dbg_coefs;
  a.T = t.T;
  a.cfwd = t.cfwd;
  a.bop = bop;
  a.counters = t.counters;
  a.width = t.width;
  a.nblocks = t.nblocks;
  a.ntiles = (t.nblocks + kPmBlocks - 1) / kPmBlocks;
  a.guard = guard;
  a.guard_rem = guard_rem;
  a.iv_hi = t.iv_hi;
  a.iv_lo = t.iv_lo;
  for (int i = 0; i < 44; ++i) a.rk[i] = t.rk[i];
  if (debug) return pm_launch_k<5, true>(a, s, sms);
  switch (t.k) {
    case 0: return pm_launch_k<0, false>(a, s, sms);
    case 5: return pm_launch_k<5, false>(a, s, sms);
    default: return cudaErrorInvalidValue;
  }
}

bool mma_supports_k(int k) { return k == 0 || k == 5; }

}  // namespace fds
