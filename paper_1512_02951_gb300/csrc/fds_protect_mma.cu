// Warp-specialised tensor-core protect kernel (Sect. 6.3.1, Fig. 6): 8x8 DCT-II of every
// channel-block as tcgen05 MMAs, exact int16 rounding, zigzag fragmentation and
// AES-128-CTR of the confidential fragment, one persistent CTA per SM.
//
// The transform as a matrix product.  For channel c of the 128 pixel blocks of a tile,
// D[128 x 128] = A[128 x 64] B[128 x 64]^T with
//   A[b][8y + x] = p - 128 of pixel (y, x) of block b (f16, exact),
//   B[64 l + z][8y + x] = limb l of 2^13 b_u(y) b_v(x), (u, v) the zigzag position z, split
//     as L0 + L1 2^-11 with integer limbs |L0| <= 1970, |L1| <= 1024 (exact in f16),
// so accumulator column 64 l + z of lane b is the exact integer sum over the block's 64
// pixels of (p - 128) L_l: every product and partial sum is an integer below 2^24, whatever
// order the tensor core adds them in.  The coefficient is F = (D0 + D1 2^-11) 2^-13; its
// error (limb remainder + one rounding) is below a bound the host proves when it builds B;
// values within that guard of a half-integer are re-decided exactly from integer
// coordinates in Z[cos(pi/16)] (Sect. 6.4.3 reading: round half away from zero of the exact
// value).  The four rational coefficients ((u, v) in {0, 4}^2, B = +-1/8) come out of limb 0
// as exact integers 8F and are rounded in integer arithmetic.  The columns are in zigzag
// order, so the rounded values leave in fragment order without any permutation.
//
// Warps (one CTA per SM, tiles of 128 consecutive pixel blocks, tile g of the image at
// blockIdx.x + i * gridDim.x):
//   0       producer: the tile's 8 pixel rows into a two-slot ring (bulk copies when the tile
//           lies in one block row and is 16-byte aligned, else cp.async pieces)
//   1       MMA: one elected thread issues 4 MMAs (K = 64) per channel into a 4-slot TMEM
//           ring (128 columns each) and commits them to mbarriers
//   2..9    transform, two warps per TMEM lane quadrant, one thread per pixel block (TMEM
//           lane = block): the first warp of a pair de-interleaves pixel rows 0-3 of the
//           block's three channels into A and rounds zigzag coefficients 0-31, the second rows
//           4-7 and coefficients 32-63; each writes its int16 pairs to the pair's staging area
//           in fragment layout (private words XORed with the keystream), and the pair's 32
//           blocks of public and private fragment leave by bulk store
//   10..13  AES: the CTR keystream of the tiles' private ranges (data-independent, so it is
//           generated ahead into a two-slot ring), one thread per 16-byte keystream block
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
constexpr int kPmTransWarps = 8;
constexpr int kPmAesWarps = 4;
constexpr int kPmWarps = 2 + kPmTransWarps + kPmAesWarps;
constexpr int kPmThreads = 32 * kPmWarps;
constexpr int kPmStageWarp = 32 * 3 * 128;           // one quadrant's staging: 12 KB
constexpr int kPmListCap = 512;                      // recorded near ties per CTA
constexpr int kPmMaxK = 15;                          // largest selection this kernel takes
constexpr int kPmTmemCols = 512;                     // 4 accumulator slots of 128 columns

template <int K>
struct PmSmem {
  static constexpr int kKsTile = 768 * (K + 1);      // keystream bytes of one tile
  static constexpr int kB = 0;                       // B operand, 16 KB
  static constexpr int kA = kB + 16384;              // A operands, 3 x 16 KB
  static constexpr int kPix = kA + 3 * 16384;        // pixel ring, 2 x 24 KB
  static constexpr int kStage = kPix + 2 * kPmPixBytes;
  static constexpr int kKs = kStage + 4 * kPmStageWarp;
  static constexpr int kT = kKs + 2 * kKsTile;
  static constexpr int kList = kT + 4096;
  static constexpr int kBar = kList + 8 * kPmListCap;
  static constexpr int kMisc = kBar + 256;
  static constexpr int kBytes = kMisc + 64 + 1024;   // + slack for the 1024-byte alignment
};
static_assert(PmSmem<kPmMaxK>::kBytes <= 227 * 1024, "shared memory");

// mbarriers (index into the barrier array)
enum : int {
  kBarPixFull = 0,     // [2] producer -> transform (32 arrivals + bytes)
  kBarPixEmpty = 2,    // [2] transform -> producer (8)
  kBarAFull = 4,       // [3] transform -> MMA (8)
  kBarAEmpty = 7,      // [3] MMA commit -> transform (1)
  kBarAccFull = 10,    // [4] MMA commit -> transform (1)
  kBarAccEmpty = 14,   // [4] transform -> MMA (8)
  kBarKsFull = 18,     // [2] AES -> transform (kPmAesWarps)
  kBarKsEmpty = 20,    // [2] transform warps of coefficients 0-31 -> AES (4)
  kBarStageFree = 22,  // [4] per quadrant: the previous tile's bulk stores have read the staging (1)
  kBarStageFull = 26,  // [4] per quadrant: coefficients 32-63 are in the staging (1)
  kBarCount = 30
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
  float guard;                   // proven bound on |computed F - exact F|
  uint64_t iv_hi, iv_lo;
  uint32_t rk[44];
};

// One coefficient Z from its limb accumulators: the bits of F + 1.5 2^23 (their low 16 bits
// are the int16 result), the residual r = F - round(F) (0 for the rational positions, which
// are rounded exactly in integer arithmetic) and (DEBUG) F itself.
template <int Z>
__device__ __forceinline__ uint32_t coef_bits(float d0, float d1, float& r, float& F) {
  if constexpr (zz_rational(Z)) {
    const int T8 = __float2int_rn(d0 * (1.0f / 1024.0f));   // 8F (level-shifted for the DC), exact
    int q;
    if constexpr (Z == 0) {
      q = (T8 + 8192 + 4) >> 3;
      F = (float)(T8 + 8192) * 0.125f;
    } else {
      q = (T8 + 4 - (T8 < 0 ? 1 : 0)) >> 3;
      F = (float)T8 * 0.125f;
    }
    r = 0.0f;
    return (uint32_t)q;
  } else {
    const float t = fmaf(d1, 1.0f / 2048.0f, d0);            // 2^13 F, one rounding
    const float y = fmaf(t, 1.0f / 8192.0f, kMagic);          // round to nearest integer
    r = fmaf(t, 1.0f / 8192.0f, -(y - kMagic));               // F - round(F), exact
    F = t * (1.0f / 8192.0f);
    return __float_as_uint(y);
  }
}

// the pair (Z, Z + 1), on packed f32x2 instructions when both are irrational
template <int Z>
__device__ __forceinline__ void coef_pair(float a0, float a1, float b0, float b1, uint32_t& qa, uint32_t& qb,
                                          float& ra, float& rb, float& Fa, float& Fb) {
  if constexpr (!zz_rational(Z) && !zz_rational(Z + 1)) {
    const float2 t = __ffma2_rn(make_float2(a1, b1), make_float2(1.0f / 2048.0f, 1.0f / 2048.0f), make_float2(a0, b0));
    const float2 y = __ffma2_rn(t, make_float2(1.0f / 8192.0f, 1.0f / 8192.0f), make_float2(kMagic, kMagic));
    const float2 ym = __fadd2_rn(y, make_float2(-kMagic, -kMagic));
    const float2 r = __ffma2_rn(t, make_float2(1.0f / 8192.0f, 1.0f / 8192.0f), make_float2(-ym.x, -ym.y));
    qa = __float_as_uint(y.x);
    qb = __float_as_uint(y.y);
    ra = r.x;
    rb = r.y;
    Fa = t.x * (1.0f / 8192.0f);
    Fb = t.y * (1.0f / 8192.0f);
  } else {
    qa = coef_bits<Z>(a0, a1, ra, Fa);
    qb = coef_bits<Z + 1>(b0, b1, rb, Fb);
  }
}

// The 32 coefficients z = 32 H .. 32 H + 31 of one channel-block from their limb accumulators.
template <int H, int... P>
__device__ __forceinline__ void round_half_seq(const uint32_t (&d0)[32], const uint32_t (&d1)[32], uint32_t (&q)[32],
                                               float (&r)[32], float (&F)[32], std::integer_sequence<int, P...>) {
  (coef_pair<32 * H + 2 * P>(__uint_as_float(d0[2 * P]), __uint_as_float(d1[2 * P]), __uint_as_float(d0[2 * P + 1]),
                             __uint_as_float(d1[2 * P + 1]), q[2 * P], q[2 * P + 1], r[2 * P], r[2 * P + 1], F[2 * P],
                             F[2 * P + 1]),
   ...);
}
template <int H>
__device__ __forceinline__ void round_half(const uint32_t (&d0)[32], const uint32_t (&d1)[32], uint32_t (&q)[32],
                                           float (&r)[32], float (&F)[32]) {
  round_half_seq<H>(d0, d1, q, r, F, std::make_integer_sequence<int, 16>{});
}

// Decide coefficient z of channel c of image block gb exactly, from the image in global memory.
__device__ __forceinline__ int decide_exact(const PmArgs& a, long long gb, int c, int z, int* esc, bool* fail) {
  int n[9];
  const int pos = 8 * zz_u(z) + zz_v(z);
  coords_fwd_global(a.pixels + block_offset(a.width, (int)gb), 3ull * (uint64_t)a.width, c, pos, a.cfwd, n);
  return exact_round(n, esc, fail);
}

// Transform warp (quadrant q, coefficient half H): per tile, pixel rows 4H..4H+3 of its 32
// blocks into the three A operands, then zigzag coefficients 32H..32H+31 of every channel from
// the accumulators to the staging area.
template <int K, bool DEBUG, int H>
__device__ __forceinline__ void pm_transform(const PmArgs& a, uint8_t* smem, uint64_t* bar, int* misc,
                                             volatile int* abort, uint2* list, uint32_t tmem, int nt) {
  using Sm = PmSmem<K>;
  constexpr int kPubCb = 2 * (63 - K), kPrivCb = 2 * (K + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;                     // TMEM lane quadrant (the warp's SM sub-partition)
  const int bl = 32 * q + lane;               // block inside the tile
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
  uint8_t* stage = smem + Sm::kStage + q * kPmStageWarp;
  uint8_t* st_pub = stage;                    // 32 blocks x 3 x kPubCb
  uint8_t* st_priv = stage + 32 * 3 * kPubCb; // 32 blocks x 3 x kPrivCb
  const float thr = 0.5f - a.guard;
  const int G = (int)gridDim.x;
  int esc = 0;
  bool fail = false;
  int n = 0;
  for (int i = 0; i < nt; ++i) {
    const int s = i & 1;
    const int g = (int)blockIdx.x + i * G;
    const int b0 = g * kPmBlocks, nb = min(kPmBlocks, a.nblocks - b0);
    if (!mbar_wait_abort(bar + kBarPixFull + s, (i >> 1) & 1, abort)) break;
    // ---- A operands: pixel rows 4H .. 4H + 3 of the three channels
    {
      const uint8_t* pix = smem + Sm::kPix + s * kPmPixBytes + bl * 24;
      uint32_t w[4][6];
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) {
        const uint2* rp = reinterpret_cast<const uint2*>(pix + (4 * H + yy) * kPmRowBytes);
        const uint2 p01 = rp[0], p23 = rp[1], p45 = rp[2];
        w[yy][0] = p01.x, w[yy][1] = p01.y, w[yy][2] = p23.x, w[yy][3] = p23.y, w[yy][4] = p45.x, w[yy][5] = p45.y;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar + kBarPixEmpty + s);      // the ring slot may be refilled
      bool ok = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (i >= 1 && !mbar_wait_abort(bar + kBarAEmpty + c, (i - 1) & 1, abort)) { ok = false; break; }
        uint8_t* A = smem + Sm::kA + c * 16384;
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) {
          uint32_t lo, hi;
          if (c == 0) {
            lo = gather4<0>(w[yy][0], w[yy][1], w[yy][2]);
            hi = gather4<0>(w[yy][3], w[yy][4], w[yy][5]);
          } else if (c == 1) {
            lo = gather4<1>(w[yy][0], w[yy][1], w[yy][2]);
            hi = gather4<1>(w[yy][3], w[yy][4], w[yy][5]);
          } else {
            lo = gather4<2>(w[yy][0], w[yy][1], w[yy][2]);
            hi = gather4<2>(w[yy][3], w[yy][4], w[yy][5]);
          }
          uint4 v;
          bytes_to_f16x2(lo, v.x, v.y);
          bytes_to_f16x2(hi, v.z, v.w);
          *reinterpret_cast<uint4*>(A + sw128_offset(bl, 4 * H + yy)) = v;
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar + kBarAFull + c);
      }
      if (!ok) break;
    }
    // ---- epilogue: accumulators -> int16 fragments in the staging area
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
      const int slot = n & 3;
      if (!mbar_wait_abort(bar + kBarAccFull + slot, (n >> 2) & 1, abort)) { ok = false; break; }
      tc_fence_after_sync();
      uint32_t d0[32], d1[32];
      tmem_ld32(tl + (uint32_t)(slot * 128 + 32 * H), d0);
      tmem_ld32(tl + (uint32_t)(slot * 128 + 64 + 32 * H), d1);
      tmem_ld_wait();
      tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar + kBarAccEmpty + slot);   // the registers hold the slot now
      uint32_t qv[32];
      float r[32], F[32];
      round_half<H>(d0, d1, qv, r, F);
      if (bl >= nb) continue;
      const long long gb = (long long)b0 + bl;               // block of the image
      if (DEBUG) {
        float* out = a.dbg + (uint64_t)(3 * gb + c) * 64ull;
#pragma unroll
        for (int i2 = 0; i2 < 32; ++i2) {
          const int z = 32 * H + i2;
          out[8 * zz_u(z) + zz_v(z)] = F[i2];
        }
        continue;
      }
      const int cbw = 3 * lane + c;                          // channel-block inside the quadrant
      const int cbt = 3 * bl + c;                            // channel-block inside the tile
      uint16_t* pub16 = reinterpret_cast<uint16_t*>(st_pub + cbw * kPubCb);
      uint16_t* priv16 = reinterpret_cast<uint16_t*>(st_priv + cbw * kPrivCb);
      const uint16_t* kc16 = ks16 + cbt * (K + 1);
#pragma unroll
      for (int i2 = 0; i2 < 32; i2 += 2) {
        const int z = 32 * H + i2;
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
      bool near = false;
#pragma unroll
      for (int i2 = 0; i2 < 32; ++i2) near = near || fabsf(r[i2]) > thr;
      if (near) {   // rare: record the positions (or decide them now if the list is full)
        uint32_t m = 0;
#pragma unroll
        for (int i2 = 0; i2 < 32; ++i2) m |= (fabsf(r[i2]) > thr ? 1u : 0u) << i2;
        while (m) {
          const int i2 = __ffs(m) - 1;
          m &= m - 1;
          const int z = 32 * H + i2;
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
    if (!ok) break;
    if (DEBUG) continue;
    if (H == 0) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar + kBarKsEmpty + s);
    }
    fence_proxy_async();
    __syncwarp();
    if (H == 1) {
      if (lane == 0) mbar_arrive(bar + kBarStageFull + q);   // coefficients 32-63 are in place
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
  constexpr int NB = 48 * (K + 1);                    // keystream blocks of a full tile
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
  for (int i = t; i < 1024; i += kPmThreads) Ts[i] = a.T[i];
  for (int i = t; i < 1024; i += kPmThreads) reinterpret_cast<uint4*>(smem + Sm::kB)[i] = a.bop[i];
  if (t < 8) misc[t] = 0;
  if (t == 0) {
    const uint32_t counts[kBarCount] = {32, 32, 8, 8, 8, 8, 8, 1, 1, 1, 1, 1, 1, 1, 8, 8, 8, 8,
                                        kPmAesWarps, kPmAesWarps, 4, 4, 1, 1, 1, 1, 1, 1, 1, 1};
    for (int i = 0; i < kBarCount; ++i) mbar_init_n(bar + i, counts[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<kPmTmemCols>(reinterpret_cast<uint32_t*>(misc + kMiscTmem));
  fence_proxy_async();                                 // the B operand, for the tensor core
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = static_cast<uint32_t>(misc[kMiscTmem]);
  auto tile_of = [&](int i) { return (int)blockIdx.x + i * G; };

  if (warp == 0) {
    // ================= producer: pixel tiles into the two-slot ring =================
    int i = 0;
    for (; i < nt; ++i) {
      const int s = i & 1;
      if (i >= 2 && !mbar_wait_abort(bar + kBarPixEmpty + s, ((i >> 1) - 1) & 1, abort)) break;
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
    }
    // copies still in flight into the ring must land before the CTA can exit
    for (int j = max(0, i - 2); j < i; ++j) mbar_wait_abort(bar + kBarPixFull + (j & 1), (j >> 1) & 1, abort);
  } else if (warp == 1) {
    // ================= MMA issuer =================
    const uint32_t idesc = idesc_f16(128, false);
    const uint64_t db = sw128_kmajor_desc(smem_u32(smem + Sm::kB));
    int n = 0;
    bool ok = true;
    for (int i = 0; i < nt && ok; ++i) {
      for (int c = 0; c < 3; ++c, ++n) {
        const int slot = n & 3;
        if (!mbar_wait_abort(bar + kBarAFull + c, i & 1, abort)) { ok = false; break; }
        if (n >= 4 && !mbar_wait_abort(bar + kBarAccEmpty + slot, ((n >> 2) - 1) & 1, abort)) { ok = false; break; }
        tc_fence_after_sync();
        if (lane == 0) {
          const uint64_t da = sw128_kmajor_desc(smem_u32(smem + Sm::kA + c * 16384));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_f16(tmem + (uint32_t)(slot * 128), da + 2 * ks, db + 2 * ks, idesc, ks > 0 ? 1u : 0u);
          mma_commit(bar + kBarAccFull + slot);
          mma_commit(bar + kBarAEmpty + c);
        }
        __syncwarp();
      }
    }
    // the last MMA must have completed before TMEM is freed
    if (n > 0) mbar_wait_abort(bar + kBarAccFull + ((n - 1) & 3), ((n - 1) >> 2) & 1, abort);
  } else if (warp < 2 + kPmTransWarps) {
    // ================= transform =================
    if (warp < 6)
      pm_transform<K, DEBUG, 0>(a, smem, bar, misc, abort, list, tmem, nt);
    else
      pm_transform<K, DEBUG, 1>(a, smem, bar, misc, abort, list, tmem, nt);
  } else if (!DEBUG) {
    // ================= AES: keystream of the private ranges, two tiles ahead =================
    const int aw = warp - 2 - kPmTransWarps;
    int arrived = 0, ready = 0;                 // tiles this warp has signalled / may write
    auto make_ready = [&](int upto) {           // slots of tiles < upto are free
      for (; ready < upto; ++ready)
        if (ready >= 2 && !mbar_wait_abort(bar + kBarKsEmpty + (ready & 1), ((ready >> 1) - 1) & 1, abort))
          return false;
      return true;
    };
    // This warp will not touch tiles < upto again: arrive for each of them, tile by tile.  The
    // arrival for tile t waits until tile t - 2 (same slot) was consumed, so that it counts
    // toward tile t's phase of the barrier; it never waits for anything that needs this
    // warp's own arrival for an earlier tile.
    auto signal_upto = [&](int upto) {
      for (; arrived < upto; ++arrived) {
        if (!make_ready(arrived + 1)) return false;
        __syncwarp();
        if (lane == 0) mbar_arrive(bar + kBarKsFull + (arrived & 1));
      }
      return true;
    };
    const long long total = (long long)nt * NB;
    bool ok = true;
    for (long long ch = aw; 32 * ch < total && ok; ch += kPmAesWarps) {
      const long long v0 = 32 * ch;
      const int tlo = (int)(v0 / NB), thi = (int)min((long long)nt - 1, (v0 + 31) / NB);
      if (!signal_upto(tlo) || !make_ready(thi + 1)) { ok = false; break; }
      const long long v = v0 + lane;
      if (v < total) {
        const int ti = (int)(v / NB), j = (int)(v - (long long)ti * NB);
        uint32_t st[4];
        ctr_block(a.iv_hi, a.iv_lo, (uint64_t)tile_of(ti) * NB + (uint64_t)j, st);
        aes128_encrypt(st, a.rk, Ts);
        *reinterpret_cast<uint4*>(smem + Sm::kKs + (ti & 1) * Sm::kKsTile + 16 * j) = make_uint4(st[0], st[1], st[2], st[3]);
      }
    }
    if (ok) signal_upto(nt);
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
  if (warp == 1) {
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
cudaError_t launch_protect_mma(const TileArgs& t, const uint4* bop, float guard, cudaStream_t s, bool debug,
                               int sms) {
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
