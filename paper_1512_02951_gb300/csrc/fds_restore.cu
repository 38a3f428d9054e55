// Fused restore kernel (defragmentation, Sect. 3.2, Fig. 3; inverse of Sect. 6.3.1): CTR
// decryption of the confidential fragment, merge with the public fragment by zigzag
// position, inverse 8x8 DCT, round half away from zero (exact), clamp to [0, 255].
//
// Persistent CTAs over a tile schedule (one image, or every tile of a batch of images in one
// launch); per tile (see fds_tile.cuh for the decomposition):
//   A. the tile's fragments are in shared memory, already decrypted; the next tile's start
//      loading (one bulk copy per fragment range, or cp.async pieces)
//   1. per channel-block: column then row float32 inverse butterflies (the column pass and
//      the rounding on pairs with packed f32x2 instructions, bit-identical per lane), round +
//      clamp, bytes into the interleaved pixel tile; values within the float32 error guard of
//      a half-integer are queued
//   B. 2. queued pixels are re-decided exactly (integer coordinates in Z[cos(pi/16)]) by the
//      last threads while the first ones decrypt the next tile's private range in place
//      (AES-128-CTR)
//   C. 3. the pixel tile goes to global memory: one bulk (TMA engine) store per pixel row when
//      the tile's rows are contiguous and 16-byte aligned, else 8-byte stores.  The pixel tile
//      is double-buffered so the bulk stores overlap the next tile.
//
// Packed storage (PACK = 11 or 8 bits per AC field, Sect. 6.4.3): the tile's part of the two
// packed streams lands in a separate shared-memory area (bulk copies when 16-byte aligned,
// else 8-byte cp.async pieces), its private bytes are decrypted there and both parts are
// unpacked into the int16 staging area, all one tile ahead, before the transform reads it.
//
// Public-image form (PUBIMG; the paper's public fragment as an image, Sect. 6.5.1 Fig. 10):
// the same kernel with the private positions "padded with zeros" -- the private staging
// holds the constant (1024, 0, .., 0) per channel-block (DC 8 x 128: the zero-mean block
// shifted to mid-grey), nothing private is loaded or decrypted.
#include "fds_mma.cuh"

namespace fds {

constexpr int kRCtasPerSm = 2;
constexpr int kSmemCoef = 0;                                 // 2 fragment staging areas
constexpr int kSmemPix = kSmemCoef + 2 * kCoefBytes;         // 2 pixel tiles
constexpr int kSmemQueue = kSmemPix + 2 * kPixBytes;
constexpr int kSmemSlot = kSmemQueue + 4 * kQueueCap;        // 3 tile slots (ring)
constexpr int kSlotBytes = (sizeof(TileSlot) + 15) & ~15;
constexpr int kSmemBar = kSmemSlot + 3 * kSlotBytes;         // 2 mbarriers (staging areas)
constexpr int kSmemMisc = kSmemBar + 16;
constexpr int kSmemBytes = kSmemMisc + 32;
// packed storage: one landing area for a tile's packed public and private parts, 24 (63 w + 11)
// bytes at most (w = 11) plus 16 for aligning the private part
constexpr int kLandBytes = 24 * (63 * 11 + 11) + 32;
constexpr int kSmemLand = kSmemBytes;
constexpr int kSmemBytesPacked = kSmemLand + kLandBytes;
// one image in int16 storage: the lane-replicated AES table (32 KB; conflict-free lookups)
// after the rest (measured: 88.7 -> 86.7 us on 4096 x 4096 at k = 5; the batched form, whose
// tiles mostly carry little keystream, was slower with it, 2.96 -> 3.11 ms on 2000 images)
constexpr int kSmemTrep = kSmemBytes;
constexpr int kSmemBytesRep = kSmemTrep + 4 * kTrepWords;
// tensor-core inverse (TC): after the rest, on a 1024-byte boundary, the A operand (256 rows
// of 64 f16 coefficients: the tile's 192 channel-blocks as two MMA row blocks of 128) and the
// B operand (the inverse basis, three f16 limbs x 64 pixels), an mbarrier and the TMEM address
constexpr int kTcA = 256 * 128;
constexpr int kSmemBytesTc = kSmemBytesRep + 1024 + kTcA + kMmaInvBytes + 16;
constexpr int kTcCols = 2 * 192;                       // accumulator columns: 2 row blocks x 3 limbs x 64
static_assert(kTcCols <= 512, "TMEM columns");
constexpr uint32_t kTcInvIdesc = idesc_f16(192, false);
// guard of the TC inverse, per channel-block with S = sum |q|: S 2^-24 + 2^-22 (the host
// proves, when it builds the limb table, that split remainder plus combining roundings stay
// below S 2^-24, and refuses otherwise; 2^-22 covers the roundings of the guard itself)
constexpr float kTcInvGuardS = 1.0f / 16777216.0f;
constexpr float kTcInvGuard0 = 1.0f / 4194304.0f;

// ---- packed storage: land, decrypt, unpack one tile
template <int W>
__device__ __forceinline__ int land_private_offset(int k) {
  return ((24 * (63 - k) * W) + 15) & ~15;
}
// true if both packed parts of slot sl's tile arrive as one bulk copy each
template <int W>
__device__ __forceinline__ bool packed_bulk(const TileSlot* sl) {
  uint64_t po, vo;
  int pb, vb;
  packed_extent<W>(sl, false, po, pb);
  packed_extent<W>(sl, true, vo, vb);
  return ((reinterpret_cast<uintptr_t>(sl->pub_in + po) | reinterpret_cast<uintptr_t>(sl->priv_in + vo) |
           (uintptr_t)pb | (uintptr_t)vb) & 15) == 0;
}
// the packed parts of slot sl's tile into the landing area (all threads; thread 0 issues the
// bulk copies); the streams are 8-byte aligned, so are the tiles' offsets
template <int W>
__device__ __forceinline__ void load_packed(const TileSlot* sl, uint8_t* land, uint64_t* bar) {
  const int t = threadIdx.x;
  uint64_t po, vo;
  int pb, vb;
  packed_extent<W>(sl, false, po, pb);
  packed_extent<W>(sl, true, vo, vb);
  const uint8_t* psrc = sl->pub_in + po;
  const uint8_t* vsrc = sl->priv_in + vo;
  uint8_t* vdst = land + land_private_offset<W>(sl->k);
  if (packed_bulk<W>(sl)) {
    if (t == 0) {
      mbar_expect_tx(bar, (uint32_t)(pb + vb));
      if (pb) bulk_load(land, psrc, (uint32_t)pb, bar);
      if (vb) bulk_load(vdst, vsrc, (uint32_t)vb, bar);
    }
    return;
  }
  const int p8 = pb >> 3, v8 = vb >> 3;
  for (int i = t; i < p8 + v8; i += kThreads) {
    if (i < p8)
      cp_async8(land + 8 * i, psrc + 8 * i);
    else
      cp_async8(vdst + 8 * (i - p8), vsrc + 8 * (i - p8));
  }
  if (t < (pb & 7)) land[(pb & ~7) + t] = psrc[(pb & ~7) + t];
  if (t < (vb & 7)) vdst[(vb & ~7) + t] = vsrc[(vb & ~7) + t];
  cp_async_commit();
}
template <int W>
__device__ __forceinline__ void wait_packed(const TileSlot* sl, uint64_t* bar, uint32_t& phase, int& lost) {
  if (packed_bulk<W>(sl)) {
    if (!mbar_wait(bar, phase)) ++lost;
    phase ^= 1u;
  } else {
    cp_async_wait_all();
  }
}
// AES-128-CTR over the landed private part (all threads; a barrier must follow)
template <int W>
__device__ __forceinline__ void decrypt_packed(const TileSlot* sl, uint8_t* land, const uint32_t* rk,
                                               const uint32_t* Ts) {
  uint64_t vo;
  int vb;
  packed_extent<W>(sl, true, vo, vb);
  ctr_tile_packed(reinterpret_cast<uint32_t*>(land + land_private_offset<W>(sl->k)), vo, vb, sl, rk, Ts,
                  (int)threadIdx.x);
}
// the landed (decrypted) parts -> int16 staging st, public [cb][63 - k], private [cb][k + 1]
// (all threads): a public thread unpacks 32 fields (W words), a private thread one
// channel-block (11 + k W bits)
template <int W>
__device__ __forceinline__ void unpack_tile(const TileSlot* sl, const uint8_t* land, uint8_t* st) {
  const int t = threadIdx.x;
  const int k = sl->k, nb = sl->nb, npub = 63 - k;
  const int nf = 3 * nb * npub, ngroups = (nf + 31) >> 5;
  const uint32_t* pw = reinterpret_cast<const uint32_t*>(land);
  int16_t* pub16 = reinterpret_cast<int16_t*>(st);
  for (int g = t; g < ngroups; g += kThreads) {
    uint32_t word[W];
#pragma unroll
    for (int j = 0; j < W; ++j) word[j] = pw[W * g + j];
    int v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int b = W * i;
      uint32_t c = word[b >> 5] >> (b & 31);
      if ((b & 31) + W > 32) c |= word[(b >> 5) + 1] << (32 - (b & 31));
      const int mag = (int)(c & ((1u << (W - 1)) - 1u));
      v[i] = (c >> (W - 1)) & 1u ? -mag : mag;
    }
    const int f0 = 32 * g;
    if (f0 + 32 <= nf) {
      uint4* dst = reinterpret_cast<uint4*>(pub16 + f0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t u[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          u[m] = ((uint32_t)v[8 * q + 2 * m] & 0xffffu) | ((uint32_t)v[8 * q + 2 * m + 1] << 16);
        dst[q] = make_uint4(u[0], u[1], u[2], u[3]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (f0 + i < nf) pub16[f0 + i] = (int16_t)v[i];
    }
  }
  if (t < 3 * nb) {
    const uint32_t* vw = reinterpret_cast<const uint32_t*>(land + land_private_offset<W>(k));
    int16_t* dst = reinterpret_cast<int16_t*>(st + kTileCb * 2 * npub) + t * (k + 1);
    int pos = t * (kDcBits + k * W);
    for (int z = 0; z <= k; ++z) {
      const int fw = z == 0 ? kDcBits : W;
      const int sh = pos & 31;
      uint32_t c = vw[pos >> 5] >> sh;
      if (sh + fw > 32) c |= vw[(pos >> 5) + 1] << (32 - sh);
      c &= (1u << fw) - 1u;
      if (z == 0) {
        dst[0] = (int16_t)c;
      } else {
        const int mag = (int)(c & ((1u << (W - 1)) - 1u));
        dst[z] = (int16_t)((c >> (W - 1)) & 1u ? -mag : mag);
      }
      pos += fw;
    }
  }
}

// gather the 64 int16 coefficients of tile channel-block cb in zigzag order, two per word
__device__ __forceinline__ void gather_coefs(const int16_t* pubst, const int16_t* privst, int cb,
                                             int k, uint32_t (&Q)[32]) {
  const uint16_t* pu = reinterpret_cast<const uint16_t*>(pubst) + cb * (63 - k) - (k + 1);
  const uint16_t* pv = reinterpret_cast<const uint16_t*>(privst) + cb * (k + 1);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const uint32_t lo = 2 * i <= k ? pv[2 * i] : pu[2 * i];
    const uint32_t hi = 2 * i + 1 <= k ? pv[2 * i + 1] : pu[2 * i + 1];
    Q[i] = lo | (hi << 16);
  }
}

// cp.async the public and private ranges of slot sl's tile into staging area st
// True if both fragment ranges of the tile are whole 16-byte units (then each arrives as one
// bulk copy completing on an mbarrier; else as 16-byte cp.async pieces)
// PUB_ONLY: the public range alone
template <bool PUB_ONLY = false>
__device__ __forceinline__ bool frag_bulk(const TileSlot* sl) {
  const int k = sl->k, nb = sl->nb;
  return ((nb * 6 * (63 - k)) & 15) == 0 && (PUB_ONLY || ((nb * 6 * (k + 1)) & 15) == 0);
}
// Load the public and private ranges of slot sl's tile into staging area st (all threads call
// it; thread 0 issues the bulk copies)
template <bool PUB_ONLY = false>
__device__ __forceinline__ void load_fragments(const TileSlot* sl, uint8_t* st, uint64_t* bar) {
  const int t = threadIdx.x;
  const int k = sl->k, npub = 63 - k, nb = sl->nb;
  const int pub_bytes = nb * 6 * npub, priv_bytes = PUB_ONLY ? 0 : nb * 6 * (k + 1);
  const uint8_t* psrc = sl->pub_in + (uint64_t)sl->local * kTileBlocks * 6ull * npub;
  const uint8_t* vsrc = sl->priv_in + (uint64_t)sl->local * kTileBlocks * 6ull * (k + 1);
  uint8_t* vdst = st + kTileCb * 2 * npub;
  if (frag_bulk<PUB_ONLY>(sl)) {
    if (t == 0) {
      mbar_expect_tx(bar, (uint32_t)(pub_bytes + priv_bytes));
      if (pub_bytes) bulk_load(st, psrc, (uint32_t)pub_bytes, bar);
      if (priv_bytes) bulk_load(vdst, vsrc, (uint32_t)priv_bytes, bar);
    }
    return;
  }
  const int p16 = pub_bytes >> 4, v16 = priv_bytes >> 4;
  for (int i = t; i < p16 + v16; i += kThreads) {
    if (i < p16)
      cp_async16(st + 16 * i, psrc + 16 * i);
    else
      cp_async16(vdst + 16 * (i - p16), vsrc + 16 * (i - p16));
  }
  for (int j = (p16 << 4) + 2 * t; j < pub_bytes; j += 2 * kThreads)
    *reinterpret_cast<uint16_t*>(st + j) = *reinterpret_cast<const uint16_t*>(psrc + j);
  for (int j = (v16 << 4) + 2 * t; j < priv_bytes; j += 2 * kThreads)
    *reinterpret_cast<uint16_t*>(vdst + j) = *reinterpret_cast<const uint16_t*>(vsrc + j);
  cp_async_commit();
}
// Wait until this thread may read what load_fragments loaded (a barrier must follow);
// phase: the next phase of bar; lost counts bulk loads that did not complete in time
template <bool PUB_ONLY = false>
__device__ __forceinline__ void wait_fragments(const TileSlot* sl, uint64_t* bar, uint32_t& phase, int& lost) {
  if (frag_bulk<PUB_ONLY>(sl)) {
    if (!mbar_wait(bar, phase)) ++lost;
    phase ^= 1u;
  } else {
    cp_async_wait_all();
  }
}

// CTR decryption of the private range of slot sl's tile, in staging area st; REP: Ts is the
// lane-replicated table, else the four T-tables
template <bool REP>
__device__ __forceinline__ void decrypt_fragments(const TileSlot* sl, const uint32_t* rk, uint8_t* st,
                                                  const uint32_t* Ts, bool aes_pair = false) {
  const int k = sl->k;
  const int bytes = sl->nb * 6 * (k + 1);
  const uint64_t first = ((uint64_t)sl->local * kTileBlocks * 6ull * (uint64_t)(k + 1)) >> 4;
  if constexpr (REP)
    ctr_tile_rep(st + kTileCb * 2 * (63 - k), bytes, first, sl, rk, Ts, aes_pair, (int)threadIdx.x);
  else
    ctr_tile(st + kTileCb * 2 * (63 - k), bytes, first, sl, rk, Ts, aes_pair, (int)threadIdx.x);
}

// BATCH: tiles of many images (round keys from the slot); else one image (round keys read
// from the kernel parameters, which AES then takes as constant-bank operands)
// TC: the inverse transform as tcgen05 MMAs (one image, int16 storage; a.tc_b = the inverse
// basis table); a tile holding a coefficient of magnitude 2048 or more takes the float32
// butterflies instead.
template <int K, bool BATCH, bool PUBIMG = false, int PACK = 0, bool TC = false>
__global__ void __launch_bounds__(kThreads, TC ? 1 : kRCtasPerSm) restore_kernel(const __grid_constant__ TileArgs a) {
  static_assert(!TC || (!BATCH && !PUBIMG && PACK == 0), "tensor-core inverse: one image, int16 storage");
  extern __shared__ __align__(128) uint8_t smem[];
  // AES tables: T0 replicated per lane (one image, int16 storage, private fragment decrypted),
  // else the four T-tables
  constexpr bool REP = !BATCH && PACK == 0 && !PUBIMG;
  __shared__ __align__(16) uint32_t T4[REP ? 4 : 1024];
  uint32_t* Ts = REP ? reinterpret_cast<uint32_t*>(smem + kSmemTrep) : T4;
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + kSmemQueue);
  // misc: [0] queue size, [1] queued total, [2] escalations, [3] failures, [4..5] schedule
  int* misc = reinterpret_cast<int*>(smem + kSmemMisc);
  const int t = threadIdx.x;
  const int ntiles = a.images ? a.total_tiles : (a.nblocks + kTileBlocks - 1) / kTileBlocks;
  if ((int)blockIdx.x >= ntiles) return;
  auto slot = [&](int i) { return reinterpret_cast<TileSlot*>(smem + kSmemSlot + i * kSlotBytes); };
  auto stage = [&](int i) { return smem + kSmemCoef + i * kCoefBytes; };

  if constexpr (REP) {
    for (int i = t; i < kTrepWords; i += kThreads) Ts[i] = __ldg(a.T + (i >> 5));
  } else {
    for (int i = t; i < 1024; i += kThreads) Ts[i] = a.T[i];
  }
  if (t < 4) misc[t] = 0;
  if (t == 0) {
    misc[6] = 0;                         // TC: a tensor-core wait gave up
    misc[4] = next_tile(a, 0, blockIdx.x, gridDim.x);
    misc[5] = next_tile(a, 1, blockIdx.x, gridDim.x);
  }
  if (t < kTileBlocks) fill_slot(a, blockIdx.x, slot(0), t);
  __syncthreads();
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  uint32_t phase[2] = {0u, 0u};
  int lost = 0;
  // TC: operands, MMA barrier, TMEM (kTcCols columns rounded up to 512)
  uint8_t* const tcbase = TC ? reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem + kSmemBytesRep) + 1023) &
                                                          ~(uintptr_t)1023)
                             : nullptr;
  uint8_t* const tA = tcbase;
  uint8_t* const tB = TC ? tcbase + kTcA : nullptr;
  uint64_t* const tbar = TC ? reinterpret_cast<uint64_t*>(tcbase + kTcA + kMmaInvBytes) : nullptr;
  uint32_t* const tslot = TC ? reinterpret_cast<uint32_t*>(tcbase + kTcA + kMmaInvBytes + 8) : nullptr;
  if constexpr (TC) {
    for (int i = t; i < kMmaInvBytes / 16; i += kThreads) reinterpret_cast<uint4*>(tB)[i] = a.tc_b[i];
    for (int i = t; i < 64 * 128 / 16; i += kThreads)    // A rows 192..255 (never a channel-block)
      reinterpret_cast<uint4*>(tA + 192 * 128)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (t < 32) tmem_alloc<512>(tslot);
    fence_proxy_async();
  }
  if (t == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
    if constexpr (TC) mbar_init(tbar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (PUBIMG) {   // the private staging of both areas: (1024, 0, .., 0) per channel-block
    const int kk = a.k, np = kTileCb * (kk + 1);
    for (int i = t; i < 2 * np; i += kThreads) {
      const int j = i < np ? i : i - np;
      reinterpret_cast<int16_t*>(stage(i < np ? 0 : 1) + kTileCb * 2 * (63 - kk))[j] =
          (int16_t)(j % (kk + 1) == 0 ? 1024 : 0);
    }
  }
  __syncthreads();
  uint8_t* land = smem + kSmemLand;   // PACK only
  if constexpr (PACK != 0) {
    load_packed<PACK>(slot(0), land, bars);
    wait_packed<PACK>(slot(0), bars, phase[0], lost);
    __syncthreads();
    decrypt_packed<PACK>(slot(0), land, a.rk, Ts);
    __syncthreads();
    unpack_tile<PACK>(slot(0), land, stage(0));
  } else {
    load_fragments<PUBIMG>(slot(0), stage(0), bars);
    wait_fragments<PUBIMG>(slot(0), bars, phase[0], lost);
    __syncthreads();
    if (!PUBIMG && !a.plain_private)
      decrypt_fragments<REP>(slot(0), BATCH ? slot(0)->rk : a.rk, stage(0), Ts, BATCH && a.aes_pair);
  }
  int esc = 0;
  bool fail = false;
  // a fragment load that did not complete in time leaves its tile's pixels unwritten (the
  // failure counter records it): cur_lost for the tile being transformed, lost counts them all
  int cur_lost = lost;
  uint32_t tmem = 0, tphase = 0;
  if constexpr (TC) {
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    tmem = *tslot;
  }
  for (int it = 0;; ++it) {
    const int buf = it & 1;
    const int cur = misc[4 + buf], nxt = misc[4 + (buf ^ 1)];
    if (cur >= ntiles) break;
    const TileSlot* sl = slot(it % 3);
    if (nxt < ntiles && t < kTileBlocks) fill_slot(a, nxt, slot((it + 1) % 3), t);
    uint8_t* pix = smem + kSmemPix + buf * kPixBytes;
    if (t == 0) {
      misc[0] = 0;
      // the stores of two tiles ago have read pix (each tile commits one bulk group)
      asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
    }
    __syncthreads();                                                       // A
    if (t == 0) misc[4 + buf] = nxt < ntiles ? next_tile(a, it + 2, blockIdx.x, gridDim.x) : ntiles;
    if (nxt < ntiles) {
      if constexpr (PACK != 0)
        load_packed<PACK>(slot((it + 1) % 3), land, bars + (buf ^ 1));
      else
        load_fragments<PUBIMG>(slot((it + 1) % 3), stage(buf ^ 1), bars + (buf ^ 1));
    }
    const int k = K >= 0 ? K : sl->k;
    const int npub = 63 - k;
    const int nb = sl->nb;
    const int16_t* pubst = reinterpret_cast<const int16_t*>(stage(buf));
    const int16_t* privst = reinterpret_cast<const int16_t*>(stage(buf) + kTileCb * 2 * npub);
    const int cb = t, b = t / 3, c = t - 3 * (t / 3);
    uint8_t* out = pix + b * 24 + c;
    uint32_t mlo = 0, mhi = 0;
    // one row of restored values: clamp, round, mark the values within the guard of a
    // half-integer, bytes into the interleaved pixel tile
    auto emit_row = [&](int y, const float (&row)[8], float thr) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 pc = make_float2(fminf(fmaxf(row[2 * j], 0.0f), 255.0f), fminf(fmaxf(row[2 * j + 1], 0.0f), 255.0f));
        const float2 yv = add2(pc, make_float2(kMagic, kMagic));
        const float2 r = sub2(pc, add2(yv, make_float2(-kMagic, -kMagic)));
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int x = 2 * j + l;
          if (fabsf(l ? r.y : r.x) > thr) {
            if (8 * y + x < 32)
              mlo |= 1u << (8 * y + x);
            else
              mhi |= 1u << (8 * y + x - 32);
          }
          out[y * kRowBytes + 3 * x] = (uint8_t)__float_as_uint(l ? yv.y : yv.x);
        }
      }
    };
    bool tc_done = false;
    if constexpr (TC) {
      // A row t: the channel-block's 64 coefficients in zigzag order (the K order of the
      // basis table), as f16 -- exact for |q| < 2048; S = sum |q| sizes the guard
      int S = 0;
      bool big = false;
      if (b < nb) {
        const int16_t* pub_cb = pubst + cb * npub;
        const int16_t* priv_cb = privst + cb * (k + 1);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          uint32_t w[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int z0 = 8 * j + 2 * m, z1 = z0 + 1;
            const int q0 = z0 <= k ? priv_cb[z0] : pub_cb[z0 - k - 1];
            const int q1 = z1 <= k ? priv_cb[z1] : pub_cb[z1 - k - 1];
            const int m0 = q0 < 0 ? -q0 : q0, m1 = q1 < 0 ? -q1 : q1;
            S += m0 + m1;
            big |= (m0 | m1) >= 2048;
            const __half2 h = __floats2half2_rn((float)q0, (float)q1);
            w[m] = *reinterpret_cast<const uint32_t*>(&h);
          }
          *reinterpret_cast<uint4*>(tA + sw128_offset(t, j)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      fence_proxy_async();
      if (!__syncthreads_or(big || misc[6] != 0)) {                           // A2
        if (t == 0) {
          tc_fence_after_sync();
          const uint32_t a0 = smem_u32(tA), b0 = smem_u32(tB);
#pragma unroll
          for (int rb = 0; rb < 2; ++rb)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_f16(tmem + 192u * rb, sw128_kmajor_desc(a0 + rb * 128 * 128) + 2 * ks, sw128_kmajor_desc(b0) + 2 * ks,
                      kTcInvIdesc, ks > 0 ? 1u : 0u);
          mma_commit(tbar);
        }
        const bool ok = __all_sync(0xffffffffu, mbar_wait(tbar, tphase));
        tphase ^= 1u;
        tc_fence_after_sync();
        if (!ok) {                               // the tile's pixels stay unwritten; later
          ++cur_lost;                            // tiles take the float32 path
          ++lost;
          if ((t & 31) == 0) misc[6] = 1;
        }
        // this warp's TMEM lanes: row block t / 128, lanes 32 (warp % 4) ..
        const int warp = t >> 5;
        const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (warp >= 4 ? 192u : 0u);
        const float thr = 0.5f - fmaf((float)S, kTcInvGuardS, kTcInvGuard0);
#pragma unroll
        for (int h = 0; h < 4; ++h) {          // pixel rows 2h and 2h + 1
          uint32_t d0[16], d1[16], d2[16];
          tmem_ld16(tl + 16 * h, d0);
          tmem_ld16(tl + 64 + 16 * h, d1);
          tmem_ld16(tl + 128 + 16 * h, d2);
          tmem_ld_wait();
          if (ok && b < nb) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
              float row[8];
#pragma unroll
              for (int x = 0; x < 8; ++x) {
                const int i = 8 * rr + x;
                row[x] = fmaf(fmaf(__uint_as_float(d2[i]), 1.0f / 256.0f, __uint_as_float(d1[i])), 1.0f / 256.0f,
                              __uint_as_float(d0[i])) * (1.0f / 512.0f);
              }
              emit_row(2 * h + rr, row, thr);
            }
          }
        }
        tc_fence_before_sync();
        tc_done = true;
      }
    }
    if (!tc_done && b < nb) {
      const int16_t* pub_cb = pubst + cb * npub;
      const int16_t* priv_cb = privst + cb * (k + 1);
      // coefficients as pairs of adjacent columns: the column pass runs on two columns per
      // packed f32x2 instruction
      float2 G[8][4];
      float l1 = 0.0f;  // sum |F|, exact (integers below 2^24)
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int z0 = zigzag_of(u, 2 * j), z1 = zigzag_of(u, 2 * j + 1);
          const int q0 = z0 <= k ? priv_cb[z0] : pub_cb[z0 - k - 1];
          const int q1 = z1 <= k ? priv_cb[z1] : pub_cb[z1 - k - 1];
          G[u][j] = add2(make_float2(__int_as_float(kMagicBits + q0), __int_as_float(kMagicBits + q1)),
                         make_float2(-kMagic, -kMagic));
          l1 += fabsf(G[u][j].x);
          l1 += fabsf(G[u][j].y);
        }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 col[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) col[u] = G[u][j];
        idct8_2(col);
#pragma unroll
        for (int y = 0; y < 8; ++y) G[y][j] = col[y];
      }
      const float thr = 0.5f - l1 * kGuardInvScale;
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        float row[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          row[2 * j] = G[y][j].x;
          row[2 * j + 1] = G[y][j].y;
        }
        idct8(row);
        emit_row(y, row, thr);
      }
    }
    if (b < nb) {
      uint64_t mask = ((uint64_t)mhi << 32) | mlo;
      while (mask) {
        const int pos = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const int idx = atomicAdd(&misc[0], 1);
        if (idx < kQueueCap) {
          queue[idx] = ((uint32_t)cb << 8) | (uint32_t)pos;
        } else {  // queue full: decide here
          uint32_t Q[32];
          int n[9];
          gather_coefs(pubst, privst, cb, k, Q);
          coords_inv(Q, pos, a.cinv, n);
          const int p = exact_round(n, &esc, &fail);
          out[(pos >> 3) * kRowBytes + 3 * (pos & 7)] = (uint8_t)(p < 0 ? 0 : (p > 255 ? 255 : p));
        }
      }
    }
    const int lost_before_next = lost;
    if (nxt < ntiles) {
      if constexpr (PACK != 0)
        wait_packed<PACK>(slot((it + 1) % 3), bars + (buf ^ 1), phase[buf ^ 1], lost);
      else
        wait_fragments<PUBIMG>(slot((it + 1) % 3), bars + (buf ^ 1), phase[buf ^ 1], lost);
    }
    __syncthreads();                                                       // B
    {
      // queued pixels (from the last thread down) re-decided exactly while the first threads
      // decrypt the next tile's private range
      const int nq = min(misc[0], kQueueCap);
      for (int i = kThreads - 1 - t; i < nq; i += kThreads) {
        const uint32_t e = queue[i];
        const int ecb = (int)(e >> 8), pos = (int)(e & 255);
        const int eb = ecb / 3, ec = ecb - 3 * eb;
        uint32_t Q[32];
        int n[9];
        gather_coefs(pubst, privst, ecb, k, Q);
        coords_inv(Q, pos, a.cinv, n);
        const int p = exact_round(n, &esc, &fail);
        pix[(pos >> 3) * kRowBytes + eb * 24 + 3 * (pos & 7) + ec] = (uint8_t)(p < 0 ? 0 : (p > 255 ? 255 : p));
      }
      if (t == 0) misc[1] += misc[0];
    }
    if constexpr (PACK != 0) {
      if (nxt < ntiles) {
        decrypt_packed<PACK>(slot((it + 1) % 3), land, a.rk, Ts);
        __syncthreads();                                                   // B2
        unpack_tile<PACK>(slot((it + 1) % 3), land, stage(buf ^ 1));
      }
    } else if (!PUBIMG && nxt < ntiles && !a.plain_private) {
      decrypt_fragments<REP>(slot((it + 1) % 3), BATCH ? slot((it + 1) % 3)->rk : a.rk, stage(buf ^ 1), Ts,
                        BATCH && a.aes_pair);
    }
    fence_proxy_async();                                  // pixel writes before the bulk stores
    const bool skip = __syncthreads_or(cur_lost != 0);                     // C
    cur_lost = lost - lost_before_next;                   // the next tile's fragments
    if (skip) {
      if (t == 0) bulk_commit();                 // an empty group keeps one group per tile
    } else {
      // the pixel tile to global memory: one bulk (TMA engine) store per pixel row when the
      // tile's blocks are contiguous and 16-byte aligned in every row, else 8-byte stores
      const uint64_t w3 = (uint64_t)sl->width * 3ull;
      uint8_t* row0 = sl->px_out + sl->blk[0];
      if (sl->px_flags & kPxOut16) {
        if (t == 0) {
#pragma unroll 1
          for (int y = 0; y < 8; ++y) bulk_store(row0 + y * w3, pix + y * kRowBytes, (uint32_t)(nb * 24));
          bulk_commit();
        }
      } else {
        if (t == 0) bulk_commit();               // an empty group keeps one group per tile
        for (int i = t; i < 8 * kTileBlocks * 3; i += kThreads) {
          const int y = i / (kTileBlocks * 3), rem = i - y * (kTileBlocks * 3);
          const int bb = rem / 3, q = rem - 3 * bb;
          if (bb < nb)
            *reinterpret_cast<uint2*>(sl->px_out + sl->blk[bb] + y * w3 + 8 * q) =
                *reinterpret_cast<const uint2*>(pix + y * kRowBytes + bb * 24 + 8 * q);
        }
      }
    }
  }
  if (esc) atomicAdd(&misc[2], esc);
  if (fail || lost) atomicAdd(&misc[3], 1);
  if constexpr (TC) tc_fence_before_sync();
  __syncthreads();
  if constexpr (TC) {
    tc_fence_after_sync();
    if (t < 32) tmem_dealloc<512>(tmem);
  }
  if (t == 0) bulk_wait_all();
  if (t == 0 && a.counters) {
    if (misc[1]) atomicAdd(&a.counters[0], (unsigned long long)misc[1]);
    if (misc[2]) atomicAdd(&a.counters[1], (unsigned long long)misc[2]);
    if (misc[3]) atomicAdd(&a.counters[2], (unsigned long long)misc[3]);
  }
}

template <int K, bool BATCH, bool PUBIMG = false, int PACK = 0, bool TC = false>
static cudaError_t launch_k(const TileArgs& a, cudaStream_t s, int sms, int per_sm) {
  static bool attr[kMaxAttrDevices];
  static int resident[kMaxAttrDevices];
  constexpr int smem = TC ? kSmemBytesTc : (PACK ? kSmemBytesPacked : (BATCH || PUBIMG ? kSmemBytes : kSmemBytesRep));
  cudaError_t e = smem_attr_once(restore_kernel<K, BATCH, PUBIMG, PACK, TC>, smem, attr);
  if (e != cudaSuccess) return e;
  const int ntiles = total_tiles(a);
  const int r = resident_ctas(restore_kernel<K, BATCH, PUBIMG, PACK, TC>, kThreads, smem, resident);
  const int cap = (per_sm >= 1 && per_sm < r ? per_sm : r) * sms;
  const int grid = ntiles < cap ? ntiles : cap;
  if (grid > 0) restore_kernel<K, BATCH, PUBIMG, PACK, TC><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// the tensor-core inverse form (one image, int16 storage; a.tc_b = the inverse basis table),
// one CTA per SM (the operands and TMEM take what a second CTA would need)
cudaError_t launch_restore_tc(const TileArgs& a, cudaStream_t s, int sms) {
  if (a.images || a.k < 0 || a.public_image || a.pack || a.plain_private || !a.tc_b) return cudaErrorInvalidValue;
  if (a.k == 0) return launch_k<0, false, false, 0, true>(a, s, sms, 1);
  if (a.k == 5) return launch_k<5, false, false, 0, true>(a, s, sms, 1);
  return launch_k<-1, false, false, 0, true>(a, s, sms, 1);
}

// k is uniform over the launch when a.k >= 0; a.k < 0 (batches of mixed k) reads k per tile;
// a.public_image (one image) selects the public-image form
cudaError_t launch_restore(const TileArgs& a, cudaStream_t s, int sms, int per_sm) {
  if (a.pack) {   // one image, packed streams in pub_in / priv_in
    if (a.images || a.k < 0 || a.public_image || (a.pack != 11 && a.pack != 8)) return cudaErrorInvalidValue;
    if (a.pack == 11) return a.k == 5 ? launch_k<5, false, false, 11>(a, s, sms, per_sm)
                                      : launch_k<-1, false, false, 11>(a, s, sms, per_sm);
    return a.k == 5 ? launch_k<5, false, false, 8>(a, s, sms, per_sm) : launch_k<-1, false, false, 8>(a, s, sms, per_sm);
  }
  if (a.public_image) {
    if (a.images || a.k < 0) return cudaErrorInvalidValue;
    return a.k == 5 ? launch_k<5, false, true>(a, s, sms, per_sm) : launch_k<-1, false, true>(a, s, sms, per_sm);
  }
  if (a.images) {
    if (a.k == 0) return launch_k<0, true>(a, s, sms, per_sm);
    if (a.k == 5) return launch_k<5, true>(a, s, sms, per_sm);
    return launch_k<-1, true>(a, s, sms, per_sm);
  }
  if (a.k == 0) return launch_k<0, false>(a, s, sms, per_sm);
  if (a.k == 5) return launch_k<5, false>(a, s, sms, per_sm);
  return launch_k<-1, false>(a, s, sms, per_sm);
}

}  // namespace fds
