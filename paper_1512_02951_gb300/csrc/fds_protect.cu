// Fused protect kernel (Sect. 6.3.1, Fig. 6): 8x8 DCT-II per channel, int16 rounding,
// zigzag fragmentation, AES-128-CTR of the confidential fragment.
//
// Persistent CTAs over a tile schedule (one image, or every tile of a batch of images in one
// launch); per tile (see fds_tile.cuh for the decomposition):
//   A. the tile's pixels (prefetched with cp.async during the previous tile) are in shared
//      memory; the previous tile's fragments leave through bulk (TMA engine) stores and the
//      next tile's pixels start loading
//   1. per channel-block: row then column float32 butterflies (the column pass and the
//      rounding on pairs of columns with packed f32x2 instructions, bit-identical per lane);
//      every coefficient rounded to int16 and written to the public or private staging area
//      at its zigzag position; coefficients within the float32 error guard of a half-integer
//      are recorded (below)
//   C. 2. the public fragment leaves (bulk store) while AES-128-CTR encrypts the private
//      staging area, one thread per 16-byte keystream block
// One CTA per SM holds three independent tile groups of 192 threads (each with its own
// tiles, named barrier and shared-memory area, like three CTAs) and one AES table, T0
// replicated per lane (32 KB; conflict-free lookups), that the groups share: a table per
// group would not fit, and four separate 1 KB T-tables per CTA made the keystream bound by
// bank conflicts (14.9 against 8.2 SM cycles per keystream block measured alone).  Measured on
// 4096 x 4096, k = 5: 78.5 us with four CTAs of 192 threads and the four 1 KB tables, 76.4 us
// with three groups and the shared table, 86.7 us with four groups and T0 in 16 copies (80
// registers: more spills), 78.5 us with two groups.  One staging area per group: the previous
// tile's bulk stores must have read it before the transform writes it again.
//
// Near ties are not decided inside the tile loop (one exact decision there held every thread
// of the CTA at a barrier): each is recorded (tile, channel-block, position, the
// float32-rounded value that was stored; 192 per CTA) and, when the list is half full at the
// start of a tile (int16 storage) and once the CTA's tiles have all left, decided exactly
// (integer coordinates in Z[cos(pi/16)]) from the image in global memory, after the recorded
// tiles' fragments have landed; a changed value is patched into the fragment by XOR with
// (old ^ new), which is right for the public int16 and, CTR being a stream cipher, for the
// private ciphertext alike.  The packed forms patch the field's code difference into the bit
// streams (one thread per CTA: fields share bytes) at the end only.  A full list means the
// value is decided in place, from the tile in shared memory.
//
// Packed storage (Sect. 6.4.3, Table 5; PACK = 11 or 8 bits per AC field): after step 1 the
// staging area is packed in place into the tile's part of the two bit streams (DC unsigned in
// 11 bits, AC sign-magnitude in PACK bits, least significant bit first, channel-blocks in
// stream order), and AES-128-CTR runs over the packed private bytes at their offset in the
// image's private stream.  A full tile holds 192 channel-blocks, a multiple of 8, so every
// tile's part of either stream starts on a byte boundary.
#include "fds_aux.h"
#include "fds_tile.cuh"

namespace fds {

// one group's area, in two parts: the large one (pixel tiles and staging) and the small one
// (near-tie list, tile slots, counters)
constexpr int kSmemPix = 0;                                  // 2 pixel tiles
constexpr int kSmemStage = kSmemPix + 2 * kPixBytes;         // 1 staging area
constexpr int kBigBytes = kSmemStage + kCoefBytes;
constexpr int kSmemQueue = 0;                                // near-tie list
constexpr int kDeferCap = 192;                               // recorded near ties per group
constexpr int kSmemSlot = kSmemQueue + 8 * kDeferCap;        // 3 tile slots (ring)
constexpr int kSlotBytes = (sizeof(TileSlot) + 15) & ~15;
constexpr int kSmemMisc = kSmemSlot + 3 * kSlotBytes;
constexpr int kSmallBytes = (kSmemMisc + 32 + 127) & ~127;
// One image: one CTA per SM of three groups and the AES pair table they share (64 KB at
// shared-window address kTpairWin = 64 KB).  The window is laid out around the table: below
// it the large part of group 0 and the small parts of all groups, above it the large parts
// of groups 1 and 2; the dynamic area must start at or below kPreWin (it starts at 1 KB, after
// the memory the hardware reserves for each CTA) and reach kEndWin.
// Batches: up to four CTAs per SM of one group each, the large part, the small part and the
// four 1 KB T-tables one after the other (a batch's tiles mostly carry little keystream --
// k = 0: 24 blocks a tile).
constexpr int kPreWin = (int)((kTpairWin - kBigBytes - 3 * kSmallBytes) & ~127u);
constexpr int kEndWin = (int)kTpairWin + kTpairBytes + 2 * kBigBytes;
template <bool BATCH>
struct PLayout {
  static constexpr int kGroups = BATCH ? 1 : 3;
  static constexpr int kCtasPerSm = BATCH ? 4 : 1;
  static constexpr bool kSharedT = !BATCH;
  // batches: the group's T-tables after its two parts
  static constexpr int kT = kBigBytes + kSmallBytes;
  static constexpr int kBytes = kSharedT ? kEndWin : kT + 4096;
};
static_assert(kBigBytes % 128 == 0 && kPreWin >= 2048 && kPreWin + kBigBytes + 3 * kSmallBytes <= (int)kTpairWin &&
                  PLayout<false>::kBytes <= 227 * 1024 && PLayout<true>::kBytes <= 227 * 1024,
              "protect shared memory");

// the public / private fragment staged for slot sl (staging area st) to global memory, one
// bulk group each; one thread
__device__ __forceinline__ void store_public(const TileSlot* sl, const uint8_t* st) {
  const int k = sl->k, npub = 63 - k, nb = sl->nb;
  const int pub_bytes = nb * 6 * npub;
  uint8_t* pdst = sl->pub_out + (uint64_t)sl->local * kTileBlocks * 6ull * npub;
  if (pub_bytes >> 4) bulk_store(pdst, st, (uint32_t)(pub_bytes & ~15));
  bulk_commit();
  for (int j = pub_bytes & ~15; j < pub_bytes; j += 2)
    *reinterpret_cast<uint16_t*>(pdst + j) = *reinterpret_cast<const uint16_t*>(st + j);
}
__device__ __forceinline__ void store_private(const TileSlot* sl, const uint8_t* st) {
  const int k = sl->k, npub = 63 - k, nb = sl->nb;
  const int priv_bytes = nb * 6 * (k + 1);
  uint8_t* vdst = sl->priv_out + (uint64_t)sl->local * kTileBlocks * 6ull * (k + 1);
  const uint8_t* vsrc = st + kTileCb * 2 * npub;
  if (priv_bytes >> 4) bulk_store(vdst, vsrc, (uint32_t)(priv_bytes & ~15));
  bulk_commit();
  for (int j = priv_bytes & ~15; j < priv_bytes; j += 2)
    *reinterpret_cast<uint16_t*>(vdst + j) = *reinterpret_cast<const uint16_t*>(vsrc + j);
}

// ---- packed storage ---------------------------------------------------------------------

// field code of AC value v in W bits: sign-magnitude, the magnitude saturated to W - 1 bits
template <int W>
__device__ __forceinline__ uint32_t ac_code(int v) {
  const uint32_t mag_max = (1u << (W - 1)) - 1u;
  uint32_t mag = (uint32_t)(v < 0 ? -v : v);
  if (mag > mag_max) mag = mag_max;
  return v < 0 ? ((1u << (W - 1)) | mag) : mag;
}

// Pack the staged tile in place (all threads; contains barriers, so every thread calls it).
// Public: fields f (stream order, int16 at st + 2 f) in groups of 32; group g fills words
// [W g, W g + W) of the packed public part at st.  Private: word j of the packed private part
// (at the private staging offset) gathers the fields overlapping bits [32 j, 32 j + 32); a
// channel-block takes 11 + k W bits.  Each round reads its inputs into registers, waits at a
// barrier and writes; the words a round writes lie below every input a later round reads
// (a word of 32 bits holds at least 2.9 fields of at most 11 bits, which took 5.8 bytes as
// int16), and the packed public part ends below the private staging offset (W <= 11 < 16).
template <int W>
__device__ __forceinline__ void pack_tile(uint8_t* st, int nb, int k, int t, int bar) {
  const int npub = 63 - k;
  const int nf = 3 * nb * npub;
  const int ngroups = (nf + 31) >> 5;
  const int period = kDcBits + k * W;
  const int pbits = 3 * nb * period;
  const int nwords = (pbits + 31) >> 5;
  const int16_t* pub16 = reinterpret_cast<const int16_t*>(st);
  uint32_t* pubw = reinterpret_cast<uint32_t*>(st);
  uint8_t* pv = st + kTileCb * 2 * npub;
  const int16_t* priv16 = reinterpret_cast<const int16_t*>(pv);
  uint32_t* privw = reinterpret_cast<uint32_t*>(pv);
  const int nrounds = ngroups > nwords ? ngroups : nwords;
  for (int r0 = 0; r0 < nrounds; r0 += kThreads) {
    const int g = r0 + t;
    uint32_t pw[W];
#pragma unroll
    for (int j = 0; j < W; ++j) pw[j] = 0;
    if (g < ngroups) {
      const int f0 = 32 * g;
      int v[32];
      if (f0 + 32 <= nf) {
        const uint4* src = reinterpret_cast<const uint4*>(pub16 + f0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 x = src[q];
          const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            v[8 * q + 2 * m] = (int16_t)(u[m] & 0xffffu);
            v[8 * q + 2 * m + 1] = (int16_t)(u[m] >> 16);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = f0 + i < nf ? pub16[f0 + i] : 0;   // zero padding
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const uint32_t c = ac_code<W>(v[i]);
        const int b = W * i;
        pw[b >> 5] |= c << (b & 31);
        if ((b & 31) + W > 32) pw[(b >> 5) + 1] |= c >> (32 - (b & 31));
      }
    }
    uint32_t vw = 0;
    if (g < nwords) {
      const int bit = 32 * g;
      const int end = bit + 32 < pbits ? bit + 32 : pbits;
      int cb = bit / period;
      const int r = bit - cb * period;
      int z = r < kDcBits ? 0 : 1 + (r - kDcBits) / W;
      int pos = cb * period + (z == 0 ? 0 : kDcBits + (z - 1) * W);
      while (pos < end) {
        const int v = priv16[cb * (k + 1) + z];
        const uint32_t c = z == 0 ? ((uint32_t)v & 0x7ffu) : ac_code<W>(v);
        const int sh = pos - bit;   // in (-11, 32)
        vw |= sh >= 0 ? c << sh : c >> (-sh);
        pos += z == 0 ? kDcBits : W;
        if (++z > k) {
          z = 0;
          ++cb;
        }
      }
    }
    group_sync(bar);
    if (g < ngroups) {
      if constexpr (W == 8) {
        uint4* d = reinterpret_cast<uint4*>(pubw + W * g);
        d[0] = make_uint4(pw[0], pw[1], pw[2], pw[3]);
        d[1] = make_uint4(pw[4], pw[5], pw[6], pw[7]);
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j) pubw[W * g + j] = pw[j];
      }
    }
    if (g < nwords) privw[g] = vw;
  }
}

// the packed public part of slot sl (at st) to global memory (all threads): one bulk store
// when its destination is 16-byte aligned, else 4-byte or byte stores
template <int W>
__device__ __forceinline__ void store_public_packed(const TileSlot* sl, const uint8_t* st, int t) {
  uint64_t off;
  int bytes;
  packed_extent<W>(sl, false, off, bytes);
  uint8_t* dst = sl->pub_out + off;
  const uintptr_t al = reinterpret_cast<uintptr_t>(dst);
  if ((al & 15) == 0) {
    if (t == 0 && (bytes >> 4)) {
      bulk_store(dst, st, (uint32_t)(bytes & ~15));
      bulk_commit();
    }
    if (t < (bytes & 15)) dst[(bytes & ~15) + t] = st[(bytes & ~15) + t];
  } else if ((al & 3) == 0) {
    for (int i = t; i < (bytes >> 2); i += kThreads)
      reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(st)[i];
    if (t < (bytes & 3)) dst[(bytes & ~3) + t] = st[(bytes & ~3) + t];
  } else {
    for (int i = t; i < bytes; i += kThreads) dst[i] = st[i];
  }
}

// the packed (encrypted) private part of slot sl to global memory (all threads); the private
// stream is 16-byte aligned and a tile's offset is a multiple of 8
template <int W>
__device__ __forceinline__ void store_private_packed(const TileSlot* sl, const uint8_t* st, int t) {
  uint64_t off;
  int bytes;
  packed_extent<W>(sl, true, off, bytes);
  uint8_t* dst = sl->priv_out + off;
  const uint8_t* src = st + kTileCb * 2 * (63 - sl->k);
  for (int i = t; i < (bytes >> 2); i += kThreads)
    reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(src)[i];
  if (t < (bytes & 3)) dst[(bytes & ~3) + t] = src[(bytes & ~3) + t];
}

// A recorded near tie: x = the tile, y = channel-block | position << 8 | stored int16 << 16.
// Decide it exactly from the image and patch the fragment in global memory if it changes.
// a patch of the packed streams: XOR bytes p[0], p[1], p[2] with bytes 0, 1, 2 of v
struct BitPatch {
  uint8_t* p;
  uint32_t v;
};

template <bool BATCH, int PACK>
__device__ __forceinline__ void resolve_deferred(const TileArgs& a, uint2 e, int* esc, bool* fail, BitPatch* bp) {
  const int g = (int)e.x;
  const int cb = (int)(e.y & 255u), pos = (int)((e.y >> 8) & 63u);
  const int q0 = (int)(int16_t)(uint16_t)(e.y >> 16);
  int width, k, local;
  const uint8_t* px;
  uint8_t* pub;
  uint8_t* priv;
  if (!BATCH) {
    width = a.width, k = a.k, local = g;
    px = a.pixels_in;
    pub = reinterpret_cast<uint8_t*>(a.pub_out);
    priv = a.priv_out;
  } else {
    int lo = 0, hi = a.n_images;                 // tile_start[lo] <= g < tile_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(a.tile_start + mid) <= g)
        lo = mid;
      else
        hi = mid;
    }
    const BatchImage& im = a.images[lo];
    width = im.width, k = im.k, local = g - __ldg(a.tile_start + lo);
    px = a.pixels_in + im.pixel_offset;
    pub = reinterpret_cast<uint8_t*>(a.pub_out) + im.public_offset;
    priv = a.priv_out + im.private_offset;
  }
  const int b = cb / 3, c = cb - 3 * b;
  int n[9];
  coords_fwd_global(px + block_offset(width, local * kTileBlocks + b), 3ull * (uint64_t)width, c, pos, a.cfwd, n);
  const int q = exact_round(n, esc, fail);
  const int z = zigzag_of(pos >> 3, pos & 7);
  const uint64_t cbg = (uint64_t)local * kTileCb + (uint64_t)cb;    // channel-block of the image
  if constexpr (PACK == 0) {
    if (q == q0) return;
    uint16_t* p = z <= k ? reinterpret_cast<uint16_t*>(priv) + cbg * (uint64_t)(k + 1) + z
                         : reinterpret_cast<uint16_t*>(pub) + cbg * (uint64_t)(63 - k) + (z - k - 1);
    *p ^= (uint16_t)(q0 ^ q);
  } else {   // an AC field of PACK bits (a near tie is never the DC coefficient)
    const uint64_t bit = z <= k ? cbg * (uint64_t)(kDcBits + k * PACK) + kDcBits + (uint64_t)(z - 1) * PACK
                                : (cbg * (uint64_t)(63 - k) + (uint64_t)(z - k - 1)) * PACK;
    bp->p = (z <= k ? priv : pub) + (bit >> 3);   // written for every entry: v = 0, nothing to do
    bp->v = (ac_code<PACK>(q0) ^ ac_code<PACK>(q)) << (bit & 7);
  }
}

// cp.async the pixels of slot sl into pixel tile pix (all threads of the group; t = index)
__device__ __forceinline__ void load_pixels(const TileSlot* sl, uint8_t* pix, int t) {
  const uint64_t w3 = (uint64_t)sl->width * 3ull;
  const int nb = sl->nb;
  if (sl->px_flags & kPxIn16) {              // whole rows of the tile: 16-byte pieces
    constexpr int kPieces = kRowBytes / 16;
    const uint8_t* row0 = sl->px_in + sl->blk[0];
    for (int i = t; i < 8 * kPieces; i += kThreads) {
      const int y = i / kPieces, x = i - y * kPieces;
      cp_async16(pix + y * kRowBytes + 16 * x, row0 + y * w3 + 16 * x);
    }
    cp_async_commit();
    return;
  }
  for (int i = t; i < 8 * kTileBlocks * 3; i += kThreads) {
    const int y = i / (kTileBlocks * 3), rem = i - y * (kTileBlocks * 3);
    const int b = rem / 3, q = rem - 3 * b;
    if (b < nb) cp_async8(pix + y * kRowBytes + b * 24 + 8 * q, sl->px_in + sl->blk[b] + y * w3 + 8 * q);
  }
  cp_async_commit();
}

// column pairs of the packed column pass: (0, 4), (1, 2), (3, 5), (6, 7)
__host__ __device__ constexpr int pair_of(int v) { return (v == 0 || v == 4) ? 0 : (v < 3 ? 1 : ((v == 3 || v == 5) ? 2 : 3)); }
__host__ __device__ constexpr int pair_lane(int v) { return (v == 4 || v == 2 || v == 5 || v == 7) ? 1 : 0; }
__host__ __device__ constexpr int pair_col(int j, int l) {
  return j == 0 ? (l ? 4 : 0) : (j == 1 ? (l ? 2 : 1) : (j == 2 ? (l ? 5 : 3) : (l ? 7 : 6)));
}

// BATCH: tiles of many images (round keys from the slot); else one image (round keys read
// from the kernel parameters, which AES then takes as constant-bank operands).
// PACK: 0 = int16 fragments; 11 or 8 = packed streams (one image)
template <int K, bool DEBUG, bool BATCH, int PACK = 0>
__global__ void __launch_bounds__(kThreads * PLayout<BATCH>::kGroups, PLayout<BATCH>::kCtasPerSm)
    protect_kernel(const __grid_constant__ TileArgs a) {
  using L = PLayout<BATCH>;
  constexpr int kPGroups = L::kGroups;
  extern __shared__ __align__(128) uint8_t smem_cta[];
  // shared-window address of the dynamic area, and this thread's tile group
  const uint32_t win0 = smem_u32(smem_cta);
  const int grp = (int)threadIdx.x / kThreads;
  const int t = (int)threadIdx.x - grp * kThreads;
  uint8_t* gbig;     // the group's pixel tiles and staging area
  uint8_t* gsmall;   // its near-tie list, tile slots and counters
  const uint32_t* Ts = nullptr;   // batches: the group's four T-tables
  if constexpr (L::kSharedT) {
    // the layout needs the dynamic area to start at or below kPreWin; elsewhere (never on
    // sm_103a) the launch records a failure and does nothing
    if (win0 > (uint32_t)kPreWin) {
      if (threadIdx.x == 0 && a.counters) atomicAdd(&a.counters[2], 1ull);
      return;
    }
    fill_pair_table(smem_cta + (kTpairWin - win0), a.T, (int)threadIdx.x, kThreads * kPGroups);
    gbig = smem_cta + ((grp == 0 ? (uint32_t)kPreWin : kTpairWin + kTpairBytes + (grp - 1) * kBigBytes) - win0);
    gsmall = smem_cta + ((uint32_t)(kPreWin + kBigBytes + grp * kSmallBytes) - win0);
  } else {                       // each group's four T-tables
    for (int i = threadIdx.x; i < kPGroups * 1024; i += kThreads * kPGroups)
      reinterpret_cast<uint32_t*>(smem_cta + (i >> 10) * L::kBytes + L::kT)[i & 1023] = a.T[i & 1023];
    gbig = smem_cta + grp * L::kBytes;
    gsmall = gbig + kBigBytes;
    Ts = reinterpret_cast<const uint32_t*>(gbig + L::kT);
  }
  __syncthreads();
  const int ng = a.groups >= 1 && a.groups < kPGroups ? a.groups : kPGroups;
  if (grp >= ng) return;
  const int vb = (int)blockIdx.x * ng + grp, vgrid = (int)gridDim.x * ng;
  const int gbar = 1 + grp;
  uint2* deferred = reinterpret_cast<uint2*>(gsmall + kSmemQueue);   // near ties, after the tile loop
  // misc: [0] queue size, [1] queued total, [2] escalations, [3] failures, [4..5] schedule
  int* misc = reinterpret_cast<int*>(gsmall + kSmemMisc);
  const int ntiles = a.images ? a.total_tiles : (a.nblocks + kTileBlocks - 1) / kTileBlocks;
  if (vb >= ntiles) return;
  auto slot = [&](int i) { return reinterpret_cast<TileSlot*>(gsmall + kSmemSlot + i * kSlotBytes); };

  if (t < 4) misc[t] = 0;
  if (t == 0) {
    misc[4] = next_tile(a, 0, vb, vgrid);
    misc[5] = next_tile(a, 1, vb, vgrid);
  }
  if (t < kTileBlocks) fill_slot(a, vb, slot(0), t);
  group_sync(gbar);
  load_pixels(slot(0), gbig + kSmemPix, t);

  int it = 0;
  bool have_prev = false;
  for (;; ++it) {
    const int buf = it & 1;
    // slots: tile it in it % 3, it + 1 in (it + 1) % 3, the one being stored in (it + 2) % 3
    const int s_cur = it % 3, s_nxt = (it + 1) % 3, s_prev = (it + 2) % 3;
    const int cur = misc[4 + buf], nxt = misc[4 + (buf ^ 1)];
    if (cur >= ntiles) break;
    const TileSlot* sl = slot(s_cur);
    if (nxt < ntiles && t < kTileBlocks) fill_slot(a, nxt, slot(s_nxt), t);
    cp_async_wait_all();
    group_sync(gbar);                                                       // A
    if (t == 0) misc[4 + buf] = nxt < ntiles ? next_tile(a, it + 2, vb, vgrid) : ntiles;
    if constexpr (PACK != 0) {
      if (have_prev) store_private_packed<PACK>(slot(s_prev), gbig + kSmemStage, t);
      if (t == 0) bulk_wait_read_all();      // the staging area may be written again
    } else if (!DEBUG && t == 0 && have_prev) {
      store_private(slot(s_prev), gbig + kSmemStage);   // the public part left before its AES
      bulk_wait_read_all();                  // the staging area may be written again
    }
    group_sync(gbar);                                                       // A'
    if constexpr (PACK == 0 && !DEBUG) {
      // the near-tie list half full: every earlier tile's fragments have been stored (the last
      // private part just above), so the recorded values are decided and patched now
      const int nrec = misc[0];
      if (nrec >= kDeferCap / 2) {
        if (t == 0) {
          bulk_wait_all();
          asm volatile("fence.proxy.async.global;\n" ::: "memory");   // bulk writes, then the patches
        }
        group_sync(gbar);                 // every thread has read misc[0] before arriving here
        if (t == 0) {
          misc[1] += nrec;
          misc[0] = 0;
        }
        int esc = 0;
        bool fail = false;
        for (int i = t; i < min(nrec, kDeferCap); i += kThreads)
          resolve_deferred<BATCH, 0>(a, deferred[i], &esc, &fail, nullptr);
        if (esc) atomicAdd(&misc[2], esc);
        if (fail) atomicAdd(&misc[3], 1);
        group_sync(gbar);
      }
    }

    if (nxt < ntiles) load_pixels(slot(s_nxt), gbig + kSmemPix + (buf ^ 1) * kPixBytes, t);

    const int k = K >= 0 ? K : sl->k;
    const int npub = 63 - k;
    const int nb = sl->nb;
    const uint8_t* tile_px = gbig + kSmemPix + buf * kPixBytes;
    int16_t* pubst = reinterpret_cast<int16_t*>(gbig + kSmemStage);
    int16_t* privst = reinterpret_cast<int16_t*>(gbig + kSmemStage + kTileCb * 2 * npub);
    const int cb = t, b = t / 3, c = t - 3 * (t / 3);
    if (b < nb) {
      // row outputs kept as pairs of columns (0, 4), (1, 2), (3, 5), (6, 7), so that the
      // column pass runs on two columns per packed f32x2 instruction
      float2 P[8][4];
      float V = 0.0f, W = 0.0f;   // error weights of the row passes and of columns 0, 4
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        uint32_t w[6];
        load_row_shifted(tile_px, y, b, c, w);
        float X[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int byte = 3 * x;
          X[x] = __int_as_float(__byte_perm(w[byte >> 2], 0x4B000000u, 0x7440u | (byte & 3)));
        }
        float fr[8];
        V += dct8_row_bytes_w(X, fr);
        P[y][0] = make_float2(fr[0], fr[4]);
        P[y][1] = make_float2(fr[1], fr[2]);
        P[y][2] = make_float2(fr[3], fr[5]);
        P[y][3] = make_float2(fr[6], fr[7]);
      }
      {   // columns 0 and 4 hold unscaled (exact integer) row outputs
        float2 col[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) col[y] = P[y][0];
        W += dct8_rat_w2(col);
#pragma unroll
        for (int u = 0; u < 8; ++u) P[u][0] = col[u];
      }
#pragma unroll
      for (int j = 1; j < 4; ++j) {
        float2 col[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) col[y] = P[y][j];
        dct8_2<false, false>(col);
#pragma unroll
        for (int u = 0; u < 8; ++u) P[u][j] = col[u];
      }
#define F(u, v) (pair_lane(v) ? P[u][pair_of(v)].y : P[u][pair_of(v)].x)
      if (DEBUG) {
        float* out = a.dbg_coefs + ((uint64_t)sl->local * kTileBlocks * 3 + cb) * 64;
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            float val = F(u, v);
            if (u == 0 && v == 0)
              val = (val + 8192.0f) * 0.125f;
            else if ((u == 0 || u == 4) && (v == 0 || v == 4))
              val *= 0.125f;
            out[8 * u + v] = val;
          }
      } else {
        // rounding: the four rational positions exactly in integers; the rest to nearest in
        // float32 (two at a time), residual checked against the guard (near ties marked in a
        // 64-bit mask)
        int16_t* pub_cb = pubst + cb * npub;
        int16_t* priv_cb = privst + cb * (k + 1);
        uint32_t mlo = 0, mhi = 0;
        const float thr = 0.5f - fminf(fmaf(V, kGuardV, fmaf(W, kGuardW, kGuardU)), kGuardFwd);
        auto put = [&](int u, int v, uint32_t q) {
          const int z = zigzag_of(u, v);
          if (z <= k)
            priv_cb[z] = (int16_t)q;
          else
            pub_cb[z - k - 1] = (int16_t)q;
        };
        auto mark = [&](int u, int v) {
          if (8 * u + v < 32)
            mlo |= 1u << (8 * u + v);
          else
            mhi |= 1u << (8 * u + v - 32);
        };
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if ((u == 0 || u == 4) && j == 0) {
#pragma unroll
              for (int l = 0; l < 2; ++l) {
                const int v = pair_col(0, l);
                const int T = __float_as_int(F(u, v) + kMagic) - kMagicBits;  // 8 F, exact
                put(u, v, (uint32_t)((u == 0 && v == 0) ? ((T + 4) >> 3) + 1024 : (T + 4 - (T < 0 ? 1 : 0)) >> 3));
              }
            } else {
              const float2 yv = add2(P[u][j], make_float2(kMagic, kMagic));
              const float2 r = sub2(P[u][j], add2(yv, make_float2(-kMagic, -kMagic)));
              put(u, pair_col(j, 0), __float_as_uint(yv.x));   // low 16 bits: the int16 result
              put(u, pair_col(j, 1), __float_as_uint(yv.y));
              if (fabsf(r.x) > thr) mark(u, pair_col(j, 0));
              if (fabsf(r.y) > thr) mark(u, pair_col(j, 1));
            }
          }
        }
#undef F
        uint64_t mask = ((uint64_t)mhi << 32) | mlo;
        while (mask) {
          const int pos = __ffsll((long long)mask) - 1;
          mask &= mask - 1;
          const int idx = atomicAdd(&misc[0], 1);
          if (idx < kDeferCap) {
            const int z = zigzag_of(pos >> 3, pos & 7);
            const uint32_t q0 = (uint16_t)(z <= k ? priv_cb[z] : pub_cb[z - k - 1]);
            deferred[idx] = make_uint2((uint32_t)cur, (uint32_t)cb | ((uint32_t)pos << 8) | (q0 << 16));
          } else {  // list full: decide here
            int n[9], esc = 0;
            bool fail = false;
            coords_fwd(tile_px, b, c, pos, a.cfwd, n);
            const int q = exact_round(n, &esc, &fail);
            const int z = zigzag_of(pos >> 3, pos & 7);
            if (z <= k)
              priv_cb[z] = (int16_t)q;
            else
              pub_cb[z - k - 1] = (int16_t)q;
            if (esc) atomicAdd(&misc[2], esc);
            if (fail) atomicAdd(&misc[3], 1);
          }
        }
      }
    }
    if (DEBUG) {
      group_sync(gbar);   // publishes the schedule entry written after barrier A
      continue;
    }
    if constexpr (PACK != 0) {
      group_sync(gbar);                                 // every staged coefficient is final
      pack_tile<PACK>(gbig + kSmemStage, nb, k, t, gbar);
    }
    fence_proxy_async();                   // every thread's staging writes, before the bulk store
    group_sync(gbar);                                                       // C
    if constexpr (PACK != 0) {
      store_public_packed<PACK>(sl, gbig + kSmemStage, t);   // it leaves during the AES
      uint64_t off;
      int bytes;
      packed_extent<PACK>(sl, true, off, bytes);
      ctr_tile_packed<L::kSharedT ? kTabPair : 0>(reinterpret_cast<uint32_t*>(privst), off, bytes, sl, a.rk, Ts, t);
    } else {
      if (t == 0) store_public(sl, gbig + kSmemStage);   // final: it leaves during the AES
      if (!a.plain_private)
      {
        const uint64_t first = ((uint64_t)sl->local * kTileBlocks * 6ull * (uint64_t)(k + 1)) >> 4;
        if constexpr (L::kSharedT)
          ctr_tile_pair(reinterpret_cast<uint8_t*>(privst), nb * 6 * (k + 1), first, sl, a.rk, t);
        else
          ctr_tile(reinterpret_cast<uint8_t*>(privst), nb * 6 * (k + 1), first, sl, sl->rk, Ts, a.aes_pair, t);
      }
    }
    fence_proxy_async();
    have_prev = true;
  }
  if (DEBUG) return;
  group_sync(gbar);
  if constexpr (PACK != 0) {
    if (have_prev) store_private_packed<PACK>(slot((it + 2) % 3), gbig + kSmemStage, t);
  }
  if (t == 0) {
    if (PACK == 0 && have_prev) store_private(slot((it + 2) % 3), gbig + kSmemStage);
    bulk_wait_all();
    asm volatile("fence.proxy.async.global;\n" ::: "memory");   // bulk writes, then the patches
  }
  {
    group_sync(gbar);                                   // every fragment of the CTA is in memory
    const int nd = min(misc[0], kDeferCap);
    int esc = 0;
    bool fail = false;
    // packed-stream patches are applied by one thread (fields share bytes; the pixel tiles are
    // free now and hold them); patches never cross into another tile's bytes or CTA
    BitPatch* bp = reinterpret_cast<BitPatch*>(gbig + kSmemPix);
    for (int i = t; i < nd; i += kThreads) resolve_deferred<BATCH, PACK>(a, deferred[i], &esc, &fail, bp + i);
    if constexpr (PACK != 0) {
      group_sync(gbar);
      if (t == 0)
        for (int i = 0; i < nd; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            if ((bp[i].v >> (8 * j)) & 0xffu) bp[i].p[j] ^= (uint8_t)(bp[i].v >> (8 * j));
    }
    if (esc) atomicAdd(&misc[2], esc);
    if (fail) atomicAdd(&misc[3], 1);
    group_sync(gbar);
    if (t == 0) misc[1] += misc[0];
  }
  if (t == 0) {
    if (a.counters) {
      if (misc[1]) atomicAdd(&a.counters[0], (unsigned long long)misc[1]);
      if (misc[2]) atomicAdd(&a.counters[1], (unsigned long long)misc[2]);
      if (misc[3]) atomicAdd(&a.counters[2], (unsigned long long)misc[3]);
    }
  }
}

template <int K, bool DEBUG, bool BATCH, int PACK = 0>
static cudaError_t launch_k(const TileArgs& a, cudaStream_t s, int sms, int per_sm) {
  static bool attr[kMaxAttrDevices];
  using L = PLayout<BATCH>;
  static bool window_ok[kMaxAttrDevices];
  cudaError_t e;
  if constexpr (L::kSharedT) {   // the groups' areas and the pair table at fixed window addresses
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxAttrDevices) return cudaErrorInvalidDevice;
    if (!window_ok[dev]) {
      if ((e = smem_window_start_ok(protect_kernel<K, DEBUG, BATCH, PACK>, (uint32_t)kPreWin)) != cudaSuccess) return e;
      window_ok[dev] = true;
    }
  }
  e = smem_attr_once(protect_kernel<K, DEBUG, BATCH, PACK>, L::kBytes, attr);
  if (e != cudaSuccess) return e;
  const int ntiles = total_tiles(a);
  // per_sm: tile groups working on each SM (one image: groups of the one CTA; batches: CTAs)
  TileArgs b = a;
  const int want = per_sm >= 1 && per_sm < L::kGroups * L::kCtasPerSm ? per_sm : L::kGroups * L::kCtasPerSm;
  b.groups = want < L::kGroups ? want : L::kGroups;
  const int need = (ntiles + b.groups - 1) / b.groups;
  const int cap = sms * (want / b.groups);
  const int grid = need < cap ? need : cap;
  if (grid > 0) protect_kernel<K, DEBUG, BATCH, PACK><<<grid, kThreads * L::kGroups, L::kBytes, s>>>(b);
  return cudaGetLastError();
}

// k is uniform over the launch when a.k >= 0; a.k < 0 (batches of mixed k) reads k per tile;
// a.pack (11 or 8: packed streams) is for one image
cudaError_t launch_protect(const TileArgs& a, cudaStream_t s, bool debug, int sms, int per_sm) {
  if (a.pack) {
    if (debug || a.images || a.k < 0 || (a.pack != 11 && a.pack != 8)) return cudaErrorInvalidValue;
    if (a.pack == 11) return a.k == 5 ? launch_k<5, false, false, 11>(a, s, sms, per_sm)
                                      : launch_k<-1, false, false, 11>(a, s, sms, per_sm);
    return a.k == 5 ? launch_k<5, false, false, 8>(a, s, sms, per_sm)
                    : launch_k<-1, false, false, 8>(a, s, sms, per_sm);
  }
  if (debug) return launch_k<-1, true, false>(a, s, sms, per_sm);
  if (a.images) {
    if (a.k == 0) return launch_k<0, false, true>(a, s, sms, per_sm);
    if (a.k == 5) return launch_k<5, false, true>(a, s, sms, per_sm);
    return launch_k<-1, false, true>(a, s, sms, per_sm);
  }
  if (a.k == 0) return launch_k<0, false, false>(a, s, sms, per_sm);
  if (a.k == 5) return launch_k<5, false, false>(a, s, sms, per_sm);
  return launch_k<-1, false, false>(a, s, sms, per_sm);
}

}  // namespace fds
