// Tile machinery shared by the fused protect and restore kernels.
//
// Work decomposition: a tile is 64 consecutive 8x8 pixel blocks (row-major over an image's
// block grid); one thread per channel-block (cb = 3 * block + channel, 192 threads per CTA).
// A tile's public and private outputs are contiguous, 16-byte aligned byte ranges
// (64 blocks x 3 channels x 2(63-k) or 2(k+1) bytes), so a tile stages them in shared memory
// and moves them with 16-byte (or bulk) copies; the tile's private range is a whole number of
// AES blocks, so CTR needs nothing from neighbouring tiles.
//
// The kernels are persistent: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and prefetches the next tile's input with cp.async while it transforms the current one.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fds_device.cuh"

namespace fds {

constexpr int kTileBlocks = 64;                // pixel blocks per tile
constexpr int kTileCb = 3 * kTileBlocks;       // channel-blocks per tile
constexpr int kThreads = kTileCb;              // one thread per channel-block
constexpr int kRowBytes = kTileBlocks * 24;    // one pixel row of the tile (8 px x 3 ch per block)
constexpr int kPixBytes = 8 * kRowBytes;       // 12 KB
constexpr int kCoefBytes = kTileCb * 128;      // public + private int16 staging (64 per cb)
constexpr int kQueueCap = 256;                 // near-tie entries per tile

// tensor-core form: bytes of the B operand (basis limbs) in shared memory
constexpr int kTcBBytesBf16 = 192 * 128;      // 3 limbs x 64 rows x 64 bf16
constexpr int kTcBBytesTf32 = 2 * 128 * 128;  // 2 limbs x 64 rows x 64 tf32, as two K atoms
// warp-specialised form: FDS_MMA_LIMBS f16 limbs of the basis (2 or 3) x 64 rows x 64 f16
#ifndef FDS_MMA_LIMBS
#define FDS_MMA_LIMBS 3
#endif
constexpr int kMmaFwdLimbs = FDS_MMA_LIMBS;
constexpr int kMmaFwdBytes = kMmaFwdLimbs * 64 * 128;
// tensor-core inverse transform (restore): three f16 limbs x 64 pixel rows x 64 f16 (K in
// zigzag order); coefficients |q| < 2048 go in exactly as f16
constexpr int kMmaInvBytes = 3 * 64 * 128;

// Forward guard.  On level-shifted pixels |p - 128| <= 128 the butterflies are within
// 1.11e-3 of the exact coefficient (first-order bound: every rounded operation and every
// rounded constant, each weighted by the output's sensitivity to it).  2^-9 = 1.95e-3.
constexpr float kGuardFwd = 1.0f / 512.0f;
// Tighter per channel-block forward guard, from the data.  With u = 2^-24, V = sum over the 8
// rows of the row pass's error weight and W = the weights of the column passes of columns 0
// and 4 (exact integer inputs; see pass_weight):
//  - a row pass output is exact (columns 0, 4) or within 2.46 u V_y of exact, and its
//    magnitude is at most 0.4904 V_y;
//  - a column pass over columns 1-3, 5-7 adds at most 0.4904 sum_y 2.46 u V_y for its
//    inputs' errors and 2.95 u sum_y |input| <= 1.45 u V of its own, so |F - exact| <= 2.65 u V;
//  - columns 0 and 4 start from exact integers: |F - exact| <= 0.87 u W (scaled constants).
// G = u (2.7 V + 0.9 W + 1) bounds every coefficient's error (the extra u covers the rounding
// of 0.5 - G and of G itself); min(G, kGuardFwd) is used.
constexpr float kGuardV = 2.7f / 16777216.0f;
constexpr float kGuardW = 0.9f / 16777216.0f;
constexpr float kGuardU = 1.0f / 16777216.0f;
// Inverse guard per channel-block: error <= 2.89 u sum|F| (u = 2^-24); 2^-22 sum|F| is used.
constexpr float kGuardInvScale = 1.0f / 4194304.0f;

// One image of a batch as the kernels read it (device copy of struct fds_image).
struct BatchImage {
  uint64_t pixel_offset, public_offset, private_offset;
  int32_t width, height, k, key_slot;
  uint64_t iv_hi, iv_lo;
};
static_assert(sizeof(BatchImage) == 56 && offsetof(BatchImage, width) == 24 && offsetof(BatchImage, iv_hi) == 40,
              "BatchImage layout");

// Kernel arguments.  Single image: `images` is null and the image fields describe it.
// Batch: the pointers are the batch buffers, images[i] gives each image's offsets, and
// global tile g belongs to the image i with tile_start[i] <= g < tile_start[i + 1].
struct TileArgs {
  const uint8_t* pixels_in;
  uint8_t* pixels_out;
  const int16_t* pub_in;
  int16_t* pub_out;
  const uint8_t* priv_in;
  uint8_t* priv_out;
  float* dbg_coefs;               // protect debug export, or null
  const uint32_t* T;              // AES T-tables, 4 x 256 words (device)
  const uint32_t* cfwd;           // exact-coordinate tables (device), see fds_api.cu
  const uint32_t* cinv;
  unsigned long long* counters;   // 3 counters (device)
  int32_t width, bx_count, nblocks, k;
  uint64_t iv_hi, iv_lo;          // initial counter block, big-endian halves
  uint32_t rk[44];                // AES-128 round keys
  // batch mode
  const BatchImage* images;       // device, n_images entries; null for a single image
  const int32_t* tile_start;      // device, n_images + 1 prefix sums of tiles per image
  const uint32_t* round_keys;     // device, FDS_MAX_KEYS x 44 words
  unsigned int* dispenser;        // device tile counter (dynamic dispatch), or null (static)
  int32_t n_images, total_tiles;
  // tensor-core form: the B operand (basis limbs) in its shared-memory byte order (device)
  const uint4* tc_b;
  // nonzero: the private fragment stays in plaintext (protect does not encrypt it, restore
  // does not decrypt it); the packed-storage entry points encrypt the packed stream instead
  int32_t plain_private;
  // protect of one image into packed streams: 11 or 8 bits per AC field (pub_out / priv_out
  // then point to the packed public stream and the packed private stream); 0 = int16
  int32_t pack;
  // restore in the public-image form (one image): private positions zero, DC 1024
  int32_t public_image;
  // AES lane schedule of the batched form: nonzero = two keystream blocks per thread
  int32_t aes_pair;
  // protect: tile groups that work in each CTA (1 .. the kernel's groups; 0 = all of them)
  int32_t groups;
};

// What a CTA knows about the tile it is working on (shared memory, filled one tile ahead).
struct TileSlot {
  uint64_t blk[kTileBlocks];      // byte offset of each block's top-left pixel in the image
  uint32_t rk[44];                // the image's AES-128 round keys
  const uint8_t* px_in;           // the image's pixels, public and private fragments
  uint8_t* px_out;
  const uint8_t* pub_in;
  uint8_t* pub_out;
  const uint8_t* priv_in;
  uint8_t* priv_out;
  uint64_t iv_hi, iv_lo;
  int32_t width, k, local, nb;    // local = tile index inside the image; nb = its blocks
  // the tile's 8 pixel rows are contiguous runs of nb * 24 bytes in the image, 16-byte aligned
  // (kPxIn16: in px_in, a whole tile; kPxOut16: in px_out)
  int32_t px_flags;
};
constexpr int32_t kPxIn16 = 1, kPxOut16 = 2;

// launchers (one translation unit each); `sms` = number of SMs of the device, `per_sm` =
// tile groups per SM to launch, at most the kernel's residency (protect: 3 groups of one CTA
// for one image, 4 CTAs for batches; restore: 2 CTAs); 0 = that residency
cudaError_t launch_protect(const TileArgs& a, cudaStream_t s, bool debug, int sms, int per_sm = 0);
cudaError_t launch_restore(const TileArgs& a, cudaStream_t s, int sms, int per_sm = 0);
// restore with the inverse transform on tensor cores (one image, int16 storage)
cudaError_t launch_restore_tc(const TileArgs& a, cudaStream_t s, int sms);
// tensor-core protect of one image (form 0: BF16 three limbs, 1: TF32 two limbs); tiles of
// 128 channel-blocks, two CTAs per SM
cudaError_t launch_protect_tc(const TileArgs& a, cudaStream_t s, int form, bool debug, int sms);

// Raise a kernel's dynamic shared-memory limit once per device (the attribute is per
// device; `done` is the launcher's own record)
constexpr int kMaxAttrDevices = 64;
template <typename Kernel>
inline cudaError_t smem_attr_once(Kernel kernel, int bytes, bool (&done)[kMaxAttrDevices]) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxAttrDevices) return cudaErrorInvalidDevice;
  if (!done[dev]) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

// Resident CTAs per SM of `kernel` at `threads` threads and `bytes` dynamic shared memory on
// the current device (at least 1), cached per device in `cache` (0 = not yet asked)
template <typename Kernel>
inline int resident_ctas(Kernel kernel, int threads, int bytes, int (&cache)[kMaxAttrDevices]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxAttrDevices) return 1;
  if (!cache[dev]) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, bytes) != cudaSuccess || n < 1) n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

inline int total_tiles(const TileArgs& a) {
  return a.images ? a.total_tiles : (a.nblocks + kTileBlocks - 1) / kTileBlocks;
}

// barrier of one 192-thread tile group of a CTA (named barrier `id`, never 0: that is the
// CTA-wide __syncthreads)
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kThreads) : "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// bulk (TMA engine) copies shared -> global; sizes and addresses multiples of 16
__device__ __forceinline__ void bulk_store(void* gmem, const void* smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem),
               "r"(smem_u32(smem)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to later bulk copies
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// mbarriers (one arrival per phase) and bulk (TMA engine) loads that complete on them
constexpr uint32_t kMbarSpinLimit = 1u << 22;   // bounded waits (seconds at most): give up, flag it
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait for phase `parity`; false if it did not complete in time (about 2 s of wall
// clock, or kMbarSpinLimit polls)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  uint64_t t0 = 0;
  for (uint32_t i = 0; i < kMbarSpinLimit && !ok; ++i) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    if (!ok && (i & 255u) == 0u) {
      uint64_t now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (i == 0)
        t0 = now;
      else if (now - t0 > 2000000000ull)
        break;
    }
  }
  return ok != 0;
}
// the one arrival of the phase, announcing `bytes` of bulk loads
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy (addresses and size multiples of 16) completing on bar
__device__ __forceinline__ void bulk_load(void* smem, const void* gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(smem)),
               "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// byte offset of block gb's top-left pixel in an H x W x 3 image
__device__ __forceinline__ uint64_t block_offset(int width, int gb) {
  const int bxc = width >> 3;
  const int by = gb / bxc, bx = gb - by * bxc;
  return (uint64_t)by * 8ull * (uint64_t)width * 3ull + (uint64_t)bx * 24ull;
}

// Fill slot s for global tile g.  Called by threads t = 0 .. kTileBlocks-1 of the tile group
// (each writes its own fields); the caller publishes the slot with a barrier.
__device__ __forceinline__ void fill_slot(const TileArgs& a, int g, TileSlot* s, int t) {
  int width, nblocks, k, local;
  uint64_t iv_hi, iv_lo, pxo = 0, puo = 0, pro = 0;
  const uint32_t* rk;
  if (a.images == nullptr) {
    width = a.width, nblocks = a.nblocks, k = a.k, local = g;
    iv_hi = a.iv_hi, iv_lo = a.iv_lo;
    rk = a.rk;
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
    nblocks = (im.width >> 3) * (im.height >> 3);
    iv_hi = im.iv_hi, iv_lo = im.iv_lo;
    pxo = im.pixel_offset, puo = im.public_offset, pro = im.private_offset;
    rk = a.round_keys + 44 * im.key_slot;
  }
  const int nb = min(kTileBlocks, nblocks - local * kTileBlocks);
  if (t == 0) {
    s->px_in = a.pixels_in + pxo;
    s->px_out = a.pixels_out + pxo;
    s->pub_in = reinterpret_cast<const uint8_t*>(a.pub_in) + puo;
    s->pub_out = reinterpret_cast<uint8_t*>(a.pub_out) + puo;
    s->priv_in = a.priv_in + pro;
    s->priv_out = a.priv_out + pro;
    s->iv_hi = iv_hi;
    s->iv_lo = iv_lo;
    s->width = width;
    s->k = k;
    s->local = local;
    s->nb = nb;
    const int bxc = width >> 3;
    const uint64_t w3 = 3ull * (uint64_t)width, b0 = block_offset(width, local * kTileBlocks);
    const bool rows = (local * kTileBlocks) % bxc + nb <= bxc && ((nb * 24) & 15) == 0 && (w3 & 15) == 0;
    int32_t f = 0;
    if (rows && nb == kTileBlocks && (reinterpret_cast<uintptr_t>(a.pixels_in + pxo + b0) & 15) == 0) f |= kPxIn16;
    if (rows && (reinterpret_cast<uintptr_t>(a.pixels_out + pxo + b0) & 15) == 0) f |= kPxOut16;
    s->px_flags = f;
  }
  if (t < 44) s->rk[t] = rk[t];
  if (t < nb) s->blk[t] = block_offset(width, local * kTileBlocks + t);
}

// Tile schedule of a persistent tile group (vb = its index among the launch's vgrid groups;
// a group is a CTA, or one of the CTA's independent 192-thread groups): the i-th tile is
// vb + i * vgrid (static), or for i >= 1 the value of an atomic counter plus vgrid (dynamic,
// a.dispenser non-null; the counter must be zero at launch).  Called by one thread.
__device__ __forceinline__ int next_tile(const TileArgs& a, int i, int vb, int vgrid) {
  if (a.dispenser == nullptr || i == 0) return vb + i * vgrid;
  return (int)atomicAdd(a.dispenser, 1u) + vgrid;
}

// 24-byte block row of the pixel tile shifted right by `c` bytes: channel c's pixel x is
// then byte 3x of the result (w[0..5] little-endian)
template <int ROWB = kRowBytes>
__device__ __forceinline__ void load_row_shifted(const uint8_t* tile, int y, int b, int c,
                                                 uint32_t (&w)[6]) {
  const uint2* rp = reinterpret_cast<const uint2*>(tile + y * ROWB + b * 24);
  const uint2 w01 = rp[0], w23 = rp[1], w45 = rp[2];
  const uint32_t r[7] = {w01.x, w01.y, w23.x, w23.y, w45.x, w45.y, 0u};
#pragma unroll
  for (int i = 0; i < 6; ++i) w[i] = __funnelshift_r(r[i], r[i + 1], 8 * c);
}

// AES-128-CTR over `bytes` bytes of a 16-byte aligned staging area whose first byte is byte
// 16 * first_block of the image's private message.
// The IV comes from the tile's slot; rk are the 44 round keys.  aes_pair: each thread takes
// two keystream blocks, i and i + kThreads, encrypted interleaved (the lane schedule the
// batched form's autotuner can choose), instead of one.
__device__ __forceinline__ void ctr_tile(uint8_t* st, int bytes, uint64_t first_block,
                                         const TileSlot* sl, const uint32_t* rk, const uint32_t* Ts,
                                         bool aes_pair, int t) {
  const int nblk = (bytes + 15) >> 4;
  if (aes_pair) {
    for (int i = t; i < nblk; i += 2 * kThreads) {
      const bool two = i + kThreads < nblk;
      uint32_t s[2][4];
      ctr_block(sl->iv_hi, sl->iv_lo, first_block + i, s[0]);
      ctr_block(sl->iv_hi, sl->iv_lo, first_block + i + kThreads, s[1]);
      aes128_encrypt_n<2>(s, rk, Ts);
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        if (m == 1 && !two) break;
        uint4* p = reinterpret_cast<uint4*>(st + 16 * (i + m * kThreads));
        uint4 d = *p;
        d.x ^= s[m][0];
        d.y ^= s[m][1];
        d.z ^= s[m][2];
        d.w ^= s[m][3];
        *p = d;
      }
    }
    return;
  }
  for (int i = t; i < nblk; i += kThreads) {
    uint32_t s[4];
    ctr_block(sl->iv_hi, sl->iv_lo, first_block + i, s);
    aes128_encrypt(s, rk, Ts);
    uint4* p = reinterpret_cast<uint4*>(st + 16 * i);
    uint4 d = *p;
    d.x ^= s[0];
    d.y ^= s[1];
    d.z ^= s[2];
    d.w ^= s[3];
    *p = d;
  }
}

// ctr_tile with a replicated T0 table (2^(SH-2) copies at Trep, entry x of copy c at word
// 2^(SH-2) x + c; SH = 7: every lookup of a warp hits 32 distinct banks).  aes_pair as in
// ctr_tile; t = the thread's index in its 192-thread tile group.
template <int SH = 7>
__device__ __forceinline__ void ctr_tile_rep(uint8_t* st, int bytes, uint64_t first_block, const TileSlot* sl,
                                             const uint32_t* rk, const uint32_t* Trep, bool aes_pair, int t) {
  const int nblk = (bytes + 15) >> 4;
  const uint32_t Tl = smem_u32(Trep) + 4u * (t & ((1 << (SH - 2)) - 1));
  const int step = aes_pair ? 2 * kThreads : kThreads;
  for (int i = t; i < nblk; i += step) {
    const int m_n = aes_pair && i + kThreads < nblk ? 2 : 1;
    uint32_t s[2][4];
    ctr_block(sl->iv_hi, sl->iv_lo, first_block + i, s[0]);
    if (aes_pair) {
      ctr_block(sl->iv_hi, sl->iv_lo, first_block + i + kThreads, s[1]);
      aes128_encrypt_rep_n<2, SH>(s, rk, Tl);
    } else {
      aes128_encrypt_rep<SH>(s[0], rk, Tl);
    }
    for (int m = 0; m < m_n; ++m) {
      uint4* p = reinterpret_cast<uint4*>(st + 16 * (i + m * kThreads));
      uint4 d = *p;
      d.x ^= s[m][0];
      d.y ^= s[m][1];
      d.z ^= s[m][2];
      d.w ^= s[m][3];
      *p = d;
    }
  }
}

// ctr_tile with the pair table (window address kTpairWin, see aes128_encrypt_pair), one
// keystream block per thread; t = the thread's index in its 192-thread tile group.
__device__ __forceinline__ void ctr_tile_pair(uint8_t* st, int bytes, uint64_t first_block, const TileSlot* sl,
                                              const uint32_t* rk, int t) {
  const int nblk = (bytes + 15) >> 4;
  const PairLanes lc = pair_lanes();
  for (int i = t; i < nblk; i += kThreads) {
    uint32_t s[4];
    ctr_block(sl->iv_hi, sl->iv_lo, first_block + i, s);
    aes128_encrypt_pair(s, rk, lc);
    uint4* p = reinterpret_cast<uint4*>(st + 16 * i);
    uint4 d = *p;
    d.x ^= s[0];
    d.y ^= s[1];
    d.z ^= s[2];
    d.w ^= s[3];
    *p = d;
  }
}

// ---- packed storage (Sect. 6.4.3): a full tile's 192 channel-blocks are a multiple of 8,
// so its part of either bit stream starts on a byte boundary
constexpr int kDcBits = 11;

// bytes of a tile's packed public / private part and their offsets in the image's streams
// (a full tile: 24 (63 - k) W and 24 (11 + k W) bytes)
template <int W>
__device__ __forceinline__ void packed_extent(const TileSlot* sl, bool priv, uint64_t& off, int& bytes) {
  const int k = sl->k;
  const int per_cb = priv ? kDcBits + k * W : (63 - k) * W;   // bits per channel-block
  off = (uint64_t)sl->local * 24ull * (uint64_t)per_cb;
  bytes = (3 * sl->nb * per_cb + 7) >> 3;
}

// AES-128-CTR over the tile's packed private part (words at w, stream bytes [off, off +
// bytes), off a multiple of 4): one thread per keystream block the part overlaps; a block
// that straddles two tiles is generated by both, each XORing its own words
// SH = 0: the four T-tables at Ts; SH = kTabPair: the pair table (Ts unused); else a
// replicated T0 as in ctr_tile_rep
constexpr int kTabPair = -1;
template <int SH = 0>
__device__ __forceinline__ void ctr_tile_packed(uint32_t* w, uint64_t off, int bytes, const TileSlot* sl,
                                                const uint32_t* rk, const uint32_t* Ts, int t) {
  const uint64_t b0 = off >> 4;
  const int nblk = (int)(((off + (uint64_t)bytes + 15) >> 4) - b0);
  const int nw = (bytes + 3) >> 2;
  const int skew = (int)((off & 15) >> 2);
  const uint32_t Tl = SH > 0 ? smem_u32(Ts) + 4u * (t & ((1 << (SH > 2 ? SH - 2 : 0)) - 1)) : 0u;
  const PairLanes lc = pair_lanes();
  for (int i = t; i < nblk; i += kThreads) {
    uint32_t s[4];
    ctr_block(sl->iv_hi, sl->iv_lo, b0 + i, s);
    if constexpr (SH == kTabPair)
      aes128_encrypt_pair(s, rk, lc);
    else if constexpr (SH != 0)
      aes128_encrypt_rep<SH>(s, rk, Tl);
    else
      aes128_encrypt(s, rk, Ts);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int wi = 4 * i + m - skew;
      if (wi >= 0 && wi < nw) w[wi] ^= s[m];
    }
  }
}

// Exact integer coordinates of 8 F[u][v] (pos = 8u+v) of channel c of tile block b:
// n[j] = sum over the 64 pixels of pixel * K_j, with the signed-byte weights K_j of
// table[pos][j][16 words] (word w covers pixels x = 4(w&1) .. +3 of row w>>1).
// ROWB: bytes per pixel row of the tile
// the dot products of coords_fwd: P[16] = the 64 pixels of the channel-block as bytes (word
// w covers pixels x = 4(w&1) .. +3 of row w>>1)
__device__ __forceinline__ void coords_from_pixels(const uint32_t (&P)[16], int pos, const uint32_t* table,
                                                   int (&n)[9]) {
  const uint4* t4 = reinterpret_cast<const uint4*>(table + pos * 128);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int acc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 tw = __ldg(t4 + 4 * j + q);
      acc = dp4a_us(P[4 * q + 0], tw.x, acc);
      acc = dp4a_us(P[4 * q + 1], tw.y, acc);
      acc = dp4a_us(P[4 * q + 2], tw.z, acc);
      acc = dp4a_us(P[4 * q + 3], tw.w, acc);
    }
    n[j] = acc;
  }
  n[8] = 0;
}

// bytes 0, 3, 6, 9 and 12, 15, 18, 21 of a row's six words (channel c already shifted to byte 0)
__device__ __forceinline__ void row_pixels(const uint32_t (&w)[6], uint32_t& lo, uint32_t& hi) {
  lo = __byte_perm(__byte_perm(w[0], w[1], 0x0630u), w[2], 0x5210u);
  hi = __byte_perm(__byte_perm(w[3], w[4], 0x0630u), w[5], 0x5210u);
}

// Exact integer coordinates of 8 F[u][v] (pos = 8u+v) of channel c of tile block b:
// n[j] = sum over the 64 pixels of pixel * K_j, with the signed-byte weights K_j of
// table[pos][j][16 words] (word w covers pixels x = 4(w&1) .. +3 of row w>>1).
// ROWB: bytes per pixel row of the tile
template <int ROWB = kRowBytes>
__device__ __forceinline__ void coords_fwd(const uint8_t* tile, int b, int c, int pos,
                                           const uint32_t* table, int (&n)[9]) {
  uint32_t P[16];
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    uint32_t w[6];
    load_row_shifted<ROWB>(tile, y, b, c, w);
    row_pixels(w, P[2 * y], P[2 * y + 1]);
  }
  coords_from_pixels(P, pos, table, n);
}

// the same from the image in global memory: blk = the block's top-left pixel (8-byte
// aligned), row = bytes per image row
__device__ __forceinline__ void coords_fwd_global(const uint8_t* blk, uint64_t row, int c, int pos,
                                                  const uint32_t* table, int (&n)[9]) {
  uint32_t P[16];
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    const uint2* rp = reinterpret_cast<const uint2*>(blk + y * row);
    const uint2 w01 = __ldg(rp), w23 = __ldg(rp + 1), w45 = __ldg(rp + 2);
    const uint32_t r[7] = {w01.x, w01.y, w23.x, w23.y, w45.x, w45.y, 0u};
    uint32_t w[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) w[i] = __funnelshift_r(r[i], r[i + 1], 8 * c);
    row_pixels(w, P[2 * y], P[2 * y + 1]);
  }
  coords_from_pixels(P, pos, table, n);
}

// Exact integer coordinates of 8 p[y][x] (pos = 8y+x) from int16 coefficients in zigzag
// order, packed two per word (Q[i] = q(2i) | q(2i+1) << 16), with the weights of
// table[pos][j][16 words] (word t covers zigzag indices 4t .. 4t+3).
__device__ __forceinline__ void coords_inv(const uint32_t (&Q)[32], int pos, const uint32_t* table,
                                           int (&n)[9]) {
  const uint4* t4 = reinterpret_cast<const uint4*>(table + pos * 128);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int acc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 tw = __ldg(t4 + 4 * j + q);
      acc = dp2a_lo(Q[8 * q + 0], tw.x, acc);
      acc = dp2a_hi(Q[8 * q + 1], tw.x, acc);
      acc = dp2a_lo(Q[8 * q + 2], tw.y, acc);
      acc = dp2a_hi(Q[8 * q + 3], tw.y, acc);
      acc = dp2a_lo(Q[8 * q + 4], tw.z, acc);
      acc = dp2a_hi(Q[8 * q + 5], tw.z, acc);
      acc = dp2a_lo(Q[8 * q + 6], tw.w, acc);
      acc = dp2a_hi(Q[8 * q + 7], tw.w, acc);
    }
    n[j] = acc;
  }
  n[8] = 0;
}

}  // namespace fds
