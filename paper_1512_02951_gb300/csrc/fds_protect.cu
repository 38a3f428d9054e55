// Fused protect kernel (Sect. 6.3.1, Fig. 6): 8x8 DCT-II per channel, int16 rounding,
// zigzag fragmentation, AES-128-CTR of the confidential fragment.
//
// Persistent CTAs over a tile schedule (one image, or every tile of a batch of images in one
// launch); per tile (see fds_tile.cuh for the decomposition):
//   A. the tile's pixels (prefetched with cp.async during the previous tile) are in shared
//      memory; the previous tile's fragments leave through bulk (TMA engine) stores and the
//      next tile's pixels start loading
//   1. per channel-block: row then column float32 butterflies; every coefficient rounded to
//      int16 and written to the public or private staging area at its zigzag position;
//      coefficients within the float32 error guard of a half-integer are queued
//   B. 2. queued coefficients are re-decided exactly (integer coordinates in Z[cos(pi/16)])
//   C. 3. the public fragment leaves (bulk store) while AES-128-CTR encrypts the private
//      staging area, one thread per 16-byte keystream block
// One staging area (so that three CTAs fit on an SM): the previous tile's bulk stores must
// have read it before the transform writes it again.
#include "fds_tile.cuh"

namespace fds {

constexpr int kPCtasPerSm = 3;
constexpr int kSmemPix = 0;                                  // 2 pixel tiles
constexpr int kSmemStage = kSmemPix + 2 * kPixBytes;         // 1 staging area
constexpr int kSmemT = kSmemStage + kCoefBytes;              // AES tables, 4 KB
constexpr int kSmemQueue = kSmemT + 4096;                    // near-tie queue
constexpr int kSmemSlot = kSmemQueue + 4 * kQueueCap;        // 3 tile slots (ring)
constexpr int kSlotBytes = (sizeof(TileSlot) + 15) & ~15;
constexpr int kSmemMisc = kSmemSlot + 3 * kSlotBytes;
constexpr int kSmemBytes = kSmemMisc + 32;

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

// cp.async the pixels of slot sl into pixel tile pix (all threads)
__device__ __forceinline__ void load_pixels(const TileSlot* sl, uint8_t* pix) {
  const uint64_t w3 = (uint64_t)sl->width * 3ull;
  const int nb = sl->nb;
  for (int i = threadIdx.x; i < 8 * kTileBlocks * 3; i += kThreads) {
    const int y = i / (kTileBlocks * 3), rem = i - y * (kTileBlocks * 3);
    const int b = rem / 3, q = rem - 3 * b;
    if (b < nb) cp_async8(pix + y * kRowBytes + b * 24 + 8 * q, sl->px_in + sl->blk[b] + y * w3 + 8 * q);
  }
  cp_async_commit();
}

// BATCH: tiles of many images (round keys from the slot); else one image (round keys read
// from the kernel parameters, which AES then takes as constant-bank operands)
template <int K, bool DEBUG, bool BATCH>
__global__ void __launch_bounds__(kThreads, kPCtasPerSm) protect_kernel(const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* Ts = reinterpret_cast<uint32_t*>(smem + kSmemT);
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + kSmemQueue);
  // misc: [0] queue size, [1] queued total, [2] escalations, [3] failures, [4..5] schedule
  int* misc = reinterpret_cast<int*>(smem + kSmemMisc);
  const int t = threadIdx.x;
  const int ntiles = a.images ? a.total_tiles : (a.nblocks + kTileBlocks - 1) / kTileBlocks;
  if ((int)blockIdx.x >= ntiles) return;
  auto slot = [&](int i) { return reinterpret_cast<TileSlot*>(smem + kSmemSlot + i * kSlotBytes); };

  for (int i = t; i < 1024; i += kThreads) Ts[i] = a.T[i];
  if (t < 4) misc[t] = 0;
  if (t == 0) {
    misc[4] = next_tile(a, 0);
    misc[5] = next_tile(a, 1);
  }
  if (t < kTileBlocks) fill_slot(a, blockIdx.x, slot(0));
  __syncthreads();
  load_pixels(slot(0), smem + kSmemPix);

  int it = 0;
  bool have_prev = false;
  for (;; ++it) {
    const int buf = it & 1;
    // slots: tile it in it % 3, it + 1 in (it + 1) % 3, the one being stored in (it + 2) % 3
    const int s_cur = it % 3, s_nxt = (it + 1) % 3, s_prev = (it + 2) % 3;
    const int cur = misc[4 + buf], nxt = misc[4 + (buf ^ 1)];
    if (cur >= ntiles) break;
    const TileSlot* sl = slot(s_cur);
    if (nxt < ntiles && t < kTileBlocks) fill_slot(a, nxt, slot(s_nxt));
    cp_async_wait_all();
    if (t == 0) misc[0] = 0;
    __syncthreads();                                                       // A
    if (t == 0) misc[4 + buf] = nxt < ntiles ? next_tile(a, it + 2) : ntiles;
    if (!DEBUG && t == 0 && have_prev) {
      store_private(slot(s_prev), smem + kSmemStage);   // the public part left before its AES
      bulk_wait_read_all();                  // the staging area may be written again
    }
    __syncthreads();                                                       // A'

    if (nxt < ntiles) load_pixels(slot(s_nxt), smem + kSmemPix + (buf ^ 1) * kPixBytes);

    const int k = K >= 0 ? K : sl->k;
    const int npub = 63 - k;
    const int nb = sl->nb;
    const uint8_t* tile_px = smem + kSmemPix + buf * kPixBytes;
    int16_t* pubst = reinterpret_cast<int16_t*>(smem + kSmemStage);
    int16_t* privst = reinterpret_cast<int16_t*>(smem + kSmemStage + kTileCb * 2 * npub);
    const int cb = t, b = t / 3, c = t - 3 * (t / 3);
    if (b < nb) {
      float f[8][8];
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
        V += dct8_row_bytes_w(X, f[y]);
      }
      // columns; columns 0 and 4 hold unscaled (exact integer) row outputs
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        float col[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) col[y] = f[y][v];
        if (v == 0 || v == 4)
          W += dct8_rat_w(col);
        else
          dct8<false, false>(col);
#pragma unroll
        for (int u = 0; u < 8; ++u) f[u][v] = col[u];
      }
      if (DEBUG) {
        float* out = a.dbg_coefs + ((uint64_t)sl->local * kTileBlocks * 3 + cb) * 64;
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            float val = f[u][v];
            if (u == 0 && v == 0)
              val = (val + 8192.0f) * 0.125f;
            else if ((u == 0 || u == 4) && (v == 0 || v == 4))
              val *= 0.125f;
            out[8 * u + v] = val;
          }
      } else {
        // rounding: the four rational positions exactly in integers; the rest to nearest in
        // float32, residual checked against the guard (near ties marked in a 64-bit mask)
        int16_t* pub_cb = pubst + cb * npub;
        int16_t* priv_cb = privst + cb * (k + 1);
        uint32_t mlo = 0, mhi = 0;
        const float thr = 0.5f - fminf(fmaf(V, kGuardV, fmaf(W, kGuardW, kGuardU)), kGuardFwd);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const int z = zigzag_of(u, v);
            uint32_t q;
            if ((u == 0 || u == 4) && (v == 0 || v == 4)) {
              const int T = __float_as_int(f[u][v] + kMagic) - kMagicBits;  // 8 F, exact
              q = (uint32_t)((u == 0 && v == 0) ? ((T + 4) >> 3) + 1024 : (T + 4 - (T < 0 ? 1 : 0)) >> 3);
            } else {
              const float yv = f[u][v] + kMagic;
              q = __float_as_uint(yv);                 // low 16 bits: the int16 result
              if (fabsf(f[u][v] - (yv - kMagic)) > thr) {
                if (8 * u + v < 32)
                  mlo |= 1u << (8 * u + v);
                else
                  mhi |= 1u << (8 * u + v - 32);
              }
            }
            if (z <= k)
              priv_cb[z] = (int16_t)q;
            else
              pub_cb[z - k - 1] = (int16_t)q;
          }
        }
        uint64_t mask = ((uint64_t)mhi << 32) | mlo;
        while (mask) {
          const int pos = __ffsll((long long)mask) - 1;
          mask &= mask - 1;
          const int idx = atomicAdd(&misc[0], 1);
          if (idx < kQueueCap) {
            queue[idx] = ((uint32_t)cb << 8) | (uint32_t)pos;
          } else {  // queue full: decide here
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
      __syncthreads();   // publishes the schedule entry written after barrier A
      continue;
    }
    __syncthreads();                                                       // B
    {
      const int nq = min(misc[0], kQueueCap);
      int esc = 0;
      bool fail = false;
      for (int i = t; i < nq; i += kThreads) {
        const uint32_t e = queue[i];
        const int ecb = (int)(e >> 8), pos = (int)(e & 255);
        const int eb = ecb / 3, ec = ecb - 3 * eb;
        int n[9];
        coords_fwd(tile_px, eb, ec, pos, a.cfwd, n);
        const int q = exact_round(n, &esc, &fail);
        const int z = zigzag_of(pos >> 3, pos & 7);
        if (z <= k)
          privst[ecb * (k + 1) + z] = (int16_t)q;
        else
          pubst[ecb * npub + z - k - 1] = (int16_t)q;
      }
      if (esc) atomicAdd(&misc[2], esc);
      if (fail) atomicAdd(&misc[3], 1);
      if (t == 0) misc[1] += misc[0];
    }
    fence_proxy_async();                   // every thread's staging writes, before the bulk store
    __syncthreads();                                                       // C
    if (t == 0) store_public(sl, smem + kSmemStage);   // final: it leaves during the AES
    if (!a.plain_private)
      ctr_tile(reinterpret_cast<uint8_t*>(privst), nb * 6 * (k + 1),
               ((uint64_t)sl->local * kTileBlocks * 6ull * (uint64_t)(k + 1)) >> 4, sl,
               BATCH ? sl->rk : a.rk, Ts);
    fence_proxy_async();
    have_prev = true;
  }
  if (DEBUG) return;
  __syncthreads();
  if (t == 0) {
    if (have_prev) store_private(slot((it + 2) % 3), smem + kSmemStage);
    bulk_wait_all();
    if (a.counters) {
      if (misc[1]) atomicAdd(&a.counters[0], (unsigned long long)misc[1]);
      if (misc[2]) atomicAdd(&a.counters[1], (unsigned long long)misc[2]);
      if (misc[3]) atomicAdd(&a.counters[2], (unsigned long long)misc[3]);
    }
  }
}

template <int K, bool DEBUG, bool BATCH>
static cudaError_t launch_k(const TileArgs& a, cudaStream_t s, int sms, int per_sm) {
  static bool attr[kMaxAttrDevices];
  cudaError_t e = smem_attr_once(protect_kernel<K, DEBUG, BATCH>, kSmemBytes, attr);
  if (e != cudaSuccess) return e;
  const int ntiles = total_tiles(a);
  const int cap = (per_sm == 1 ? 1 : kPCtasPerSm) * sms;
  const int grid = ntiles < cap ? ntiles : cap;
  if (grid > 0) protect_kernel<K, DEBUG, BATCH><<<grid, kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

// k is uniform over the launch when a.k >= 0; a.k < 0 (batches of mixed k) reads k per tile
cudaError_t launch_protect(const TileArgs& a, cudaStream_t s, bool debug, int sms, int per_sm) {
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
