// Fused protect kernel (Sect. 6.3.1, Fig. 6): 8x8 DCT-II per channel, int16 rounding,
// zigzag fragmentation, AES-128-CTR of the confidential fragment.  Per tile:
//   1. cp.async the pixels (8 rows x 24 bytes per block) into shared memory
//   2. per channel-block: row then column float32 butterflies, round every coefficient to
//      int16, write it to the public or private staging area at its zigzag position;
//      coefficients within the float32 error guard of a half-integer go to a queue
//   3. the queue is resolved exactly (64-bit fixed point; exact arithmetic in Z[cos(pi/16)]
//      when that is still ambiguous)
//   4. AES-128-CTR over the private staging area, one thread per 16-byte keystream block
//   5. coalesced 16-byte stores of both staging areas
#include "fds_tile.cuh"

namespace fds {

// Exact rounding of coefficient `pos` = 8u+v of channel c of tile block b.
__device__ __noinline__ int resolve_fwd(const uint8_t* tile, int b, int c, int pos, float v,
                                        const int32_t* bfwd, int* n3, bool* fail) {
  const int m = (int)floorf(v);
  const uint8_t* px = tile + b * 24 + c;
  // stage 2: 64-bit fixed point; |acc - 8F 2^28| <= (1/2 + tiny) sum p
  long long acc = 0, err = 0;
  const int32_t* row = bfwd + pos * 64;
  for (int y = 0; y < 8; ++y) {
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int p = px[y * kRowBytes + 3 * x];
      acc += (long long)p * row[8 * y + x];
      err += p;
    }
  }
  const long long d = acc - ((long long)(8 * m + 4) << kFixShift);
  if (d > err + 1) return m + 1;
  if (d < -err - 1) return m;
  // stage 3: exact coordinates in Z[cos(pi/16)]
  ++*n3;
  const int u = pos >> 3, vv = pos & 7;
  int n[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) n[j] = 0;
  for (int y = 0; y < 8; ++y) {
    const int al = u == 0 ? 4 : (2 * y + 1) * u;
    for (int x = 0; x < 8; ++x) {
      const int be = vv == 0 ? 4 : (2 * x + 1) * vv;
      const int p = px[y * kRowBytes + 3 * x];
      add_cos_term(n, al - be, p);
      add_cos_term(n, al + be, p);
    }
  }
  return pick(m, exact_sign(n[0] - 8 * m - 4, n, fail));
}

template <int K, bool DEBUG>
__global__ void __launch_bounds__(kThreads) protect_kernel(const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* tile = smem + kSmemPix;
  uint8_t* coef = smem + kSmemCoef;
  const uint32_t* T0s = reinterpret_cast<const uint32_t*>(smem + kSmemT0);
  QEntry* queue = reinterpret_cast<QEntry*>(smem + kSmemQueue);
  const uint64_t* blk = reinterpret_cast<const uint64_t*>(smem + kSmemBlk);
  int* misc = reinterpret_cast<int*>(smem + kSmemMisc);

  const int k = K >= 0 ? K : a.k;
  const int npub = 63 - k;
  const int t = threadIdx.x;
  const int b0 = blockIdx.x * kTileBlocks;
  const int nb = min(kTileBlocks, a.nblocks - b0);
  const uint64_t w3 = (uint64_t)a.width * 3ull;

  tile_prologue(a, smem, b0, nb);
  __syncthreads();
  for (int i = t; i < 8 * kTileBlocks * 3; i += kThreads) {
    const int y = i / (kTileBlocks * 3), rem = i - y * (kTileBlocks * 3);
    const int b = rem / 3, q = rem - 3 * b;
    if (b < nb) cp_async8(tile + y * kRowBytes + b * 24 + 8 * q, a.pixels_in + blk[b] + y * w3 + 8 * q);
  }
  cp_async_wait_all();
  __syncthreads();

  int16_t* pubst = reinterpret_cast<int16_t*>(coef);
  int16_t* privst = reinterpret_cast<int16_t*>(coef + kTileCb * 2 * npub);
  int n3 = 0;
  bool fail = false;
  const int cb = t, b = t / 3, c = t - 3 * (t / 3);

  if (b < nb) {
    float f[8][8];
    // rows: channel c's bytes of the block row, level-shifted by 128 (exact)
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      uint32_t w[6];
      load_row_shifted(tile, y, b, c, w);
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const int byte = 3 * x;
        f[y][x] = __int_as_float(__byte_perm(w[byte >> 2], 0x4B000000u, 0x7440u | (byte & 3))) -
                  8388736.0f;
      }
      dct8<true, false>(f[y]);
    }
    // columns; columns 0 and 4 hold unscaled (exact integer) row outputs
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      float col[8];
#pragma unroll
      for (int y = 0; y < 8; ++y) col[y] = f[y][v];
      if (v == 0 || v == 4)
        dct8<true, true>(col);
      else
        dct8<false, false>(col);
#pragma unroll
      for (int u = 0; u < 8; ++u) f[u][v] = col[u];
    }
    if (DEBUG) {
      float* out = a.dbg_coefs + ((uint64_t)b0 * 3 + cb) * 64;
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
      // rounding: the four rational positions exactly in integers, the rest to nearest in
      // float32 with the residual checked against the guard
      int16_t* pub_cb = pubst + cb * npub;
      int16_t* priv_cb = privst + cb * (k + 1);
      float maxr = 0.0f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int z = zigzag_of(u, v);
          int q;
          if ((u == 0 || u == 4) && (v == 0 || v == 4)) {
            const int T = __float_as_int(f[u][v] + kMagic) - kMagicBits;  // 8 F, exact
            q = (u == 0 && v == 0) ? ((T + 4) >> 3) + 1024 : (T + 4 - (T < 0 ? 1 : 0)) >> 3;
          } else {
            const float yv = f[u][v] + kMagic;
            q = __float_as_int(yv) - kMagicBits;
            maxr = fmaxf(maxr, fabsf(f[u][v] - (yv - kMagic)));
          }
          if (z <= k)
            priv_cb[z] = (int16_t)q;
          else
            pub_cb[z - k - 1] = (int16_t)q;
        }
      }
      if (maxr > 0.5f - kGuardFwd) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            if ((u == 0 || u == 4) && (v == 0 || v == 4)) continue;
            const float yv = f[u][v] + kMagic;
            if (fabsf(f[u][v] - (yv - kMagic)) > 0.5f - kGuardFwd) {
              const int idx = atomicAdd(&misc[0], 1);
              if (idx < kQueueCap) {
                queue[idx] = QEntry{(uint16_t)cb, (uint8_t)(8 * u + v), 0, f[u][v]};
              } else {  // queue full: resolve here
                const int q = resolve_fwd(tile, b, c, 8 * u + v, f[u][v], a.bfwd, &n3, &fail);
                const int z = zigzag_of(u, v);
                if (z <= k)
                  priv_cb[z] = (int16_t)q;
                else
                  pub_cb[z - k - 1] = (int16_t)q;
              }
            }
          }
        }
      }
    }
  }
  if (DEBUG) return;
  __syncthreads();
  const int nq = min(misc[0], kQueueCap);
  for (int i = t; i < nq; i += kThreads) {
    const QEntry e = queue[i];
    const int eb = e.cb / 3, ec = e.cb - 3 * eb;
    const int q = resolve_fwd(tile, eb, ec, e.pos, e.v, a.bfwd, &n3, &fail);
    const int z = zigzag_of(e.pos >> 3, e.pos & 7);
    if (z <= k)
      privst[e.cb * (k + 1) + z] = (int16_t)q;
    else
      pubst[e.cb * npub + z - k - 1] = (int16_t)q;
  }
  if (n3) atomicAdd(&misc[1], n3);
  if (fail) atomicAdd(&misc[2], 1);
  __syncthreads();

  // AES-128-CTR over the private staging area
  const int priv_bytes = nb * 6 * (k + 1);
  const uint64_t priv_off = (uint64_t)b0 * 6ull * (uint64_t)(k + 1);  // multiple of 16
  ctr_tile(reinterpret_cast<uint8_t*>(privst), priv_bytes, priv_off >> 4, a, T0s);
  __syncthreads();

  // coalesced stores
  {
    const int bytes = nb * 6 * npub;
    uint8_t* dst = reinterpret_cast<uint8_t*>(a.pub_out) + (uint64_t)b0 * 6ull * (uint64_t)npub;
    const uint8_t* src = reinterpret_cast<const uint8_t*>(pubst);
    const int n16 = bytes >> 4;
    for (int i = t; i < n16; i += kThreads)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    for (int j = (n16 << 4) + 2 * t; j < bytes; j += 2 * kThreads)
      *reinterpret_cast<uint16_t*>(dst + j) = *reinterpret_cast<const uint16_t*>(src + j);
  }
  {
    uint8_t* dst = a.priv_out + priv_off;
    const uint8_t* src = reinterpret_cast<const uint8_t*>(privst);
    const int n16 = priv_bytes >> 4;
    for (int i = t; i < n16; i += kThreads)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    for (int j = (n16 << 4) + 2 * t; j < priv_bytes; j += 2 * kThreads)
      *reinterpret_cast<uint16_t*>(dst + j) = *reinterpret_cast<const uint16_t*>(src + j);
  }
  tile_epilogue_counters(a, smem);
}

cudaError_t launch_protect(const TileArgs& a, cudaStream_t s, bool debug) {
  const int grid = (a.nblocks + kTileBlocks - 1) / kTileBlocks;
  if (debug)
    protect_kernel<-1, true><<<grid, kThreads, kSmemBytes, s>>>(a);
  else if (a.k == 0)
    protect_kernel<0, false><<<grid, kThreads, kSmemBytes, s>>>(a);
  else if (a.k == 5)
    protect_kernel<5, false><<<grid, kThreads, kSmemBytes, s>>>(a);
  else
    protect_kernel<-1, false><<<grid, kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fds
