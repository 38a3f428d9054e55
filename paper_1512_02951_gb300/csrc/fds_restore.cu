// Fused restore kernel (defragmentation, Sect. 3.2, Fig. 3; inverse of Sect. 6.3.1): CTR
// decryption of the confidential fragment, merge with the public fragment by zigzag
// position, inverse 8x8 DCT, round half away from zero (exact), clamp to [0, 255].  Per tile:
//   1. cp.async the public and private fragment ranges of the tile into shared memory
//   2. AES-128-CTR decryption of the private range in place
//   3. per channel-block: column then row float32 inverse butterflies, round + clamp, write
//      the bytes into the interleaved pixel tile; values within the float32 error guard of a
//      half-integer go to a queue, resolved exactly afterwards
//   4. coalesced 8-byte stores of the pixel tile
#include "fds_tile.cuh"

namespace fds {

// Exact rounding of pixel `pos` = 8y+x of tile channel-block cb from its int16 coefficients.
__device__ __noinline__ int resolve_inv(const int16_t* pubst, const int16_t* privst, int cb,
                                        int pos, float v, int k, const int32_t* binv, int* n3,
                                        bool* fail) {
  const int m = (int)floorf(v);
  // stage 2: 64-bit fixed point; |acc - 8p 2^28| <= (1/2 + tiny) sum |F|
  long long acc = 0, err = 0;
  const int32_t* row = binv + pos * 64;
  for (int z = 0; z < 64; ++z) {
    const int q = coef_at(pubst, privst, cb, z, k);
    acc += (long long)q * row[z];
    err += q < 0 ? -q : q;
  }
  const long long d = acc - ((long long)(8 * m + 4) << kFixShift);
  if (d > err + 1) return m + 1;
  if (d < -err - 1) return m;
  // stage 3: exact coordinates in Z[cos(pi/16)]
  ++*n3;
  const int y = pos >> 3, x = pos & 7;
  int n[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) n[j] = 0;
  for (int u = 0; u < 8; ++u) {
    const int al = u == 0 ? 4 : (2 * y + 1) * u;
    for (int vv = 0; vv < 8; ++vv) {
      const int be = vv == 0 ? 4 : (2 * x + 1) * vv;
      const int q = coef_at(pubst, privst, cb, zigzag_of(u, vv), k);
      add_cos_term(n, al - be, q);
      add_cos_term(n, al + be, q);
    }
  }
  return pick(m, exact_sign(n[0] - 8 * m - 4, n, fail));
}

template <int K>
__global__ void __launch_bounds__(kThreads) restore_kernel(const __grid_constant__ TileArgs a) {
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

  int16_t* pubst = reinterpret_cast<int16_t*>(coef);
  int16_t* privst = reinterpret_cast<int16_t*>(coef + kTileCb * 2 * npub);
  const int pub_bytes = nb * 6 * npub;
  const int priv_bytes = nb * 6 * (k + 1);
  const uint64_t pub_off = (uint64_t)b0 * 6ull * (uint64_t)npub;
  const uint64_t priv_off = (uint64_t)b0 * 6ull * (uint64_t)(k + 1);

  tile_prologue(a, smem, b0, nb);
  {
    const uint8_t* src = reinterpret_cast<const uint8_t*>(a.pub_in) + pub_off;
    uint8_t* dst = reinterpret_cast<uint8_t*>(pubst);
    const int n16 = pub_bytes >> 4;
    for (int i = t; i < n16; i += kThreads) cp_async16(dst + 16 * i, src + 16 * i);
    for (int j = (n16 << 4) + 2 * t; j < pub_bytes; j += 2 * kThreads)
      *reinterpret_cast<uint16_t*>(dst + j) = *reinterpret_cast<const uint16_t*>(src + j);
  }
  {
    const uint8_t* src = a.priv_in + priv_off;
    uint8_t* dst = reinterpret_cast<uint8_t*>(privst);
    const int n16 = priv_bytes >> 4;
    for (int i = t; i < n16; i += kThreads) cp_async16(dst + 16 * i, src + 16 * i);
    for (int j = (n16 << 4) + 2 * t; j < priv_bytes; j += 2 * kThreads)
      *reinterpret_cast<uint16_t*>(dst + j) = *reinterpret_cast<const uint16_t*>(src + j);
  }
  cp_async_wait_all();
  __syncthreads();
  ctr_tile(reinterpret_cast<uint8_t*>(privst), priv_bytes, priv_off >> 4, a, T0s);
  __syncthreads();

  int n3 = 0;
  bool fail = false;
  const int cb = t, b = t / 3, c = t - 3 * (t / 3);
  if (b < nb) {
    const int16_t* pub_cb = pubst + cb * npub;
    const int16_t* priv_cb = privst + cb * (k + 1);
    float f[8][8];
    float l1 = 0.0f;  // sum |F|, exact (integers below 2^24)
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const int z = zigzag_of(u, v);
        const int q = z <= k ? priv_cb[z] : pub_cb[z - k - 1];
        f[u][v] = __int_as_float(kMagicBits + q) - kMagic;
        l1 += fabsf(f[u][v]);
      }
    // columns (over u), then rows (over v)
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      float col[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) col[u] = f[u][v];
      idct8(col);
#pragma unroll
      for (int y = 0; y < 8; ++y) f[y][v] = col[y];
    }
#pragma unroll
    for (int y = 0; y < 8; ++y) idct8(f[y]);
    const float thr = 0.5f - l1 * kGuardInvScale;
    uint8_t* out = tile + b * 24 + c;
    float maxr = 0.0f;
#pragma unroll
    for (int y = 0; y < 8; ++y)
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const float pc = fminf(fmaxf(f[y][x], 0.0f), 255.0f);
        const float yv = pc + kMagic;
        maxr = fmaxf(maxr, fabsf(pc - (yv - kMagic)));
        out[y * kRowBytes + 3 * x] = (uint8_t)(__float_as_uint(yv) & 0xffu);
      }
    if (maxr > thr) {
#pragma unroll
      for (int y = 0; y < 8; ++y)
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const float pc = fminf(fmaxf(f[y][x], 0.0f), 255.0f);
          const float yv = pc + kMagic;
          if (fabsf(pc - (yv - kMagic)) > thr) {
            const int idx = atomicAdd(&misc[0], 1);
            if (idx < kQueueCap) {
              queue[idx] = QEntry{(uint16_t)cb, (uint8_t)(8 * y + x), 0, pc};
            } else {  // queue full: resolve here
              int p = resolve_inv(pubst, privst, cb, 8 * y + x, pc, k, a.binv, &n3, &fail);
              out[y * kRowBytes + 3 * x] = (uint8_t)(p < 0 ? 0 : (p > 255 ? 255 : p));
            }
          }
        }
    }
  }
  __syncthreads();
  const int nq = min(misc[0], kQueueCap);
  for (int i = t; i < nq; i += kThreads) {
    const QEntry e = queue[i];
    const int eb = e.cb / 3, ec = e.cb - 3 * eb;
    const int p = resolve_inv(pubst, privst, e.cb, e.pos, e.v, k, a.binv, &n3, &fail);
    tile[(e.pos >> 3) * kRowBytes + eb * 24 + 3 * (e.pos & 7) + ec] =
        (uint8_t)(p < 0 ? 0 : (p > 255 ? 255 : p));
  }
  if (n3) atomicAdd(&misc[1], n3);
  if (fail) atomicAdd(&misc[2], 1);
  __syncthreads();
  for (int i = t; i < 8 * kTileBlocks * 3; i += kThreads) {
    const int y = i / (kTileBlocks * 3), rem = i - y * (kTileBlocks * 3);
    const int bb = rem / 3, q = rem - 3 * bb;
    if (bb < nb)
      *reinterpret_cast<uint2*>(a.pixels_out + blk[bb] + y * w3 + 8 * q) =
          *reinterpret_cast<const uint2*>(tile + y * kRowBytes + bb * 24 + 8 * q);
  }
  tile_epilogue_counters(a, smem);
}

cudaError_t launch_restore(const TileArgs& a, cudaStream_t s) {
  const int grid = (a.nblocks + kTileBlocks - 1) / kTileBlocks;
  if (a.k == 0)
    restore_kernel<0><<<grid, kThreads, kSmemBytes, s>>>(a);
  else if (a.k == 5)
    restore_kernel<5><<<grid, kThreads, kSmemBytes, s>>>(a);
  else
    restore_kernel<-1><<<grid, kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fds
