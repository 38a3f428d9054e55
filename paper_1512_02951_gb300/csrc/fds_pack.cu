// Bit-packed coefficient storage (Sect. 6.4.3, Table 5), the unpacking direction: the
// paper's 11-bit storage (DC unsigned in 11 bits, AC as a sign bit and a 10-bit magnitude) and
// 8-bit storage (AC as a sign bit and a 7-bit magnitude) back to int16 fragments.  (Packing
// happens inside the protect kernel.)
//
// A field of width w takes the next w bits of its stream, least significant bit first;
// stream bit b is bit b % 8 of byte b / 8 (so, little-endian, bit b % 32 of 32-bit word
// b / 32).  Channel-blocks follow each other in [by][bx][c] order, each with its fields in
// fragment order; the last byte is padded with zero bits.
//
// An HBM-bound streaming pass, laid out so that every thread issues its loads up front:
//   public stream  all fields have the AC width w, so 32 fields fill exactly w words: a
//                  thread unpacks words [w t, w t + w) into fields [32 t, 32 t + 32), with
//                  shifts fixed at compile time;
//   private stream the period is 11 + k w bits per channel-block: one thread per
//                  channel-block (its fields start at bit cb (11 + k w)).
// One launch does both streams: the first blocks of the grid take the public stream, the
// rest the private one.
#include "fds_tile.cuh"
#include "fds_aux.h"

namespace fds {

constexpr int kPackThreads = 256;

__device__ __forceinline__ int ac_value(uint32_t code, int w) {
  const int mag = (int)(code & ((1u << (w - 1)) - 1u));
  return (code >> (w - 1)) & 1u ? -mag : mag;
}

// 32-bit word j of a byte stream of `nbytes` bytes (bytes past the end read as zero);
// `aligned` = the stream's base is 4-byte aligned
__device__ __forceinline__ uint32_t load_word(const uint8_t* in, long long j, long long nbytes, bool aligned) {
  const long long b = 4 * j;
  if (aligned && b + 4 <= nbytes) return *reinterpret_cast<const uint32_t*>(in + b);
  uint32_t v = 0;
  for (int q = 0; q < 4; ++q)
    if (b + q < nbytes) v |= (uint32_t)in[b + q] << (8 * q);
  return v;
}

struct PackArgs {
  const uint8_t* pub;     // packed public stream, pub_bytes
  const uint8_t* priv;    // packed private stream, priv_bytes
  long long nfields;      // ncb (63 - k)
  long long ncb;
  long long pub_bytes, priv_bytes;
  int k;
  int pub_blocks;         // blocks [0, pub_blocks) take the public stream
  bool pub_aligned, priv_aligned;
};

template <int W>
__device__ __forceinline__ void unpack_public(const PackArgs& a, long long t, int16_t* pub16) {
  const long long f0 = 32 * t;
  if (f0 >= a.nfields) return;
  uint32_t word[W];
#pragma unroll
  for (int j = 0; j < W; ++j) word[j] = load_word(a.pub, W * t + j, a.pub_bytes, a.pub_aligned);
  int v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int b = W * i;
    uint32_t c = word[b >> 5] >> (b & 31);
    if ((b & 31) + W > 32) c |= word[(b >> 5) + 1] << (32 - (b & 31));
    v[i] = ac_value(c & ((1u << W) - 1u), W);
  }
  if (f0 + 32 <= a.nfields) {
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
      if (f0 + i < a.nfields) pub16[f0 + i] = (int16_t)v[i];
  }
}

// private: thread per channel-block; its fields start at bit cb (11 + k w)
__device__ __forceinline__ void unpack_private(const PackArgs& a, long long cb, int w, int16_t* priv16) {
  if (cb >= a.ncb) return;
  const long long period = kDcBits + (long long)a.k * w;
  long long pos = cb * period;
  int16_t* dst = priv16 + cb * (a.k + 1);
  for (int z = 0; z <= a.k; ++z) {
    const int fw = z == 0 ? kDcBits : w;
    const long long j = pos >> 5;
    const int sh = (int)(pos & 31);
    uint64_t x = load_word(a.priv, j, a.priv_bytes, a.priv_aligned);
    if (sh + fw > 32) x |= (uint64_t)load_word(a.priv, j + 1, a.priv_bytes, a.priv_aligned) << 32;
    const uint32_t c = (uint32_t)(x >> sh) & ((1u << fw) - 1u);
    dst[z] = (int16_t)(z == 0 ? (int)c : ac_value(c, w));
    pos += fw;
  }
}

template <int W>
__global__ void __launch_bounds__(kPackThreads) unpack_kernel(const __grid_constant__ PackArgs a, int16_t* pub16,
                                                              int16_t* priv16) {
  if ((int)blockIdx.x < a.pub_blocks)
    unpack_public<W>(a, (long long)blockIdx.x * kPackThreads + threadIdx.x, pub16);
  else
    unpack_private(a, (long long)(blockIdx.x - a.pub_blocks) * kPackThreads + threadIdx.x, W, priv16);
}

static PackArgs pack_args(const uint8_t* pub, const uint8_t* priv, long long ncb, int k, int w) {
  PackArgs a{};
  a.pub = pub;
  a.priv = priv;
  a.ncb = ncb;
  a.k = k;
  a.nfields = ncb * (63 - k);
  a.pub_bytes = (a.nfields * w + 7) / 8;
  a.priv_bytes = (ncb * (kDcBits + (long long)k * w) + 7) / 8;
  a.pub_aligned = (reinterpret_cast<uintptr_t>(pub) & 3) == 0;
  a.priv_aligned = (reinterpret_cast<uintptr_t>(priv) & 3) == 0;
  a.pub_blocks = (int)((a.nfields + 32ll * kPackThreads - 1) / (32ll * kPackThreads));
  return a;
}

// packed streams -> int16 fragments (pub16 16-byte aligned)
cudaError_t launch_unpack(const uint8_t* pub_in, const uint8_t* priv_in, int16_t* pub16, int16_t* priv16,
                          long long ncb, int k, int w, cudaStream_t s) {
  const PackArgs a = pack_args(pub_in, priv_in, ncb, k, w);
  const long long grid = a.pub_blocks + (ncb + kPackThreads - 1) / kPackThreads;
  if (grid == 0) return cudaSuccess;
  if (w == 11)
    unpack_kernel<11><<<(unsigned)grid, kPackThreads, 0, s>>>(a, pub16, priv16);
  else
    unpack_kernel<8><<<(unsigned)grid, kPackThreads, 0, s>>>(a, pub16, priv16);
  return cudaGetLastError();
}

}  // namespace fds
