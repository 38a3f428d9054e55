// Bit-packed coefficient storage (Sect. 6.4.3, Table 5): the paper's 11-bit storage (DC
// unsigned in 11 bits, AC as a sign bit and a 10-bit magnitude) and 8-bit storage (AC as a
// sign bit and a 7-bit magnitude, saturated), for both fragments.
//
// A field of width w takes the next w bits of its stream, least significant bit first;
// stream bit b is bit b % 8 of byte b / 8.  Channel-blocks follow each other in [by][bx][c]
// order, each with its fields in fragment order.  Eight channel-blocks always end on a byte
// boundary (8 w (63 - k) and 8 (11 + k w) bits), so one thread packs or unpacks a group of
// eight channel-blocks and owns its bytes.
#include "fds_tile.cuh"

namespace fds {

constexpr int kPackThreads = 256;
constexpr int kDcBits = 11;

// field code of value v: DC unsigned; AC sign-magnitude of width w (8-bit storage saturates)
__device__ __forceinline__ uint32_t ac_code(int v, int w) {
  const uint32_t mag_max = (1u << (w - 1)) - 1u;
  uint32_t mag = (uint32_t)(v < 0 ? -v : v);
  if (mag > mag_max) mag = mag_max;
  return v < 0 ? ((1u << (w - 1)) | mag) : mag;
}

__device__ __forceinline__ int ac_value(uint32_t code, int w) {
  const int mag = (int)(code & ((1u << (w - 1)) - 1u));
  return (code >> (w - 1)) & 1u ? -mag : mag;
}

// Append a field to a byte stream: bits accumulate in acc (nbits of them), whole bytes go out.
struct BitWriter {
  uint8_t* out;
  uint64_t acc;
  int nbits;
  __device__ __forceinline__ void put(uint32_t code, int w) {
    acc |= (uint64_t)code << nbits;
    nbits += w;
    while (nbits >= 8) {
      *out++ = (uint8_t)acc;
      acc >>= 8;
      nbits -= 8;
    }
  }
  __device__ __forceinline__ void flush() {
    if (nbits > 0) *out++ = (uint8_t)acc;
    nbits = 0;
  }
};

struct BitReader {
  const uint8_t* in;
  uint64_t acc;
  int nbits;
  __device__ __forceinline__ uint32_t get(int w) {
    while (nbits < w) {
      acc |= (uint64_t)(*in++) << nbits;
      nbits += 8;
    }
    const uint32_t code = (uint32_t)(acc & ((1ull << w) - 1ull));
    acc >>= w;
    nbits -= w;
    return code;
  }
};

// int16 fragments ([ncb][63 - k] public, [ncb][k + 1] private plaintext) -> packed streams
__global__ void __launch_bounds__(kPackThreads) pack_kernel(const int16_t* pub16, const int16_t* priv16,
                                                            uint8_t* pub_out, uint8_t* priv_out, long long ncb,
                                                            int k, int w) {
  const long long g = (long long)blockIdx.x * kPackThreads + threadIdx.x;
  const long long c0 = 8 * g;
  if (c0 >= ncb) return;
  const int n = (int)min(8ll, ncb - c0);
  const int npub = 63 - k;
  if (npub > 0) {
    BitWriter bw{pub_out + g * (long long)(npub * w), 0, 0};
    const int16_t* src = pub16 + c0 * npub;
    for (int i = 0; i < n * npub; ++i) bw.put(ac_code(src[i], w), w);
    bw.flush();
  }
  BitWriter bv{priv_out + g * (long long)(kDcBits + k * w), 0, 0};
  const int16_t* src = priv16 + c0 * (k + 1);
  for (int c = 0; c < n; ++c) {
    bv.put((uint32_t)src[c * (k + 1)] & 0x7ffu, kDcBits);
    for (int z = 1; z <= k; ++z) bv.put(ac_code(src[c * (k + 1) + z], w), w);
  }
  bv.flush();
}

// packed streams -> int16 fragments
__global__ void __launch_bounds__(kPackThreads) unpack_kernel(const uint8_t* pub_in, const uint8_t* priv_in,
                                                              int16_t* pub16, int16_t* priv16, long long ncb, int k,
                                                              int w) {
  const long long g = (long long)blockIdx.x * kPackThreads + threadIdx.x;
  const long long c0 = 8 * g;
  if (c0 >= ncb) return;
  const int n = (int)min(8ll, ncb - c0);
  const int npub = 63 - k;
  if (npub > 0) {
    BitReader br{pub_in + g * (long long)(npub * w), 0, 0};
    int16_t* dst = pub16 + c0 * npub;
    for (int i = 0; i < n * npub; ++i) dst[i] = (int16_t)ac_value(br.get(w), w);
  }
  BitReader bv{priv_in + g * (long long)(kDcBits + k * w), 0, 0};
  int16_t* dst = priv16 + c0 * (k + 1);
  for (int c = 0; c < n; ++c) {
    dst[c * (k + 1)] = (int16_t)bv.get(kDcBits);
    for (int z = 1; z <= k; ++z) dst[c * (k + 1) + z] = (int16_t)ac_value(bv.get(w), w);
  }
}

cudaError_t launch_pack(const int16_t* pub16, const int16_t* priv16, uint8_t* pub_out, uint8_t* priv_out,
                        long long ncb, int k, int w, cudaStream_t s) {
  const long long groups = (ncb + 7) / 8;
  const unsigned grid = (unsigned)((groups + kPackThreads - 1) / kPackThreads);
  if (grid) pack_kernel<<<grid, kPackThreads, 0, s>>>(pub16, priv16, pub_out, priv_out, ncb, k, w);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t* pub_in, const uint8_t* priv_in, int16_t* pub16, int16_t* priv16,
                          long long ncb, int k, int w, cudaStream_t s) {
  const long long groups = (ncb + 7) / 8;
  const unsigned grid = (unsigned)((groups + kPackThreads - 1) / kPackThreads);
  if (grid) unpack_kernel<<<grid, kPackThreads, 0, s>>>(pub_in, priv_in, pub16, priv16, ncb, k, w);
  return cudaGetLastError();
}

}  // namespace fds
