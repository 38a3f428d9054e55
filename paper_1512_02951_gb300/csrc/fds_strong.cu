// Strong level of protection (Sect. 6.3.2, Fig. 8; Fig. 7 (d)): the public image of every
// channel-block is XORed with the SHA-512 digest of the block's selected coefficients (Part 1:
// k + 1 int16 little-endian, plaintext), digest byte 8 y + x onto pixel (y, x) of the block --
// 512 bits for 64 pixels.  The XOR is its own inverse, so the same kernel masks and unmasks.
//
// SHA-512 (fds_sha.cuh) is written from FIPS 180-4; its constants (the first 64 fraction bits
// of the cube roots of the first 80 primes and of the square roots of the first 8) are
// computed here on the host with exact integer roots and uploaded once per device.  One
// thread per channel-block; the message of a channel-block (2 (k + 1) bytes) takes one
// 1024-bit block up to k = 54, two beyond.
#include "fds_tile.cuh"
#include "fds_aux.h"
#include "fds_sha.cuh"

namespace fds {

constexpr int kMaskThreads = 128;

// padded message byte m of the L-byte message msg (one or two 128-byte blocks)
__device__ __forceinline__ uint32_t msg_byte(const uint8_t* msg, int L, int m, int nblk) {
  if (m < L) return msg[m];
  if (m == L) return 0x80u;
  const int end = 128 * nblk;                // the last 16 bytes: the bit length, big-endian
  if (m >= end - 8) {
    const uint64_t bits = 8ull * (uint64_t)L;
    return (uint32_t)(bits >> (8 * (end - 1 - m))) & 0xffu;
  }
  return 0u;
}

// SHA-512 of the L-byte message at msg (L <= 128 - 17 + 128); digest words in h
template <int K>
__device__ __forceinline__ void sha512_part1(const uint8_t* msg, int k, uint64_t (&h)[8]) {
  const int L = 2 * ((K >= 0 ? K : k) + 1);
  const int nblk = L + 17 <= 128 ? 1 : 2;
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = c_sha512_h0[i];
  for (int blk = 0; blk < nblk; ++blk) {
    uint64_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      uint64_t x = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) x = (x << 8) | msg_byte(msg, L, 128 * blk + 8 * i + b, nblk);
      w[i] = x;
    }
    sha512_compress(h, w);
  }
}

// out = in XOR mask for every channel-block (in may equal out); plain: [ncb][k + 1] int16
template <int K>
__global__ void __launch_bounds__(kMaskThreads) strong_mask_kernel(const uint8_t* __restrict__ plain,
                                                                   const uint8_t* in, uint8_t* out, int width,
                                                                   int bx_count, long long ncb, int k) {
  const long long cb = (long long)blockIdx.x * kMaskThreads + threadIdx.x;
  if (cb >= ncb) return;
  const int L = 2 * ((K >= 0 ? K : k) + 1);
  uint64_t h[8];
  sha512_part1<K>(plain + cb * L, k, h);
  const long long blk = cb / 3;
  const int c = (int)(cb - 3 * blk);
  const long long by = blk / bx_count, bx = blk - by * bx_count;
  const long long base = ((8 * by) * (long long)width + 8 * bx) * 3 + c;
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    const long long row = base + (long long)y * width * 3;
#pragma unroll
    for (int x = 0; x < 8; ++x)   // digest bytes 8 y .. 8 y + 7 are word y, most significant first
      out[row + 3 * x] = in[row + 3 * x] ^ (uint8_t)(h[y] >> (8 * (7 - x)));
  }
}

cudaError_t launch_strong_mask(const uint8_t* plain, const uint8_t* in, uint8_t* out, int width, int height, int k,
                               cudaStream_t s) {
  const int bxc = width / 8;
  const long long ncb = 3ll * bxc * (height / 8);
  const long long grid = (ncb + kMaskThreads - 1) / kMaskThreads;
  if (grid == 0) return cudaSuccess;
  if (k == 5)
    strong_mask_kernel<5><<<(unsigned)grid, kMaskThreads, 0, s>>>(plain, in, out, width, bxc, ncb, k);
  else if (k == 0)
    strong_mask_kernel<0><<<(unsigned)grid, kMaskThreads, 0, s>>>(plain, in, out, width, bxc, ncb, k);
  else
    strong_mask_kernel<-1><<<(unsigned)grid, kMaskThreads, 0, s>>>(plain, in, out, width, bxc, ncb, k);
  return cudaGetLastError();
}

// ---- the constants, from their definition: floor(frac(p^(1/e)) 2^64) for prime p
namespace {

struct U256 {
  uint64_t w[4];   // little-endian limbs
};

// a * b for a < 2^128, b < 2^128
U256 mul128(unsigned __int128 a, unsigned __int128 b) {
  const uint64_t al[2] = {(uint64_t)a, (uint64_t)(a >> 64)}, bl[2] = {(uint64_t)b, (uint64_t)(b >> 64)};
  U256 r{};
  for (int i = 0; i < 2; ++i) {
    unsigned __int128 carry = 0;
    for (int j = 0; j < 2; ++j) {
      const unsigned __int128 cur = (unsigned __int128)al[i] * bl[j] + r.w[i + j] + carry;
      r.w[i + j] = (uint64_t)cur;
      carry = cur >> 64;
    }
    r.w[i + 2] += (uint64_t)carry;
  }
  return r;
}

// a * b for a < 2^256 (result assumed < 2^256), b < 2^64
U256 mul_small(const U256& a, uint64_t b) {
  U256 r{};
  unsigned __int128 carry = 0;
  for (int i = 0; i < 4; ++i) {
    const unsigned __int128 cur = (unsigned __int128)a.w[i] * b + carry;
    r.w[i] = (uint64_t)cur;
    carry = cur >> 64;
  }
  return r;
}

bool le(const U256& a, const U256& b) {
  for (int i = 3; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return true;
}

// floor(p^(1/e) 2^64) mod 2^64, e = 2 or 3: the largest r with r^e <= p 2^(64 e)
uint64_t root_fraction(uint64_t p, int e) {
  U256 n{};
  n.w[e] = p;                                   // p 2^(64 e)
  unsigned __int128 lo = 0, hi = (unsigned __int128)1 << 72;   // p < 2^9: the root is < 2^(64 + 3)
  while (hi - lo > 1) {
    const unsigned __int128 mid = (lo + hi) >> 1;
    U256 pw = mul128(mid, mid);                 // < 2^144
    if (e == 3) {                               // mid^3 = mid^2 * mid, mid < 2^72: two steps
      const U256 lo_part = mul_small(pw, (uint64_t)mid);
      const U256 hi_part = mul_small(pw, (uint64_t)(mid >> 64));
      U256 sum = lo_part;
      unsigned __int128 carry = 0;
      for (int i = 1; i < 4; ++i) {
        const unsigned __int128 cur = (unsigned __int128)sum.w[i] + hi_part.w[i - 1] + carry;
        sum.w[i] = (uint64_t)cur;
        carry = cur >> 64;
      }
      pw = sum;
    }
    if (le(pw, n))
      lo = mid;
    else
      hi = mid;
  }
  return (uint64_t)lo;
}

}  // namespace

void sha512_constants(uint64_t k[80], uint64_t h0[8]) {
  int found = 0;
  for (uint64_t p = 2; found < 80; ++p) {
    bool prime = true;
    for (uint64_t q = 2; q * q <= p; ++q)
      if (p % q == 0) {
        prime = false;
        break;
      }
    if (!prime) continue;
    k[found] = root_fraction(p, 3);
    if (found < 8) h0[found] = root_fraction(p, 2);
    ++found;
  }
}

cudaError_t upload_sha512_constants() { return upload_sha_tables(); }

}  // namespace fds
