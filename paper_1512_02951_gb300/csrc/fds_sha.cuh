// SHA-256 and SHA-512 compression functions written from FIPS 180-4, for the strong level and
// the DWT scheme.  Each translation unit that includes this header holds its own copy of the
// round constants in constant memory and uploads it with upload_sha_tables() (the constants
// come from sha512_constants(), which computes them from their definition; the SHA-256 ones
// are the first 32 of those fraction bits).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fds_aux.h"

namespace fds {

static __constant__ uint64_t c_sha512_k[80];
static __constant__ uint64_t c_sha512_h0[8];
static __constant__ uint32_t c_sha256_k[64];
static __constant__ uint32_t c_sha256_h0[8];

__device__ __forceinline__ uint64_t rotr64(uint64_t x, int n) { return (x >> n) | (x << (64 - n)); }
__device__ __forceinline__ uint32_t rotr32(uint32_t x, int n) { return __funnelshift_r(x, x, n); }

// SHA-512 rounds R0..79 of one compression on the working variables v = (a, .., h) entering
// round R0, with the 16 big-endian message words w (all 16 are needed for the schedule).  The
// rounds run as passes of 16 (the schedule ring index is then fixed in each unrolled round, and
// the code stays small enough for the instruction cache).
template <int R0 = 0>
__device__ __forceinline__ void sha512_rounds(uint64_t (&v)[8], uint64_t (&w)[16]) {
  uint64_t a = v[0], b = v[1], c = v[2], d = v[3], e = v[4], f = v[5], g = v[6], hh = v[7];
  auto round = [&](int t, uint64_t wt) {
    const uint64_t S1 = rotr64(e, 14) ^ rotr64(e, 18) ^ rotr64(e, 41);
    const uint64_t ch = (e & f) ^ (~e & g);
    const uint64_t t1 = hh + S1 + ch + c_sha512_k[t] + wt;
    const uint64_t S0 = rotr64(a, 28) ^ rotr64(a, 34) ^ rotr64(a, 39);
    const uint64_t maj = (a & b) ^ (a & c) ^ (b & c);
    const uint64_t t2 = S0 + maj;
    hh = g;
    g = f;
    f = e;
    e = d + t1;
    d = c;
    c = b;
    b = a;
    a = t1 + t2;
  };
  // from round 0 the first pass is the loop's (one copy of the body); from a later round it
  // is unrolled ahead of the loop
  if constexpr (R0 > 0) {
#pragma unroll
    for (int j = R0; j < 16; ++j) round(j, w[j]);
  }
#pragma unroll 1
  for (int t0 = R0 > 0 ? 16 : 0; t0 < 80; t0 += 16) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (t0 > 0) {   // w[t] = sigma1(w[t-2]) + w[t-7] + sigma0(w[t-15]) + w[t-16], in the ring
        const uint64_t x15 = w[(j + 1) & 15], x2 = w[(j + 14) & 15];
        const uint64_t s0 = rotr64(x15, 1) ^ rotr64(x15, 8) ^ (x15 >> 7);
        const uint64_t s1 = rotr64(x2, 19) ^ rotr64(x2, 61) ^ (x2 >> 6);
        w[j] += s0 + w[(j + 9) & 15] + s1;
      }
      round(t0 + j, w[j]);
    }
  }
  v[0] = a;
  v[1] = b;
  v[2] = c;
  v[3] = d;
  v[4] = e;
  v[5] = f;
  v[6] = g;
  v[7] = hh;
}

// one SHA-512 compression of the 16 big-endian words w into state h
__device__ __forceinline__ void sha512_compress(uint64_t (&h)[8], uint64_t (&w)[16]) {
  uint64_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = h[i];
  sha512_rounds<0>(v, w);
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] += v[i];
}

// SHA-256 rounds R0..63 on the working variables v entering round R0 (as sha512_rounds)
template <int R0 = 0>
__device__ __forceinline__ void sha256_rounds(uint32_t (&v)[8], uint32_t (&w)[16]) {
  uint32_t a = v[0], b = v[1], c = v[2], d = v[3], e = v[4], f = v[5], g = v[6], hh = v[7];
  auto round = [&](int t, uint32_t wt) {
    const uint32_t S1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
    const uint32_t ch = (e & f) ^ (~e & g);
    const uint32_t t1 = hh + S1 + ch + c_sha256_k[t] + wt;
    const uint32_t S0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
    const uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
    const uint32_t t2 = S0 + maj;
    hh = g;
    g = f;
    f = e;
    e = d + t1;
    d = c;
    c = b;
    b = a;
    a = t1 + t2;
  };
  if constexpr (R0 > 0) {
#pragma unroll
    for (int j = R0; j < 16; ++j) round(j, w[j]);
  }
#pragma unroll 1
  for (int t0 = R0 > 0 ? 16 : 0; t0 < 64; t0 += 16) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (t0 > 0) {
        const uint32_t x15 = w[(j + 1) & 15], x2 = w[(j + 14) & 15];
        const uint32_t s0 = rotr32(x15, 7) ^ rotr32(x15, 18) ^ (x15 >> 3);
        const uint32_t s1 = rotr32(x2, 17) ^ rotr32(x2, 19) ^ (x2 >> 10);
        w[j] += s0 + w[(j + 9) & 15] + s1;
      }
      round(t0 + j, w[j]);
    }
  }
  v[0] = a;
  v[1] = b;
  v[2] = c;
  v[3] = d;
  v[4] = e;
  v[5] = f;
  v[6] = g;
  v[7] = hh;
}

// one SHA-256 compression of the 16 big-endian words w into state h
__device__ __forceinline__ void sha256_compress(uint32_t (&h)[8], uint32_t (&w)[16]) {
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = h[i];
  sha256_rounds<0>(v, w);
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] += v[i];
}

// this translation unit's copy of the constants, to the current device
static cudaError_t upload_sha_tables() {
  uint64_t k[80], h0[8];
  sha512_constants(k, h0);
  uint32_t k32[64], h32[8];
  for (int i = 0; i < 64; ++i) k32[i] = (uint32_t)(k[i] >> 32);
  for (int i = 0; i < 8; ++i) h32[i] = (uint32_t)(h0[i] >> 32);
  cudaError_t e = cudaMemcpyToSymbol(c_sha512_k, k, sizeof(k));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sha512_h0, h0, sizeof(h0));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sha256_k, k32, sizeof(k32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sha256_h0, h32, sizeof(h32));
  return e;
}

}  // namespace fds
