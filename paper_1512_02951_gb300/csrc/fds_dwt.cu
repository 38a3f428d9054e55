// Selective encryption with the DWT (Sect. 6.8-6.12, Figs. 16-18): any data read as an H x W
// matrix of bytes, per 8x8 block a two-level reversible Le Gall 5/3 DWT by integer lifting,
//   level 1 = the second-level LL (4 coefficients), AES-128-CTR encrypted,
//   level 2 = the second-level HL, LH, HH (12), XORed with SHA-256(key, IV, block, level 1),
//   level 3 = the first-level HL, LH, HH (48), XORed with SHA-512(key, IV, block, level 2).
// Lifting (the invertible JPEG 2000 form of Eqs. 1-2): d[n] = x[2n+1] - floor((x[2n] +
// x[2n+2]) / 2), s[n] = x[2n] + floor((d[n-1] + d[n] + 2) / 4), whole-sample symmetric
// extension (x[8] = x[6], d[-1] = d[0]); rows first, then columns; input shifted by -128.
// Fields: two's complement, 10 bits (11 for the second-level HH), least significant bit
// first; per block level 1 takes 5 bytes, level 2 16 (124 bits), level 3 60.  Hashed
// messages: key || IV || block index (8 bytes, big-endian) || the previous level's packed
// plaintext; level 2 takes digest bytes 0..15, level 3 digest bytes 0..59.
//
// One thread per block, 128 blocks per CTA.  A CTA's level-1 bytes (5 per block, 640 per CTA,
// so every CTA starts on a 16-byte keystream boundary) are staged in shared memory and
// encrypted there by one thread per keystream block; level 3 is staged for coalesced stores.
// The transform and both hashes stay in registers.  Restore runs the same steps backwards.
#include "fds_tile.cuh"
#include "fds_aux.h"
#include "fds_sha.cuh"

namespace fds {

constexpr int kDwtThreads = 128;
constexpr int kL1Bytes = 5, kL2Bytes = 16, kL3Words = 15;

struct DwtArgs {
  const uint8_t* data_in;      // protect: H x W bytes
  uint8_t* data_out;           // restore
  const uint8_t* l1_in;
  const uint8_t* l2_in;
  const uint8_t* l3_in;
  uint8_t* l1_out;
  uint8_t* l2_out;
  uint8_t* l3_out;
  const uint32_t* T;           // AES T-tables (device)
  long long nblocks;
  int width, bx_count;
  uint64_t iv_hi, iv_lo;
  uint32_t kiv[8];             // key and IV as big-endian words (the hashed prefix)
  uint32_t rk[44];
  // the hashes' working variables after the rounds that read only key || IV: SHA-256 after
  // rounds 0..7 (message words 0..7), SHA-512 after rounds 0..3 (words 0..3)
  uint32_t mid256[8];
  uint64_t mid512[8];
};
constexpr int kMid256 = 8, kMid512 = 4;

// one level of lifting on 2m samples v[0], v[s], .., v[(2m-1) s] -> [low | high] in place
template <int M>
__device__ __forceinline__ void lift_fwd(int* v, int s) {
  int e[M], o[M];
#pragma unroll
  for (int n = 0; n < M; ++n) {
    e[n] = v[(2 * n) * s];
    o[n] = v[(2 * n + 1) * s];
  }
  int d[M];
#pragma unroll
  for (int n = 0; n < M; ++n) d[n] = o[n] - ((e[n] + e[n + 1 < M ? n + 1 : M - 1]) >> 1);
#pragma unroll
  for (int n = 0; n < M; ++n) {
    v[n * s] = e[n] + ((d[n > 0 ? n - 1 : 0] + d[n] + 2) >> 2);
    v[(M + n) * s] = d[n];
  }
}

template <int M>
__device__ __forceinline__ void lift_inv(int* v, int s) {
  int sl[M], d[M];
#pragma unroll
  for (int n = 0; n < M; ++n) {
    sl[n] = v[n * s];
    d[n] = v[(M + n) * s];
  }
  int e[M];
#pragma unroll
  for (int n = 0; n < M; ++n) e[n] = sl[n] - ((d[n > 0 ? n - 1 : 0] + d[n] + 2) >> 2);
#pragma unroll
  for (int n = 0; n < M; ++n) {
    v[(2 * n) * s] = e[n];
    v[(2 * n + 1) * s] = d[n] + ((e[n] + e[n + 1 < M ? n + 1 : M - 1]) >> 1);
  }
}

// two-level forward / inverse DWT of c[8][8] (row-major, c[8 y + x])
__device__ __forceinline__ void dwt_forward(int* c) {
#pragma unroll
  for (int y = 0; y < 8; ++y) lift_fwd<4>(c + 8 * y, 1);
#pragma unroll
  for (int x = 0; x < 8; ++x) lift_fwd<4>(c + x, 8);
#pragma unroll
  for (int y = 0; y < 4; ++y) lift_fwd<2>(c + 8 * y, 1);
#pragma unroll
  for (int x = 0; x < 4; ++x) lift_fwd<2>(c + x, 8);
}

__device__ __forceinline__ void dwt_inverse(int* c) {
#pragma unroll
  for (int x = 0; x < 4; ++x) lift_inv<2>(c + x, 8);
#pragma unroll
  for (int y = 0; y < 4; ++y) lift_inv<2>(c + 8 * y, 1);
#pragma unroll
  for (int x = 0; x < 8; ++x) lift_inv<4>(c + x, 8);
#pragma unroll
  for (int y = 0; y < 8; ++y) lift_inv<4>(c + 8 * y, 1);
}

// field f of a level (row-major quadrant order) -> index into c[64]
__device__ __forceinline__ constexpr int l1_pos(int f) { return 8 * (f >> 1) + (f & 1); }
__device__ __forceinline__ constexpr int l2_pos(int f) {   // 2nd HL, LH, HH
  return f < 4 ? 8 * (f >> 1) + 2 + (f & 1) : (f < 8 ? 8 * (2 + ((f - 4) >> 1)) + ((f - 4) & 1)
                                                      : 8 * (2 + ((f - 8) >> 1)) + 2 + ((f - 8) & 1));
}
__device__ __forceinline__ constexpr int l3_pos(int f) {   // 1st HL, LH, HH, 4 x 4 each
  return f < 16 ? 8 * (f >> 2) + 4 + (f & 3)
                : (f < 32 ? 8 * (4 + ((f - 16) >> 2)) + ((f - 16) & 3) : 8 * (4 + ((f - 32) >> 2)) + 4 + ((f - 32) & 3));
}
__device__ __forceinline__ constexpr int l2_width(int f) { return f < 8 ? 10 : 11; }
__device__ __forceinline__ constexpr int l2_bit(int f) { return f < 8 ? 10 * f : 80 + 11 * (f - 8); }

// append the w-bit two's complement field v at bit b of the little-endian words out[]
template <int NW>
__device__ __forceinline__ void put_field(uint32_t (&out)[NW], int b, int w, int v) {
  const uint32_t u = (uint32_t)v & ((1u << w) - 1u);
  out[b >> 5] |= u << (b & 31);
  if ((b & 31) + w > 32) out[(b >> 5) + 1] |= u >> (32 - (b & 31));
}
template <int NW>
__device__ __forceinline__ int get_field(const uint32_t (&in)[NW], int b, int w) {
  uint32_t u = in[b >> 5] >> (b & 31);
  if ((b & 31) + w > 32) u |= in[(b >> 5) + 1] << (32 - (b & 31));
  return (int)(u << (32 - w)) >> (32 - w);   // sign-extend the w-bit field
}

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0u, 0x0123u); }

// SHA-256(key || IV || block index || 5 bytes of level 1): digest as little-endian words of
// its bytes 0..15 (the level-2 mask)
__device__ __forceinline__ void mask2(const DwtArgs& a, long long b, uint64_t l1, uint32_t (&m)[4]) {
  uint32_t w[16];
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = a.kiv[i];
  w[8] = (uint32_t)((uint64_t)b >> 32);
  w[9] = (uint32_t)b;
  // bytes 40..44: level 1 (little-endian bytes of l1), then 0x80, zeros, bit length 360
  w[10] = bswap32((uint32_t)l1);
  w[11] = ((uint32_t)(l1 >> 32) & 0xffu) << 24 | 0x00800000u;
  w[12] = w[13] = w[14] = 0u;
  w[15] = 8u * (32u + 8u + 5u);
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = a.mid256[i];
  sha256_rounds<kMid256>(v, w);
#pragma unroll
  for (int i = 0; i < 4; ++i) m[i] = bswap32(c_sha256_h0[i] + v[i]);
}

// SHA-512(key || IV || block index || 16 bytes of level 2): digest bytes 0..59 as 15 words
__device__ __forceinline__ void mask3(const DwtArgs& a, long long b, const uint32_t (&l2)[4],
                                      uint32_t (&m)[kL3Words]) {
  uint64_t w[16];
#pragma unroll
  for (int i = 0; i < 4; ++i) w[i] = ((uint64_t)a.kiv[2 * i] << 32) | a.kiv[2 * i + 1];
  w[4] = (uint64_t)b;
  w[5] = ((uint64_t)bswap32(l2[0]) << 32) | bswap32(l2[1]);
  w[6] = ((uint64_t)bswap32(l2[2]) << 32) | bswap32(l2[3]);
  w[7] = 0x80ull << 56;
#pragma unroll
  for (int i = 8; i < 15; ++i) w[i] = 0;
  w[15] = 8ull * (32 + 8 + 16);
  uint64_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = a.mid512[i];
  sha512_rounds<kMid512>(v, w);
#pragma unroll
  for (int i = 0; i < kL3Words; ++i) {
    const uint64_t x = c_sha512_h0[i >> 1] + v[i >> 1];
    m[i] = bswap32((i & 1) ? (uint32_t)x : (uint32_t)(x >> 32));
  }
}

// AES-128-CTR over the CTA's level-1 bytes in shared memory (n bytes from stream offset off,
// off a multiple of 16), one thread per keystream block
__device__ __forceinline__ void ctr_l1(uint8_t* buf, int n, long long off, const DwtArgs& a, const uint32_t* Ts) {
  const int nblk = (n + 15) >> 4;
  for (int i = threadIdx.x; i < nblk; i += kDwtThreads) {
    uint32_t s[4];
    ctr_block(a.iv_hi, a.iv_lo, (uint64_t)(off >> 4) + i, s);
    aes128_encrypt(s, a.rk, Ts);
    uint4* p = reinterpret_cast<uint4*>(buf + 16 * i);
    uint4 d = *p;
    d.x ^= s[0];
    d.y ^= s[1];
    d.z ^= s[2];
    d.w ^= s[3];
    *p = d;
  }
}

__global__ void __launch_bounds__(kDwtThreads) dwt_protect_kernel(const __grid_constant__ DwtArgs a) {
  __shared__ uint32_t Ts[1024];
  __shared__ __align__(16) uint8_t l1s[kDwtThreads * kL1Bytes];
  __shared__ uint32_t l3s[kDwtThreads * kL3Words];
  const int t = threadIdx.x;
  for (int i = t; i < 1024; i += kDwtThreads) Ts[i] = a.T[i];
  const long long b0 = (long long)blockIdx.x * kDwtThreads;
  const int nvalid = (int)min((long long)kDwtThreads, a.nblocks - b0);
  const long long b = b0 + t;
  if (t < nvalid) {
    const long long by = b / a.bx_count, bx = b - by * a.bx_count;
    const uint8_t* src = a.data_in + (8 * by) * (long long)a.width + 8 * bx;
    int c[64];
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const uint2 r = *reinterpret_cast<const uint2*>(src + (long long)y * a.width);
#pragma unroll
      for (int x = 0; x < 8; ++x) c[8 * y + x] = (int)(((x < 4 ? r.x : r.y) >> (8 * (x & 3))) & 0xffu) - 128;
    }
    dwt_forward(c);
    uint64_t l1 = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) l1 |= (uint64_t)((uint32_t)c[l1_pos(f)] & 0x3ffu) << (10 * f);
    uint32_t l2[4] = {0, 0, 0, 0};
#pragma unroll
    for (int f = 0; f < 12; ++f) put_field(l2, l2_bit(f), l2_width(f), c[l2_pos(f)]);
    uint32_t l3[kL3Words];
#pragma unroll
    for (int i = 0; i < kL3Words; ++i) l3[i] = 0;
#pragma unroll
    for (int f = 0; f < 48; ++f) put_field(l3, 10 * f, 10, c[l3_pos(f)]);
#pragma unroll
    for (int q = 0; q < kL1Bytes; ++q) l1s[kL1Bytes * t + q] = (uint8_t)(l1 >> (8 * q));
    uint32_t m2[4];
    mask2(a, b, l1, m2);
    *reinterpret_cast<uint4*>(a.l2_out + kL2Bytes * b) =
        make_uint4(l2[0] ^ m2[0], l2[1] ^ m2[1], l2[2] ^ m2[2], l2[3] ^ m2[3]);
    uint32_t m3[kL3Words];
    mask3(a, b, l2, m3);
#pragma unroll
    for (int i = 0; i < kL3Words; ++i) l3s[kL3Words * t + i] = l3[i] ^ m3[i];
  }
  __syncthreads();
  const int n1 = kL1Bytes * nvalid;
  ctr_l1(l1s, n1, kL1Bytes * b0, a, Ts);
  __syncthreads();
  uint8_t* d1 = a.l1_out + kL1Bytes * b0;
  for (int i = t; i < (n1 >> 4); i += kDwtThreads)
    reinterpret_cast<uint4*>(d1)[i] = reinterpret_cast<const uint4*>(l1s)[i];
  for (int i = (n1 & ~15) + t; i < n1; i += kDwtThreads) d1[i] = l1s[i];
  uint32_t* d3 = reinterpret_cast<uint32_t*>(a.l3_out + 4ll * kL3Words * b0);
  for (int i = t; i < kL3Words * nvalid; i += kDwtThreads) d3[i] = l3s[i];
}

__global__ void __launch_bounds__(kDwtThreads) dwt_restore_kernel(const __grid_constant__ DwtArgs a) {
  __shared__ uint32_t Ts[1024];
  __shared__ __align__(16) uint8_t l1s[kDwtThreads * kL1Bytes];
  __shared__ uint32_t l3s[kDwtThreads * kL3Words];
  const int t = threadIdx.x;
  for (int i = t; i < 1024; i += kDwtThreads) Ts[i] = a.T[i];
  const long long b0 = (long long)blockIdx.x * kDwtThreads;
  const int nvalid = (int)min((long long)kDwtThreads, a.nblocks - b0);
  const int n1 = kL1Bytes * nvalid;
  const uint8_t* s1 = a.l1_in + kL1Bytes * b0;
  for (int i = t; i < (n1 >> 4); i += kDwtThreads)
    reinterpret_cast<uint4*>(l1s)[i] = reinterpret_cast<const uint4*>(s1)[i];
  for (int i = (n1 & ~15) + t; i < n1; i += kDwtThreads) l1s[i] = s1[i];
  const uint32_t* s3 = reinterpret_cast<const uint32_t*>(a.l3_in + 4ll * kL3Words * b0);
  for (int i = t; i < kL3Words * nvalid; i += kDwtThreads) l3s[i] = s3[i];
  __syncthreads();
  ctr_l1(l1s, n1, kL1Bytes * b0, a, Ts);
  __syncthreads();
  if (t >= nvalid) return;
  const long long b = b0 + t;
  uint64_t l1 = 0;
#pragma unroll
  for (int q = 0; q < kL1Bytes; ++q) l1 |= (uint64_t)l1s[kL1Bytes * t + q] << (8 * q);
  uint32_t m2[4];
  mask2(a, b, l1, m2);
  const uint4 v2 = *reinterpret_cast<const uint4*>(a.l2_in + kL2Bytes * b);
  const uint32_t l2[4] = {v2.x ^ m2[0], v2.y ^ m2[1], v2.z ^ m2[2], v2.w ^ m2[3]};
  uint32_t m3[kL3Words];
  mask3(a, b, l2, m3);
  uint32_t l3[kL3Words];
#pragma unroll
  for (int i = 0; i < kL3Words; ++i) l3[i] = l3s[kL3Words * t + i] ^ m3[i];
  int c[64];
#pragma unroll
  for (int f = 0; f < 4; ++f) c[l1_pos(f)] = (int)((uint32_t)(l1 >> (10 * f)) << 22) >> 22;
#pragma unroll
  for (int f = 0; f < 12; ++f) c[l2_pos(f)] = get_field(l2, l2_bit(f), l2_width(f));
#pragma unroll
  for (int f = 0; f < 48; ++f) c[l3_pos(f)] = get_field(l3, 10 * f, 10);
  dwt_inverse(c);
  const long long by = b / a.bx_count, bx = b - by * a.bx_count;
  uint8_t* dst = a.data_out + (8 * by) * (long long)a.width + 8 * bx;
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      lo |= (uint32_t)(c[8 * y + x] + 128) << (8 * x);
      hi |= (uint32_t)(c[8 * y + 4 + x] + 128) << (8 * x);
    }
    *reinterpret_cast<uint2*>(dst + (long long)y * a.width) = make_uint2(lo, hi);
  }
}

// The rounds of SHA-256 and SHA-512 (FIPS 180-4) that read only key || IV, the same for every
// block of a launch, run once here on the host; the kernels go on from the state they leave.
struct ShaConsts {
  uint64_t k[80], h0[8];
};
static void hash_midstates(DwtArgs& a) {
  static const ShaConsts sc = [] {
    ShaConsts c;
    sha512_constants(c.k, c.h0);
    return c;
  }();
  auto r32 = [](uint32_t x, int n) { return (x >> n) | (x << (32 - n)); };
  auto r64 = [](uint64_t x, int n) { return (x >> n) | (x << (64 - n)); };
  uint32_t v[8];
  for (int i = 0; i < 8; ++i) v[i] = (uint32_t)(sc.h0[i] >> 32);   // SHA-256's: the top 32 bits
  for (int t = 0; t < kMid256; ++t) {
    const uint32_t e = v[4], f = v[5], g = v[6], av = v[0], b = v[1], c = v[2];
    const uint32_t t1 = v[7] + (r32(e, 6) ^ r32(e, 11) ^ r32(e, 25)) + ((e & f) ^ (~e & g)) +
                        (uint32_t)(sc.k[t] >> 32) + a.kiv[t];
    const uint32_t t2 = (r32(av, 2) ^ r32(av, 13) ^ r32(av, 22)) + ((av & b) ^ (av & c) ^ (b & c));
    for (int i = 7; i > 0; --i) v[i] = v[i - 1];
    v[4] += t1;
    v[0] = t1 + t2;
  }
  for (int i = 0; i < 8; ++i) a.mid256[i] = v[i];
  uint64_t u[8];
  for (int i = 0; i < 8; ++i) u[i] = sc.h0[i];
  for (int t = 0; t < kMid512; ++t) {
    const uint64_t e = u[4], f = u[5], g = u[6], av = u[0], b = u[1], c = u[2];
    const uint64_t wt = ((uint64_t)a.kiv[2 * t] << 32) | a.kiv[2 * t + 1];
    const uint64_t t1 = u[7] + (r64(e, 14) ^ r64(e, 18) ^ r64(e, 41)) + ((e & f) ^ (~e & g)) + sc.k[t] + wt;
    const uint64_t t2 = (r64(av, 28) ^ r64(av, 34) ^ r64(av, 39)) + ((av & b) ^ (av & c) ^ (b & c));
    for (int i = 7; i > 0; --i) u[i] = u[i - 1];
    u[4] += t1;
    u[0] = t1 + t2;
  }
  for (int i = 0; i < 8; ++i) a.mid512[i] = u[i];
}

static void dwt_args(DwtArgs& a, int width, int height, const uint8_t key[16], const uint8_t iv[16],
                     const uint32_t rk[44], const uint32_t* T) {
  a.width = width;
  a.bx_count = width / 8;
  a.nblocks = (long long)(width / 8) * (height / 8);
  a.T = T;
  for (int i = 0; i < 4; ++i) {
    a.kiv[i] = (uint32_t)key[4 * i] << 24 | (uint32_t)key[4 * i + 1] << 16 | (uint32_t)key[4 * i + 2] << 8 | key[4 * i + 3];
    a.kiv[4 + i] = (uint32_t)iv[4 * i] << 24 | (uint32_t)iv[4 * i + 1] << 16 | (uint32_t)iv[4 * i + 2] << 8 | iv[4 * i + 3];
  }
  a.iv_hi = ((uint64_t)a.kiv[4] << 32) | a.kiv[5];
  a.iv_lo = ((uint64_t)a.kiv[6] << 32) | a.kiv[7];
  for (int i = 0; i < 44; ++i) a.rk[i] = rk[i];
  hash_midstates(a);
}

cudaError_t launch_dwt_protect(const uint8_t* data, int width, int height, const uint8_t key[16],
                               const uint8_t iv[16], const uint32_t rk[44], const uint32_t* T, uint8_t* l1,
                               uint8_t* l2, uint8_t* l3, cudaStream_t s) {
  DwtArgs a{};
  dwt_args(a, width, height, key, iv, rk, T);
  a.data_in = data;
  a.l1_out = l1;
  a.l2_out = l2;
  a.l3_out = l3;
  const long long grid = (a.nblocks + kDwtThreads - 1) / kDwtThreads;
  if (grid > 0) dwt_protect_kernel<<<(unsigned)grid, kDwtThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dwt_restore(const uint8_t* l1, const uint8_t* l2, const uint8_t* l3, int width, int height,
                               const uint8_t key[16], const uint8_t iv[16], const uint32_t rk[44],
                               const uint32_t* T, uint8_t* data, cudaStream_t s) {
  DwtArgs a{};
  dwt_args(a, width, height, key, iv, rk, T);
  a.l1_in = l1;
  a.l2_in = l2;
  a.l3_in = l3;
  a.data_out = data;
  const long long grid = (a.nblocks + kDwtThreads - 1) / kDwtThreads;
  if (grid > 0) dwt_restore_kernel<<<(unsigned)grid, kDwtThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t upload_dwt_constants() { return upload_sha_tables(); }

}  // namespace fds
