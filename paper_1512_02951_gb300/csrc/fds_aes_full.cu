// Full encryption, the paper's comparator for selective encryption (Sect. 6.5, Tables 7, 9,
// 11: the whole bitmap encrypted with AES): AES-128-CTR over an entire byte buffer.
//
// One thread per 16-byte block, grid-stride over the buffer: the block is read with one
// 16-byte load, XORed with AES_K(IV + i) and written with one 16-byte store (coalesced).
// With one block per thread and every thread in the AES, the T-table lookups would be
// shared-memory bound by bank conflicts, so the table is replicated per bank (32 KB per CTA,
// filled once by the persistent CTAs).  The round keys sit in the kernel's parameter space.
// A trailing partial block is handled byte by byte.
#include "fds_tile.cuh"
#include "fds_aux.h"

namespace fds {

constexpr int kFullThreads = 512;
constexpr int kTrepWords = 256 * 32;   // T0 replicated: entry x of copy L at word 32 x + L

struct FullArgs {
  const uint8_t* in;
  uint8_t* out;
  uint64_t bytes;
  uint64_t iv_hi, iv_lo;
  const uint32_t* T;
  uint32_t rk[44];
};

// AES-128 with one T-table, T0, replicated 32 times in shared memory: lane L always reads
// copy L, i.e. bank L, so a warp's 32 lookups never conflict.  Tl = the table's byte address
// plus 4 * lane (entry x of the lane's copy at Tl + 128 x).  T_r[x] = rotl(T0[x], 8 r) by
// byte permutes; S[x] is byte 1 of T0[x] (last round).
__device__ __forceinline__ void aes128_encrypt_rep(uint32_t (&s)[4], const uint32_t* rk, const char* Tl) {
  auto l0 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tl + ((w << 7) & 0x7f80u)); };
  auto l1 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tl + ((w >> 1) & 0x7f80u)); };
  auto l2 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tl + ((w >> 9) & 0x7f80u)); };
  auto l3 = [&](uint32_t w) { return *reinterpret_cast<const uint32_t*>(Tl + ((w >> 17) & 0x7f80u)); };
  auto r8 = [](uint32_t x) { return __byte_perm(x, x, 0x2103u); };
  auto r16 = [](uint32_t x) { return __byte_perm(x, x, 0x1032u); };
  auto r24 = [](uint32_t x) { return __byte_perm(x, x, 0x0321u); };
  uint32_t s0 = s[0] ^ rk[0], s1 = s[1] ^ rk[1], s2 = s[2] ^ rk[2], s3 = s[3] ^ rk[3];
#pragma unroll 1
  for (int r = 1; r < 10; ++r) {
    const uint32_t n0 = l0(s0) ^ r8(l1(s1)) ^ r16(l2(s2)) ^ r24(l3(s3)) ^ rk[4 * r];
    const uint32_t n1 = l0(s1) ^ r8(l1(s2)) ^ r16(l2(s3)) ^ r24(l3(s0)) ^ rk[4 * r + 1];
    const uint32_t n2 = l0(s2) ^ r8(l1(s3)) ^ r16(l2(s0)) ^ r24(l3(s1)) ^ rk[4 * r + 2];
    const uint32_t n3 = l0(s3) ^ r8(l1(s0)) ^ r16(l2(s1)) ^ r24(l3(s2)) ^ rk[4 * r + 3];
    s0 = n0;
    s1 = n1;
    s2 = n2;
    s3 = n3;
  }
  s[0] = (__byte_perm(l0(s0), 0u, 0x4441u) | __byte_perm(l1(s1), 0u, 0x4414u) |
          __byte_perm(l2(s2), 0u, 0x4144u) | __byte_perm(l3(s3), 0u, 0x1444u)) ^ rk[40];
  s[1] = (__byte_perm(l0(s1), 0u, 0x4441u) | __byte_perm(l1(s2), 0u, 0x4414u) |
          __byte_perm(l2(s3), 0u, 0x4144u) | __byte_perm(l3(s0), 0u, 0x1444u)) ^ rk[41];
  s[2] = (__byte_perm(l0(s2), 0u, 0x4441u) | __byte_perm(l1(s3), 0u, 0x4414u) |
          __byte_perm(l2(s0), 0u, 0x4144u) | __byte_perm(l3(s1), 0u, 0x1444u)) ^ rk[42];
  s[3] = (__byte_perm(l0(s3), 0u, 0x4441u) | __byte_perm(l1(s0), 0u, 0x4414u) |
          __byte_perm(l2(s1), 0u, 0x4144u) | __byte_perm(l3(s2), 0u, 0x1444u)) ^ rk[43];
}

__global__ void __launch_bounds__(kFullThreads) aes_ctr_full_kernel(const __grid_constant__ FullArgs a) {
  extern __shared__ __align__(16) uint32_t Trep[];
  for (int i = threadIdx.x; i < kTrepWords; i += kFullThreads) Trep[i] = __ldg(a.T + (i >> 5));
  __syncthreads();
  const char* Tl = reinterpret_cast<const char*>(Trep) + 4 * (threadIdx.x & 31);
  const uint64_t nfull = a.bytes >> 4;
  const uint64_t stride = (uint64_t)gridDim.x * kFullThreads;
  for (uint64_t i = (uint64_t)blockIdx.x * kFullThreads + threadIdx.x; i < nfull; i += stride) {
    uint32_t s[4];
    ctr_block(a.iv_hi, a.iv_lo, i, s);
    aes128_encrypt_rep(s, a.rk, Tl);
    uint4 d = *reinterpret_cast<const uint4*>(a.in + 16 * i);
    d.x ^= s[0];
    d.y ^= s[1];
    d.z ^= s[2];
    d.w ^= s[3];
    *reinterpret_cast<uint4*>(a.out + 16 * i) = d;
  }
  const int tail = (int)(a.bytes & 15);
  if (tail && blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t s[4];
    ctr_block(a.iv_hi, a.iv_lo, nfull, s);
    aes128_encrypt_rep(s, a.rk, Tl);
    for (int j = 0; j < tail; ++j)
      a.out[16 * nfull + j] = a.in[16 * nfull + j] ^ (uint8_t)(s[j >> 2] >> (8 * (j & 3)));
  }
}

// `sms` = number of SMs; grid = enough CTAs for the buffer, at most 4 per SM (32 KB table each)
cudaError_t launch_aes_full(const uint8_t* in, uint8_t* out, uint64_t bytes, uint64_t iv_hi, uint64_t iv_lo,
                            const uint32_t rk[44], const uint32_t* T, cudaStream_t s, int sms) {
  static bool attr[kMaxAttrDevices];
  constexpr int kSmem = kTrepWords * 4;
  cudaError_t e = smem_attr_once(aes_ctr_full_kernel, kSmem, attr);
  if (e != cudaSuccess) return e;
  FullArgs a{};
  a.in = in;
  a.out = out;
  a.bytes = bytes;
  a.iv_hi = iv_hi;
  a.iv_lo = iv_lo;
  a.T = T;
  for (int i = 0; i < 44; ++i) a.rk[i] = rk[i];
  const uint64_t blocks = (bytes + 15) >> 4;
  const uint64_t need = (blocks + kFullThreads - 1) / kFullThreads;
  const uint64_t cap = 4ull * (uint64_t)sms;
  const unsigned grid = (unsigned)(need < cap ? (need ? need : 1) : cap);
  aes_ctr_full_kernel<<<grid, kFullThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fds
