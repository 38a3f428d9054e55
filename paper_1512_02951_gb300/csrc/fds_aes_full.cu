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

struct FullArgs {
  const uint8_t* in;
  uint8_t* out;
  uint64_t bytes;
  uint64_t iv_hi, iv_lo;
  const uint32_t* T;
  uint32_t rk[44];
};

__global__ void __launch_bounds__(kFullThreads) aes_ctr_full_kernel(const __grid_constant__ FullArgs a) {
  extern __shared__ __align__(16) uint32_t Trep[];
  for (int i = threadIdx.x; i < kTrepWords; i += kFullThreads) Trep[i] = __ldg(a.T + (i >> 5));
  __syncthreads();
  const uint32_t Tl = (uint32_t)__cvta_generic_to_shared(Trep) + 4u * (threadIdx.x & 31);
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
