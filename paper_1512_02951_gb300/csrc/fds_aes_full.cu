// Full encryption, the paper's comparator for selective encryption (Sect. 6.5, Tables 7, 9,
// 11: the whole bitmap encrypted with AES): AES-128-CTR over an entire byte buffer.
//
// One thread per 16-byte block, grid-stride over the buffer: the block is read with one
// 16-byte load, XORed with AES_K(IV + i) and written with one 16-byte store (coalesced).
// With one block per thread and every thread in the AES, the T-table lookups would be
// shared-memory bound by bank conflicts, so the table is replicated per lane: the 64 KB pair
// table of T0 and T2 at shared-window address 64 KB (aes128_encrypt_pair), filled once by
// each persistent CTA of 1024 threads, one per SM.  The round keys sit in the kernel's
// parameter space.  A trailing partial block is handled byte by byte.
#include "fds_tile.cuh"
#include "fds_aux.h"

namespace fds {

constexpr int kFullThreads = 1024;
// dynamic shared memory: enough for the window [64 KB, 128 KB) wherever the area starts below it
constexpr int kFullSmem = (int)kTpairWin + kTpairBytes;

struct FullArgs {
  const uint8_t* in;
  uint8_t* out;
  uint64_t bytes;
  uint64_t iv_hi, iv_lo;
  const uint32_t* T;
  uint32_t rk[44];
};

__global__ void __launch_bounds__(kFullThreads, 1) aes_ctr_full_kernel(const __grid_constant__ FullArgs a,
                                                                       unsigned long long* counters) {
  extern __shared__ __align__(16) uint8_t smem_full[];
  const uint32_t win0 = smem_u32(smem_full);
  if (win0 > kTpairWin) {   // the table cannot sit at its window address (never on sm_103a)
    if (threadIdx.x == 0 && counters) atomicAdd(&counters[2], 1ull);
    return;
  }
  fill_pair_table(smem_full + (kTpairWin - win0), a.T, (int)threadIdx.x, kFullThreads);
  __syncthreads();
  const PairLanes lc = pair_lanes();
  const uint64_t nfull = a.bytes >> 4;
  const uint64_t stride = (uint64_t)gridDim.x * kFullThreads;
  for (uint64_t i = (uint64_t)blockIdx.x * kFullThreads + threadIdx.x; i < nfull; i += stride) {
    uint32_t s[4];
    ctr_block(a.iv_hi, a.iv_lo, i, s);
    aes128_encrypt_pair(s, a.rk, lc);
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
    aes128_encrypt_pair(s, a.rk, lc);
    for (int j = 0; j < tail; ++j)
      a.out[16 * nfull + j] = a.in[16 * nfull + j] ^ (uint8_t)(s[j >> 2] >> (8 * (j & 3)));
  }
}

// `sms` = number of SMs; grid = enough CTAs for the buffer, at most one per SM (the 64 KB
// table and 1024 threads fill it)
cudaError_t launch_aes_full(const uint8_t* in, uint8_t* out, uint64_t bytes, uint64_t iv_hi, uint64_t iv_lo,
                            const uint32_t rk[44], const uint32_t* T, cudaStream_t s, int sms,
                            unsigned long long* counters) {
  static bool attr[kMaxAttrDevices];
  static bool window_ok[kMaxAttrDevices];
  int dev = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxAttrDevices) return cudaErrorInvalidDevice;
  if (!window_ok[dev]) {   // the pair table at window address 64 KB
    if ((e = smem_window_start_ok(aes_ctr_full_kernel, kTpairWin)) != cudaSuccess) return e;
    window_ok[dev] = true;
  }
  e = smem_attr_once(aes_ctr_full_kernel, kFullSmem, attr);
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
  const uint64_t cap = (uint64_t)sms;
  const unsigned grid = (unsigned)(need < cap ? (need ? need : 1) : cap);
  aes_ctr_full_kernel<<<grid, kFullThreads, kFullSmem, s>>>(a, counters);
  return cudaGetLastError();
}

}  // namespace fds
