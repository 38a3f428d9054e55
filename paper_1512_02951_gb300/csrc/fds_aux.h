// Launchers of the kernels outside the tile machinery (one translation unit each): the
// full-encryption comparator, packed-storage unpacking, image statistics and the strong
// level's SHA-512 masks.  Host code only needs <cuda_runtime.h>.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fds {

// Kernels that lay their shared memory out at fixed shared-window addresses need their dynamic
// area to start at or below max_start.  The area starts after the memory the device reserves
// for each CTA and the kernel's static shared memory (128-byte aligned); this checks that on
// the current device (the kernels check it again and, should it ever fail there, count a
// failure and do nothing).
template <typename Kernel>
inline cudaError_t smem_window_start_ok(Kernel kernel, uint32_t max_start) {
  int dev = 0, reserved = 0;
  cudaFuncAttributes fa{};
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
  const size_t start = (size_t)reserved + ((fa.sharedSizeBytes + 127) & ~(size_t)127);
  return start <= max_start ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// AES-128-CTR over a whole buffer (the full-encryption comparator); counters: the device's
// three counters (the failure counter records a launch that could not place its table)
cudaError_t launch_aes_full(const uint8_t* in, uint8_t* out, uint64_t bytes, uint64_t iv_hi, uint64_t iv_lo,
                            const uint32_t rk[44], const uint32_t* T, cudaStream_t s, int sms,
                            unsigned long long* counters);
// histogram and adjacent-pair sums of an H x W x 3 image (hist [3][256], sums [3][3][6],
// both zero on entry)
cudaError_t launch_image_stats(const uint8_t* img, int width, int height, unsigned long long* hist, long long* sums,
                               cudaStream_t s, int sms);
// strong level: out = in XOR (per channel-block SHA-512 of its Part 1 plaintext, [ncb][k+1]
// int16); the constants are uploaded once per device by upload_sha512_constants
cudaError_t launch_strong_mask(const uint8_t* plain, const uint8_t* in, uint8_t* out, int width, int height, int k,
                               cudaStream_t s);
cudaError_t upload_sha512_constants();
void sha512_constants(uint64_t k[80], uint64_t h0[8]);
// the DWT scheme: per 8x8 block of an H x W byte matrix, level 1 (5 bytes, AES-CTR), level 2
// (16 bytes, SHA-256 masked), level 3 (60 bytes, SHA-512 masked); constants uploaded once per
// device by upload_dwt_constants
cudaError_t launch_dwt_protect(const uint8_t* data, int width, int height, const uint8_t key[16],
                               const uint8_t iv[16], const uint32_t rk[44], const uint32_t* T, uint8_t* l1,
                               uint8_t* l2, uint8_t* l3, cudaStream_t s);
cudaError_t launch_dwt_restore(const uint8_t* l1, const uint8_t* l2, const uint8_t* l3, int width, int height,
                               const uint8_t key[16], const uint8_t iv[16], const uint32_t rk[44],
                               const uint32_t* T, uint8_t* data, cudaStream_t s);
cudaError_t upload_dwt_constants();
// bit-packed storage: packed streams -> int16 fragments, w = 11 or 8 bits per AC field
// tensor-core protect / restore of one image (warp-specialised, tiles of 128 pixel blocks);
// bop: the B operand image in shared-memory byte order; the TileArgs fields of the image, keys and tables as for the other
// kernels.  k must be one of the instantiated selections (mma_supports_k).
struct TileArgs;
bool mma_supports_k(int k);
// guard: the fixed bound on the error of any pre-rounding value; guard_rem: its part that does
// not scale with the value (the kernel adds |2^13 F| 2^-37 per value)
cudaError_t launch_protect_mma(const TileArgs& t, const uint4* bop, float guard, float guard_rem, cudaStream_t s,
                               bool debug, int sms);
cudaError_t launch_unpack(const uint8_t* pub_in, const uint8_t* priv_in, int16_t* pub16, int16_t* priv16,
                          long long ncb, int k, int w, cudaStream_t s);
}  // namespace fds
