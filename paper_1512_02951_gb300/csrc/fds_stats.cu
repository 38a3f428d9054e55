// Statistics of an RGB image used to judge a protected image (Sect. 6.6): the histogram of
// every channel (Sect. 6.6.1) and, for the correlation coefficient of adjacent pixels
// (Sect. 6.6.2), exact integer sums over every pair of a pixel and its right, lower and
// lower-right neighbour: n, sum x, sum y, sum x^2, sum y^2, sum x y per direction and channel.
//
// Persistent CTAs over the pixel rows; 384 threads (a multiple of 3), so a thread always sees
// the same channel of the interleaved row.  Per-thread 64-bit accumulators and a shared
// histogram, reduced per CTA in shared memory and added to the device outputs with atomics.
#include "fds_tile.cuh"
#include "fds_aux.h"

namespace fds {

constexpr int kStatThreads = 384;

__global__ void __launch_bounds__(kStatThreads) image_stats_kernel(const uint8_t* __restrict__ img, int width,
                                                                   int height, unsigned long long* hist,
                                                                   long long* sums) {
  __shared__ unsigned int sh_hist[3 * 256];
  __shared__ unsigned long long sh_sums[3 * 3 * 5];   // [direction][channel][sum]
  const int t = threadIdx.x;
  for (int i = t; i < 3 * 256; i += kStatThreads) sh_hist[i] = 0;
  if (t < 45) sh_sums[t] = 0;
  __syncthreads();
  const int c = t % 3;
  const long long w3 = 3ll * width;
  unsigned long long acc[3][5] = {};
  for (int y = blockIdx.x; y < height; y += gridDim.x) {
    const uint8_t* row = img + (long long)y * w3;
    const uint8_t* next = row + w3;
    const bool down = y + 1 < height;
    for (long long i = t; i < w3; i += kStatThreads) {
      const unsigned int p = row[i];
      atomicAdd(&sh_hist[c * 256 + p], 1u);
      const bool right = i + 3 < w3;
      unsigned int q[3];
      bool has[3] = {right, down, down && right};
      q[0] = right ? row[i + 3] : 0u;
      q[1] = down ? next[i] : 0u;
      q[2] = has[2] ? next[i + 3] : 0u;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (has[d]) {
          acc[d][0] += p;
          acc[d][1] += q[d];
          acc[d][2] += p * p;
          acc[d][3] += q[d] * q[d];
          acc[d][4] += p * q[d];
        }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int j = 0; j < 5; ++j)
      if (acc[d][j]) atomicAdd(&sh_sums[(d * 3 + c) * 5 + j], acc[d][j]);
  __syncthreads();
  for (int i = t; i < 3 * 256; i += kStatThreads)
    if (sh_hist[i]) atomicAdd(&hist[i], (unsigned long long)sh_hist[i]);
  if (t < 45) {
    const int d = t / 15, cc = (t / 5) % 3, j = t % 5;
    if (sh_sums[t])
      atomicAdd(reinterpret_cast<unsigned long long*>(sums) + (d * 3 + cc) * 6 + 1 + j, sh_sums[t]);
  }
  if (blockIdx.x == 0 && t < 9) {   // pair counts: (W - 1) H, W (H - 1), (W - 1)(H - 1)
    const int d = t / 3;
    const long long wn = d == 1 ? width : width - 1, hn = d == 0 ? height : height - 1;
    sums[t * 6] = wn * hn;
  }
}

// hist [3][256] and sums [3][3][6] must be zero on entry (the caller clears them on s)
cudaError_t launch_image_stats(const uint8_t* img, int width, int height, unsigned long long* hist, long long* sums,
                               cudaStream_t s, int sms) {
  const int grid = height < 4 * sms ? height : 4 * sms;
  if (grid > 0) image_stats_kernel<<<grid, kStatThreads, 0, s>>>(img, width, height, hist, sums);
  return cudaGetLastError();
}

}  // namespace fds
