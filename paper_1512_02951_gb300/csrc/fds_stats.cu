// Statistics of an RGB image used to judge a protected image (Sect. 6.6): the histogram of
// every channel (Sect. 6.6.1) and, for the correlation coefficient of adjacent pixels
// (Sect. 6.6.2), exact integer sums over every pair of a pixel and its right, lower and
// lower-right neighbour: n, sum x, sum y, sum x^2, sum y^2, sum x y per direction and channel.
//
// Two launches.  The first streams the image once: CTAs take chunks of 2048 pixels of a row,
// stage that chunk of the row and of the next row in shared memory (16-byte loads where
// aligned), and every thread walks 16 consecutive pixels of one channel, accumulating the
// histogram (equal neighbours merged into one shared-memory atomic), sum p, sum p^2 and the
// three neighbour products, and the sums of p and p^2 over the first and last rows and
// columns.  The per-direction sums of x, y, x^2, y^2 differ from the image totals only by
// those borders, so the second launch (one warp) writes the 54 pair sums from them.
#include "fds_tile.cuh"
#include "fds_aux.h"

namespace fds {

constexpr int kStatThreads = 384;                 // 128 pixel groups x 3 channels
constexpr int kGroupPx = 16;                      // consecutive pixels per thread
constexpr int kChunkPx = kGroupPx * (kStatThreads / 3);   // 2048 pixels of a row per chunk
constexpr int kChunkBytes = 3 * kChunkPx + 32;    // + the next pixel and a 16-byte skew

// totals[c][j], j: sum p, sum p^2, sum p * right, sum p * down, sum p * down-right; then
// borders[c][j], j: first row p, p^2; last row p, p^2; first column p, p^2; last column p, p^2
// (entries 0..14 and 15..38 of the output pair sums until the second launch)
__global__ void __launch_bounds__(kStatThreads) image_stats_kernel(const uint8_t* __restrict__ img, int width,
                                                                   int height, unsigned long long* hist,
                                                                   unsigned long long* totals) {
  __shared__ __align__(16) uint8_t rows[2][kChunkBytes];
  __shared__ unsigned int sh_hist[3 * 256];
  __shared__ unsigned long long sh_tot[15 + 24];
  const int t = threadIdx.x;
  for (int i = t; i < 3 * 256; i += kStatThreads) sh_hist[i] = 0;
  if (t < 39) sh_tot[t] = 0;
  const int c = t % 3, g = t / 3;
  const long long w3 = 3ll * width;
  const int nchunks = (width + kChunkPx - 1) / kChunkPx;
  const long long items = (long long)height * nchunks;
  unsigned long long acc[5] = {0, 0, 0, 0, 0};
  unsigned long long* bord = sh_tot + 15 + 8 * c;   // border sums: rare, straight to shared memory
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int y = (int)(item / nchunks);
    const int x0 = (int)(item - (long long)y * nchunks) * kChunkPx;
    const int npx = min(kChunkPx, width - x0);
    const bool down = y + 1 < height;
    const int nbytes = 3 * min(npx + 1, width - x0);        // the chunk and its right neighbour
    __syncthreads();                                         // the previous chunk is read
    // byte k of a row's chunk goes to rows[r][skew + k], skew = the source's offset from a
    // 16-byte boundary, so the middle moves as aligned 16-byte loads and stores
    int skew[2] = {0, 0};
    for (int r = 0; r < (down ? 2 : 1); ++r) {
      const uint8_t* src = img + (long long)(y + r) * w3 + 3ll * x0;
      skew[r] = (int)(reinterpret_cast<uintptr_t>(src) & 15);
      uint8_t* dst = rows[r] + skew[r];
      const int h = min((16 - skew[r]) & 15, nbytes);
      for (int i = t; i < h; i += kStatThreads) dst[i] = src[i];
      const int n16 = (nbytes - h) >> 4;
      for (int i = t; i < n16; i += kStatThreads)
        *reinterpret_cast<uint4*>(dst + h + 16 * i) = *reinterpret_cast<const uint4*>(src + h + 16 * i);
      for (int i = h + 16 * n16 + t; i < nbytes; i += kStatThreads) dst[i] = src[i];
    }
    __syncthreads();
    const uint8_t* r0 = rows[0] + skew[0];
    const uint8_t* r1 = rows[1] + skew[1];
    uint32_t s[5] = {0, 0, 0, 0, 0};
    unsigned int run_v = 0, run_n = 0;
    const int xa = kGroupPx * g;
#pragma unroll 4
    for (int j = 0; j < kGroupPx; ++j) {
      const int x = xa + j;
      if (x >= npx) break;
      const int i = 3 * x + c;
      const uint32_t p = r0[i];
      if (p == run_v) {
        ++run_n;
      } else {
        if (run_n) atomicAdd(&sh_hist[c * 256 + run_v], run_n);
        run_v = p;
        run_n = 1;
      }
      const bool right = x0 + x + 1 < width;
      s[0] += p;
      s[1] += p * p;
      if (right) s[2] += p * r0[i + 3];
      if (down) s[3] += p * r1[i];
      if (down && right) s[4] += p * r1[i + 3];
    }
    if (run_n) atomicAdd(&sh_hist[c * 256 + run_v], run_n);
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] += s[q];
    if (y == 0) {                                  // this thread's pixels of the first row
      atomicAdd(&bord[0], (unsigned long long)s[0]);
      atomicAdd(&bord[1], (unsigned long long)s[1]);
    }
    if (y == height - 1) {
      atomicAdd(&bord[2], (unsigned long long)s[0]);
      atomicAdd(&bord[3], (unsigned long long)s[1]);
    }
    if (x0 == 0 && g == 0) {                       // column 0
      const uint32_t p = r0[c];
      atomicAdd(&bord[4], (unsigned long long)p);
      atomicAdd(&bord[5], (unsigned long long)(p * p));
    }
    if (x0 + npx == width && g == (npx - 1) / kGroupPx) {   // column W - 1
      const uint32_t p = r0[3 * (npx - 1) + c];
      atomicAdd(&bord[6], (unsigned long long)p);
      atomicAdd(&bord[7], (unsigned long long)(p * p));
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q)
    if (acc[q]) atomicAdd(&sh_tot[c * 5 + q], acc[q]);
  __syncthreads();
  for (int i = t; i < 3 * 256; i += kStatThreads)
    if (sh_hist[i]) atomicAdd(&hist[i], (unsigned long long)sh_hist[i]);
  if (t < 39 && sh_tot[t]) atomicAdd(&totals[t], sh_tot[t]);
}

// The 54 pair sums from the totals, the border sums and the two corner pixels (one warp).
__global__ void __launch_bounds__(32) stats_finish_kernel(const uint8_t* __restrict__ img, int width, int height,
                                                          long long* sums) {
  __shared__ long long sh[39];
  const int t = threadIdx.x;
  for (int i = t; i < 39; i += 32) sh[i] = sums[i];
  __syncwarp();
  if (t < 3) {
    const int c = t;
    const long long* b = sh + 15 + 8 * c;
    const long long S1 = sh[c * 5], S2 = sh[c * 5 + 1];
    const long long FR1 = b[0], FR2 = b[1], LR1 = b[2], LR2 = b[3];
    const long long FC1 = b[4], FC2 = b[5], LC1 = b[6], LC2 = b[7];
    const long long w3 = 3ll * width;
    const long long p00 = img[c], pll = img[(long long)(height - 1) * w3 + 3ll * (width - 1) + c];
    const long long W = width, H = height;
    long long* o = sums + 6 * c;                   // [direction][channel][6]: direction stride 18
    o[0] = (W - 1) * H;                            // right
    o[1] = S1 - LC1;
    o[2] = S1 - FC1;
    o[3] = S2 - LC2;
    o[4] = S2 - FC2;
    o[5] = sh[c * 5 + 2];
    o[18] = W * (H - 1);                           // down
    o[19] = S1 - LR1;
    o[20] = S1 - FR1;
    o[21] = S2 - LR2;
    o[22] = S2 - FR2;
    o[23] = sh[c * 5 + 3];
    o[36] = (W - 1) * (H - 1);                     // down-right
    o[37] = S1 - LR1 - LC1 + pll;
    o[38] = S1 - FR1 - FC1 + p00;
    o[39] = S2 - LR2 - LC2 + pll * pll;
    o[40] = S2 - FR2 - FC2 + p00 * p00;
    o[41] = sh[c * 5 + 4];
  }
}

// hist [3][256] and sums [3][3][6] must be zero on entry (the caller clears them on s)
cudaError_t launch_image_stats(const uint8_t* img, int width, int height, unsigned long long* hist, long long* sums,
                               cudaStream_t s, int sms) {
  const long long items = (long long)height * ((width + kChunkPx - 1) / kChunkPx);
  static const int per_sm = [] {                 // resident CTAs per SM: one full wave
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, image_stats_kernel, kStatThreads, 0) != cudaSuccess ||
        n < 1)
      n = 1;
    return n;
  }();
  const long long cap = (long long)per_sm * sms;
  const int grid = (int)(items < cap ? items : cap);
  if (grid <= 0) return cudaSuccess;
  image_stats_kernel<<<grid, kStatThreads, 0, s>>>(img, width, height, hist,
                                                   reinterpret_cast<unsigned long long*>(sums));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stats_finish_kernel<<<1, 32, 0, s>>>(img, width, height, sums);
  return cudaGetLastError();
}

}  // namespace fds
