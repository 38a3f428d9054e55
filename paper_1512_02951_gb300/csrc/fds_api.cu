// C ABI of the selective-protection library (include/fds.h): argument checks, key registry,
// device tables, and the launches of the fused protect / restore kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include <algorithm>

#include "fds.h"
#include "fds_tile.cuh"
#include "fds_aux.h"

namespace fds {

// Device tables (static, no allocation):
//  g_T        AES T-tables T[r][x] = rotl(T0[x], 8r), r = 0..3
//  g_cfwd     exact-coordinate weights of the forward transform: for coefficient 8u+v and
//             coordinate j, 64 signed bytes K_j(u,v,y,x) (16 words, word w = row w/2,
//             x = 4(w&1) .. +3)
//  g_cinv     the same for the inverse: for pixel 8y+x and coordinate j, the weight of the
//             coefficient at zigzag index z = 4t + byte (16 words)
//  g_counters exact-fallback counters
//  g_rk       round keys of the registered key slots (FDS_MAX_KEYS x 44 words)
// where 8 b_u(y) b_v(x) = sum_j K_j(u,v,y,x) cos(j pi/16), cos(0) = 1.
__device__ __align__(16) uint32_t g_T[1024];
__device__ __align__(16) uint32_t g_rk[FDS_MAX_KEYS * 44];
__device__ __align__(16) uint32_t g_cfwd[64 * 128];
__device__ __align__(16) uint32_t g_cinv[64 * 128];
__device__ unsigned long long g_counters[3];
//  g_tcb0/1   tensor-core B operands (basis limbs, BF16 / TF32) in shared-memory byte order
__device__ __align__(16) uint4 g_tcb0[kTcBBytesBf16 / 16];
__device__ __align__(16) uint4 g_tcb1[kTcBBytesTf32 / 16];
//  g_mma_fwd  B operand of the warp-specialised tensor-core protect (f16, three limbs, rows in
//             zigzag order), in shared-memory byte order
__device__ __align__(16) uint4 g_mma_fwd[kMmaFwdBytes / 16];
//  g_mma_inv  B operand of the tensor-core inverse transform (restore; f16, three limbs, K in
//             zigzag order), in shared-memory byte order
__device__ __align__(16) uint4 g_mma_inv[kMmaInvBytes / 16];

// The exact rounding step alone: out[i] = round half away from zero of V_i, 8 V_i =
// coords[8i] + sum_j coords[8i + j] cos(j pi/16); escalations and failures are counted like
// the fused kernels count them
__global__ void debug_exact_round_kernel(const int32_t* coords, int32_t* out, int32_t n,
                                         unsigned long long* counters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[9];
#pragma unroll
  for (int j = 0; j < 8; ++j) c[j] = coords[8 * i + j];
  c[8] = 0;
  int esc = 0;
  bool fail = false;
  out[i] = exact_round(c, &esc, &fail);
  if (esc) atomicAdd(&counters[1], (unsigned long long)esc);
  if (fail) atomicAdd(&counters[2], 1ull);
}

__global__ void init_tables_kernel() {
  const int t = threadIdx.x;
  const uint32_t t0 = aes_t0((uint8_t)t);
  g_T[t] = t0;
  g_T[256 + t] = (t0 << 8) | (t0 >> 24);
  g_T[512 + t] = (t0 << 16) | (t0 >> 16);
  g_T[768 + t] = (t0 << 24) | (t0 >> 8);
  if (t < 3) g_counters[t] = 0;
}

// ------------------------------------------------------------------------------------------
// host side
namespace {

thread_local std::string t_err;
std::mutex g_mu;
constexpr int kMaxDevices = 64;
bool g_ready[kMaxDevices];
struct DevTables {
  const uint32_t* T;
  const uint32_t* cfwd;
  const uint32_t* cinv;
  const uint32_t* round_keys;
  unsigned long long* counters;
  const uint4* tc_b[2];
  const uint4* mma_fwd;
  float mma_fwd_guard, mma_fwd_guard_rem;
  const uint4* mma_inv;
  int sms;
};
DevTables g_tables[kMaxDevices];

struct KeySlot {
  bool used;
  uint32_t rk[44];
};
KeySlot g_slots[FDS_MAX_KEYS];

int set_err(int code, const std::string& msg) {
  t_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return set_err(FDS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// FIPS-197 Sect. 5.2 key expansion, words little-endian over bytes 4i .. 4i+3
void expand_key(const uint8_t key[16], uint32_t rk[44]) {
  for (int i = 0; i < 4; ++i)
    rk[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) | ((uint32_t)key[4 * i + 2] << 16) |
            ((uint32_t)key[4 * i + 3] << 24);
  uint8_t rcon = 1;
  for (int i = 4; i < 44; ++i) {
    uint32_t t = rk[i - 1];
    if (i % 4 == 0) {
      t = (t >> 8) | (t << 24);   // RotWord
      t = (uint32_t)aes_sbox((uint8_t)t) | ((uint32_t)aes_sbox((uint8_t)(t >> 8)) << 8) |
          ((uint32_t)aes_sbox((uint8_t)(t >> 16)) << 16) | ((uint32_t)aes_sbox((uint8_t)(t >> 24)) << 24);
      t ^= rcon;
      rcon = gf_xtime(rcon);
    }
    rk[i] = rk[i - 4] ^ t;
  }
}

void iv_words(const uint8_t iv[16], uint64_t* hi, uint64_t* lo) {
  uint64_t h = 0, l = 0;
  for (int i = 0; i < 8; ++i) h = (h << 8) | iv[i];
  for (int i = 8; i < 16; ++i) l = (l << 8) | iv[i];
  *hi = h;
  *lo = l;
}

// Tensor-core B operand of form 0 (BF16, limbs 2^9, 2^8, 2^8) or 1 (TF32, limbs 2^12, 2^11):
// row n = 64 l + (8u + v) holds limb l of b_u(y) b_v(x) at K index 8y + x, laid out as the
// kernel's 128-byte swizzled K-major shared-memory image.  Returns false (with a message)
// unless every assumption of the kernel's exactness argument holds: limbs exact in the
// operand type, integer accumulators below 2^24, rational coefficients in limb 0 alone, and
// split remainder + combining roundings below the kernel's rounding guard.
bool build_tc_b(int form, std::vector<uint8_t>& img, std::string& why, double* bound_out = nullptr) {
  const int nl = form == 0 ? 3 : 2;
  const int sh[3] = {form == 0 ? 9 : 12, form == 0 ? 8 : 11, 8};
  const int tot = form == 0 ? 25 : 23;                // sum of the shifts
  const double guard = form == 0 ? 1.0 / 2048 : 1.0 / 1024;
  const double lmax = form == 0 ? 256.0 : 2048.0;      // integers exact in bf16 / tf32
  img.assign(form == 0 ? kTcBBytesBf16 : kTcBBytesTf32, 0);
  double b[8][8];
  for (int u = 0; u < 8; ++u)
    for (int y = 0; y < 8; ++y) b[u][y] = (u == 0 ? std::sqrt(0.5) : 1.0) * 0.5 * std::cos((2 * y + 1) * u * std::acos(-1.0) / 16);
  double rem_max = 0, fmax = 0, accmax = 0;
  for (int pos = 0; pos < 64; ++pos) {
    const int u = pos >> 3, v = pos & 7;
    const bool rational = (u == 0 || u == 4) && (v == 0 || v == 4);
    double rem = 0, fpos = 0, fneg = 0, lsum[3] = {0, 0, 0};
    for (int kk = 0; kk < 64; ++kk) {
      const double B = b[u][kk >> 3] * b[v][kk & 7];
      (B > 0 ? fpos : fneg) += std::fabs(B);
      double r = std::ldexp(B, sh[0]);
      double L[3] = {0, 0, 0};
      for (int l = 0; l < nl; ++l) {
        if (l) r = std::ldexp(r, sh[l]);
        L[l] = std::nearbyint(r);
        r -= L[l];
        lsum[l] += std::fabs(L[l]);
        if (std::fabs(L[l]) > lmax) return (why = "limb not exact in the operand type"), false;
      }
      if (rational && (std::fabs(L[0]) != std::ldexp(1.0, sh[0] - 3) || L[1] != 0 || L[2] != 0))
        return (why = "rational coefficient not carried by limb 0 alone"), false;
      rem += std::ldexp(std::fabs(r), -tot);
      for (int l = 0; l < nl; ++l) {
        const int n = 64 * l + pos;
        if (form == 0) {
          const float f = (float)L[l];
          uint32_t bits;
          std::memcpy(&bits, &f, 4);
          const uint16_t h = (uint16_t)(bits >> 16);
          const int off = n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2;
          std::memcpy(&img[off], &h, 2);
        } else {
          const float f = (float)L[l];
          const int atom = kk >> 5, k2 = kk & 31;
          const int off = atom * 128 * 128 + n * 128 + (((k2 >> 2) ^ (n & 7)) << 4) + (k2 & 3) * 4;
          std::memcpy(&img[off], &f, 4);
        }
      }
    }
    rem_max = std::max(rem_max, 255.0 * rem);
    if (!rational) fmax = std::max(fmax, 255.0 * std::max(fpos, fneg));
    for (int l = 0; l < nl; ++l) accmax = std::max(accmax, 255.0 * lsum[l]);
  }
  if (accmax >= 16777216.0) return (why = "accumulator may exceed 2^24"), false;
  // combining roundings: half an ulp of s = F 2^sh0 (and of the inner sum, BF16), scaled back
  auto half_ulp = [](double x) { return std::ldexp(1.0, (int)std::floor(std::log2(x)) - 24); };
  double comb = std::ldexp(half_ulp(fmax * std::ldexp(1.0, sh[0]) * 1.001), -sh[0]);
  if (form == 0) comb += std::ldexp(half_ulp(accmax * 1.004), -17);
  const double slack = 64.0 * 255.0 * std::ldexp(1.0, -50);   // cos() and B in double
  if (bound_out) *bound_out = rem_max + comb + slack;
  if (rem_max + comb + slack >= guard) return (why = "limb split exceeds the rounding guard"), false;
  return true;
}

// f16 bit pattern of an integer |v| <= 2048 (exact)
uint16_t f16_of_int(int v) {
  if (v == 0) return 0;
  const uint16_t sign = v < 0 ? 0x8000u : 0u;
  unsigned m = (unsigned)(v < 0 ? -v : v);
  int e = 0;
  while ((m >> e) > 1) ++e;                            // m in [2^e, 2^(e+1))
  const unsigned frac = (m << (10 - e)) & 0x3FFu;      // exact: m has at most 11 significant bits
  return (uint16_t)(sign | (unsigned)((e + 15) << 10) | frac);
}

// B operand of the tensor-core protect (f16, three limbs): row n = 64 l + z holds limb l of
// s = 2^13 b_u(y) b_v(x) ((u, v) the zigzag position z) at K index 8y + x, the split being
// s ~ L0 + L1 2^-11 + L2 2^-22 with integer limbs, laid out as the kernel's 128-byte swizzled
// K-major shared-memory image.  Returns false (with a message) unless the kernel's exactness
// argument holds: limbs exact in f16, every accumulator an integer below 2^24 for inputs
// |p - 128| <= 128, the rational coefficients carried by limb 0 alone.  The kernel forms
// t = D1 + D2 2^-11 (|t| < 2^23: error <= 1/2) and S = D0 + t 2^-11 = 2^13 F (error <= half an
// ulp of S, at most |S| 2^-24), then rounds S 2^-13 exactly.  *bound_rem: the limb remainder
// over |p - 128| <= 128, plus t's rounding (2^-25 in units of F), plus the error of cos() in
// double; the error of a value F is at most bound_rem + |F| 2^-24.  *bound: that bound for the
// largest |F| of an irrational coefficient of 8-bit pixels.
bool build_mma_fwd(std::vector<uint8_t>& img, double* bound, double* bound_rem, std::string& why) {
  img.assign(kMmaFwdBytes, 0);
  double b[8][8];
  for (int u = 0; u < 8; ++u)
    for (int y = 0; y < 8; ++y) b[u][y] = (u == 0 ? std::sqrt(0.5) : 1.0) * 0.5 * std::cos((2 * y + 1) * u * std::acos(-1.0) / 16);
  int uz[64], vz[64];
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v) uz[zigzag_of(u, v)] = u, vz[zigzag_of(u, v)] = v;
  double rem_max = 0, tmax = 0, fmax = 0;
  for (int z = 0; z < 64; ++z) {
    const int u = uz[z], v = vz[z];
    const bool rational = (u == 0 || u == 4) && (v == 0 || v == 4);
    constexpr int NL = kMmaFwdLimbs;
    double rem = 0, fsum = 0, lsum[3] = {0, 0, 0};
    for (int kk = 0; kk < 64; ++kk) {
      const double B = b[u][kk >> 3] * b[v][kk & 7];
      fsum += std::fabs(B);
      double r = std::ldexp(B, 13);
      double L[3] = {0, 0, 0};
      for (int l = 0; l < NL; ++l) {
        if (l) r = std::ldexp(r, 11);
        L[l] = std::nearbyint(r);
        r -= L[l];
      }
      rem += std::ldexp(std::fabs(r), -13 - 11 * (NL - 1));
      for (int l = 0; l < NL; ++l) {
        if (std::fabs(L[l]) > 2048.0) return (why = "limb not exact in f16"), false;
        lsum[l] += std::fabs(L[l]);
        const int n = 64 * l + z;
        const uint16_t h = f16_of_int((int)L[l]);
        std::memcpy(&img[n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + (kk & 7) * 2], &h, 2);
      }
      if (rational && (std::fabs(L[0]) != 1024.0 || L[1] != 0.0 || L[2] != 0.0))
        return (why = "rational coefficient not carried by limb 0 alone"), false;
    }
    for (int l = 0; l < NL; ++l)
      if (128.0 * lsum[l] >= 16777216.0) return (why = "accumulator may exceed 2^24"), false;
    rem_max = std::max(rem_max, 128.0 * rem);
    tmax = std::max(tmax, 128.0 * (lsum[1] + std::ldexp(lsum[2], -11)));
    if (!rational) fmax = std::max(fmax, 128.0 * fsum);
  }
  if (tmax >= 8388608.0) return (why = "the residual sum may reach 2^23"), false;
  if (fmax * 8192.0 >= 8388608.0) return (why = "a coefficient may reach 2^23 in units of 2^-13"), false;
  // (two limbs: S = D0 + D1 2^-11 is the only rounding, relative; three limbs add t's)
  *bound_rem = rem_max + (kMmaFwdLimbs == 3 ? std::ldexp(1.0, -25) : 0.0) + 64.0 * 255.0 * std::ldexp(1.0, -50);
  *bound = *bound_rem + std::ldexp(fmax, -24);
  if (*bound >= std::ldexp(1.0, -10)) return (why = "limb split too coarse"), false;
  return true;
}

// B operand of the tensor-core inverse transform: row n = 64 l + 8 y + x holds, at K index z
// (the zigzag index), limb l of s = 2^9 b_u(y) b_v(x), (u, v) the position of z, split as
// s ~ L0 + L1 2^-8 + L2 2^-16 with integer limbs |L| <= 128; f16, laid out as the kernel's
// 128-byte swizzled K-major shared-memory image.  Returns false (with a message) unless the
// kernel's exactness argument holds: limbs exact in f16 and at most 128 in magnitude (so that
// for coefficients |q| < 2048 every product and partial sum is an integer below 2^24), the
// rational coefficients carried by limb 0 alone, and the per-coefficient bound the kernel's
// guard uses, (split remainder + combining roundings) per unit of sum |q|, below 2^-24.
// *bound gets that bound.
bool build_mma_inv(std::vector<uint8_t>& img, double* bound, std::string& why) {
  img.assign(kMmaInvBytes, 0);
  double b[8][8];
  for (int u = 0; u < 8; ++u)
    for (int y = 0; y < 8; ++y) b[u][y] = (u == 0 ? std::sqrt(0.5) : 1.0) * 0.5 * std::cos((2 * y + 1) * u * std::acos(-1.0) / 16);
  int uz[64], vz[64];
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v) uz[zigzag_of(u, v)] = u, vz[zigzag_of(u, v)] = v;
  double rem_max = 0;
  for (int p = 0; p < 64; ++p) {
    const int y = p >> 3, x = p & 7;
    for (int z = 0; z < 64; ++z) {
      const int u = uz[z], v = vz[z];
      const bool rational = (u == 0 || u == 4) && (v == 0 || v == 4);
      double r = std::ldexp(b[u][y] * b[v][x], 9);
      double L[3];
      for (int l = 0; l < 3; ++l) {
        if (l) r = std::ldexp(r, 8);
        L[l] = std::nearbyint(r);
        r -= L[l];
        if (std::fabs(L[l]) > 128.0) return (why = "inverse limb above 128"), false;
      }
      if (rational && (std::fabs(L[0]) != 64.0 || L[1] != 0.0 || L[2] != 0.0))
        return (why = "rational coefficient not carried by limb 0 alone"), false;
      rem_max = std::max(rem_max, std::ldexp(std::fabs(r), -25));   // |basis - limbs|
      for (int l = 0; l < 3; ++l) {
        const int n = 64 * l + p;
        const uint16_t h = f16_of_int((int)L[l]);
        std::memcpy(&img[n * 128 + (((z >> 3) ^ (n & 7)) << 4) + (z & 7) * 2], &h, 2);
      }
    }
  }
  // per unit of sum |q|: the split remainder, and the two fused multiply-adds that combine the
  // limb accumulators (each accumulator at most 128 sum |q|; half an ulp relative, 2^-24, of
  // t1 = D1 + D2 2^-8 and of t2 = D0 + t1 2^-8, then scaled by 2^-9), plus cos() in double
  const double comb = std::ldexp(128.0 * (1.0 + 2.0 / 256.0 + 1.0 / 65536.0), -24 - 9);
  *bound = rem_max + comb + std::ldexp(1.0, -45);
  if (*bound >= std::ldexp(1.0, -24)) return (why = "inverse limb split too coarse"), false;
  return true;
}

// Initialise the current device (once) and return its index in *dev_out.
int ensure_init(int* dev_out = nullptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_err(FDS_E_INVALID, "device index out of range");
  if (dev_out) *dev_out = dev;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ready[dev]) return FDS_OK;
  // exact-coordinate tables: fold cos(m pi/16) to +-cos(j pi/16), j = 0..8 (cos(8 pi/16) = 0)
  auto fold = [](int m, int* j, int* sgn) {
    m &= 31;
    if (m > 16) m = 32 - m;
    *sgn = 1;
    if (m > 8) {
      m = 16 - m;
      *sgn = -1;
    }
    *j = m;
  };
  static int8_t K[8][8][8][8][8];  // [u][v][y][x][j]
  std::memset(K, 0, sizeof(K));
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v)
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) {
          const int al = u == 0 ? 4 : (2 * y + 1) * u, be = v == 0 ? 4 : (2 * x + 1) * v;
          for (int m : {al - be, al + be}) {
            int j, sg;
            fold(m, &j, &sg);
            if (j < 8) K[u][v][y][x][j] = (int8_t)(K[u][v][y][x][j] + sg);
          }
        }
  static uint32_t hf[64 * 128], hinv[64 * 128];
  std::memset(hf, 0, sizeof(hf));
  std::memset(hinv, 0, sizeof(hinv));
  int uz[64], vz[64];
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v) {
      uz[zigzag_of(u, v)] = u;
      vz[zigzag_of(u, v)] = v;
    }
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v)
      for (int j = 0; j < 8; ++j)
        for (int w = 0; w < 16; ++w)
          for (int i = 0; i < 4; ++i)
            hf[(8 * u + v) * 128 + 16 * j + w] |=
                (uint32_t)(uint8_t)K[u][v][w >> 1][4 * (w & 1) + i][j] << (8 * i);
  for (int y = 0; y < 8; ++y)
    for (int x = 0; x < 8; ++x)
      for (int j = 0; j < 8; ++j)
        for (int tw = 0; tw < 16; ++tw)
          for (int i = 0; i < 4; ++i) {
            const int z = 4 * tw + i;
            hinv[(8 * y + x) * 128 + 16 * j + tw] |= (uint32_t)(uint8_t)K[uz[z]][vz[z]][y][x][j] << (8 * i);
          }
  if ((e = cudaMemcpyToSymbol(g_cfwd, hf, sizeof(hf))) != cudaSuccess) return cuda_fail(e, "table upload");
  if ((e = cudaMemcpyToSymbol(g_cinv, hinv, sizeof(hinv))) != cudaSuccess) return cuda_fail(e, "table upload");
  init_tables_kernel<<<1, 256>>>();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "init kernel launch");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "init kernel");
  DevTables& tb = g_tables[dev];
  void* p = nullptr;
  if ((e = cudaGetSymbolAddress(&p, g_T)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.T = static_cast<const uint32_t*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_cfwd)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.cfwd = static_cast<const uint32_t*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_cinv)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.cinv = static_cast<const uint32_t*>(p);
  if ((e = cudaDeviceGetAttribute(&tb.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaGetSymbolAddress(&p, g_counters)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.counters = static_cast<unsigned long long*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_rk)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.round_keys = static_cast<const uint32_t*>(p);
  {
    static std::vector<uint8_t> tcb[2];
    static bool tcb_ok[2];
    static std::string tcb_why[2];
    for (int f = 0; f < 2; ++f) {
      if (tcb[f].empty()) tcb_ok[f] = build_tc_b(f, tcb[f], tcb_why[f]);
      if (!tcb_ok[f]) return set_err(FDS_E_INVALID, "tensor-core table: " + tcb_why[f]);
    }
    if ((e = cudaMemcpyToSymbol(g_tcb0, tcb[0].data(), tcb[0].size())) != cudaSuccess) return cuda_fail(e, "table upload");
    if ((e = cudaMemcpyToSymbol(g_tcb1, tcb[1].data(), tcb[1].size())) != cudaSuccess) return cuda_fail(e, "table upload");
    if ((e = cudaGetSymbolAddress(&p, g_tcb0)) != cudaSuccess) return cuda_fail(e, "symbol address");
    tb.tc_b[0] = static_cast<const uint4*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_tcb1)) != cudaSuccess) return cuda_fail(e, "symbol address");
    tb.tc_b[1] = static_cast<const uint4*>(p);
  }
  {
    static std::vector<uint8_t> mf;
    static double mf_bound = 0, mf_rem = 0;
    static bool mf_ok = false;
    static std::string mf_why;
    if (mf.empty()) mf_ok = build_mma_fwd(mf, &mf_bound, &mf_rem, mf_why);
    if (!mf_ok) return set_err(FDS_E_INVALID, "tensor-core table: " + mf_why);
    if ((e = cudaMemcpyToSymbol(g_mma_fwd, mf.data(), mf.size())) != cudaSuccess) return cuda_fail(e, "table upload");
    if ((e = cudaGetSymbolAddress(&p, g_mma_fwd)) != cudaSuccess) return cuda_fail(e, "symbol address");
    tb.mma_fwd = static_cast<const uint4*>(p);
    // the guard the kernel compares with, rounded up: float(bound) * (1 + 2^-20)
    tb.mma_fwd_guard = (float)(mf_bound * (1.0 + std::ldexp(1.0, -20)));
    tb.mma_fwd_guard_rem = (float)(mf_rem * (1.0 + std::ldexp(1.0, -20)));
  }
  {
    static std::vector<uint8_t> mi;
    static double mi_bound = 0;
    static bool mi_ok = false;
    static std::string mi_why;
    if (mi.empty()) mi_ok = build_mma_inv(mi, &mi_bound, mi_why);
    if (!mi_ok) return set_err(FDS_E_INVALID, "tensor-core inverse table: " + mi_why);
    if ((e = cudaMemcpyToSymbol(g_mma_inv, mi.data(), mi.size())) != cudaSuccess) return cuda_fail(e, "table upload");
    if ((e = cudaGetSymbolAddress(&p, g_mma_inv)) != cudaSuccess) return cuda_fail(e, "symbol address");
    tb.mma_inv = static_cast<const uint4*>(p);
  }
  if ((e = upload_sha512_constants()) != cudaSuccess) return cuda_fail(e, "SHA-512 constants upload");
  if ((e = upload_dwt_constants()) != cudaSuccess) return cuda_fail(e, "SHA constants upload");
  for (int i = 0; i < FDS_MAX_KEYS; ++i)   // keys registered before this device was ready
    if (g_slots[i].used &&
        (e = cudaMemcpyToSymbol(g_rk, g_slots[i].rk, sizeof(g_slots[i].rk), 44 * 4 * i)) != cudaSuccess)
      return cuda_fail(e, "key upload");
  g_ready[dev] = true;
  return FDS_OK;
}

bool bad_dims(int32_t w, int32_t h) {
  return w <= 0 || h <= 0 || (w & 7) || (h & 7) || (int64_t)(w / 8) * (int64_t)(h / 8) > (1ll << 30);
}

void set_tables(TileArgs& a, int dev) {
  a.T = g_tables[dev].T;
  a.cfwd = g_tables[dev].cfwd;
  a.cinv = g_tables[dev].cinv;
  a.round_keys = g_tables[dev].round_keys;
  a.counters = g_tables[dev].counters;
}

int run_protect(TileArgs& a, int dev, cudaStream_t s, bool debug, int per_sm = 0) {
  set_tables(a, dev);
  const cudaError_t e = launch_protect(a, s, debug, g_tables[dev].sms, per_sm);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "protect launch");
}

int run_restore(TileArgs& a, int dev, cudaStream_t s, int per_sm = 0) {
  set_tables(a, dev);
  const cudaError_t e = launch_restore(a, s, g_tables[dev].sms, per_sm);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "restore launch");
}

void fill_geometry(TileArgs& a, int32_t w, int32_t h, int32_t k) {
  a.width = w;
  a.bx_count = w / 8;
  a.nblocks = (w / 8) * (h / 8);
  a.k = k;
}

bool misaligned(const void* p, uintptr_t align) { return ((uintptr_t)p & (align - 1)) != 0; }

// Failure counter value (counter 2 of fds_counters) already reported per device: fds_sync
// returns FDS_E_TIMEOUT once for every increase.
uint64_t g_failures_seen[kMaxDevices];

}  // namespace
}  // namespace fds

using namespace fds;

extern "C" int fds_status_of_failures(uint64_t seen, uint64_t now);

namespace fds {
namespace {
// the status of a failure-counter reading on device dev, and the watermark moved past it
int failure_status(int dev, uint64_t now) {
  uint64_t seen;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    seen = g_failures_seen[dev];
    if (now > seen) g_failures_seen[dev] = now;
  }
  return fds_status_of_failures(seen, now);
}
}  // namespace
}  // namespace fds

extern "C" {

int fds_init(int device) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return ensure_init();
}

int fds_key_register(const uint8_t key[16], int32_t* slot_out) {
  if (!key || !slot_out) return set_err(FDS_E_INVALID, "null key or slot pointer");
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < FDS_MAX_KEYS; ++i) {
    if (!g_slots[i].used) {
      expand_key(key, g_slots[i].rk);
      // device copy now if the current device is initialised, else when it is
      int dev = -1;
      if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices && g_ready[dev]) {
        const cudaError_t e = cudaMemcpyToSymbol(g_rk, g_slots[i].rk, sizeof(g_slots[i].rk), 44 * 4 * i);
        if (e != cudaSuccess) return cuda_fail(e, "key upload");
      }
      g_slots[i].used = true;
      *slot_out = i;
      return FDS_OK;
    }
  }
  return set_err(FDS_E_BUSY, "all key slots are in use");
}

int fds_key_release(int32_t slot) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot < 0 || slot >= FDS_MAX_KEYS || !g_slots[slot].used) return set_err(FDS_E_NO_KEY, "key slot not registered");
  g_slots[slot].used = false;
  std::memset(g_slots[slot].rk, 0, sizeof(g_slots[slot].rk));
  return FDS_OK;
}

int fds_sizes(int32_t width, int32_t height, int32_t k, uint64_t* public_bytes, uint64_t* private_bytes) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  const uint64_t ncb = (uint64_t)(width / 8) * (uint64_t)(height / 8) * 3ull;
  if (public_bytes) *public_bytes = ncb * 2ull * (uint64_t)(63 - k);
  if (private_bytes) *private_bytes = ncb * 2ull * (uint64_t)(k + 1);
  return FDS_OK;
}

int fds_protect_image(const uint8_t* pixels, int32_t width, int32_t height, int32_t k,
                      const uint8_t key[16], const uint8_t iv[16], int16_t* public_out,
                      uint8_t* private_out, void* stream) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (!pixels || !key || !iv || !private_out || (k < 63 && !public_out))
    return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(pixels, 8) || misaligned(public_out, 16) || misaligned(private_out, 16))
    return set_err(FDS_E_INVALID, "pixels must be 8-byte aligned, fragments 16-byte aligned");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pixels_in = pixels;
  a.pub_out = public_out;
  a.priv_out = private_out;
  fill_geometry(a, width, height, k);
  expand_key(key, a.rk);
  iv_words(iv, &a.iv_hi, &a.iv_lo);
  return run_protect(a, dev, (cudaStream_t)stream, false);
}

int fds_restore_image(const int16_t* public_in, const uint8_t* private_in, int32_t width,
                      int32_t height, int32_t k, const uint8_t key[16], const uint8_t iv[16],
                      uint8_t* pixels_out, void* stream) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (!pixels_out || !key || !iv || !private_in || (k < 63 && !public_in))
    return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(pixels_out, 8) || misaligned(public_in, 16) || misaligned(private_in, 16))
    return set_err(FDS_E_INVALID, "pixels must be 8-byte aligned, fragments 16-byte aligned");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pub_in = public_in;
  a.priv_in = private_in;
  a.pixels_out = pixels_out;
  fill_geometry(a, width, height, k);
  expand_key(key, a.rk);
  iv_words(iv, &a.iv_hi, &a.iv_lo);
  return run_restore(a, dev, (cudaStream_t)stream);
}

static int check_batch(const fds_image* images, int32_t n, const void* px, const void* pub,
                       const void* priv) {
  if (n < 0 || (n > 0 && !images)) return set_err(FDS_E_INVALID, "bad descriptor array");
  for (int32_t i = 0; i < n; ++i) {
    const fds_image& d = images[i];
    if (bad_dims(d.width, d.height)) return set_err(FDS_E_INVALID, "image " + std::to_string(i) + ": bad size");
    if (d.k < 0 || d.k > 63) return set_err(FDS_E_INVALID, "image " + std::to_string(i) + ": k out of range");
    if ((d.pixel_offset & 7) || (d.public_offset & 15) || (d.private_offset & 15))
      return set_err(FDS_E_INVALID, "image " + std::to_string(i) + ": misaligned offset");
    if (d.key_slot < 0 || d.key_slot >= FDS_MAX_KEYS || !g_slots[d.key_slot].used)
      return set_err(FDS_E_NO_KEY, "image " + std::to_string(i) + ": key slot not registered");
  }
  if (n > 0 && (!px || !priv)) return set_err(FDS_E_INVALID, "null buffer");
  if (misaligned(px, 8) || misaligned(pub, 16) || misaligned(priv, 16))
    return set_err(FDS_E_INVALID, "misaligned buffer");
  return FDS_OK;
}

int fds_protect(const uint8_t* pixels, int16_t* public_out, uint8_t* private_out,
                const fds_image* images, int32_t n, void* stream) {
  int rc = check_batch(images, n, pixels, public_out, private_out);
  if (rc) return rc;
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  for (int32_t i = 0; i < n; ++i) {
    const fds_image& d = images[i];
    TileArgs a{};
    a.pixels_in = pixels + d.pixel_offset;
    a.pub_out = reinterpret_cast<int16_t*>(reinterpret_cast<uint8_t*>(public_out) + d.public_offset);
    a.priv_out = private_out + d.private_offset;
    fill_geometry(a, d.width, d.height, d.k);
    std::memcpy(a.rk, g_slots[d.key_slot].rk, sizeof(a.rk));
    iv_words(d.iv, &a.iv_hi, &a.iv_lo);
    if ((rc = run_protect(a, dev, (cudaStream_t)stream, false))) return rc;
  }
  return FDS_OK;
}

int fds_restore(const int16_t* public_in, const uint8_t* private_in, uint8_t* pixels_out,
                const fds_image* images, int32_t n, void* stream) {
  int rc = check_batch(images, n, pixels_out, public_in, private_in);
  if (rc) return rc;
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  for (int32_t i = 0; i < n; ++i) {
    const fds_image& d = images[i];
    TileArgs a{};
    a.pub_in = reinterpret_cast<const int16_t*>(reinterpret_cast<const uint8_t*>(public_in) + d.public_offset);
    a.priv_in = private_in + d.private_offset;
    a.pixels_out = pixels_out + d.pixel_offset;
    fill_geometry(a, d.width, d.height, d.k);
    std::memcpy(a.rk, g_slots[d.key_slot].rk, sizeof(a.rk));
    iv_words(d.iv, &a.iv_hi, &a.iv_lo);
    if ((rc = run_restore(a, dev, (cudaStream_t)stream))) return rc;
  }
  return FDS_OK;
}

int fds_debug_dct_f32(const uint8_t* pixels, int32_t width, int32_t height, float* coefs_out,
                      void* stream) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (!pixels || !coefs_out) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(pixels, 8) || misaligned(coefs_out, 4)) return set_err(FDS_E_INVALID, "misaligned buffer");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pixels_in = pixels;
  a.dbg_coefs = coefs_out;
  fill_geometry(a, width, height, 0);
  return run_protect(a, dev, (cudaStream_t)stream, true);
}

int fds_protect_image_tc(int32_t form, const uint8_t* pixels, int32_t width, int32_t height, int32_t k,
                         const uint8_t key[16], const uint8_t iv[16], int16_t* public_out,
                         uint8_t* private_out, void* stream) {
  if (form != FDS_TC_BF16 && form != FDS_TC_TF32 && form != FDS_TC_F16)
    return set_err(FDS_E_INVALID, "unknown tensor-core form");
  if (form == FDS_TC_F16 && k >= 0 && k <= 63 && !mma_supports_k(k))
    return set_err(FDS_E_INVALID, "FDS_TC_F16 takes k = " + std::string(FDS_TC_F16_K_LIST));
  if (bad_dims(width, height) || 3ll * (width / 8) * (height / 8) >= (1ll << 31))
    return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8, 3 W H / 64 < 2^31");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (!pixels || !key || !iv || !private_out || (k < 63 && !public_out))
    return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(pixels, 8) || misaligned(public_out, 16) || misaligned(private_out, 16))
    return set_err(FDS_E_INVALID, "pixels must be 8-byte aligned, fragments 16-byte aligned");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pixels_in = pixels;
  a.pub_out = public_out;
  a.priv_out = private_out;
  fill_geometry(a, width, height, k);
  expand_key(key, a.rk);
  iv_words(iv, &a.iv_hi, &a.iv_lo);
  set_tables(a, dev);
  cudaError_t e;
  if (form == FDS_TC_F16) {
    e = launch_protect_mma(a, g_tables[dev].mma_fwd, g_tables[dev].mma_fwd_guard, g_tables[dev].mma_fwd_guard_rem,
                           (cudaStream_t)stream, false, g_tables[dev].sms);
  } else {
    a.tc_b = g_tables[dev].tc_b[form];
    e = launch_protect_tc(a, (cudaStream_t)stream, form, false, g_tables[dev].sms);
  }
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "tensor-core protect launch");
}

int fds_restore_image_tc(int32_t form, const int16_t* public_in, const uint8_t* private_in, int32_t width,
                         int32_t height, int32_t k, const uint8_t key[16], const uint8_t iv[16],
                         uint8_t* pixels_out, void* stream) {
  if (form != FDS_TC_F16) return set_err(FDS_E_INVALID, "the tensor-core inverse takes form FDS_TC_F16");
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (!pixels_out || !key || !iv || !private_in || (k < 63 && !public_in))
    return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(pixels_out, 8) || misaligned(public_in, 16) || misaligned(private_in, 16))
    return set_err(FDS_E_INVALID, "pixels must be 8-byte aligned, fragments 16-byte aligned");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pub_in = public_in;
  a.priv_in = private_in;
  a.pixels_out = pixels_out;
  fill_geometry(a, width, height, k);
  expand_key(key, a.rk);
  iv_words(iv, &a.iv_hi, &a.iv_lo);
  set_tables(a, dev);
  a.tc_b = g_tables[dev].mma_inv;
  const cudaError_t e = launch_restore_tc(a, (cudaStream_t)stream, g_tables[dev].sms);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "tensor-core restore launch");
}

int fds_encrypt_full(const uint8_t* in, uint8_t* out, uint64_t bytes, const uint8_t key[16], const uint8_t iv[16],
                     void* stream) {
  if (!key || !iv || (bytes && (!in || !out))) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(in, 16) || misaligned(out, 16)) return set_err(FDS_E_INVALID, "buffers must be 16-byte aligned");
  if (in != out && bytes && (const uint8_t*)out < in + bytes && in < (const uint8_t*)out + bytes)
    return set_err(FDS_E_INVALID, "buffers overlap without being the same");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  if (!bytes) return FDS_OK;
  uint32_t rk[44];
  expand_key(key, rk);
  uint64_t hi, lo;
  iv_words(iv, &hi, &lo);
  const cudaError_t e = launch_aes_full(in, out, bytes, hi, lo, rk, g_tables[dev].T, (cudaStream_t)stream,
                                        g_tables[dev].sms, g_tables[dev].counters);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "full encryption launch");
}

// ---- bit-packed storage (Sect. 6.4.3, Table 5)
static uint64_t align16u(uint64_t x) { return (x + 15) & ~15ull; }

int fds_sizes_packed(int32_t form, int32_t width, int32_t height, int32_t k, uint64_t* public_bytes,
                     uint64_t* private_bytes, uint64_t* scratch_bytes) {
  if (form != FDS_PACK_11 && form != FDS_PACK_8) return set_err(FDS_E_INVALID, "form must be 11 or 8");
  uint64_t pub16 = 0, priv16 = 0;
  int rc = fds_sizes(width, height, k, &pub16, &priv16);
  if (rc) return rc;
  const uint64_t ncb = (uint64_t)(width / 8) * (uint64_t)(height / 8) * 3ull;
  const uint64_t pub = (ncb * (uint64_t)(63 - k) * (uint64_t)form + 7) / 8;
  const uint64_t priv = (ncb * (11ull + (uint64_t)k * (uint64_t)form) + 7) / 8;
  if (public_bytes) *public_bytes = pub;
  if (private_bytes) *private_bytes = priv;
  if (scratch_bytes) *scratch_bytes = align16u(pub16) + align16u(priv16) + align16u(priv);
  return FDS_OK;
}

static int packed_checks(int32_t form, int32_t width, int32_t height, int32_t k, const void* px, const void* pub,
                         const void* priv, const void* scratch, uint64_t* pub16, uint64_t* priv16,
                         uint64_t* priv_packed) {
  if (form != FDS_PACK_11 && form != FDS_PACK_8) return set_err(FDS_E_INVALID, "form must be 11 or 8");
  int rc = fds_sizes_packed(form, width, height, k, nullptr, priv_packed, nullptr);
  if (rc) return rc;
  if ((rc = fds_sizes(width, height, k, pub16, priv16))) return rc;
  if (!px || !priv || !scratch || (k < 63 && !pub)) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(px, 8) || misaligned(priv, 16) || misaligned(scratch, 16))
    return set_err(FDS_E_INVALID, "pixels must be 8-byte aligned, private and scratch 16-byte aligned");
  return FDS_OK;
}

int fds_protect_image_packed(int32_t form, const uint8_t* pixels, int32_t width, int32_t height, int32_t k,
                             const uint8_t key[16], const uint8_t iv[16], uint8_t* public_out, uint8_t* private_out,
                             void* scratch, void* stream) {
  uint64_t pub16 = 0, priv16 = 0, vpk = 0;
  int rc = packed_checks(form, width, height, k, pixels, public_out, private_out, scratch, &pub16, &priv16, &vpk);
  if (rc) return rc;
  if (!key || !iv) return set_err(FDS_E_INVALID, "null pointer argument");
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  TileArgs a{};                                  // one launch: transform, pack, encrypt
  a.pixels_in = pixels;
  a.pub_out = reinterpret_cast<int16_t*>(public_out);
  a.priv_out = private_out;
  a.pack = form;
  fill_geometry(a, width, height, k);
  expand_key(key, a.rk);
  iv_words(iv, &a.iv_hi, &a.iv_lo);
  return run_protect(a, dev, (cudaStream_t)stream, false);
}

int fds_restore_image_packed(int32_t form, const uint8_t* public_in, const uint8_t* private_in, int32_t width,
                             int32_t height, int32_t k, const uint8_t key[16], const uint8_t iv[16],
                             uint8_t* pixels_out, void* scratch, void* stream) {
  uint64_t pub16 = 0, priv16 = 0, vpk = 0;
  int rc = packed_checks(form, width, height, k, pixels_out, public_in, private_in, scratch, &pub16, &priv16, &vpk);
  if (rc) return rc;
  if (!key || !iv) return set_err(FDS_E_INVALID, "null pointer argument");
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (!misaligned(public_in, 8)) {               // one launch: land, decrypt, unpack, restore
    TileArgs a{};
    a.pub_in = reinterpret_cast<const int16_t*>(public_in);
    a.priv_in = private_in;
    a.pixels_out = pixels_out;
    a.pack = form;
    fill_geometry(a, width, height, k);
    expand_key(key, a.rk);
    iv_words(iv, &a.iv_hi, &a.iv_lo);
    return run_restore(a, dev, s);
  }
  int16_t* s_pub = static_cast<int16_t*>(scratch);   // a public stream at any alignment
  uint8_t* s_priv = static_cast<uint8_t*>(scratch) + align16u(pub16);
  uint8_t* s_plain = s_priv + align16u(priv16);
  uint32_t rk[44];
  expand_key(key, rk);
  uint64_t hi, lo;
  iv_words(iv, &hi, &lo);
  cudaError_t e = launch_aes_full(private_in, s_plain, vpk, hi, lo, rk, g_tables[dev].T, s,
                                  g_tables[dev].sms, g_tables[dev].counters);   // 1. decrypt the packed private stream
  if (e != cudaSuccess) return cuda_fail(e, "decryption launch");
  const long long ncb = 3ll * (width / 8) * (long long)(height / 8);
  e = launch_unpack(public_in, s_plain, s_pub, reinterpret_cast<int16_t*>(s_priv), ncb, k, form, s);
  if (e != cudaSuccess) return cuda_fail(e, "unpack launch");   // 2. back to int16
  TileArgs a{};                                  // 3. the inverse transform from plaintext
  a.pub_in = s_pub;
  a.priv_in = s_priv;
  a.pixels_out = pixels_out;
  a.plain_private = 1;
  fill_geometry(a, width, height, k);
  std::memcpy(a.rk, rk, sizeof(rk));
  a.iv_hi = hi;
  a.iv_lo = lo;
  return run_restore(a, dev, s);
}

// ---- protect / restore with host buffers: copies overlapped with the kernels, by strips
namespace {
struct HostLanes {
  cudaStream_t in = nullptr, out = nullptr;   // host -> device and device -> host copies
};
// One pair of copy streams per device and caller stream, so that calls on one stream keep
// their copies in order while calls on different streams overlap theirs.  Beyond
// kLaneStreams caller streams on a device, further streams share one pair.
constexpr size_t kLaneStreams = 16;
std::map<std::pair<int, cudaStream_t>, HostLanes> g_lanes;   // guarded by g_mu
size_t g_lane_count[kMaxDevices];

int host_lanes(int dev, cudaStream_t caller, HostLanes** lanes) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, caller);
  if (!g_lanes.count(key)) {
    if (g_lane_count[dev] >= kLaneStreams) key.second = nullptr;
    if (!g_lanes.count(key)) ++g_lane_count[dev];
  }
  HostLanes& l = g_lanes[key];
  cudaError_t e = cudaSuccess;
  if (!l.in && (e = cudaStreamCreateWithFlags(&l.in, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "copy stream");
  if (!l.out && (e = cudaStreamCreateWithFlags(&l.out, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "copy stream");
  *lanes = &l;
  return FDS_OK;
}

// A strip is a run of block rows, a multiple of 8 of them: its private bytes, bx * 3 * 2 (k+1)
// per block row, then start on a keystream-block boundary.
struct Strip {
  int r0, rows;
};
std::vector<Strip> make_strips(int by, int strips) {
  int rows = (by + strips - 1) / strips;
  rows = ((rows + 7) / 8) * 8;
  std::vector<Strip> out;
  for (int r0 = 0; r0 < by; r0 += rows) out.push_back({r0, by - r0 < rows ? by - r0 : rows});
  return out;
}

// the counter block `blocks` keystream blocks after (hi, lo): a 128-bit big-endian addition
void iv_advance(uint64_t* hi, uint64_t* lo, uint64_t blocks) {
  const uint64_t l = *lo + blocks;
  if (l < *lo) ++*hi;
  *lo = l;
}

// events recorded while enqueuing; destroyed once enqueued (the runtime keeps them alive
// until they complete)
struct EventSet {
  std::vector<cudaEvent_t> ev;
  ~EventSet() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  cudaError_t record(cudaStream_t s, cudaEvent_t* out) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    *out = e;
    return cudaEventRecord(e, s);
  }
};

int host_checks(int32_t width, int32_t height, int32_t k, int32_t strips, const void* a, const void* b,
                const void* c, const void* d, const void* key, const void* iv) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (strips < 1 || strips > 64) return set_err(FDS_E_INVALID, "strips must be in 1..64");
  if (!a || !b || !c || !d || !key || !iv) return set_err(FDS_E_INVALID, "null pointer argument");
  return FDS_OK;
}
}  // namespace

int fds_protect_image_host(const uint8_t* host_pixels, uint8_t* dev_pixels, int32_t width, int32_t height,
                           int32_t k, const uint8_t key[16], const uint8_t iv[16], int16_t* dev_public,
                           uint8_t* dev_private, int16_t* host_public, uint8_t* host_private, int32_t strips,
                           void* stream) {
  int rc = host_checks(width, height, k, strips, host_pixels, dev_pixels, dev_private, host_private, key, iv);
  if (rc) return rc;
  if (k < 63 && (!dev_public || !host_public)) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(dev_pixels, 8) || misaligned(dev_public, 16) || misaligned(dev_private, 16))
    return set_err(FDS_E_INVALID, "device pixels must be 8-byte aligned, fragments 16-byte aligned");
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  HostLanes* ln = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = host_lanes(dev, s, &ln))) return rc;
  const uint64_t w3 = 3ull * (uint64_t)width, bx = (uint64_t)(width / 8);
  const uint64_t pub_row = bx * 3ull * (uint64_t)(63 - k), priv_row = bx * 3ull * 2ull * (uint64_t)(k + 1);
  uint32_t rk[44];
  expand_key(key, rk);
  uint64_t hi0, lo0;
  iv_words(iv, &hi0, &lo0);
  EventSet evs;
  cudaEvent_t e0;
  cudaError_t e = evs.record(s, &e0);   // earlier work on the caller's stream comes first
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ln->in, e0, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ln->out, e0, 0);
  for (const Strip& st : make_strips(height / 8, strips)) {
    if (e != cudaSuccess) break;
    const uint64_t px0 = (uint64_t)st.r0 * 8ull * w3, pxn = (uint64_t)st.rows * 8ull * w3;
    e = cudaMemcpyAsync(dev_pixels + px0, host_pixels + px0, pxn, cudaMemcpyHostToDevice, ln->in);
    cudaEvent_t ein, ek;
    if (e == cudaSuccess) e = evs.record(ln->in, &ein);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ein, 0);
    if (e != cudaSuccess) break;
    TileArgs a{};
    a.pixels_in = dev_pixels + px0;
    a.pub_out = dev_public ? dev_public + (uint64_t)st.r0 * pub_row : nullptr;
    a.priv_out = dev_private + (uint64_t)st.r0 * priv_row;
    fill_geometry(a, width, st.rows * 8, k);
    std::memcpy(a.rk, rk, sizeof(rk));
    a.iv_hi = hi0;
    a.iv_lo = lo0;
    iv_advance(&a.iv_hi, &a.iv_lo, (uint64_t)st.r0 * priv_row / 16);
    if ((rc = run_protect(a, dev, s, false))) return rc;
    e = evs.record(s, &ek);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ln->out, ek, 0);
    if (e == cudaSuccess && k < 63)
      e = cudaMemcpyAsync(host_public + (uint64_t)st.r0 * pub_row, a.pub_out, (uint64_t)st.rows * pub_row * 2ull,
                          cudaMemcpyDeviceToHost, ln->out);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host_private + (uint64_t)st.r0 * priv_row, a.priv_out, (uint64_t)st.rows * priv_row,
                          cudaMemcpyDeviceToHost, ln->out);
  }
  cudaEvent_t ed;
  if (e == cudaSuccess) e = evs.record(ln->out, &ed);   // the caller's stream completes after the copies
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ed, 0);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "host pipeline");
}

int fds_restore_image_host(const int16_t* dev_public, const uint8_t* dev_private, uint8_t* dev_pixels,
                           uint8_t* host_pixels, int32_t width, int32_t height, int32_t k, const uint8_t key[16],
                           const uint8_t iv[16], int32_t strips, void* stream) {
  int rc = host_checks(width, height, k, strips, dev_private, dev_pixels, host_pixels, host_pixels, key, iv);
  if (rc) return rc;
  if (k < 63 && !dev_public) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(dev_pixels, 8) || misaligned(dev_public, 16) || misaligned(dev_private, 16))
    return set_err(FDS_E_INVALID, "device pixels must be 8-byte aligned, fragments 16-byte aligned");
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  HostLanes* ln = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = host_lanes(dev, s, &ln))) return rc;
  const uint64_t w3 = 3ull * (uint64_t)width, bx = (uint64_t)(width / 8);
  const uint64_t pub_row = bx * 3ull * (uint64_t)(63 - k), priv_row = bx * 3ull * 2ull * (uint64_t)(k + 1);
  uint32_t rk[44];
  expand_key(key, rk);
  uint64_t hi0, lo0;
  iv_words(iv, &hi0, &lo0);
  EventSet evs;
  cudaError_t e = cudaSuccess;
  for (const Strip& st : make_strips(height / 8, strips)) {
    const uint64_t px0 = (uint64_t)st.r0 * 8ull * w3, pxn = (uint64_t)st.rows * 8ull * w3;
    TileArgs a{};
    a.pub_in = dev_public ? dev_public + (uint64_t)st.r0 * pub_row : nullptr;
    a.priv_in = dev_private + (uint64_t)st.r0 * priv_row;
    a.pixels_out = dev_pixels + px0;
    fill_geometry(a, width, st.rows * 8, k);
    std::memcpy(a.rk, rk, sizeof(rk));
    a.iv_hi = hi0;
    a.iv_lo = lo0;
    iv_advance(&a.iv_hi, &a.iv_lo, (uint64_t)st.r0 * priv_row / 16);
    if ((rc = run_restore(a, dev, s))) return rc;
    cudaEvent_t ek;
    e = evs.record(s, &ek);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ln->out, ek, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host_pixels + px0, dev_pixels + px0, pxn, cudaMemcpyDeviceToHost, ln->out);
    if (e != cudaSuccess) break;
  }
  cudaEvent_t ed;
  if (e == cudaSuccess) e = evs.record(ln->out, &ed);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ed, 0);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "host pipeline");
}

// ---- the paper-form public fragment and the statistics of Sect. 6.6
int fds_public_image(const int16_t* public_in, int32_t width, int32_t height, int32_t k, uint8_t* image_out,
                     void* stream) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (!image_out || (k < 63 && !public_in)) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(image_out, 8) || misaligned(public_in, 16))
    return set_err(FDS_E_INVALID, "image must be 8-byte aligned, the fragment 16-byte aligned");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pub_in = public_in;
  a.pixels_out = image_out;
  a.public_image = 1;
  fill_geometry(a, width, height, k);
  return run_restore(a, dev, (cudaStream_t)stream);
}

int fds_image_stats(const uint8_t* image, int32_t width, int32_t height, uint64_t* histogram_out,
                    int64_t* pair_sums_out, void* stream) {
  if (width <= 0 || height <= 0) return set_err(FDS_E_INVALID, "width and height must be positive");
  if (!image || !histogram_out || !pair_sums_out) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(histogram_out, 8) || misaligned(pair_sums_out, 8))
    return set_err(FDS_E_INVALID, "outputs must be 8-byte aligned");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(histogram_out, 0, 3 * 256 * sizeof(uint64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pair_sums_out, 0, 3 * 3 * 6 * sizeof(int64_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "clearing the statistics");
  e = launch_image_stats(image, width, height, reinterpret_cast<unsigned long long*>(histogram_out),
                         reinterpret_cast<long long*>(pair_sums_out), s, g_tables[dev].sms);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "statistics launch");
}

// ---- strong level of protection (Sect. 6.3.2, Fig. 8)
int fds_sizes_strong(int32_t width, int32_t height, int32_t k, uint64_t* public_bytes, uint64_t* private_bytes,
                     uint64_t* scratch_bytes) {
  uint64_t pub16 = 0, priv16 = 0;
  int rc = fds_sizes(width, height, k, &pub16, &priv16);
  if (rc) return rc;
  const uint64_t px = (uint64_t)width * (uint64_t)height * 3ull;
  if (public_bytes) *public_bytes = px;
  if (private_bytes) *private_bytes = priv16;
  // restore: Part 1 plaintext, the public image, its int16 public fragment, a private sink
  if (scratch_bytes) *scratch_bytes = align16u(priv16) + align16u(px) + align16u(pub16) + align16u(priv16);
  return FDS_OK;
}

static int strong_checks(int32_t width, int32_t height, int32_t k, const void* px, const void* img,
                         const void* priv, const void* scratch, const void* key, const void* iv) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (k < 0 || k > 63) return set_err(FDS_E_INVALID, "k must be in 0..63");
  if (!px || !img || !priv || !scratch || !key || !iv) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(px, 8) || misaligned(img, 8) || misaligned(priv, 16) || misaligned(scratch, 16))
    return set_err(FDS_E_INVALID, "images must be 8-byte aligned, private and scratch 16-byte aligned");
  return FDS_OK;
}

int fds_protect_image_strong(const uint8_t* pixels, int32_t width, int32_t height, int32_t k, const uint8_t key[16],
                             const uint8_t iv[16], uint8_t* public_image_out, uint8_t* private_out, void* scratch,
                             void* stream) {
  int rc = strong_checks(width, height, k, pixels, public_image_out, private_out, scratch, key, iv);
  if (rc) return rc;
  uint64_t pub16 = 0, priv16 = 0;
  fds_sizes(width, height, k, &pub16, &priv16);
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int16_t* s_pub = static_cast<int16_t*>(scratch);
  uint8_t* s_plain = static_cast<uint8_t*>(scratch) + align16u(pub16);
  TileArgs a{};                                  // 1. transform, Part 1 left in plaintext
  a.pixels_in = pixels;
  a.pub_out = s_pub;
  a.priv_out = s_plain;
  a.plain_private = 1;
  fill_geometry(a, width, height, k);
  expand_key(key, a.rk);
  iv_words(iv, &a.iv_hi, &a.iv_lo);
  if ((rc = run_protect(a, dev, s, false))) return rc;
  TileArgs b{};                                  // 2. the public image
  b.pub_in = s_pub;
  b.pixels_out = public_image_out;
  b.public_image = 1;
  fill_geometry(b, width, height, k);
  if ((rc = run_restore(b, dev, s))) return rc;
  cudaError_t e = launch_strong_mask(s_plain, public_image_out, public_image_out, width, height, k, s);
  if (e != cudaSuccess) return cuda_fail(e, "mask launch");   // 3. XOR the SHA-512 masks
  e = launch_aes_full(s_plain, private_out, priv16, a.iv_hi, a.iv_lo, a.rk, g_tables[dev].T, s,
                      g_tables[dev].sms, g_tables[dev].counters);        // 4. encrypt Part 1
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "encryption launch");
}

int fds_restore_image_strong(const uint8_t* public_image_in, const uint8_t* private_in, int32_t width,
                             int32_t height, int32_t k, const uint8_t key[16], const uint8_t iv[16],
                             uint8_t* pixels_out, void* scratch, void* stream) {
  int rc = strong_checks(width, height, k, pixels_out, public_image_in, private_in, scratch, key, iv);
  if (rc) return rc;
  uint64_t pub16 = 0, priv16 = 0;
  fds_sizes(width, height, k, &pub16, &priv16);
  const uint64_t px = (uint64_t)width * (uint64_t)height * 3ull;
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* s_plain = static_cast<uint8_t*>(scratch);
  uint8_t* s_img = s_plain + align16u(priv16);
  int16_t* s_pub = reinterpret_cast<int16_t*>(s_img + align16u(px));
  uint8_t* s_sink = reinterpret_cast<uint8_t*>(s_pub) + align16u(pub16);
  uint32_t rk[44];
  expand_key(key, rk);
  uint64_t hi, lo;
  iv_words(iv, &hi, &lo);
  cudaError_t e = launch_aes_full(private_in, s_plain, priv16, hi, lo, rk, g_tables[dev].T, s,
                                  g_tables[dev].sms, g_tables[dev].counters);   // 1. decrypt Part 1
  if (e != cudaSuccess) return cuda_fail(e, "decryption launch");
  e = launch_strong_mask(s_plain, public_image_in, s_img, width, height, k, s);
  if (e != cudaSuccess) return cuda_fail(e, "mask launch");   // 2. remove the masks
  TileArgs a{};                                  // 3. the public coefficients of the public image
  a.pixels_in = s_img;
  a.pub_out = s_pub;
  a.priv_out = s_sink;
  a.plain_private = 1;
  fill_geometry(a, width, height, k);
  if ((rc = run_protect(a, dev, s, false))) return rc;
  TileArgs b{};                                  // 4. restore from plaintext Part 1
  b.pub_in = s_pub;
  b.priv_in = s_plain;
  b.pixels_out = pixels_out;
  b.plain_private = 1;
  fill_geometry(b, width, height, k);
  return run_restore(b, dev, s);
}

// ---- the DWT scheme (Sect. 6.8-6.12, Fig. 18)
int fds_dwt_sizes(int32_t width, int32_t height, uint64_t* level1_bytes, uint64_t* level2_bytes,
                  uint64_t* level3_bytes) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  const uint64_t nb = (uint64_t)(width / 8) * (uint64_t)(height / 8);
  if (level1_bytes) *level1_bytes = 5 * nb;
  if (level2_bytes) *level2_bytes = 16 * nb;
  if (level3_bytes) *level3_bytes = 60 * nb;
  return FDS_OK;
}

static int dwt_checks(int32_t width, int32_t height, const void* data, const void* l1, const void* l2,
                      const void* l3, const void* key, const void* iv) {
  if (bad_dims(width, height)) return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8");
  if (!data || !l1 || !l2 || !l3 || !key || !iv) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(data, 8) || misaligned(l1, 16) || misaligned(l2, 16) || misaligned(l3, 16))
    return set_err(FDS_E_INVALID, "data must be 8-byte aligned, the level streams 16-byte aligned");
  return FDS_OK;
}

int fds_dwt_protect(const uint8_t* data, int32_t width, int32_t height, const uint8_t key[16], const uint8_t iv[16],
                    uint8_t* level1_out, uint8_t* level2_out, uint8_t* level3_out, void* stream) {
  int rc = dwt_checks(width, height, data, level1_out, level2_out, level3_out, key, iv);
  if (rc) return rc;
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  uint32_t rk[44];
  expand_key(key, rk);
  const cudaError_t e = launch_dwt_protect(data, width, height, key, iv, rk, g_tables[dev].T, level1_out,
                                           level2_out, level3_out, (cudaStream_t)stream);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "DWT protect launch");
}

int fds_dwt_restore(const uint8_t* level1_in, const uint8_t* level2_in, const uint8_t* level3_in, int32_t width,
                    int32_t height, const uint8_t key[16], const uint8_t iv[16], uint8_t* data_out, void* stream) {
  int rc = dwt_checks(width, height, data_out, level1_in, level2_in, level3_in, key, iv);
  if (rc) return rc;
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  uint32_t rk[44];
  expand_key(key, rk);
  const cudaError_t e = launch_dwt_restore(level1_in, level2_in, level3_in, width, height, key, iv, rk,
                                           g_tables[dev].T, data_out, (cudaStream_t)stream);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "DWT restore launch");
}

int fds_sha512_constants(uint64_t k_out[80], uint64_t h0_out[8]) {
  if (!k_out || !h0_out) return set_err(FDS_E_INVALID, "null pointer argument");
  sha512_constants(k_out, h0_out);
  return FDS_OK;
}

int fds_tc_basis(int32_t form, uint8_t* out, uint64_t bytes, double* error_bound) {
  if (form != FDS_TC_BF16 && form != FDS_TC_TF32 && form != FDS_TC_F16 && form != FDS_TC_F16_INVERSE)
    return set_err(FDS_E_INVALID, "unknown tensor-core form");
  std::vector<uint8_t> img;
  std::string why;
  double bound = 0;
  double rem = 0;
  const bool ok = form == FDS_TC_F16_INVERSE ? build_mma_inv(img, &bound, why)
                  : form == FDS_TC_F16       ? build_mma_fwd(img, &bound, &rem, why)
                                             : build_tc_b(form, img, why, &bound);
  if (error_bound) *error_bound = bound;
  if (!ok) return set_err(FDS_E_INVALID, "tensor-core table: " + why);
  if (out) {
    if (bytes < img.size()) return set_err(FDS_E_INVALID, "output buffer too small");
    std::memcpy(out, img.data(), img.size());
  }
  return FDS_OK;
}

int fds_debug_dct_tc(int32_t form, const uint8_t* pixels, int32_t width, int32_t height, float* coefs_out,
                     void* stream) {
  if (form != FDS_TC_BF16 && form != FDS_TC_TF32 && form != FDS_TC_F16)
    return set_err(FDS_E_INVALID, "unknown tensor-core form");
  if (bad_dims(width, height) || 3ll * (width / 8) * (height / 8) >= (1ll << 31))
    return set_err(FDS_E_INVALID, "width and height must be positive multiples of 8, 3 W H / 64 < 2^31");
  if (!pixels || !coefs_out) return set_err(FDS_E_INVALID, "null pointer argument");
  if (misaligned(pixels, 8) || misaligned(coefs_out, 4)) return set_err(FDS_E_INVALID, "misaligned buffer");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  TileArgs a{};
  a.pixels_in = pixels;
  a.dbg_coefs = coefs_out;
  fill_geometry(a, width, height, 0);
  set_tables(a, dev);
  cudaError_t e;
  if (form == FDS_TC_F16) {
    e = launch_protect_mma(a, g_tables[dev].mma_fwd, g_tables[dev].mma_fwd_guard, g_tables[dev].mma_fwd_guard_rem,
                           (cudaStream_t)stream, true, g_tables[dev].sms);
  } else {
    a.tc_b = g_tables[dev].tc_b[form];
    e = launch_protect_tc(a, (cudaStream_t)stream, form, true, g_tables[dev].sms);
  }
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "tensor-core debug launch");
}

int fds_debug_exact_round(const int32_t* coords, int32_t* out, int32_t n) {
  if (n < 0) return set_err(FDS_E_INVALID, "negative count");
  if (n > 0 && (!coords || !out)) return set_err(FDS_E_INVALID, "null pointer argument");
  // the range in which the device decision is proven exact (the fused kernels stay far
  // inside it): |N_0| < 2^26 and sum_j>=1 |N_j| < 2^26
  for (int32_t i = 0; i < n; ++i) {
    int64_t s = 0;
    for (int j = 1; j < 8; ++j) s += std::llabs((int64_t)coords[8 * i + j]);
    if (std::llabs((int64_t)coords[8 * i]) >= (1ll << 26) || s >= (1ll << 26))
      return set_err(FDS_E_INVALID, "coordinate vector " + std::to_string(i) + " outside |N_0|, sum |N_j| < 2^26");
  }
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  if (n == 0) return FDS_OK;
  int32_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int32_t) * 9ull * (size_t)n);
  if (e != cudaSuccess) return set_err(FDS_E_NOMEM, "device allocation failed");
  e = cudaMemcpy(d, coords, sizeof(int32_t) * 8ull * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    debug_exact_round_kernel<<<(n + 127) / 128, 128>>>(d, d + 8ull * (size_t)n, n, g_tables[dev].counters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 8ull * (size_t)n, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost);
  const cudaError_t ef = cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "exact-round diagnostic");
  return ef == cudaSuccess ? FDS_OK : cuda_fail(ef, "cudaFree");
}

int fds_counters(uint64_t* out, int reset) {
  if (!out) return set_err(FDS_E_INVALID, "null output");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  unsigned long long h[3];
  if ((e = cudaMemcpyFromSymbol(h, g_counters, sizeof(h))) != cudaSuccess) return cuda_fail(e, "counter read");
  for (int i = 0; i < 3; ++i) out[i] = h[i];
  if (reset) {
    const unsigned long long z[3] = {0, 0, 0};
    if ((e = cudaMemcpyToSymbol(g_counters, z, sizeof(z))) != cudaSuccess) return cuda_fail(e, "counter reset");
    std::lock_guard<std::mutex> lk(g_mu);
    g_failures_seen[dev] = 0;
  }
  return FDS_OK;
}

int fds_status_of_failures(uint64_t seen, uint64_t now) {
  if (now > seen)
    return set_err(FDS_E_TIMEOUT, std::to_string(now - seen) +
                                      " bounded device wait(s) gave up since the last check: the outputs of the "
                                      "launches involved are incomplete");
  return FDS_OK;
}

int fds_debug_set_counters(const uint64_t* values) {
  if (!values) return set_err(FDS_E_INVALID, "null pointer argument");
  int rc = ensure_init();
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  unsigned long long h[3] = {values[0], values[1], values[2]};
  if ((e = cudaMemcpyToSymbol(g_counters, h, sizeof(h))) != cudaSuccess) return cuda_fail(e, "counter write");
  return FDS_OK;
}

int fds_sync(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "asynchronous error");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  unsigned long long h[3];
  if ((e = cudaMemcpyFromSymbol(h, g_counters, sizeof(h))) != cudaSuccess) return cuda_fail(e, "counter read");
  return failure_status(dev, h[2]);
}

const char* fds_last_error(void) { return t_err.c_str(); }

int fds_copy_many(const uint64_t* dsts, const uint64_t* srcs, const uint64_t* bytes, int32_t n, void* stream) {
  if (n < 0 || (n > 0 && (!dsts || !srcs || !bytes))) return set_err(FDS_E_INVALID, "fds_copy_many: bad arguments");
  for (int32_t i = 0; i < n; ++i) {
    if (!bytes[i]) continue;
    if (!dsts[i] || !srcs[i]) return set_err(FDS_E_INVALID, "fds_copy_many: null address in copy " + std::to_string(i));
    const cudaError_t e = cudaMemcpyAsync(reinterpret_cast<void*>(dsts[i]), reinterpret_cast<const void*>(srcs[i]),
                                          (size_t)bytes[i], cudaMemcpyDefault, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, ("fds_copy_many: copy " + std::to_string(i)).c_str());
  }
  return FDS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// batch plans: one persistent launch over every tile of every image
struct fds_plan {
  int dev = 0;
  std::vector<fds_image> images;        // host copy, caller's order
  int32_t n = 0, total_tiles = 0, k_uniform = -1, capacity = 0;
  // schedule per direction (0 protect, 1 restore); per_sm 0 = the kernel's residency
  int32_t per_sm[2] = {0, 0}, dynamic[2] = {0, 0}, aes_pair[2] = {0, 0}, largest_first = 0;
  std::string tuning;                   // JSON list of the last autotune's candidates
  void* mem = nullptr;                  // device: BatchImage[cap], tile_start[cap+1], counter
  void* host = nullptr;                 // pinned staging of reusable plans (fds_plan_reserve)
  cudaEvent_t staged = nullptr;         // the last asynchronous update has left `host`
  fds::BatchImage* d_images = nullptr;
  int32_t* d_tile_start = nullptr;
  unsigned int* d_dispenser = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // protect, restore
  const void* graph_bufs[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  cudaStream_t graph_stream[2] = {nullptr, nullptr};
};

namespace fds {
namespace {

int check_descs(const fds_image* images, int32_t n) {
  if (n <= 0 || !images) return set_err(FDS_E_INVALID, "a plan needs at least one image");
  for (int32_t i = 0; i < n; ++i) {
    const fds_image& d = images[i];
    if (bad_dims(d.width, d.height)) return set_err(FDS_E_INVALID, "image " + std::to_string(i) + ": bad size");
    if (d.k < 0 || d.k > 63) return set_err(FDS_E_INVALID, "image " + std::to_string(i) + ": k out of range");
    if ((d.pixel_offset & 7) || (d.public_offset & 15) || (d.private_offset & 15))
      return set_err(FDS_E_INVALID, "image " + std::to_string(i) + ": misaligned offset");
    if (d.key_slot < 0 || d.key_slot >= FDS_MAX_KEYS || !g_slots[d.key_slot].used)
      return set_err(FDS_E_NO_KEY, "image " + std::to_string(i) + ": key slot not registered");
  }
  return FDS_OK;
}

void drop_graphs(fds_plan* p) {
  for (int i = 0; i < 2; ++i) {
    if (p->graph[i]) cudaGraphExecDestroy(p->graph[i]);
    p->graph[i] = nullptr;
  }
}

// the plan's tables in its current order, into host arrays bi[n] and ts[n + 1]
int build_tables(fds_plan* p, BatchImage* bi, int32_t* ts) {
  std::vector<int> order(p->n);
  for (int i = 0; i < p->n; ++i) order[i] = i;
  if (p->largest_first)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return (int64_t)p->images[x].width * p->images[x].height > (int64_t)p->images[y].width * p->images[y].height;
    });
  int64_t acc = 0;
  for (int j = 0; j < p->n; ++j) {
    const fds_image& d = p->images[order[j]];
    BatchImage& b = bi[j];
    b.pixel_offset = d.pixel_offset;
    b.public_offset = d.public_offset;
    b.private_offset = d.private_offset;
    b.width = d.width;
    b.height = d.height;
    b.k = d.k;
    b.key_slot = d.key_slot;
    iv_words(d.iv, &b.iv_hi, &b.iv_lo);
    ts[j] = (int32_t)acc;
    acc += ((int64_t)(d.width / 8) * (d.height / 8) + kTileBlocks - 1) / kTileBlocks;
  }
  if (acc > (1ll << 30)) return set_err(FDS_E_INVALID, "batch too large");
  ts[p->n] = (int32_t)acc;
  p->total_tiles = (int32_t)acc;
  p->k_uniform = p->n ? p->images[0].k : 0;
  for (int32_t i = 1; i < p->n; ++i)
    if (p->images[i].k != p->k_uniform) p->k_uniform = -1;
  return FDS_OK;
}

// device tables of the plan in its current order (synchronous copy)
int upload_schedule(fds_plan* p) {
  std::vector<BatchImage> bi(p->n + 1);
  std::vector<int32_t> ts(p->n + 1);
  int rc = build_tables(p, bi.data(), ts.data());
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (p->staged) e = cudaEventSynchronize(p->staged);   // an update may still be copying
  if (e == cudaSuccess && p->n)
    e = cudaMemcpy(p->d_images, bi.data(), sizeof(BatchImage) * p->n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tile_start, ts.data(), sizeof(int32_t) * (p->n + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "plan upload");
  drop_graphs(p);
  return FDS_OK;
}

int plan_device(const fds_plan* p) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != p->dev) return set_err(FDS_E_INVALID, "the plan belongs to another device");
  return FDS_OK;
}

TileArgs plan_args(const fds_plan* p, int dir) {
  TileArgs a{};
  a.images = p->d_images;
  a.tile_start = p->d_tile_start;
  a.n_images = p->n;
  a.total_tiles = p->total_tiles;
  a.k = p->k_uniform;
  a.dispenser = p->dynamic[dir] ? p->d_dispenser : nullptr;
  a.aes_pair = p->aes_pair[dir];
  return a;
}

// enqueue one protect (dir 0) or restore (dir 1) of the whole plan on s
int plan_enqueue(fds_plan* p, int dir, const void* b0, const void* b1, const void* b2, cudaStream_t s) {
  TileArgs a = plan_args(p, dir);
  if (p->dynamic[dir]) {
    const cudaError_t e = cudaMemsetAsync(p->d_dispenser, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
  }
  if (dir == 0) {
    a.pixels_in = static_cast<const uint8_t*>(b0);
    a.pub_out = static_cast<int16_t*>(const_cast<void*>(b1));
    a.priv_out = static_cast<uint8_t*>(const_cast<void*>(b2));
    return run_protect(a, p->dev, s, false, p->per_sm[0]);
  }
  a.pub_in = static_cast<const int16_t*>(b0);
  a.priv_in = static_cast<const uint8_t*>(b1);
  a.pixels_out = static_cast<uint8_t*>(const_cast<void*>(b2));
  return run_restore(a, p->dev, s, p->per_sm[1]);
}

// size class of a batch, the key of stored schedules: the median image's tiles and the
// batch's tiles, each rounded up to a power of two, and k when it is uniform
std::string size_class(const fds_plan* p) {
  std::vector<int64_t> t(p->n);
  for (int i = 0; i < p->n; ++i)
    t[i] = ((int64_t)(p->images[i].width / 8) * (p->images[i].height / 8) + kTileBlocks - 1) / kTileBlocks;
  int64_t med = 0;
  if (p->n) {
    std::nth_element(t.begin(), t.begin() + p->n / 2, t.end());
    med = t[p->n / 2];
  }
  auto lg = [](int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
  };
  std::string c = "t" + std::to_string(lg(med)) + "-T" + std::to_string(lg(p->total_tiles)) + "-k";
  return c + (p->k_uniform >= 0 ? std::to_string(p->k_uniform) : std::string("mixed"));
}

std::string dir_json(const fds_plan* p, int dir) {
  return "{\"ctas_per_sm\": " + std::to_string(p->per_sm[dir]) + ", \"dynamic\": " + std::to_string(p->dynamic[dir]) +
         ", \"aes_pair\": " + std::to_string(p->aes_pair[dir]) + "}";
}

std::string schedule_json(const fds_plan* p) {
  return "{\"size_class\": \"" + size_class(p) + "\", \"largest_first\": " + std::to_string(p->largest_first) +
         ", \"protect\": " + dir_json(p, 0) + ", \"restore\": " + dir_json(p, 1) + ", \"candidates\": [" +
         p->tuning + "]}";
}

int plan_buffers_ok(const void* px, const void* pub, const void* priv) {
  if (!px || !priv) return set_err(FDS_E_INVALID, "null buffer");
  if (misaligned(px, 8) || misaligned(pub, 16) || misaligned(priv, 16))
    return set_err(FDS_E_INVALID, "misaligned buffer");
  return FDS_OK;
}

int plan_graph(fds_plan* p, int dir, const void* b0, const void* b1, const void* b2, cudaStream_t s) {
  if (s == nullptr) return set_err(FDS_E_INVALID, "graph launches need a created stream, not the default stream");
  const void* bufs[3] = {b0, b1, b2};
  if (!p->graph[dir] || std::memcmp(bufs, p->graph_bufs[dir], sizeof(bufs)) != 0) {
    if (p->graph[dir]) cudaGraphExecDestroy(p->graph[dir]);
    p->graph[dir] = nullptr;
    int rc = plan_enqueue(p, dir, b0, b1, b2, s);   // plain launch first: sets kernel attributes
    if (rc) return rc;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    rc = plan_enqueue(p, dir, b0, b1, b2, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&p->graph[dir], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    std::memcpy(p->graph_bufs[dir], bufs, sizeof(bufs));
  }
  const cudaError_t e = cudaGraphLaunch(p->graph[dir], s);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "graph launch");
}

// mean time of one launch of direction dir in the plan's current schedule (one warm-up)
int time_direction(fds_plan* p, int dir, const void* b0, const void* b1, const void* b2, int reps, cudaStream_t s,
                   cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  int rc = plan_enqueue(p, dir, b0, b1, b2, s);
  if (rc) return rc;
  cudaError_t e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && !rc && e == cudaSuccess; ++r) rc = plan_enqueue(p, dir, b0, b1, b2, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  if (rc) return rc;
  cudaEventElapsedTime(ms, e0, e1);
  *ms /= (float)reps;
  return FDS_OK;
}

// Time every schedule of protect (and of restore when px_out is given) on this batch and keep
// the fastest.  Tile order is shared by the directions: the order with the smaller sum of the
// two directions' best times wins.  Every candidate and its time is kept for the JSON export.
int plan_autotune(fds_plan* p, const uint8_t* px, int16_t* pub, uint8_t* priv, uint8_t* px_out, int reps,
                  cudaStream_t s) {
  if (!p) return set_err(FDS_E_INVALID, "null plan");
  if (reps < 1) return set_err(FDS_E_INVALID, "reps must be >= 1");
  int rc = plan_device(p);
  if (!rc) rc = plan_buffers_ok(px, pub, priv);
  if (!rc && px_out) rc = plan_buffers_ok(px_out, pub, priv);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return set_err(FDS_E_CUDA, "event creation failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_err(FDS_E_CUDA, "event creation failed");
  }
  const int ndir = px_out ? 2 : 1;
  struct Best {
    float ms = 1e30f;
    int ps = 0, dyn = 0, aes = 0;
  } best[2][2];
  std::string list;
  for (int lf = 0; lf < 2 && !rc; ++lf) {
    if (lf != p->largest_first) {
      p->largest_first = lf;
      const cudaError_t e = cudaDeviceSynchronize();   // in-flight launches read the tables
      rc = e != cudaSuccess ? cuda_fail(e, "synchronize") : upload_schedule(p);
    }
    for (int dir = 0; dir < ndir && !rc; ++dir) {
      const int cap = dir == 0 ? FDS_PROTECT_MAX_CTAS_PER_SM : FDS_RESTORE_MAX_CTAS_PER_SM;
      for (int ps = 1; ps <= cap && !rc; ++ps)
        for (int dyn = 0; dyn < 2 && !rc; ++dyn)
          for (int aes = 0; aes < 2 && !rc; ++aes) {
            p->per_sm[dir] = ps, p->dynamic[dir] = dyn, p->aes_pair[dir] = aes;
            float ms = 0.0f;
            rc = dir == 0 ? time_direction(p, 0, px, pub, priv, reps, s, e0, e1, &ms)
                          : time_direction(p, 1, pub, priv, px_out, reps, s, e0, e1, &ms);
            if (rc) break;
            if (ms < best[lf][dir].ms) best[lf][dir] = {ms, ps, dyn, aes};
            char row[192];
            std::snprintf(row, sizeof(row),
                          "%s{\"direction\": \"%s\", \"largest_first\": %d, \"ctas_per_sm\": %d, \"dynamic\": %d, "
                          "\"aes_pair\": %d, \"ms\": %.5f}",
                          list.empty() ? "" : ", ", dir ? "restore" : "protect", lf, ps, dyn, aes, ms);
            list += row;
          }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  float t0 = 0.0f, t1 = 0.0f;
  for (int dir = 0; dir < ndir; ++dir) t0 += best[0][dir].ms, t1 += best[1][dir].ms;
  const int lf = t1 < t0 ? 1 : 0;
  for (int dir = 0; dir < ndir; ++dir) {
    p->per_sm[dir] = best[lf][dir].ps;
    p->dynamic[dir] = best[lf][dir].dyn;
    p->aes_pair[dir] = best[lf][dir].aes;
  }
  p->tuning = list;
  if (lf != p->largest_first) {
    p->largest_first = lf;
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return upload_schedule(p);
  }
  drop_graphs(p);
  return FDS_OK;
}

}  // namespace
}  // namespace fds

extern "C" {

int fds_plan_create(const fds_image* images, int32_t n, fds_plan** plan_out) {
  if (!plan_out) return set_err(FDS_E_INVALID, "null plan pointer");
  *plan_out = nullptr;
  int rc;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((rc = check_descs(images, n))) return rc;
  }
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  fds_plan* p = new (std::nothrow) fds_plan();
  if (!p) return set_err(FDS_E_NOMEM, "host allocation failed");
  p->dev = dev;
  p->n = n;
  p->capacity = n;
  p->images.assign(images, images + n);
  const size_t img_bytes = (sizeof(BatchImage) * n + 255) & ~(size_t)255;
  const size_t ts_bytes = (sizeof(int32_t) * (n + 1) + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&p->mem, img_bytes + ts_bytes + 256);
  if (e != cudaSuccess) {
    delete p;
    return set_err(FDS_E_NOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  p->d_images = static_cast<BatchImage*>(p->mem);
  p->d_tile_start = reinterpret_cast<int32_t*>(static_cast<char*>(p->mem) + img_bytes);
  p->d_dispenser = reinterpret_cast<unsigned int*>(static_cast<char*>(p->mem) + img_bytes + ts_bytes);
  if ((rc = upload_schedule(p))) {
    cudaFree(p->mem);
    delete p;
    return rc;
  }
  *plan_out = p;
  return FDS_OK;
}

int fds_plan_destroy(fds_plan* plan) {
  if (!plan) return FDS_OK;
  cudaDeviceSynchronize();
  drop_graphs(plan);
  cudaFree(plan->mem);
  if (plan->host) cudaFreeHost(plan->host);
  if (plan->staged) cudaEventDestroy(plan->staged);
  delete plan;
  return FDS_OK;
}

int fds_plan_reserve(int32_t capacity, fds_plan** plan_out) {
  if (!plan_out) return set_err(FDS_E_INVALID, "null plan pointer");
  *plan_out = nullptr;
  if (capacity < 1 || capacity > (1 << 20)) return set_err(FDS_E_INVALID, "capacity must be 1 .. 2^20");
  int dev = 0;
  int rc = ensure_init(&dev);
  if (rc) return rc;
  fds_plan* p = new (std::nothrow) fds_plan();
  if (!p) return set_err(FDS_E_NOMEM, "host allocation failed");
  p->dev = dev;
  p->capacity = capacity;
  const size_t img_bytes = (sizeof(BatchImage) * capacity + 255) & ~(size_t)255;
  const size_t ts_bytes = (sizeof(int32_t) * (capacity + 1) + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&p->mem, img_bytes + ts_bytes + 256);
  if (e == cudaSuccess) e = cudaMallocHost(&p->host, img_bytes + ts_bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->staged, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fds_plan_destroy(p);
    return set_err(FDS_E_NOMEM, std::string("plan allocation failed: ") + cudaGetErrorString(e));
  }
  p->d_images = static_cast<BatchImage*>(p->mem);
  p->d_tile_start = reinterpret_cast<int32_t*>(static_cast<char*>(p->mem) + img_bytes);
  p->d_dispenser = reinterpret_cast<unsigned int*>(static_cast<char*>(p->mem) + img_bytes + ts_bytes);
  *plan_out = p;
  return FDS_OK;
}

int fds_plan_update(fds_plan* plan, const fds_image* images, int32_t n, void* stream) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  if (!plan->host) return set_err(FDS_E_INVALID, "only plans made by fds_plan_reserve can be updated");
  if (n < 0 || n > plan->capacity) return set_err(FDS_E_INVALID, "more images than the plan's capacity");
  int rc = plan_device(plan);
  if (rc) return rc;
  if (n > 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((rc = check_descs(images, n))) return rc;
  }
  cudaError_t e = cudaEventSynchronize(plan->staged);   // previous copy has left the staging
  if (e != cudaSuccess) return cuda_fail(e, "staging wait");
  plan->images.assign(images, images + n);
  plan->n = n;
  const size_t img_bytes = (sizeof(BatchImage) * plan->capacity + 255) & ~(size_t)255;
  BatchImage* bi = static_cast<BatchImage*>(plan->host);
  int32_t* ts = reinterpret_cast<int32_t*>(static_cast<char*>(plan->host) + img_bytes);
  if ((rc = build_tables(plan, bi, ts))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (n) e = cudaMemcpyAsync(plan->d_images, bi, sizeof(BatchImage) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_tile_start, ts, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(plan->staged, s);
  if (e != cudaSuccess) return cuda_fail(e, "plan update");
  drop_graphs(plan);
  return FDS_OK;
}

int fds_plan_set_schedule(fds_plan* plan, int32_t ctas_per_sm, int32_t dynamic, int32_t largest_first) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  if (ctas_per_sm < 0 || ctas_per_sm > FDS_PROTECT_MAX_CTAS_PER_SM)
    return set_err(FDS_E_INVALID, "ctas_per_sm must be 0 .. " + std::to_string(FDS_PROTECT_MAX_CTAS_PER_SM));
  int rc = plan_device(plan);
  if (rc) return rc;
  for (int dir = 0; dir < 2; ++dir) {
    plan->per_sm[dir] = dir == 1 && ctas_per_sm > FDS_RESTORE_MAX_CTAS_PER_SM ? 0 : ctas_per_sm;
    plan->dynamic[dir] = dynamic ? 1 : 0;
    plan->aes_pair[dir] = 0;
  }
  const int lf = largest_first ? 1 : 0;
  if (lf != plan->largest_first) {
    plan->largest_first = lf;
    cudaError_t e = cudaDeviceSynchronize();   // in-flight launches read the tables
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return upload_schedule(plan);
  }
  drop_graphs(plan);
  return FDS_OK;
}

int fds_plan_get_schedule(const fds_plan* plan, int32_t* ctas_per_sm, int32_t* dynamic, int32_t* largest_first) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  if (ctas_per_sm) *ctas_per_sm = plan->per_sm[0];
  if (dynamic) *dynamic = plan->dynamic[0];
  if (largest_first) *largest_first = plan->largest_first;
  return FDS_OK;
}

int fds_plan_set_direction_schedule(fds_plan* plan, int32_t direction, int32_t ctas_per_sm, int32_t dynamic,
                                    int32_t aes_pair) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  if (direction != 0 && direction != 1) return set_err(FDS_E_INVALID, "direction must be 0 (protect) or 1 (restore)");
  const int cap = direction == 0 ? FDS_PROTECT_MAX_CTAS_PER_SM : FDS_RESTORE_MAX_CTAS_PER_SM;
  if (ctas_per_sm < 0 || ctas_per_sm > cap)
    return set_err(FDS_E_INVALID, "ctas_per_sm must be 0 .. " + std::to_string(cap) + " for this direction");
  int rc = plan_device(plan);
  if (rc) return rc;
  plan->per_sm[direction] = ctas_per_sm;
  plan->dynamic[direction] = dynamic ? 1 : 0;
  plan->aes_pair[direction] = aes_pair ? 1 : 0;
  drop_graphs(plan);
  return FDS_OK;
}

int fds_plan_get_direction_schedule(const fds_plan* plan, int32_t direction, int32_t* ctas_per_sm,
                                    int32_t* dynamic, int32_t* aes_pair) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  if (direction != 0 && direction != 1) return set_err(FDS_E_INVALID, "direction must be 0 (protect) or 1 (restore)");
  if (ctas_per_sm) *ctas_per_sm = plan->per_sm[direction];
  if (dynamic) *dynamic = plan->dynamic[direction];
  if (aes_pair) *aes_pair = plan->aes_pair[direction];
  return FDS_OK;
}

int fds_plan_protect(fds_plan* plan, const uint8_t* pixels, int16_t* public_out, uint8_t* private_out,
                     void* stream) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  int rc = plan_device(plan);
  if (!rc) rc = plan_buffers_ok(pixels, public_out, private_out);
  return rc ? rc : plan_enqueue(plan, 0, pixels, public_out, private_out, (cudaStream_t)stream);
}

int fds_plan_restore(fds_plan* plan, const int16_t* public_in, const uint8_t* private_in,
                     uint8_t* pixels_out, void* stream) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  int rc = plan_device(plan);
  if (!rc) rc = plan_buffers_ok(pixels_out, public_in, private_in);
  return rc ? rc : plan_enqueue(plan, 1, public_in, private_in, pixels_out, (cudaStream_t)stream);
}

int fds_plan_protect_graph(fds_plan* plan, const uint8_t* pixels, int16_t* public_out,
                           uint8_t* private_out, void* stream) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  int rc = plan_device(plan);
  if (!rc) rc = plan_buffers_ok(pixels, public_out, private_out);
  return rc ? rc : plan_graph(plan, 0, pixels, public_out, private_out, (cudaStream_t)stream);
}

int fds_plan_restore_graph(fds_plan* plan, const int16_t* public_in, const uint8_t* private_in,
                           uint8_t* pixels_out, void* stream) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  int rc = plan_device(plan);
  if (!rc) rc = plan_buffers_ok(pixels_out, public_in, private_in);
  return rc ? rc : plan_graph(plan, 1, public_in, private_in, pixels_out, (cudaStream_t)stream);
}

int fds_plan_autotune(fds_plan* plan, const uint8_t* pixels, int16_t* public_out, uint8_t* private_out,
                      int32_t reps, void* stream) {
  return fds::plan_autotune(plan, pixels, public_out, private_out, nullptr, reps, (cudaStream_t)stream);
}

int fds_plan_autotune_directions(fds_plan* plan, const uint8_t* pixels, int16_t* public_buf,
                                 uint8_t* private_buf, uint8_t* pixels_out, int32_t reps, void* stream) {
  if (!pixels_out) return set_err(FDS_E_INVALID, "null buffer");
  return fds::plan_autotune(plan, pixels, public_buf, private_buf, pixels_out, reps, (cudaStream_t)stream);
}

int fds_plan_schedule_json(const fds_plan* plan, char* buf, int64_t capacity, int64_t* length) {
  if (!plan) return set_err(FDS_E_INVALID, "null plan");
  const std::string j = fds::schedule_json(plan);
  if (length) *length = (int64_t)j.size() + 1;
  if (!buf) return FDS_OK;
  if (capacity < (int64_t)j.size() + 1) return set_err(FDS_E_INVALID, "buffer too small for the schedule");
  std::memcpy(buf, j.c_str(), j.size() + 1);
  return FDS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// batch protect without allocation: the batch's descriptor table, tile prefix sums and tile
// counter live in a fixed static device array instead of plan memory
namespace fds {

constexpr size_t kNoAllocImgBytes = sizeof(BatchImage) * FDS_NOALLOC_MAX_IMAGES;
constexpr size_t kNoAllocTsBytes = ((sizeof(int32_t) * (FDS_NOALLOC_MAX_IMAGES + 1)) + 255) & ~(size_t)255;
constexpr size_t kNoAllocBytes = kNoAllocImgBytes + kNoAllocTsBytes + 256;

// the scratch area; every call overwrites it (see fds.h)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
unsigned char* g_noalloc_addr[kMaxDevices];   // device address of the scratch, per device
}  // namespace

// One chunk of the batch's tables, passed BY VALUE as a kernel parameter (under the 4 KB
// parameter limit), so that nothing depends on the lifetime of a host buffer: the values
// are captured when the launch is enqueued.
constexpr int kNoAllocChunk = 64;
struct NoAllocChunk {
  BatchImage img[kNoAllocChunk];
  int32_t ts[kNoAllocChunk + 1];
  int32_t first, count, ts_count, reset_counter;
};
static_assert(sizeof(NoAllocChunk) <= 4000, "kernel parameter limit");

__global__ void noalloc_upload_kernel(const __grid_constant__ NoAllocChunk c, BatchImage* img, int32_t* ts,
                                      unsigned int* counter) {
  const int t = threadIdx.x;
  if (t < c.count) img[c.first + t] = c.img[t];
  if (t < c.ts_count) ts[c.first + t] = c.ts[t];
  if (t == 0 && c.reset_counter) *counter = 0u;   // the tile counter must start at zero
}

}  // namespace fds

extern "C" int fds_protect_batch_noalloc(const uint8_t* pixels, int16_t* public_out, uint8_t* private_out,
                                         const fds_image* images, int32_t n, void* stream) {
  if (n < 1 || n > FDS_NOALLOC_MAX_IMAGES)
    return set_err(FDS_E_INVALID, "fds_protect_batch_noalloc takes 1 to " +
                                      std::to_string(FDS_NOALLOC_MAX_IMAGES) + " images, got " +
                                      std::to_string(n));
  int rc;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((rc = check_descs(images, n))) return rc;
  }
  if ((rc = plan_buffers_ok(pixels, public_out, private_out))) return rc;
  {   // the whole batch is checked before anything is enqueued
    int64_t tiles = 0;
    for (int32_t i = 0; i < n; ++i)
      tiles += ((int64_t)(images[i].width / 8) * (images[i].height / 8) + kTileBlocks - 1) / kTileBlocks;
    if (tiles > (1ll << 30)) return set_err(FDS_E_INVALID, "batch too large");
  }
  int dev = 0;
  if ((rc = ensure_init(&dev))) return rc;
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_noalloc_addr[dev]) {   // once per device, with that device current
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "scratch address");
      g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  BatchImage* d_img = reinterpret_cast<BatchImage*>(base);
  int32_t* d_ts = reinterpret_cast<int32_t*>(base + kNoAllocImgBytes);
  unsigned int* d_counter = reinterpret_cast<unsigned int*>(base + kNoAllocImgBytes + kNoAllocTsBytes);
  // descriptors and tile prefix sums, chunk by chunk as kernel parameters
  NoAllocChunk c;
  int64_t acc = 0;
  int32_t k_uniform = images[0].k;
  for (int32_t c0 = 0; c0 < n; c0 += kNoAllocChunk) {
    const int32_t m = std::min<int32_t>(kNoAllocChunk, n - c0);
    std::memset(&c, 0, sizeof(c));
    for (int32_t j = 0; j < m; ++j) {
      const fds_image& d = images[c0 + j];
      BatchImage& b = c.img[j];
      b.pixel_offset = d.pixel_offset;
      b.public_offset = d.public_offset;
      b.private_offset = d.private_offset;
      b.width = d.width;
      b.height = d.height;
      b.k = d.k;
      b.key_slot = d.key_slot;
      iv_words(d.iv, &b.iv_hi, &b.iv_lo);
      if (d.k != k_uniform) k_uniform = -1;
      c.ts[j] = (int32_t)acc;
      acc += ((int64_t)(d.width / 8) * (d.height / 8) + kTileBlocks - 1) / kTileBlocks;
    }
    const bool last = c0 + m == n;                 // the last chunk also writes tile_start[n]
    if (last) c.ts[m] = (int32_t)acc;
    c.first = c0;
    c.count = m;
    c.ts_count = m + (last ? 1 : 0);
    c.reset_counter = last ? 1 : 0;
    noalloc_upload_kernel<<<1, kNoAllocChunk + 1, 0, s>>>(c, d_img, d_ts, d_counter);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scratch upload");
  }
  TileArgs a{};
  a.pixels_in = pixels;
  a.pub_out = public_out;
  a.priv_out = private_out;
  a.images = d_img;
  a.tile_start = d_ts;
  a.n_images = n;
  a.total_tiles = (int32_t)acc;
  a.k = k_uniform;
  a.dispenser = d_counter;
  return run_protect(a, dev, s, false);
}
