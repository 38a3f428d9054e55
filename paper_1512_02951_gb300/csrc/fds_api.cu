// C ABI of the selective-protection library (include/fds.h): argument checks, key registry,
// device tables, and the launches of the fused protect / restore kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "fds.h"
#include "fds_tile.cuh"

namespace fds {

// device tables: AES T-table, stage-2 fixed-point DCT basis tables, fallback counters
__device__ uint32_t g_T0[256];
__device__ int32_t g_bfwd[64 * 64];
__device__ int32_t g_binv[64 * 64];
__device__ unsigned long long g_counters[3];

__global__ void init_tables_kernel() {
  const int t = threadIdx.x;
  g_T0[t] = aes_t0((uint8_t)t);
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
  const uint32_t* T0;
  const int32_t* bfwd;
  const int32_t* binv;
  unsigned long long* counters;
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

// Initialise the current device (once) and return its index in *dev_out.
int ensure_init(int* dev_out = nullptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_err(FDS_E_INVALID, "device index out of range");
  if (dev_out) *dev_out = dev;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ready[dev]) return FDS_OK;
  // stage-2 tables in double precision: round(8 b_u(y) b_v(x) 2^28)
  static int32_t hf[64 * 64], hi[64 * 64];
  uint8_t zz[64];
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v) zz[8 * u + v] = (uint8_t)zigzag_of(u, v);
  const double pi = 3.14159265358979323846264338327950288;
  auto basis = [&](int u, int y) {
    return (u == 0 ? std::sqrt(0.125) : 0.5) * std::cos((2 * y + 1) * u * pi / 16.0);
  };
  for (int u = 0; u < 8; ++u)
    for (int v = 0; v < 8; ++v)
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) {
          const int32_t val = (int32_t)std::llround(8.0 * basis(u, y) * basis(v, x) * (double)(1 << kFixShift));
          hf[(8 * u + v) * 64 + 8 * y + x] = val;
          hi[(8 * y + x) * 64 + zz[8 * u + v]] = val;
        }
  if ((e = cudaMemcpyToSymbol(g_bfwd, hf, sizeof(hf))) != cudaSuccess) return cuda_fail(e, "table upload");
  if ((e = cudaMemcpyToSymbol(g_binv, hi, sizeof(hi))) != cudaSuccess) return cuda_fail(e, "table upload");
  init_tables_kernel<<<1, 256>>>();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "init kernel launch");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "init kernel");
  DevTables& tb = g_tables[dev];
  void* p = nullptr;
  if ((e = cudaGetSymbolAddress(&p, g_T0)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.T0 = static_cast<const uint32_t*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_bfwd)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.bfwd = static_cast<const int32_t*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_binv)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.binv = static_cast<const int32_t*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_counters)) != cudaSuccess) return cuda_fail(e, "symbol address");
  tb.counters = static_cast<unsigned long long*>(p);
  g_ready[dev] = true;
  return FDS_OK;
}

bool bad_dims(int32_t w, int32_t h) {
  return w <= 0 || h <= 0 || (w & 7) || (h & 7) || (int64_t)(w / 8) * (int64_t)(h / 8) > (1ll << 30);
}

int run_protect(TileArgs& a, int dev, cudaStream_t s, bool debug) {
  a.T0 = g_tables[dev].T0;
  a.bfwd = g_tables[dev].bfwd;
  a.binv = g_tables[dev].binv;
  a.counters = g_tables[dev].counters;
  const cudaError_t e = launch_protect(a, s, debug);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "protect launch");
}

int run_restore(TileArgs& a, int dev, cudaStream_t s) {
  a.T0 = g_tables[dev].T0;
  a.bfwd = g_tables[dev].bfwd;
  a.binv = g_tables[dev].binv;
  a.counters = g_tables[dev].counters;
  const cudaError_t e = launch_restore(a, s);
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "restore launch");
}

void fill_geometry(TileArgs& a, int32_t w, int32_t h, int32_t k) {
  a.width = w;
  a.bx_count = w / 8;
  a.nblocks = (w / 8) * (h / 8);
  a.k = k;
}

bool misaligned(const void* p, uintptr_t align) { return ((uintptr_t)p & (align - 1)) != 0; }

}  // namespace
}  // namespace fds

using namespace fds;

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
      g_slots[i].used = true;
      expand_key(key, g_slots[i].rk);
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

int fds_counters(uint64_t* out, int reset) {
  if (!out) return set_err(FDS_E_INVALID, "null output");
  int rc = ensure_init();
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  unsigned long long h[3];
  if ((e = cudaMemcpyFromSymbol(h, g_counters, sizeof(h))) != cudaSuccess) return cuda_fail(e, "counter read");
  for (int i = 0; i < 3; ++i) out[i] = h[i];
  if (reset) {
    const unsigned long long z[3] = {0, 0, 0};
    if ((e = cudaMemcpyToSymbol(g_counters, z, sizeof(z))) != cudaSuccess) return cuda_fail(e, "counter reset");
  }
  return FDS_OK;
}

int fds_sync(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  e = cudaGetLastError();
  return e == cudaSuccess ? FDS_OK : cuda_fail(e, "asynchronous error");
}

const char* fds_last_error(void) { return t_err.c_str(); }

}  // extern "C"
