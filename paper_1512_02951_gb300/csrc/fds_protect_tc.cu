// Tensor-core protect kernel (precision form): the 8x8 DCT-II of 128 channel-blocks at a time
// as one tcgen05 MMA, D[128 x N] = A[128 x 64] B[N x 64]^T, then the same exact rounding,
// zigzag fragmentation and AES-128-CTR as the float32 CUDA-core kernel (Sect. 6.3.1, 6.4.2).
//
// Exactness by construction.  A holds the 64 pixels of a channel-block, exact in bf16 / tf32.
// The basis matrix B[(u,v)][(y,x)] = b_u(y) b_v(x) is split into integer limbs:
//   BF16, three limbs:  B ~ (L0 + L1 2^-8 + L2 2^-16) 2^-9,  |L| <= 128
//   TF32, two limbs:    B ~ (L0 + L1 2^-11) 2^-12,           |L| <= 1024
// and each limb has its own block of 64 output columns.  Every product is an integer below
// 2^15 (2^18) and every partial sum an integer below 2^24, so the FP32 accumulators hold the
// exact integer dot products.  The CUDA cores combine the limbs with two (one) fused
// multiply-adds.  The only errors are the split remainder, 255 sum_(y,x) |B - limbs| <= 1.62e-4
// (BF16) resp. 6.56e-4 (TF32) -- the host recomputes this bound when it builds the limb
// table and refuses to run if it exceeds the budget -- and the combining roundings
// (<= 6.2e-5 for |F| <= 924, the largest AC coefficient of 8-bit pixels).  So guards of
// 2^-11 (BF16) and 2^-10 (TF32) around each half-integer are rigorous, and everything inside
// a guard is re-decided exactly from integer coordinates, as in the CUDA-core kernel.  The
// four rational coefficients (u, v in {0, 4}, B = +-1/8) come out exactly from limb 0.
//
// Per tile of 128 consecutive channel-blocks (one TMEM lane and one thread each):
//   A. pixels of the <= 44 blocks the tile touches are in shared memory (cp.async, one tile
//      ahead); each thread writes its A row (SW128 K-major layout) and the next tile's
//      pixels start loading; the previous tile's fragments leave by bulk store
//   B. one thread issues the MMA (4 or 8 k-steps) and commits it to an mbarrier
//   1. every thread reads its lane's accumulators (tcgen05.ld), combines, rounds, writes
//      int16 to the staging area by zigzag position, queues near-ties
//   C. 2. queued coefficients re-decided exactly
//   D. 3. AES-128-CTR over the private staging
#include "fds_tile.cuh"

namespace fds {

constexpr int kTcCb = 128;                    // channel-blocks per tile = MMA M
constexpr int kTcThreads = kTcCb;
constexpr int kTcMaxBlocks = 44;              // blocks a run of 128 channel-blocks can touch
constexpr int kTcRowB = kTcMaxBlocks * 24;    // one pixel row of the tile
constexpr int kTcPixBytes = 8 * kTcRowB;
constexpr int kTcCoefBytes = kTcCb * 128;     // public + private int16 staging

template <int FORM>
struct TcForm;
template <>
struct TcForm<0> {        // BF16, three limbs, kind::f16
  static constexpr int kLimbs = 3, kN = 192, kElem = 2, kKSteps = 4;
  static constexpr int kABytes = 128 * 128, kBBytes = kTcBBytesBf16, kAtomA = 128 * 128, kAtomB = 192 * 128;
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(192 >> 3) << 17) |
                                     ((uint32_t)(128 >> 4) << 24);
  static constexpr int kTmemCols = 256;
  static constexpr float kGuard = 1.0f / 2048.0f;
  static constexpr float kScale = 1.0f / 512.0f;   // B = limbs 2^-9
};
template <>
struct TcForm<1> {        // TF32, two limbs, kind::tf32
  static constexpr int kLimbs = 2, kN = 128, kElem = 4, kKSteps = 8;
  static constexpr int kABytes = 2 * 128 * 128, kBBytes = kTcBBytesTf32, kAtomA = 128 * 128, kAtomB = 128 * 128;
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                     ((uint32_t)(128 >> 4) << 24);
  static constexpr int kTmemCols = 128;
  static constexpr float kGuard = 1.0f / 1024.0f;
  static constexpr float kScale = 1.0f / 4096.0f;  // B = limbs 2^-12
};

// Shared memory, from a 1024-byte aligned base (the 128-byte swizzle repeats every 1024
// bytes): A and B operands, two pixel tiles, fragment staging (two areas in the BF16 form,
// one in the TF32 form, whose operands are twice as large), AES tables, near-tie queue, misc.
template <int FORM>
struct TcSmem {
  static constexpr int kStages = FORM == 0 ? 2 : 1;
  static constexpr int kA = 0;
  static constexpr int kB = kA + TcForm<FORM>::kABytes;
  static constexpr int kPix = kB + TcForm<FORM>::kBBytes;
  static constexpr int kStage = kPix + 2 * kTcPixBytes;
  static constexpr int kT = kStage + kStages * kTcCoefBytes;
  static constexpr int kQueue = kT + 4096;
  static constexpr int kMisc = kQueue + 4 * kQueueCap;   // ints: queue size, totals; mbarrier; TMEM
  static constexpr int kBytes = kMisc + 64 + 1024;       // + alignment slack
};
static_assert(2 * (TcSmem<0>::kBytes + 1024) <= 228 * 1024, "two BF16 CTAs per SM");
static_assert(2 * (TcSmem<1>::kBytes + 1024) <= 228 * 1024, "two TF32 CTAs per SM");

// SW128 K-major shared-memory matrix descriptor: start address, SBO = 1024 bytes between
// 8-row groups, LBO unused, descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// byte offset of the 16-byte chunk `chunk` of row `row` in a SW128 K-major atom
__device__ __forceinline__ uint32_t sw128_chunk(int row, int chunk) {
  return (uint32_t)(row * 128 + ((chunk ^ (row & 7)) << 4));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int FORM>
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  if (FORM == 0)
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem), "l"(da), "l"(db), "r"(TcForm<FORM>::kIdesc), "r"(acc)
                 : "memory");
  else
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem), "l"(da), "l"(db), "r"(TcForm<FORM>::kIdesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)) : "memory");
}
// 32 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// cp.async the pixels of the blocks that channel-blocks c0 .. c0+ncb-1 touch into `pix`
// (block j of the tile = image block c0/3 + j, rows kTcRowB bytes apart); all threads
__device__ __forceinline__ void tc_load_pixels(const TileArgs& a, long long c0, int ncb, uint8_t* pix) {
  const long long b0 = c0 / 3;
  const int nbt = (int)((c0 + ncb - 1) / 3 - b0) + 1;
  const uint64_t w3 = (uint64_t)a.width * 3ull;
  for (int p = threadIdx.x; p < 3 * nbt; p += kTcThreads) {
    const int j = p / 3, q = p - 3 * j;
    const uint8_t* src = a.pixels_in + block_offset(a.width, (int)(b0 + j)) + 8 * q;
    uint8_t* dst = pix + j * 24 + 8 * q;
#pragma unroll
    for (int y = 0; y < 8; ++y) cp_async8(dst + y * kTcRowB, src + y * w3);
  }
  cp_async_commit();
}

// Row t of the A operand: the 64 pixels (K index 8y + x) of channel ch of tile block j, as
// bf16 (one 16-byte chunk per pixel row) or tf32 (two chunks per row, rows 0-3 in the first
// 128-byte K atom, rows 4-7 in the second), in the 128-byte swizzled K-major layout.
template <int FORM>
__device__ __forceinline__ void tc_write_a(const uint8_t* pix, int j, int ch, int t, uint8_t* sA) {
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    uint32_t w[6];
    load_row_shifted<kTcRowB>(pix, y, j, ch, w);
    uint32_t X[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int byte = 3 * x;   // 2^23 + p as float bits, minus 2^23: the pixel, exactly
      X[x] = __float_as_uint(__uint_as_float(__byte_perm(w[byte >> 2], 0x4B000000u, 0x7440u | (byte & 3))) -
                             8388608.0f);
    }
    if (FORM == 0) {
      const uint4 c = make_uint4(__byte_perm(X[0], X[1], 0x7632u), __byte_perm(X[2], X[3], 0x7632u),
                                 __byte_perm(X[4], X[5], 0x7632u), __byte_perm(X[6], X[7], 0x7632u));
      *reinterpret_cast<uint4*>(sA + sw128_chunk(t, y)) = c;
    } else {
      uint8_t* atom = sA + (y >> 2) * TcForm<1>::kAtomA;
      *reinterpret_cast<uint4*>(atom + sw128_chunk(t, 2 * (y & 3))) = make_uint4(X[0], X[1], X[2], X[3]);
      *reinterpret_cast<uint4*>(atom + sw128_chunk(t, 2 * (y & 3) + 1)) = make_uint4(X[4], X[5], X[6], X[7]);
    }
  }
}

// the staged fragments of tile `tile` to global memory; one thread
__device__ __forceinline__ void tc_store(const TileArgs& a, long long tile, int k, const uint8_t* st) {
  const long long c0 = tile * kTcCb;
  const int ncb = (int)min((long long)kTcCb, 3ll * a.nblocks - c0);
  const int npub = 63 - k;
  const int pub_bytes = ncb * 2 * npub, priv_bytes = ncb * 2 * (k + 1);
  uint8_t* pdst = reinterpret_cast<uint8_t*>(a.pub_out) + (uint64_t)c0 * 2ull * (uint64_t)npub;
  uint8_t* vdst = a.priv_out + (uint64_t)c0 * 2ull * (uint64_t)(k + 1);
  const uint8_t* vsrc = st + kTcCb * 2 * npub;
  if (pub_bytes >> 4) bulk_store(pdst, st, (uint32_t)(pub_bytes & ~15));
  if (priv_bytes >> 4) bulk_store(vdst, vsrc, (uint32_t)(priv_bytes & ~15));
  bulk_commit();
  for (int j = pub_bytes & ~15; j < pub_bytes; j += 2)
    *reinterpret_cast<uint16_t*>(pdst + j) = *reinterpret_cast<const uint16_t*>(st + j);
  for (int j = priv_bytes & ~15; j < priv_bytes; j += 2)
    *reinterpret_cast<uint16_t*>(vdst + j) = *reinterpret_cast<const uint16_t*>(vsrc + j);
}

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}

// one coefficient: integer-exact accumulators d0 (d1, d2) of the limbs -> int16 (low bits of
// the returned word); `near` is set when the value is within the guard of a half-integer
// (pos is a compile-time constant after unrolling)
template <int FORM>
__device__ __forceinline__ uint32_t tc_round(int pos, float d0, float d1, float d2, bool& near, float& F) {
  const int u = pos >> 3, v = pos & 7;
  if ((u == 0 || u == 4) && (v == 0 || v == 4)) {   // d0 = (8 F) * 2^9 resp. 2^12 exactly
    const int T = __float2int_rz(d0 * (8.0f * TcForm<FORM>::kScale));
    F = (float)T * 0.125f;
    near = false;
    return (uint32_t)((T + 4 - (T < 0 ? 1 : 0)) >> 3);
  }
  const float s = FORM == 0 ? fmaf(fmaf(d2, 1.0f / 256.0f, d1), 1.0f / 256.0f, d0) : fmaf(d1, 1.0f / 2048.0f, d0);
  F = s * TcForm<FORM>::kScale;
  const float yv = F + kMagic;
  near = fabsf(F - (yv - kMagic)) > 0.5f - TcForm<FORM>::kGuard;
  return __float_as_uint(yv);
}

// FORM 0: BF16 three-limb, 1: TF32 two-limb.  K >= 0: selection fixed at compile time.
// DEBUG: write the pre-rounding coefficients to a.dbg_coefs instead of fragments.
template <int FORM, int K, bool DEBUG>
__global__ void __launch_bounds__(kTcThreads, 2) protect_tc_kernel(const __grid_constant__ TileArgs a) {
  using Fm = TcForm<FORM>;
  using Sm = TcSmem<FORM>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem + Sm::kA;
  uint8_t* sB = smem + Sm::kB;
  uint32_t* Ts = reinterpret_cast<uint32_t*>(smem + Sm::kT);
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + Sm::kQueue);
  int* misc = reinterpret_cast<int*>(smem + Sm::kMisc);   // [0] queue size [1] queued [2] escalations [3] failures
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Sm::kMisc + 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Sm::kMisc + 32);
  const int t = threadIdx.x, warp = t >> 5;
  const long long ncb_total = 3ll * a.nblocks;
  const long long ntiles = (ncb_total + kTcCb - 1) / kTcCb;
  if ((long long)blockIdx.x >= ntiles) return;
  const int k = K >= 0 ? K : a.k;
  const int npub = 63 - k;

  // setup: tables, the B operand (already in its swizzled byte order), barrier, TMEM
  for (int i = t; i < 1024; i += kTcThreads) Ts[i] = a.T[i];
  for (int i = t; i < Fm::kBBytes / 16; i += kTcThreads) reinterpret_cast<uint4*>(sB)[i] = a.tc_b[i];
  if (t < 4) misc[t] = 0;
  if (t == 0) mbar_init(mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "n"(Fm::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
  {
    const long long c0 = (long long)blockIdx.x * kTcCb;
    tc_load_pixels(a, c0, (int)min((long long)kTcCb, ncb_total - c0), smem + Sm::kPix);
  }

  int it = 0;
  bool have_prev = false, timed_out = false;
  for (;; ++it) {
    const long long tile = (long long)blockIdx.x + (long long)it * gridDim.x;
    if (tile >= ntiles) break;
    const long long nxt = tile + gridDim.x;
    const int buf = it & 1;
    const long long c0 = tile * kTcCb;
    const int ncb = (int)min((long long)kTcCb, ncb_total - c0);
    uint8_t* pix = smem + Sm::kPix + buf * kTcPixBytes;
    uint8_t* st = smem + Sm::kStage + (it % Sm::kStages) * kTcCoefBytes;
    int16_t* pubst = reinterpret_cast<int16_t*>(st);
    int16_t* privst = reinterpret_cast<int16_t*>(st + kTcCb * 2 * npub);
    cp_async_wait_all();
    if (t == 0) misc[0] = 0;
    __syncthreads();                                                       // A
    if (!DEBUG && t == 0 && have_prev)
      tc_store(a, tile - gridDim.x, k, smem + Sm::kStage + ((it - 1) % Sm::kStages) * kTcCoefBytes);
    if (nxt < ntiles)
      tc_load_pixels(a, nxt * kTcCb, (int)min((long long)kTcCb, ncb_total - nxt * kTcCb),
                     smem + Sm::kPix + (buf ^ 1) * kTcPixBytes);
    const long long g = c0 + t;
    const int j = (int)(g / 3 - c0 / 3), ch = (int)(g % 3);
    tc_write_a<FORM>(pix, j, ch, t, sA);
    fence_proxy_async();
    if (!DEBUG && t == 0) bulk_wait_read<Sm::kStages - 1>();   // staging `st` is free again
    __syncthreads();                                                       // B
    if (t == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int s = 0; s < Fm::kKSteps; ++s) {
        const int atom = FORM == 0 ? 0 : s >> 2, sub = FORM == 0 ? s : s & 3;
        tc_mma<FORM>(tmem, sw128_desc(a0 + atom * Fm::kAtomA) + 2 * sub, sw128_desc(b0 + atom * Fm::kAtomB) + 2 * sub,
                     s > 0 ? 1u : 0u);
      }
      tc_commit(mbar);
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait(mbar, (uint32_t)(it & 1)));
    if (ok) {
      tc_fence_after();
      const bool active = t < ncb;
      int16_t* pub_cb = pubst + t * npub;
      int16_t* priv_cb = privst + t * (k + 1);
      uint32_t mlo = 0, mhi = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t r0[32], r1[32], r2[32];
        tc_ld32(tlane + 32 * h, r0);
        tc_ld32(tlane + 64 + 32 * h, r1);
        if (FORM == 0) tc_ld32(tlane + 128 + 32 * h, r2);
        tc_wait_ld();
        if (active) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int pos = 32 * h + i;
            bool near;
            float F;
            const uint32_t q = tc_round<FORM>(pos, __uint_as_float(r0[i]), __uint_as_float(r1[i]),
                                              FORM == 0 ? __uint_as_float(r2[i]) : 0.0f, near, F);
            if (DEBUG) {
              a.dbg_coefs[(uint64_t)g * 64ull + pos] = F;
            } else {
              const int z = zigzag_of(pos >> 3, pos & 7);
              if (z <= k)
                priv_cb[z] = (int16_t)q;
              else
                pub_cb[z - k - 1] = (int16_t)q;
              if (near) {
                if (h == 0)
                  mlo |= 1u << i;
                else
                  mhi |= 1u << i;
              }
            }
          }
        }
      }
      uint64_t mask = ((uint64_t)mhi << 32) | mlo;
      while (mask) {
        const int pos = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const int idx = atomicAdd(&misc[0], 1);
        if (idx < kQueueCap) {
          queue[idx] = ((uint32_t)t << 8) | (uint32_t)pos;
        } else {   // queue full: decide here
          int n[9], esc = 0;
          bool fail = false;
          coords_fwd<kTcRowB>(pix, j, ch, pos, a.cfwd, n);
          const int q = exact_round(n, &esc, &fail);
          const int z = zigzag_of(pos >> 3, pos & 7);
          if (z <= k)
            priv_cb[z] = (int16_t)q;
          else
            pub_cb[z - k - 1] = (int16_t)q;
          if (esc) atomicAdd(&misc[2], esc);
          if (fail) atomicAdd(&misc[3], 1);
        }
      }
    }
    tc_fence_before();
    if (__syncthreads_or(!ok)) {                                           // C
      timed_out = true;
      break;
    }
    if (DEBUG) continue;
    {
      const int nq = min(misc[0], kQueueCap);
      int esc = 0;
      bool fail = false;
      for (int i = t; i < nq; i += kTcThreads) {
        const uint32_t e = queue[i];
        const int et = (int)(e >> 8), pos = (int)(e & 255);
        const long long eg = c0 + et;
        int n[9];
        coords_fwd<kTcRowB>(pix, (int)(eg / 3 - c0 / 3), (int)(eg % 3), pos, a.cfwd, n);
        const int q = exact_round(n, &esc, &fail);
        const int z = zigzag_of(pos >> 3, pos & 7);
        if (z <= k)
          privst[et * (k + 1) + z] = (int16_t)q;
        else
          pubst[et * npub + z - k - 1] = (int16_t)q;
      }
      if (esc) atomicAdd(&misc[2], esc);
      if (fail) atomicAdd(&misc[3], 1);
      if (t == 0) misc[1] += misc[0];
    }
    __syncthreads();                                                       // D
    {   // AES-128-CTR over the tile's private bytes (a whole number of 16-byte blocks from the
        // tile's first byte, which is 16-byte aligned in the message)
      const int nblk = (ncb * 2 * (k + 1) + 15) >> 4;
      const uint64_t first = ((uint64_t)c0 * 2ull * (uint64_t)(k + 1)) >> 4;
      for (int i = t; i < nblk; i += kTcThreads) {
        uint32_t s4[4];
        ctr_block(a.iv_hi, a.iv_lo, first + i, s4);
        aes128_encrypt(s4, a.rk, Ts);
        uint4* p = reinterpret_cast<uint4*>(privst) + i;
        uint4 d = *p;
        d.x ^= s4[0];
        d.y ^= s4[1];
        d.z ^= s4[2];
        d.w ^= s4[3];
        *p = d;
      }
    }
    fence_proxy_async();
    have_prev = true;
  }
  __syncthreads();
  if (t == 0) {
    if (!DEBUG && have_prev && !timed_out) {
      const long long last = (long long)blockIdx.x + (long long)(it - 1) * gridDim.x;
      tc_store(a, last, k, smem + Sm::kStage + ((it - 1) % Sm::kStages) * kTcCoefBytes);
    }
    bulk_wait_all();
    if (timed_out) misc[3] += 1;
    if (a.counters) {
      if (misc[1]) atomicAdd(&a.counters[0], (unsigned long long)misc[1]);
      if (misc[2]) atomicAdd(&a.counters[1], (unsigned long long)misc[2]);
      if (misc[3]) atomicAdd(&a.counters[2], (unsigned long long)misc[3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(Fm::kTmemCols)
                              : "memory");
}

template <int FORM, int K, bool DEBUG>
static cudaError_t tc_launch_k(const TileArgs& a, cudaStream_t s, int sms) {
  static bool attr[kMaxAttrDevices];
  cudaError_t e = smem_attr_once(protect_tc_kernel<FORM, K, DEBUG>, TcSmem<FORM>::kBytes, attr);
  if (e != cudaSuccess) return e;
  const long long ntiles = (3ll * a.nblocks + kTcCb - 1) / kTcCb;
  const long long grid = ntiles < 2ll * sms ? ntiles : 2ll * sms;
  if (grid > 0) protect_tc_kernel<FORM, K, DEBUG><<<(unsigned)grid, kTcThreads, TcSmem<FORM>::kBytes, s>>>(a);
  return cudaGetLastError();
}

template <int FORM>
static cudaError_t tc_launch_form(const TileArgs& a, cudaStream_t s, bool debug, int sms) {
  if (debug) return tc_launch_k<FORM, 0, true>(a, s, sms);
  if (a.k == 0) return tc_launch_k<FORM, 0, false>(a, s, sms);
  if (a.k == 5) return tc_launch_k<FORM, 5, false>(a, s, sms);
  return tc_launch_k<FORM, -1, false>(a, s, sms);
}

cudaError_t launch_protect_tc(const TileArgs& a, cudaStream_t s, int form, bool debug, int sms) {
  return form == 0 ? tc_launch_form<0>(a, s, debug, sms) : tc_launch_form<1>(a, s, debug, sms);
}

}  // namespace fds
