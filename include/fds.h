/*
 * fds.h -- C ABI of the GB300 selective-protection library.
 *
 * The library implements the "first level of protection" of selective encryption for RGB
 * bitmaps (Memmi, Kapusta, Lambein, Qiu, "Data Protection: Combining Fragmentation,
 * Encryption, and Dispersion", Sect. 6.3.1, Fig. 6):
 *
 *   protect: every 8x8 block of every colour channel gets a 2-D DCT-II (Sect. 6.4.2); each
 *            coefficient is rounded to int16 (Sect. 6.4.3); the coefficients at zigzag
 *            positions 0..k form the confidential fragment (Part 1), which is encrypted with
 *            AES-128 in counter mode (Sect. 6.12, Sect. 6.5.2); positions k+1..63 form the
 *            public fragment (Part 2).  k = 5 is the paper's default selection [0,0], [0,1],
 *            [1,0], [2,0], [1,1], [0,2]; k = 0 keeps only the DC coefficient (Sect. 6.2.1).
 *   restore: decrypt Part 1, merge it with Part 2, inverse DCT, round, clamp to [0, 255]
 *            (defragmentation, Sect. 3.2 and Sect. 5.2 Fig. 3).
 *
 * Conventions that the paper leaves open, fixed here:
 *   - DCT: orthonormal DCT-II, no level shift (the DC of an 8-bit block is at most 2040,
 *     Sect. 6.4.3); F[u][v] with u the vertical and v the horizontal frequency.
 *   - Rounding: half away from zero, decided on the exact real value of the coefficient
 *     (or pixel).  Every output is therefore a pure function of the input, bit for bit.
 *   - Zigzag: the JPEG scan (anti-diagonals u + v, alternating direction, starting
 *     [0,0], [0,1], [1,0], [2,0], ...).
 *   - Image: H x W x 3 uint8, row-major, channels interleaved; W and H multiples of 8.
 *   - Public fragment: int16 [H/8][W/8][3][63 - k], zigzag positions k+1..63 in order.
 *   - Private fragment: the little-endian int16 stream [H/8][W/8][3][k + 1] (zigzag 0..k),
 *     AES-128-CTR encrypted as one message per image: keystream block j is
 *     AES_K(IV + j), IV the 16-byte initial counter block read as a big-endian 128-bit
 *     integer, addition modulo 2^128 (OpenSSL's aes-128-ctr).  The caller must never reuse
 *     a (key, counter) pair across images.
 *
 * Memory: every pointer argument marked "device" is a CUDA device pointer on the device
 * passed to fds_init; "host" pointers are ordinary host memory.  The caller owns every
 * buffer; the library never frees or retains caller memory.  Device buffers must be
 * 16-byte aligned (pixels: 8-byte aligned).
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Kernels are enqueued
 * asynchronously; argument errors are reported synchronously by the return value, errors
 * of the enqueued work by the next call that synchronises (fds_sync) or by the CUDA
 * runtime.
 *
 * Errors: every function returns FDS_OK (0) or a negative FDS_E_* code and never aborts or
 * prints; fds_last_error() gives a message for the calling thread's last failure.
 */
#ifndef FDS_H
#define FDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDS_OK 0
#define FDS_E_INVALID (-1)  /* bad argument: size, alignment, k, null pointer, overflow */
#define FDS_E_NO_KEY (-2)   /* key slot not registered */
#define FDS_E_NOMEM (-3)    /* device or host allocation failed */
#define FDS_E_CUDA (-4)     /* CUDA runtime error; see fds_last_error() */
#define FDS_E_TIMEOUT (-5)  /* a bounded device wait gave up */
#define FDS_E_BUSY (-6)     /* no capacity to admit the work now */

#define FDS_MAX_KEYS 256

/* One image of a batch.  Offsets are in bytes from the batch buffers passed to the call. */
typedef struct fds_image {
  uint64_t pixel_offset;   /* into the pixel buffer; multiple of 8 */
  uint64_t public_offset;  /* into the public buffer; multiple of 16 */
  uint64_t private_offset; /* into the private buffer; multiple of 16 */
  int32_t width;           /* multiple of 8, >= 8 */
  int32_t height;          /* multiple of 8, >= 8 */
  int32_t k;               /* selection: zigzag positions 0..k are private, 0 <= k <= 63 */
  int32_t key_slot;        /* a slot returned by fds_key_register */
  uint8_t iv[16];          /* initial counter block of this image's private message */
} fds_image;

/* Select the CUDA device and build the library's device tables (AES tables, fixed-point
 * constants of the exact rounding path).  Idempotent per device. */
int fds_init(int device);

/* Expand an AES-128 key (FIPS-197 Sect. 5.2) and keep its round keys resident on the
 * device.  key: host, 16 bytes.  *slot_out receives the slot (0 .. FDS_MAX_KEYS-1).
 * FDS_E_BUSY when every slot is taken. */
int fds_key_register(const uint8_t key[16], int32_t* slot_out);

/* Free a key slot.  Work already enqueued with the slot must have completed. */
int fds_key_release(int32_t slot);

/* Sizes in bytes of the public and private fragments of one width x height image at
 * selection k: 2 (63 - k) and 2 (k + 1) bytes per channel-block.  Host pointers. */
int fds_sizes(int32_t width, int32_t height, int32_t k, uint64_t* public_bytes,
              uint64_t* private_bytes);

/* Protect one image (Sect. 6.3.1).  pixels: device, H x W x 3 uint8.  key, iv: host, 16
 * bytes each.  public_out, private_out: device, fds_sizes() bytes. */
int fds_protect_image(const uint8_t* pixels, int32_t width, int32_t height, int32_t k,
                      const uint8_t key[16], const uint8_t iv[16], int16_t* public_out,
                      uint8_t* private_out, void* stream);

/* Restore one image (inverse of fds_protect_image).  public_in, private_in: device.
 * pixels_out: device, H x W x 3 uint8. */
int fds_restore_image(const int16_t* public_in, const uint8_t* private_in, int32_t width,
                      int32_t height, int32_t k, const uint8_t key[16], const uint8_t iv[16],
                      uint8_t* pixels_out, void* stream);

/* Protect a batch of n images (descriptors: host array of n) whose pixels, public and
 * private fragments live at the descriptors' offsets in three device buffers.  Keys are
 * taken from registered slots.  One launch per image. */
int fds_protect(const uint8_t* pixels, int16_t* public_out, uint8_t* private_out,
                const fds_image* images, int32_t n, void* stream);

/* Restore a batch (inverse of fds_protect). */
int fds_restore(const int16_t* public_in, const uint8_t* private_in, uint8_t* pixels_out,
                const fds_image* images, int32_t n, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched form: a plan holds a batch's descriptors and tile schedule in device memory, so
 * that the whole batch runs as ONE persistent launch (every 64-block tile of every image
 * in one grid), optionally captured in a CUDA graph.  Work is the same per image as
 * fds_protect_image / fds_restore_image and so are the outputs, bit for bit.
 */
typedef struct fds_plan fds_plan;

/* Create a plan for n images (host descriptor array, keys by registered slot).  Allocates
 * the plan's device memory (descriptors, tile prefix sums, a tile counter) on the current
 * device.  The key slots must stay registered while the plan is used. */
int fds_plan_create(const fds_image* images, int32_t n, fds_plan** plan_out);

/* Free a plan (synchronises the device first). */
int fds_plan_destroy(fds_plan* plan);

/* Create an empty, reusable plan with room for `capacity` images (device tables plus pinned
 * host staging).  Fill it with fds_plan_update; launching an empty plan does nothing. */
int fds_plan_reserve(int32_t capacity, fds_plan** plan_out);

/* Replace the plan's batch with n <= capacity images.  The tables are copied
 * asynchronously on `stream`: launches of this plan must be on the same stream (or ordered
 * after it).  Waits only for the previous update's copy to have left the staging area. */
int fds_plan_update(fds_plan* plan, const fds_image* images, int32_t n, void* stream);

/* The most a plan's schedule may launch per SM: protect runs one CTA per SM holding up to
 * four independent tile groups of 192 threads (its "ctas_per_sm" counts those groups; one
 * image outside a plan runs three, which share one AES table); restore runs up to two CTAs
 * of 192 threads per SM. */
#define FDS_PROTECT_MAX_CTAS_PER_SM 4
#define FDS_RESTORE_MAX_CTAS_PER_SM 2

/* Schedule of the persistent launches, both directions at once.  ctas_per_sm: tile groups
 * (protect) or CTAs (restore) per SM, 0 = the most (protect 4, restore 2), 1 .. 4 (restore
 * takes values above 2 as 0); dynamic: 0 = static round-robin tile assignment, 1 = tiles handed
 * out by an atomic counter; largest_first: 0 = tiles in descriptor order, 1 = images by
 * decreasing size (shared by the directions).  The lane schedule of both directions goes
 * back to one keystream block per thread.  Re-uploads the tile order when it changes and
 * drops captured graphs.  FDS_E_INVALID for ctas_per_sm outside 0 .. 4. */
int fds_plan_set_schedule(fds_plan* plan, int32_t ctas_per_sm, int32_t dynamic,
                          int32_t largest_first);

/* Read the schedule (the protect direction's ctas_per_sm and dynamic; host pointers, each
 * may be NULL). */
int fds_plan_get_schedule(const fds_plan* plan, int32_t* ctas_per_sm, int32_t* dynamic,
                          int32_t* largest_first);

/* Schedule of one direction (0 = protect, 1 = restore): ctas_per_sm 0 .. the direction's
 * FDS_*_MAX_CTAS_PER_SM, dynamic as above, aes_pair: 0 = each thread of a CTA encrypts one
 * 16-byte keystream block of the tile at a time, 1 = two blocks with their AES rounds
 * interleaved (fewer threads, more independent lookups each; it pays only where a tile has
 * more keystream blocks than a CTA has threads, k > 7).  Drops captured graphs.
 * FDS_E_INVALID for a bad direction or value. */
int fds_plan_set_direction_schedule(fds_plan* plan, int32_t direction, int32_t ctas_per_sm,
                                    int32_t dynamic, int32_t aes_pair);
int fds_plan_get_direction_schedule(const fds_plan* plan, int32_t direction,
                                    int32_t* ctas_per_sm, int32_t* dynamic, int32_t* aes_pair);

/* Time every protect schedule on this batch (tile order x ctas_per_sm 1 .. 4 x dynamic x
 * aes_pair, `reps` launches each after one warm-up, on `stream`) and keep the fastest.  The
 * buffers are written to; their previous contents are lost.  Synchronises the device. */
int fds_plan_autotune(fds_plan* plan, const uint8_t* pixels, int16_t* public_out,
                      uint8_t* private_out, int32_t reps, void* stream);

/* The same for both directions, tuned separately: protect writes public_buf / private_buf,
 * restore reads them and writes pixels_out (all three overwritten).  Each direction keeps
 * its fastest ctas_per_sm / dynamic / aes_pair; the tile order, which the directions share,
 * is the one with the smaller sum of their best times. */
int fds_plan_autotune_directions(fds_plan* plan, const uint8_t* pixels, int16_t* public_buf,
                                 uint8_t* private_buf, uint8_t* pixels_out, int32_t reps,
                                 void* stream);

/* The plan's schedule as a NUL-terminated JSON object: "size_class" (the key under which a
 * caller may store it: "t<a>-T<b>-k<k>", 2^a the median image's tiles of 64 blocks and 2^b
 * the batch's tiles, each rounded up to a power of two, k the uniform k or "mixed"),
 * "largest_first", "protect" and "restore" ({"ctas_per_sm", "dynamic", "aes_pair"}), and
 * "candidates": every schedule the last autotune timed with its mean ms per launch.
 * *length (may be NULL) receives the size including the NUL; buf may be NULL to ask for it.
 * FDS_E_INVALID when capacity is smaller than that size. */
int fds_plan_schedule_json(const fds_plan* plan, char* buf, int64_t capacity, int64_t* length);

/* One persistent launch protecting / restoring every image of the plan.  Buffer pointers
 * and offsets as for fds_protect / fds_restore. */
int fds_plan_protect(fds_plan* plan, const uint8_t* pixels, int16_t* public_out,
                     uint8_t* private_out, void* stream);
int fds_plan_restore(fds_plan* plan, const int16_t* public_in, const uint8_t* private_in,
                     uint8_t* pixels_out, void* stream);

/* The same through a CUDA graph: the first call (or a call with other buffers) captures
 * the counter reset and the launch into a graph owned by the plan; later calls replay it.
 * The first call must not be inside another stream capture. */
int fds_plan_protect_graph(fds_plan* plan, const uint8_t* pixels, int16_t* public_out,
                           uint8_t* private_out, void* stream);
int fds_plan_restore_graph(fds_plan* plan, const int16_t* public_in, const uint8_t* private_in,
                           uint8_t* pixels_out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batch protect that allocates nothing (the paper has no counterpart; this is an interface
 * convenience of this library).
 *
 * Some callers cannot allocate device memory at the point where they protect a batch: a
 * host framework that owns all device memory through its own pool and forbids allocations
 * behind its back, a latency-critical loop in which cudaMalloc / cudaFree would synchronise
 * the device, or an embedded service that must not fail at run time for lack of memory.
 * fds_protect_batch_noalloc gives them the same one-launch batched protect as
 * fds_plan_protect (same outputs, bit for bit) without a plan: the batch's descriptor
 * table, tile prefix sums and tile counter live in one fixed scratch area that the library
 * holds in static device memory (about 214 KB, kept on every GPU that loads the library
 * until the process exits).
 *
 * - n must be 1 .. FDS_NOALLOC_MAX_IMAGES, else FDS_E_INVALID; buffers, offsets and keys as
 *   for fds_protect.  The caller allocates pixels, public_out and private_out.
 * - The first call on a device looks up the scratch area's device address (once per
 *   device, with that device current); make that first call before any stream capture.
 * - Every call reuses the same scratch area and overwrites it on `stream`: calls that can
 *   overlap on the GPU (other streams, other host threads) race and must be serialised by
 *   the caller.
 * - It calls no cudaMalloc, cudaFree or other allocating CUDA routine.
 */
#define FDS_NOALLOC_MAX_IMAGES 4096
int fds_protect_batch_noalloc(const uint8_t* pixels, int16_t* public_out, uint8_t* private_out,
                              const fds_image* images, int32_t n, void* stream);

/* ---------------------------------------------------------------------------------------
 * Full encryption, the paper's comparator for selective encryption (Sect. 6.5, Tables 7, 9,
 * 11: the whole bitmap encrypted): AES-128-CTR over `bytes` bytes, the same keystream
 * convention as the private fragment (block j = AES_K(IV + j), 128-bit big-endian counter).
 * in, out: device, 16-byte aligned; in == out encrypts in place, other overlaps are
 * rejected.  key, iv: host, 16 bytes each.  Decryption is the same call. */
int fds_encrypt_full(const uint8_t* in, uint8_t* out, uint64_t bytes, const uint8_t key[16],
                     const uint8_t iv[16], void* stream);

/* Diagnostics: the float32 coefficients the protect kernel computes before rounding, as
 * float [H/8][W/8][3][8][8] ([u][v] inside a block).  coefs_out: device.  Used to compare
 * the pre-rounding values with a float64 reference (Sect. 6.4.3 precision concern). */
int fds_debug_dct_f32(const uint8_t* pixels, int32_t width, int32_t height,
                      float* coefs_out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Tensor-core precision form of fds_protect_image (Sect. 6.4.2 transform as a matrix
 * product).  The 8x8 DCT-II of 128 channel-blocks at a time is one tcgen05 MMA: pixels
 * (exact in the operand type) times the orthonormal basis split into integer limbs,
 * FP32 accumulate:
 *   FDS_TC_BF16: basis = (L0 + L1 2^-8 + L2 2^-16) 2^-9, bf16 operands, three limbs
 *   FDS_TC_TF32: basis = (L0 + L1 2^-11) 2^-12, tf32 operands, two limbs
 * The accumulators hold exact integers; the coefficient error before rounding is at most
 * 2.3e-4 (BF16) resp. 7.2e-4 (TF32), and every value within 2^-11 (2^-10) of a rounding
 * boundary is re-decided exactly, so the outputs are bit-identical to fds_protect_image.
 * Arguments, layouts and errors as fds_protect_image, and 3 (W/8)(H/8) < 2^31.  A
 * tensor-core wait that gives up (bounded) adds 1 to counter 2 of fds_counters and leaves
 * the outputs incomplete. */
#define FDS_TC_BF16 0
#define FDS_TC_TF32 1
#define FDS_TC_F16 2
#define FDS_TC_F16_K_LIST "0, 5"
/* the inverse transform's table, for fds_tc_basis only */
#define FDS_TC_F16_INVERSE 3
/* FDS_TC_F16 is the warp-specialised form: one persistent CTA per SM, tiles of 128 pixel
 * blocks, thirteen warps.  A control warp moves pixel rows in with bulk copies and, from one
 * elected thread, issues the MMAs (D = A B^T per channel, A = p - 128 in f16, B = the basis
 * with rows in zigzag order split as (L0 + L1 2^-11 + L2 2^-22) 2^-13, |L| <= 2048, so the
 * FP32 accumulators are exact integer sums; the integer part is rounded from limb 0 alone and
 * limbs 1, 2 only form the residual); four work warps de-interleave the pixels into the A
 * operands and generate the CTR keystream ahead of use; eight epilogue warps (two per TMEM
 * lane quadrant, one thread per pixel block) round the accumulators and write the fragments.
 * The error of
 * a coefficient before rounding is below the bound fds_tc_basis reports (about 6e-5, and about
 * 1e-7 + |F| 2^-24 for a value F); values
 * within it of a half-integer are re-decided exactly.  Selections k in FDS_TC_F16_K_LIST,
 * else FDS_E_INVALID. */
int fds_protect_image_tc(int32_t form, const uint8_t* pixels, int32_t width, int32_t height,
                         int32_t k, const uint8_t key[16], const uint8_t iv[16],
                         int16_t* public_out, uint8_t* private_out, void* stream);

/* Restore with the inverse 8x8 transform on tensor cores (Sect. 3.2, Fig. 3; the separable
 * transform of Sect. 6.4.2 as a matrix product; form FDS_TC_F16 only, else FDS_E_INVALID).
 * Per tile of 64 pixel blocks (192 channel-blocks), D = A B^T as tcgen05 MMAs: A = each
 * channel-block's 64 coefficients in zigzag order in f16 (exact, since |q| < 2048), B = the
 * inverse basis, row 8y + x of limb l of 2^9 b_u(y) b_v(x) in zigzag column order, split as
 * L0 + L1 2^-8 + L2 2^-16 with |L| <= 128, so every product and partial sum is an integer
 * below 2^24 and the FP32 accumulators are exact.  A pixel is (D0 + D1 2^-8 + D2 2^-16) 2^-9
 * within S 2^-24 of its exact value (S = sum |q| of its channel-block; fds_tc_basis with
 * FDS_TC_F16_INVERSE reports the proven bound per unit of S); values within S 2^-24 + 2^-22 of a
 * half-integer are re-decided exactly from integer coordinates in Z[cos(pi/16)], so the
 * output equals fds_restore_image's byte for byte for any int16 fragments.  A tile holding a
 * coefficient of magnitude 2048 or more is inverted by the float32 butterflies instead.
 * Arguments, layouts, alignment and errors as fds_restore_image.  One CTA per SM; a
 * tensor-core wait that gives up (bounded) adds 1 to counter 2 of fds_counters, leaves that
 * tile's pixels unwritten and sends the CTA's later tiles to the float32 path. */
int fds_restore_image_tc(int32_t form, const int16_t* public_in, const uint8_t* private_in,
                         int32_t width, int32_t height, int32_t k, const uint8_t key[16],
                         const uint8_t iv[16], uint8_t* pixels_out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Bit-packed storage (Sect. 6.4.3, Table 5): both fragments as bit streams instead of int16
 * words.  FDS_PACK_11 ("11-bit storage", lossless for 8-bit images): DC unsigned in 11 bits,
 * every AC as a sign bit over a 10-bit magnitude.  FDS_PACK_8 ("8-bit storage", lossy): DC in
 * 11 bits, AC as a sign bit over a 7-bit magnitude saturated at 127.  A field takes the next
 * bits of its stream, least significant bit first (stream bit b = bit b % 8 of byte b / 8);
 * channel-blocks in [by][bx][c] order, each with its fields in fragment order (zigzag k+1..63,
 * resp. 0..k); the last byte is zero-padded.  The packed private stream is AES-128-CTR
 * encrypted from the IV like the int16 one.
 * Protect is one launch (the transform packs and encrypts each tile in shared memory); so is
 * restore when the packed public stream is 8-byte aligned (each tile's packed parts land in
 * shared memory, are decrypted and unpacked there), else it decrypts, unpacks to int16 in
 * scratch and runs the restore kernel.
 * fds_sizes_packed gives the packed fragment sizes and the device scratch restore needs (the
 * int16 fragments and the decrypted packed stream; protect, and restore of an 8-byte aligned
 * public stream, do not touch it).  Arguments
 * otherwise as fds_protect_image / fds_restore_image; private and scratch 16-byte aligned, the
 * packed public fragment at any alignment.  scratch: device, owned by the caller, overwritten. */
#define FDS_PACK_11 11
#define FDS_PACK_8 8
int fds_sizes_packed(int32_t form, int32_t width, int32_t height, int32_t k,
                     uint64_t* public_bytes, uint64_t* private_bytes, uint64_t* scratch_bytes);
int fds_protect_image_packed(int32_t form, const uint8_t* pixels, int32_t width, int32_t height,
                             int32_t k, const uint8_t key[16], const uint8_t iv[16],
                             uint8_t* public_out, uint8_t* private_out, void* scratch,
                             void* stream);
int fds_restore_image_packed(int32_t form, const uint8_t* public_in, const uint8_t* private_in,
                             int32_t width, int32_t height, int32_t k, const uint8_t key[16],
                             const uint8_t iv[16], uint8_t* pixels_out, void* scratch,
                             void* stream);

/* Protect / restore with host buffers, the copies overlapped with the kernels (the paper
 * overlaps host and GPU work across images, Sect. 6.5, Fig. 11, Fig. 26; here within one image).
 * The image is cut into `strips` runs of block rows (multiples of 8 rows, so each run's private
 * bytes start on a keystream block); per strip, host -> device copy, kernel and device -> host
 * copy run on three streams joined by events, so copies in both directions overlap the
 * kernels of other strips.  Results are byte-identical to fds_protect_image /
 * fds_restore_image.  fds_protect_image_host: host_pixels (pinned host, H x W x 3) is copied
 * to dev_pixels, protected into dev_public / dev_private (device, kept for later use) and
 * both fragments are copied to host_public / host_private (pinned host).
 * fds_restore_image_host: restores dev_public / dev_private into dev_pixels and copies the
 * pixels to host_pixels.  Kernels run on `stream`: earlier work on it comes
 * first (the copy streams wait for it), and when it completes every copy of the call has
 * completed.  Each caller stream has its own copy streams (up to 16 caller streams per
 * device; further ones share one pair), so calls on different streams, for example two
 * images in flight on two streams with their own buffers, overlap their copies.
 * strips: 1..64.
 * Device alignments as fds_protect_image; host buffers should be pinned (pageable memory
 * works but does not overlap). */
int fds_protect_image_host(const uint8_t* host_pixels, uint8_t* dev_pixels, int32_t width,
                           int32_t height, int32_t k, const uint8_t key[16], const uint8_t iv[16],
                           int16_t* dev_public, uint8_t* dev_private, int16_t* host_public,
                           uint8_t* host_private, int32_t strips, void* stream);
int fds_restore_image_host(const int16_t* dev_public, const uint8_t* dev_private,
                           uint8_t* dev_pixels, uint8_t* host_pixels, int32_t width, int32_t height,
                           int32_t k, const uint8_t key[16], const uint8_t iv[16], int32_t strips,
                           void* stream);

/* The paper's own form of the public fragment (Sect. 6.5.1, Fig. 10; Fig. 7 (b)): the public
 * coefficients as an image.  Per channel-block the zigzag positions 1..k are zero and the DC
 * coefficient is 1024 (= 8 x 128: the zero-mean block shifted to mid-grey), the positions
 * k+1..63 come from the int16 public fragment; the exact inverse DCT is rounded half away
 * from zero and clamped to [0, 255], as in restore.  The public coefficients come back from
 * such an image through fds_protect_image's public output (a constant shift changes only the
 * private DC coefficient).
 * public_in: device int16 [H/8][W/8][3][63-k] (16-byte aligned; may be null when k = 63);
 * image_out: device H x W x 3 uint8 (8-byte aligned), written.  No key: nothing private. */
int fds_public_image(const int16_t* public_in, int32_t width, int32_t height, int32_t k,
                     uint8_t* image_out, void* stream);

/* Statistics used to assess protected images (Sect. 6.6): the per-channel histogram (6.6.1) and
 * exact integer sums for the correlation coefficient of adjacent pixels (6.6.2), over every
 * pair of a pixel and its right, lower and lower-right neighbour:
 *   r = (n Sxy - Sx Sy) / sqrt((n Sxx - Sx^2)(n Syy - Sy^2)).
 * image: device H x W x 3 uint8, any W, H >= 1.  histogram_out: device uint64 [3][256]
 * (channel, level); pair_sums_out: device int64 [3][3][6] = [direction: right, down,
 * down-right][channel][n, Sx, Sy, Sxx, Syy, Sxy].  Both 8-byte aligned and overwritten
 * (cleared on `stream`, then accumulated). */
int fds_image_stats(const uint8_t* image, int32_t width, int32_t height, uint64_t* histogram_out,
                    int64_t* pair_sums_out, void* stream);

/* Strong level of protection (Sect. 6.3.2, Fig. 8; Fig. 7 (d)).  The public fragment is the
 * public image (as fds_public_image) with every channel-block's 64 pixels XORed with the
 * SHA-512 digest (FIPS 180-4) of that block's Part 1 plaintext -- its k+1 int16 coefficients,
 * little-endian, zigzag order -- digest byte 8y+x onto pixel (y, x) of the block, its channel.
 * Part 1 is AES-128-CTR encrypted from the IV exactly as fds_protect_image's private output.
 * Restore decrypts Part 1, removes the masks, recovers the public coefficients from the public
 * image by the forward transform (exact rounding) and restores as fds_restore_image; the
 * public image holds rounded, clamped bytes, so the result is close to, not equal to, the
 * original (its PSNR is the measure, Sect. 6.4.3).
 * fds_sizes_strong: public bytes (W x H x 3), private bytes (2 (k+1) per channel-block) and the
 * scratch both calls need.  Pointers: device; images 8-byte aligned, private and scratch
 * 16-byte aligned; scratch owned by the caller, overwritten.  Asynchronous on `stream`. */
int fds_sizes_strong(int32_t width, int32_t height, int32_t k, uint64_t* public_bytes,
                     uint64_t* private_bytes, uint64_t* scratch_bytes);
int fds_protect_image_strong(const uint8_t* pixels, int32_t width, int32_t height, int32_t k,
                             const uint8_t key[16], const uint8_t iv[16], uint8_t* public_image_out,
                             uint8_t* private_out, void* scratch, void* stream);
int fds_restore_image_strong(const uint8_t* public_image_in, const uint8_t* private_in,
                             int32_t width, int32_t height, int32_t k, const uint8_t key[16],
                             const uint8_t iv[16], uint8_t* pixels_out, void* scratch,
                             void* stream);
/* Selective encryption with the DWT (Sect. 6.8-6.12, Figs. 16-18): lossless, for any data.
 * The data is an H x W matrix of bytes (W, H multiples of 8; arbitrary bytes fill W-byte rows,
 * zero-padded to whole 8-row blocks, Sect. 6.9.3).  Per 8x8 block, in raster order: the bytes
 * minus 128 go through a two-level reversible Le Gall 5/3 DWT (integer lifting, the invertible
 * JPEG 2000 form of Eqs. 1-2: d[n] = x[2n+1] - floor((x[2n] + x[2n+2]) / 2), s[n] = x[2n] +
 * floor((d[n-1] + d[n] + 2) / 4), whole-sample symmetric extension; rows, then columns);
 *   level 1 = second-level LL (4 x 10-bit fields = 5 bytes), AES-128-CTR encrypted as one
 *             message from the IV over all blocks' level-1 bytes;
 *   level 2 = second-level HL, LH (10 bits) and HH (11 bits): 124 bits in 16 bytes, XORed
 *             with bytes 0..15 of SHA-256(key || IV || block index as 8 bytes big-endian ||
 *             level 1 plaintext);
 *   level 3 = first-level HL, LH, HH, 48 x 10 bits = 60 bytes, XORed with bytes 0..59 of
 *             SHA-512(key || IV || block index || level 2 plaintext).
 * Fields are two's complement, least significant bit first; quadrants in the order HL, LH,
 * HH, each row-major.  Levels 1 and 2 are the private fragment, level 3 the public one.
 * Restore inverts every step exactly.
 * Pointers: device; data 8-byte aligned, level streams 16-byte aligned (5, 16 and 60 bytes per
 * block: fds_dwt_sizes).  Asynchronous on `stream`; argument errors are returned at once. */
int fds_dwt_sizes(int32_t width, int32_t height, uint64_t* level1_bytes, uint64_t* level2_bytes,
                  uint64_t* level3_bytes);
int fds_dwt_protect(const uint8_t* data, int32_t width, int32_t height, const uint8_t key[16],
                    const uint8_t iv[16], uint8_t* level1_out, uint8_t* level2_out,
                    uint8_t* level3_out, void* stream);
int fds_dwt_restore(const uint8_t* level1_in, const uint8_t* level2_in, const uint8_t* level3_in,
                    int32_t width, int32_t height, const uint8_t key[16], const uint8_t iv[16],
                    uint8_t* data_out, void* stream);

/* Diagnostics (host only): the SHA-512 constants the library computes from their definition
 * (the first 64 fraction bits of the cube roots of the first 80 primes, of the square roots
 * of the first 8).  k_out: host uint64 [80]; h0_out: host uint64 [8]. */
int fds_sha512_constants(uint64_t k_out[80], uint64_t h0_out[8]);

/* Diagnostics (host only, no device needed): the tensor-core form's B operand as the kernel
 * holds it in shared memory -- row n = 64 l + 8u + v is limb l of the basis function
 * (u, v), K index 8y + x, 128-byte rows, 16-byte chunk c of row n stored at chunk c ^ (n & 7);
 * the TF32 form stores K 0..31 and K 32..63 as two consecutive 128-row blocks; the F16 form
 * has rows n = 64 l + z (z the zigzag index) of limb l of 2^13 b_u(y) b_v(x), three limbs
 * (24576 bytes); FDS_TC_F16_INVERSE gives the inverse transform's table (rows n = 64 l + 8y + x
 * of limb l of 2^9 b_u(y) b_v(x), K = the zigzag index z of (u, v), three limbs, 24576 bytes).
 * out: host, at least 24576 (BF16, F16, F16_INVERSE) or 32768 (TF32) bytes, or NULL.
 * *error_bound (host, or NULL): the proven bound on |computed - exact| of a pre-rounding
 * coefficient of 8-bit pixels; for FDS_TC_F16_INVERSE, of a restored pixel value per unit of
 * sum |q| over its channel-block's coefficients. */
int fds_tc_basis(int32_t form, uint8_t* out, uint64_t bytes, double* error_bound);

/* Diagnostics: the pre-rounding coefficients of the tensor-core form, laid out as in
 * fds_debug_dct_f32.  coefs_out: device. */
int fds_debug_dct_tc(int32_t form, const uint8_t* pixels, int32_t width, int32_t height,
                     float* coefs_out, void* stream);

/* Diagnostics: the exact rounding step of both transforms on its own (Sect. 6.4.3 reading:
 * round half away from zero of the exact value).  For each i, with c(j) = cos(j pi / 16),
 *   8 V_i = coords[8i] + sum_{j=1..7} coords[8i + j] c(j),
 * out[i] = V_i rounded half away from zero, decided exactly: a 64-bit fixed-point evaluation
 * first and, where it is too close to call, a 256-bit one that a norm bound in Z[cos(pi/16)]
 * makes exact.  This is the routine the fused kernels call for every value within their
 * float32 error guard of a half-integer; the 256-bit evaluations it needed are added to
 * counter 1 of fds_counters, failures (none can occur) to counter 2.
 * coords: host int32 [n][8]; out: host int32 [n].  Every vector must satisfy |coords[8i]| <
 * 2^26 and sum_j |coords[8i + j]| < 2^26 (the proven range; the kernels' own coordinates
 * stay below 2^23), else FDS_E_INVALID and nothing runs.  Synchronous; allocates and frees
 * its own device buffer. */
int fds_debug_exact_round(const int32_t* coords, int32_t* out, int32_t n);

/* Diagnostics: counters of the exact-rounding fallbacks taken since the last reset:
 * out[0] = values within the float32 error guard of a rounding boundary, re-decided from
 * their exact integer coordinates in Z[cos(pi/16)]; out[1] = of those, values whose 128-bit
 * fixed-point evaluation was still ambiguous and that a 256-bit evaluation decided (exact
 * ties excluded); out[2] = internal consistency failures (must stay 0).
 * Host pointer to 3 uint64.  Synchronises the device.  reset != 0 clears them. */
int fds_counters(uint64_t* out, int reset);

/* Wait for all work on `stream` and report any asynchronous CUDA error.  Also reports the
 * kernels' bounded waits: every wait in the library's kernels gives up after about 2 s (it
 * never hangs), leaves the affected outputs unwritten and adds 1 to counter 2 of
 * fds_counters; when that counter has grown since the last fds_sync (or reset) on this
 * device, fds_sync returns FDS_E_TIMEOUT once, with the count in fds_last_error(). */
int fds_sync(void* stream);

/* The status fds_sync derives from the failure counter (host only, no device needed): FDS_OK
 * when now <= seen, else FDS_E_TIMEOUT with a message giving now - seen. */
int fds_status_of_failures(uint64_t seen, uint64_t now);

/* Test hook: overwrite the three counters of fds_counters on the current device (host array of
 * 3).  Synchronises the device.  Lets a test exercise fds_sync's FDS_E_TIMEOUT without
 * making any device wait give up. */
int fds_debug_set_counters(const uint64_t* values);

/* Message describing the calling thread's last error ("" if none). */
const char* fds_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Copies of a serving batch (the paper has no counterpart: a host-side helper of the serving
 * loop).  Enqueues n asynchronous copies on `stream`, in order: copy i moves bytes[i] bytes
 * from address srcs[i] to address dsts[i].  Addresses are host or device pointers given as
 * integers (host arrays of n each, read before the call returns); the direction of each copy
 * follows from its addresses (unified addressing), and host memory should be pinned for the
 * copy to overlap other work.  One cudaMemcpyAsync per copy: a batch's inputs and outputs
 * move with one call instead of one call per request.  Copies of 0 bytes are skipped.
 * Errors: n < 0, a null array with n > 0, or a null address of a non-empty copy ->
 * FDS_E_INVALID; a copy the runtime refuses -> FDS_E_CUDA (the copies before it stay
 * enqueued). */
int fds_copy_many(const uint64_t* dsts, const uint64_t* srcs, const uint64_t* bytes, int32_t n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FDS_H */
