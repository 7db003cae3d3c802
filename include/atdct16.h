/*
 * atdct16 -- GB300 (sm_103a) library for the orthogonal 16-point approximate
 * DCT of da Silveira, Bayer, Cintra, Kulasekera, Madanayake and Kozakevicius
 * (arXiv 1606.05562).
 *
 * The transform is the 16x16 matrix T with entries in {0, +-1} (Sec. 2),
 * applied separably to every disjoint 16x16 block of an image,
 *     Y = T X T^T,
 * through the paper's 60-addition factorisation T = P2 M4 M3 M2 P1 M1
 * (Sec. 2).  The orthogonal approximation is C_hat = S T with
 * S = diag(T T^T)^(-1/2); S is folded into the quantisation step or the zonal
 * retention (Sec. 2, last paragraph), so the inverse is
 *     X_hat = T^T (S^2 Y' S^2) T.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers prefixed d_ are device pointers, h_ host pointers.  The caller
 *   owns every buffer it passes; the library never frees them.  A plan owns
 *   only its own workspace (tables, descriptors, per-tile partial sums).
 * - Images are row-major with a pitch in bytes.  Width and height must be
 *   positive multiples of 16.  Image base pointers and pitches must be
 *   16-byte aligned (the kernels move 16-byte rows of a block), and pitches
 *   of batched images must be below 2^31 bytes.
 * - Block (by, bx) covers rows 16*by..16*by+15 and columns 16*bx..16*bx+15.
 *   Within a block the coefficient index is (u, v), u = vertical frequency
 *   (row of T applied to the block's columns), v = horizontal frequency:
 *       Y[u][v] = sum_m sum_n T[u][m] X[m][n] T[v][n].
 * - Zig-zag order (Sec. 4 adapts the 8x8 JPEG scan to 16x16): the JPEG
 *   convention extended to 16x16: anti-diagonals s = u + v; on even s the
 *   scan runs with u decreasing, on odd s with v decreasing.
 * - Every compute call is asynchronous on the given stream and allocates
 *   nothing.  Argument errors are detected on the host before any launch and
 *   return ATDCT16_EINVAL; CUDA launch or copy errors return ATDCT16_ECUDA.
 * - A plan is not thread-safe: use one plan per host thread (or serialise).
 */
#ifndef ATDCT16_H
#define ATDCT16_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ATDCT16_OK = 0,
  ATDCT16_EINVAL = 1,       /* bad argument: nothing was launched */
  ATDCT16_ENOMEM = 2,       /* workspace or device memory exhausted */
  ATDCT16_ECUDA = 3,        /* a CUDA runtime call failed */
  ATDCT16_ETIMEOUT = 4,     /* a bounded device-side wait expired */
  ATDCT16_EUNSUPPORTED = 5, /* a valid request this library does not support */
  ATDCT16_EDEVICE = 6       /* a kernel's own bounds checks rejected work */
} atdct16_status;

typedef enum { ATDCT16_U8 = 0, ATDCT16_I16 = 1 } atdct16_dtype;

/* One image of a batch.  src/dst are device pointers (host pointers for the
 * *_host entry points).  r_or_qp is the zonal r (0..256) for
 * atdct16_compress_zonal and the quantisation point QP (0..63) for
 * atdct16_compress_quant. */
typedef struct {
  const void* src;
  void* dst;
  int64_t src_pitch; /* bytes */
  int64_t dst_pitch; /* bytes */
  int32_t width;
  int32_t height;
  int32_t r_or_qp;
  int32_t reserved; /* must be 0 */
} atdct16_image;

typedef struct atdct16_plan_st* atdct16_plan_t;
typedef struct atdct16_batch_st* atdct16_batch_t;

/* Library version string, e.g. "atdct16 1.0 sm_103a". */
const char* atdct16_version(void);

/* Human-readable name of a status code (static storage). */
const char* atdct16_status_string(atdct16_status s);

/* Create a plan on the current CUDA device.
 *   dtype          pixel type of the images the plan will process (U8: zonal
 *                  path, I16: quantisation path; forward/inverse accept both)
 *   max_images     largest batch size any call will pass (>= 1)
 *   workspace_budget_bytes  upper bound on device memory the plan may take
 *                  (0 = a default of 256 MiB).  The plan sizes its per-tile
 *                  partial-sum buffer from it; calls whose batches need more
 *                  tiles than fit return ATDCT16_ENOMEM.
 *   flags          0, or ATDCT16_PLAN_ZIGZAG: the 256 coefficients of every
 *                  block in atdct16_forward / atdct16_inverse and the 256
 *                  levels of every block in atdct16_compress_quant are stored
 *                  in the zig-zag scan of Sec. 4 (entry k of a block is the
 *                  coefficient (u, v) at scan position k: anti-diagonals
 *                  s = u + v in increasing order, even s with u decreasing,
 *                  odd s with v decreasing), the order an entropy coder reads
 *                  them in; without it they are row-major in (u, v).
 *                  ATDCT16_PLAN_TEST_STALL_COPIES (failure-path test hook):
 *                  atdct16_inverse announces 16 bytes more than its bulk
 *                  copies deliver, so its bounded waits expire (about 2 s per
 *                  call) and atdct16_last_device_status reports
 *                  ATDCT16_ETIMEOUT; the context stays usable.
 *                  ATDCT16_PLAN_TEST_STALL_MMA (failure-path test hook): a
 *                  batch on this plan that runs the tcgen05 kernel variant
 *                  issues no tensor-core product, so every CTA's bounded wait
 *                  on the first one expires (about half a second), the CTA
 *                  frees its tensor memory and returns, results are left
 *                  undefined and atdct16_batch_last_device_status reports
 *                  ATDCT16_ETIMEOUT; the context stays usable.  Other bits:
 *                  ATDCT16_EINVAL.
 * Allocates the plan's workspace (device tables, descriptor ring, partials)
 * with cudaMalloc and pinned host staging with cudaHostAlloc. */
#define ATDCT16_PLAN_ZIGZAG 1u
#define ATDCT16_PLAN_TEST_STALL_COPIES 0x80000000u
#define ATDCT16_PLAN_TEST_STALL_MMA 0x40000000u
atdct16_status atdct16_plan_create(atdct16_plan_t* plan, atdct16_dtype dtype, int32_t max_images,
                                   size_t workspace_budget_bytes, uint32_t flags);

/* Wait for the plan's outstanding work, then release its workspace. */
atdct16_status atdct16_plan_destroy(atdct16_plan_t plan);

/* Forward 2-D transform of every block (Sec. 2, Y = T X T^T; Sec. 4 splits
 * the image into disjoint 16x16 blocks).  S is not applied.
 *   d_src   image of `dtype` (U8 or I16) with pitch `pitch` bytes, w x h
 *   d_coef  output, block-major: block b = by*(w/16)+bx occupies
 *           d_coef[256*b .. 256*b+255], row-major in (u, v), or in zig-zag
 *           order if the plan was created with ATDCT16_PLAN_ZIGZAG.  Exact
 *           int32 (|Y| <= 65280 for U8 input, <= 256*32768 for I16 input).
 * w, h multiples of 16; d_src, d_coef and pitch 16-byte aligned (EINVAL
 * otherwise).  Asynchronous on `stream`; reads d_src once, writes d_coef once. */
atdct16_status atdct16_forward(atdct16_plan_t plan, atdct16_dtype dtype, const void* d_src,
                               int64_t pitch, int32_t w, int32_t h, int32_t* d_coef,
                               cudaStream_t stream);

/* Inverse 2-D transform (Sec. 4, A' = C_hat^T B' C_hat with S folded in),
 * computed exactly: Z = T^T (W Y W) T with the integer W = 48 S^2, then
 * X_hat = Z / 2304 rounded half to even (decided exactly from Z) and
 * clamped to the range of `dtype`.  Coefficients produced by atdct16_forward reconstruct the input
 * bit-exactly.  Layout of d_coef as for atdct16_forward (the plan's order).
 * Any int32 coefficients are accepted and give the exact result: tiles whose
 * coefficients all satisfy |Y| < 2^18 run in 32-bit integers (|Z| < 2^31),
 * others in two 32-bit halves combined in 64 bits.  d_coef, d_dst and pitch
 * 16-byte aligned, w, h multiples of 16 (EINVAL otherwise).  Each tile's
 * coefficients arrive by bulk copies whose completion every warp awaits for
 * at most about a second; an expired wait leaves that part of d_dst
 * unwritten and makes atdct16_last_device_status report ATDCT16_ETIMEOUT. */
atdct16_status atdct16_inverse(atdct16_plan_t plan, atdct16_dtype dtype, const int32_t* d_coef,
                               int32_t w, int32_t h, void* d_dst, int64_t pitch,
                               cudaStream_t stream);

/* 1-D forward transform (Sec. 2, y = T x; S is not applied) of `count`
 * contiguous vectors of 16 samples of `dtype` (U8 or I16): d_src holds
 * count * 16 samples, d_coef receives count * 16 exact int32 coefficients,
 * vector i at d_coef[16 i .. 16 i + 15] in frequency order u = 0..15
 * (|y| <= 16 * 255 for U8, <= 16 * 32768 for I16).  A packed image of width
 * w (a multiple of 16) is w / 16 vectors per row, so one call transforms
 * all its 16-sample row segments.  count = 0 does nothing; d_src and d_coef
 * 16-byte aligned (EINVAL otherwise).  Asynchronous on `stream`. */
atdct16_status atdct16_forward_1d(atdct16_plan_t plan, atdct16_dtype dtype, const void* d_src, int64_t count,
                                  int32_t* d_coef, cudaStream_t stream);

/* 1-D exact inverse (C_hat^T C_hat = T^T S^2 T = I, Sec. 2): for each of
 * `count` vectors of 16 int32 coefficients,
 *     x_n = round_half_even( sum_u T[u][n] W_u y_u / 48 ),  W = 48 S^2,
 * clamped to the range of `dtype` and stored as 16 samples of `dtype` at
 * d_dst[16 i ..].  Exact for any int32 input (64-bit arithmetic for vectors
 * with a coefficient of magnitude >= 2^24).  atdct16_forward_1d output
 * reconstructs its input bit-exactly.  Alignment and count rules as
 * atdct16_forward_1d. */
atdct16_status atdct16_inverse_1d(atdct16_plan_t plan, atdct16_dtype dtype, const int32_t* d_coef, int64_t count,
                                  void* d_dst, cudaStream_t stream);

/* Fused zonal compression of a batch of uint8 images (Sec. 4 procedure):
 * forward transform, keep the first r zig-zag coefficients of every block
 * (images[i].r_or_qp = r, 0..256), scale by S^2 on both sides, inverse,
 * store clamp(round_half_even(X_hat)) as uint8 in images[i].dst, and write
 * the per-image PSNR (Sec. 4) to d_psnr[i]:
 *     PSNR = 10 log10(255^2 * w * h / SSE),  +inf when SSE = 0,
 * with SSE the squared error of the unrounded reconstruction X_hat against
 * the input.  Every pixel crosses device memory once in and once out.
 * The reconstruction numerator Z is exact, so the stored pixels are exact;
 * SSE is accumulated in FP32 per block and FP64 per image.
 *   h_images  host array of n descriptors (device src/dst pointers)
 *   d_psnr    device array of n doubles
 *   d_sse     optional device array of n doubles (may be NULL) */
atdct16_status atdct16_compress_zonal(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                      double* d_psnr, double* d_sse, cudaStream_t stream);

/* Fused quantisation of a batch of int16 planes (Sec. 2: S absorbed into
 * the quantiser; Sec. 5.3: HEVC quantisation points):
 *     B = s_u s_v Y,  level = sign(B) floor(|B| / Qstep + 1/2),
 *     Qstep = 2^(QP/6),  B' = level * Qstep,  X_hat = C_hat^T B' C_hat,
 * stored as clamp(rint(X_hat)) int16 in images[i].dst.  The level decision
 * is taken in FP32 as fp32(|Y| * fp32(s_u s_v / Qstep)) + 0.5 (no fused
 * multiply-add).  The inverse runs in FP32.  PSNR (peak 255) of the
 * unrounded reconstruction goes to d_psnr[i].
 *   d_levels  optional (may be NULL, else 16-byte aligned): int16 levels,
 *             block-major as for atdct16_forward (row-major in (u, v), or
 *             zig-zag order with ATDCT16_PLAN_ZIGZAG), images concatenated
 *             in batch order. */
atdct16_status atdct16_compress_quant(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                      int16_t* d_levels, double* d_psnr, double* d_sse,
                                      cudaStream_t stream);

/* Zonal compression that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they compress -- programs running on a memory budget fixed at
 * start-up, latency-critical paths that cannot afford cudaMalloc's implicit
 * synchronisation, applications whose own allocator owns all device memory.
 * It computes exactly what atdct16_compress_zonal computes, without a plan.
 * Besides the caller's images and outputs it uses only a scratch area of
 * about 1 MiB that is part of the library image itself: every GPU that loads
 * the library holds it until the process exits.
 *   n <= ATDCT16_NOALLOC_MAX_IMAGES, and the batch must fit in
 *   ATDCT16_NOALLOC_MAX_TILES tiles of 16 x 128 pixels (each image takes
 *   ceil(w/128) * h/16 tiles, e.g. 128 per 512x512 image); larger requests
 *   return ATDCT16_ENOMEM and launch nothing.  Other argument rules and the
 *   meaning of d_psnr / d_sse are those of atdct16_compress_zonal.
 * The first call on each device sets that device up (looks up the scratch
 * area's device address and fills its weight table on `stream`); make that
 * first call before any stream capture (while `stream` is being captured it
 * returns ATDCT16_EUNSUPPORTED and enqueues nothing).  All calls share the scratch area and
 * it keeps the last call's contents: calls that may overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller. */
#define ATDCT16_NOALLOC_MAX_IMAGES 64
#define ATDCT16_NOALLOC_MAX_TILES 131072
atdct16_status atdct16_compress_zonal_noalloc(const atdct16_image* h_images, int32_t n, double* d_psnr,
                                              double* d_sse, cudaStream_t stream);
/* Device-side status of the last atdct16_compress_zonal_noalloc call on the
 * current device (the paper has no counterpart: the plan-free callers above
 * have no plan whose status they could read).  Synchronises `stream`, which
 * should be the stream of that call, then reads the status word of the
 * shared scratch area: ATDCT16_OK, or ATDCT16_EDEVICE when the kernel's own
 * checks rejected a descriptor.  Each call clears the word, so it reports the
 * last call only.  ATDCT16_EINVAL if no call has set this device up yet. */
atdct16_status atdct16_noalloc_last_device_status(cudaStream_t stream);

/* Exact-DCT baseline of atdct16_compress_zonal: the same Sec. 4 procedure
 * with the orthonormal 16-point DCT-II (Sec. 3.2, the transform the paper
 * measures its approximation against) as dense FP32 products: B = C A C^T,
 * the first r zig-zag coefficients kept, A' = C^T B' C, stored pixels
 * clamp(rint(A'), 0, 255) (FP32; they may differ from an exact evaluation
 * where A' lies within FP32 error of a half-integer), PSNR of the unrounded
 * A' (the dropped energy, C being orthonormal).  Arguments, ownership and
 * errors as atdct16_compress_zonal; the first call on a device uploads C and
 * synchronises `stream` (make it outside any stream capture). */
atdct16_status atdct16_compress_zonal_dct(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                          double* d_psnr, double* d_sse, cudaStream_t stream);

/* Mean SSIM (Sec. 4, the structural similarity of Wang et al. 2004 that the
 * paper cites) of n uint8 image pairs: h_images[i].src against
 * h_images[i].dst (both read; e.g. an original and its reconstruction),
 * r_or_qp ignored.  Window: 11 x 11 Gaussian of standard deviation 1.5,
 * normalised; C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2; the mean over the
 * (h - 10) x (w - 10) positions where the window lies inside the image; FP32
 * moments of the centred pixels, FP64 mean.  d_mssim: n device doubles.
 * Asynchronous on `stream`; the first call on a device uploads the window
 * weights and synchronises `stream` (make it outside any stream capture).
 * EINVAL for the argument rules of atdct16_compress_zonal, ENOMEM if the
 * batch needs more 16 x 64-position tiles than the plan's workspace holds. */
atdct16_status atdct16_ssim_batch(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n, double* d_mssim,
                                  cudaStream_t stream);

/* PSNR between two images of the same shape (Sec. 4), exact integer SSE.
 * peak 255.  d_out: one device double.  Allocates nothing: the output slot
 * doubles as the accumulator. */
atdct16_status atdct16_psnr(atdct16_dtype dtype, const void* d_a, int64_t pitch_a, const void* d_b,
                            int64_t pitch_b, int32_t w, int32_t h, double* d_out,
                            cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Resident mixed-size batches (a fixed set of images compressed repeatedly).
 * atdct16_batch_create uploads the descriptors once, sizes the batch's own
 * per-tile partials, optionally autotunes the launch shape of the fused
 * zonal kernel on the batch itself (kernel variant, warps per CTA and CTAs
 * per SM, i.e. tiles per CTA), and optionally captures the
 * fused kernel and the PSNR finalize into one CUDA graph.  Each
 * atdct16_batch_launch then re-runs the whole batch (Sec. 4 procedure on
 * every image) with one graph launch.
 * --------------------------------------------------------------------------- */
#define ATDCT16_BATCH_AUTOTUNE 1u /* time the candidate launch shapes, keep the fastest */
#define ATDCT16_BATCH_GRAPH 2u    /* capture the launches into a CUDA graph */
/* Pin the kernel variant instead (not with ATDCT16_BATCH_AUTOTUNE):
 * flags |= ATDCT16_BATCH_VARIANT(v), v = 0 (integer row pass, FP32 column
 * pass), 1 (forward transform in int16 SWAR, the default), 2 (forward
 * transform as mma.sync tensor-core products) or 3 (forward transform as
 * tcgen05 products with the accumulators in tensor memory).  All variants
 * give the same stored pixels; PSNR agrees to FP32 summation order. */
#define ATDCT16_BATCH_VARIANT_SHIFT 8
#define ATDCT16_BATCH_VARIANT_MASK (7u << ATDCT16_BATCH_VARIANT_SHIFT)
#define ATDCT16_BATCH_VARIANT(v) ((uint32_t)((v) + 1) << ATDCT16_BATCH_VARIANT_SHIFT)
/* Pin the launch shape of the kernels for r <= 36 instead (not with
 * ATDCT16_BATCH_AUTOTUNE): tiles per CTA w in {2, 4, 8}, staging depth d in
 * {1, 2, 3}, input copy width v in {8, 16} bytes (see atdct16_tune_point). */
#define ATDCT16_BATCH_SHAPE_SHIFT 12
#define ATDCT16_BATCH_SHAPE_MASK (0x3fu << ATDCT16_BATCH_SHAPE_SHIFT)
#define ATDCT16_BATCH_SHAPE(w, d, v)                                                           \
  ((uint32_t)((((w) == 2 ? 1 : (w) == 4 ? 2 : 3) | ((d) << 2) | (((v) == 8 ? 1 : 2) << 4)) \
              << ATDCT16_BATCH_SHAPE_SHIFT))

/* h_images: n zonal descriptors (device src/dst, r in 0..256).  d_psnr /
 * d_sse: caller-owned device outputs (d_sse may be NULL), written by every
 * launch.  Creation allocates the batch's device memory, copies the
 * descriptors synchronously and, with ATDCT16_BATCH_AUTOTUNE, runs the batch
 * several times on `stream` (so dst must not overlap any src: EINVAL).  The
 * tuning result is cached per (GPU, batch shape) in the plan; when the
 * environment variable ATDCT16_TUNE_CACHE names a file, results are also
 * read from and appended to it (one JSON object per line). */
atdct16_status atdct16_batch_create(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                    double* d_psnr, double* d_sse, uint32_t flags, cudaStream_t stream,
                                    atdct16_batch_t* batch);
/* Re-run the batch on `stream` (asynchronous). */
atdct16_status atdct16_batch_launch(atdct16_batch_t batch, cudaStream_t stream);
/* Chosen launch shape: variant (0: integer row pass + FP32 column pass,
 * 1: forward transform in int16 SWAR, 2: forward transform as mma.sync
 * products, 3: forward transform as tcgen05 products), warps per CTA,
 * prefetch (always 1: input rows are staged ahead), grid size, tile count
 * and the tuned time per launch in ms (0 if untuned).
 * Any pointer may be NULL. */
/* Device-side status of the batch's launches so far (sticky, first error
 * wins): waits for the last launch's stream, then ATDCT16_OK,
 * ATDCT16_ETIMEOUT (a bounded wait of a kernel expired; that launch's results
 * are undefined) or ATDCT16_EDEVICE (a kernel's own checks failed). */
atdct16_status atdct16_batch_last_device_status(atdct16_batch_t batch);
atdct16_status atdct16_batch_info(atdct16_batch_t batch, int32_t* variant, int32_t* warps, int32_t* prefetch,
                                  int32_t* grid, int64_t* tiles, float* tuned_ms);
/* One launch shape of a batch and its time.  The general kernel (jobs with
 * r = 0 or r > 36) runs in a variant (as above) with general_ctas CTAs per
 * SM; the kernels for r <= 36 (kept set inside the 8 x 8 low-frequency
 * corner) run tiles_per_cta warps per CTA (one 16 x 128 tile each at a
 * time), with the input rows of staging_depth tiles in flight per warp (1,
 * 2 or 3), copied vector_bytes (16 or 8) at a time, box_ctas CTAs per SM (0:
 * as many as fit).  ms: median time of one launch of the batch.  phase: 0
 * for a candidate of the box-kernel search, 1 of the general-kernel search
 * (which runs with the box shape found first). */
typedef struct {
  int32_t phase;
  int32_t variant;
  int32_t general_ctas;
  int32_t tiles_per_cta;
  int32_t staging_depth;
  int32_t vector_bytes;
  int32_t box_ctas;
  float ms;
} atdct16_tune_point;
/* The batch's launch shape and, after autotuning, every candidate the
 * autotuner timed (the box kernels' tiles per CTA x staging depth x vector
 * width x CTAs per SM, then the general kernel's variant x CTAs per SM), each
 * the median of five timed launches of the whole batch.  chosen may be NULL;
 * up to max_candidates entries go to candidates, *n_candidates receives
 * their total count (0 without autotuning or when the shape came from the
 * tuning cache). */
atdct16_status atdct16_batch_tuning(atdct16_batch_t batch, atdct16_tune_point* chosen,
                                    atdct16_tune_point* candidates, int32_t max_candidates,
                                    int32_t* n_candidates);
/* Waits for the batch's last launch stream, then frees it. */
atdct16_status atdct16_batch_destroy(atdct16_batch_t batch);

/* ---------------------------------------------------------------------------
 * Continuous-batching compression server (zonal path).  A scheduler thread
 * admits submitted requests in arrival order as soon as their buffers fit in
 * a device arena of memory_budget_bytes (allocated once at creation), uploads
 * them while earlier batches compute, puts every uploaded request into the
 * next fused-kernel launch on a free compute slot (up to max_batch requests
 * per launch; slots run concurrently), downloads the reconstruction and the
 * PSNR, and frees the buffers.  A request's result does not depend on the
 * batch it rode in.
 * --------------------------------------------------------------------------- */
typedef struct atdct16_server_st* atdct16_server_t;
typedef struct {
  size_t memory_budget_bytes; /* device arena for request buffers (2 bytes per pixel) */
  int32_t max_batch;          /* requests per launch, >= 1 */
  int32_t compute_slots;      /* launches that may be in flight at once, 1..16 */
  int32_t reserved;           /* 0 */
} atdct16_server_config;
/* One compression request: uint8 image in host memory (pinned memory makes
 * the copies asynchronous), reconstruction written to h_dst; r in 0..256. */
typedef struct {
  const void* h_src;
  void* h_dst;
  int64_t src_pitch; /* bytes */
  int64_t dst_pitch; /* bytes */
  int32_t width;     /* multiple of 16 */
  int32_t height;    /* multiple of 16 */
  int32_t r;
  int32_t reserved; /* 0 */
} atdct16_request;

atdct16_status atdct16_server_create(const atdct16_server_config* cfg, atdct16_server_t* server);
/* Queue a request (never blocks).  The host buffers must stay valid until the
 * request completes.  ATDCT16_ENOMEM if it can never fit in the arena. */
atdct16_status atdct16_server_submit(atdct16_server_t server, const atdct16_request* req, uint64_t* ticket);
/* Wait for a request (timeout_us < 0: no limit; ATDCT16_ETIMEOUT when it
 * expires).  On completion returns its PSNR (Sec. 4) and its latency in
 * seconds from arrival (submission, unless given to atdct16_server_submit_at)
 * to completion, and forgets the ticket. */
atdct16_status atdct16_server_wait(atdct16_server_t server, uint64_t ticket, double* psnr, double* latency_s,
                                   int64_t timeout_us);
/* Seconds on the server's clock (a steady clock; the timestamps below). */
double atdct16_server_clock(void);
/* As atdct16_server_submit, for a request that arrived at arrival_s on the
 * server's clock (<= now): its latency is measured from arrival_s. */
atdct16_status atdct16_server_submit_at(atdct16_server_t server, const atdct16_request* req, double arrival_s,
                                        uint64_t* ticket);
/* Where a request's time went, in seconds on the server's clock: arrival
 * (submission time unless given), submission, the start and end of its
 * upload, the start and end of the fused launch it rode in, the end of its
 * download, and when the scheduler saw it complete.  The device stage
 * boundaries come from timing events placed on the host clock through a
 * reference event recorded when the server was created. */
typedef struct {
  double arrival, submit, h2d_start, h2d_end, compute_start, compute_end, d2h_end, done;
} atdct16_request_timing;
/* As atdct16_server_wait, returning the request's timing as well (either
 * output may be NULL). */
atdct16_status atdct16_server_wait_timing(atdct16_server_t server, uint64_t ticket, double* psnr,
                                          atdct16_request_timing* timing, int64_t timeout_us);
/* Completed requests, kernel launches, pixels completed, seconds from the
 * first submission to the last completion, arena bytes in use. */
atdct16_status atdct16_server_stats(atdct16_server_t server, uint64_t* completed, uint64_t* launches,
                                    double* pixels, double* busy_s, size_t* arena_used);
/* Stops the scheduler after the work in flight, frees everything. */
atdct16_status atdct16_server_destroy(atdct16_server_t server);

/* Sticky device-side status of the plan: ATDCT16_OK, ATDCT16_EDEVICE when a
 * kernel's own checks rejected a descriptor, or ATDCT16_ETIMEOUT when a
 * bounded device-side wait expired (first event wins).  Synchronises the
 * plan's last stream. */
atdct16_status atdct16_last_device_status(atdct16_plan_t plan);

/* Kernel timing hook (tracing support; not part of the paper).  With
 * every = n > 0, the first fused zonal / quantisation kernel launch of the
 * plan after this call and then every n-th one is bracketed by CUDA events on
 * the launch stream (n = 1: every launch; sampling leaves the other calls
 * free of the extra stream operations, which would otherwise separate the
 * fused kernel from the finalize that overlaps its end); every = 0 turns the
 * hook off; every < 0 is EINVAL.  atdct16_plan_profile synchronises on those
 * events and returns the number of timed launches and their summed device
 * time in milliseconds, then clears the record.  At most 4096 launches are
 * recorded between two queries; later ones are not timed. */
atdct16_status atdct16_plan_set_profiling(atdct16_plan_t plan, int32_t every);
atdct16_status atdct16_plan_profile(atdct16_plan_t plan, int64_t* launches, double* kernel_ms);

/* Runs the library's 1-D butterflies on the host, for tests:
 * inverse = 0: out = T in;  inverse = 1: out = T^T in.  Same source code as
 * the device kernels.  in/out: 16 int32 each. */
atdct16_status atdct16_host_butterfly(const int32_t* in, int32_t* out, int32_t inverse);

#ifdef __cplusplus
}
#endif

#endif /* ATDCT16_H */
