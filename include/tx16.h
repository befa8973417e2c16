/*
 * libtx16 -- GB300 (sm_103a) implementation of the orthogonal 16-point DCT
 * approximation of Cintra, Bayer, Oliveira et al., "Multiplierless 16-point
 * DCT approximation for low-complexity image and video coding".
 *
 * Notation (the paper's):
 *   T        16x16 matrix with entries in {0, +1, -1}                (Sec. 2.1)
 *   S        (1/4) diag(1,1,2,r2,r2,1,2,2,1,2,2,r2,r2,2,2,2), r2 = sqrt 2
 *            = sqrt((T T^t)^-1)                                      (Sec. 2.1)
 *   C_hat    S T, orthogonal                                         (Sec. 2.1)
 *   X        one 16x16 block of samples; row index i is vertical
 *   Y        T X T^t, exact integers; Y[u][v], u vertical frequency (Sec. 3.1)
 *   Z_r      the first r cells of the zig-zag scan of a 16x16 block,
 *            JPEG convention extended to 16x16                       (Sec. 3.1)
 *
 * Every transform runs through the 44-addition factorisation
 * T = P2 M4 M3 M2 P1 M1 (Sec. 2.2), and the forward transform is exact:
 *   - the fused codec kernels evaluate the forward network on packed binary32
 *     lanes holding integers (samples enter as 2^23 + 256 x or as integers
 *     below 2^24), every intermediate an integer multiple of a power of two
 *     small enough to be represented exactly, so Y = T X T^t bit for bit;
 *     their no-quantiser inverse is exact the same way (values k / 256);
 *   - the forward-only, general and unfused kernels use int32.
 * S is merged into the quantiser (Sec. 2.1, last paragraph): with a
 * quantiser, the level is taken from one binary32 product per kept
 * coefficient, the dequantised coefficient is one binary32 product, and the
 * inverse network runs in binary32, stage by stage as factorised.
 *
 * Conventions for every call below:
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  Arrays of descriptors (tx16_image,
 *     tx16_qparams) are HOST arrays, read before the call returns.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream).  Argument errors are returned synchronously and nothing
 *     is launched.  A CUDA launch error returns TX16_ECUDA.
 *   - Coefficient / level layout ("block-major"): the blocks of image 0 in
 *     raster block order, then those of image 1, ...; block b occupies int32
 *     elements [256 b, 256 b + 256), row-major Y[u][v] at 256 b + 16 u + v.
 *   - Images: width and height are positive multiples of 16 (the paper splits
 *     images into disjoint 16x16 blocks, Sec. 3.1); pitch_bytes is a multiple
 *     of 16 and at least width * sample size; data is 16-byte aligned.
 *     bits = 8 means uint8 samples, 9..12 means uint16 samples.
 */
#ifndef TX16_H
#define TX16_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TX16_OK = 0,
  TX16_EINVAL = 1,   /* bad argument; nothing launched */
  TX16_ENOMEM = 2,   /* device or host allocation failed / admission refused */
  TX16_ECUDA = 3,    /* a CUDA runtime call or launch failed */
  TX16_ETIMEOUT = 4, /* a bounded wait ran out */
  TX16_EBUSY = 5     /* no free slot */
} tx16_status;

/* One image plane.  `data` is a device pointer: read by calls that take the
 * image as input, written by calls that take it as output. */
typedef struct {
  void* data;
  int32_t width;
  int32_t height;
  int64_t pitch_bytes;
  int32_t bits;
} tx16_image;

/* Quantiser of one image (Sec. 3.1 zonal coding; Sec. 2.1 S merged into the
 * quantiser).  r in 1..256 keeps Z_r.  q > 0: uniform step q on the
 * orthonormal coefficient c = s_u s_v Y[u][v], level = round_half_away(c / q)
 * taken in binary32 as round(fl32(Y) * f), f = fl32(s_u s_v / q).
 * q <= 0: no uniform quantiser (the paper's image experiment): the "level"
 * of a kept coefficient is Y[u][v] itself and the inverse is exact. */
typedef struct {
  float q;
  int32_t r;
} tx16_qparams;

/* Human-readable name of a status code (static storage). */
const char* tx16_status_str(tx16_status s);

/* Number of 16x16 blocks of an image (width/16 * height/16), or -1 if the
 * descriptor is invalid. */
int64_t tx16_image_blocks(const tx16_image* img);

/*
 * Forward 2-D transform Y = T X T^t of every block of n images (Sec. 3.1
 * forward transform with C = T; Sec. 2.2 fast algorithm: 16 row transforms,
 * then 16 column transforms, 44 additions each).
 *   imgs    host array of n input descriptors
 *   coeffs  device int32 array of 256 * sum(blocks) elements, block-major
 * Exact: |Y| <= 256 (2^bits - 1).
 */
tx16_status tx16_forward(const tx16_image* imgs, int32_t n, int32_t* coeffs, void* stream);

/*
 * Zonal / uniform quantisation of nblk coefficient blocks with one quantiser
 * (Sec. 3.1 zonal mask; Sec. 2.1 S merged into the quantiser).
 *   coeffs  device int32, 256 * nblk, block-major (as written by tx16_forward)
 *   levels  device int32, 256 * nblk: level inside Z_r, 0 outside
 *           (q <= 0: Y[u][v] inside Z_r, 0 outside).  May equal coeffs.
 */
tx16_status tx16_quantise(const int32_t* coeffs, int64_t nblk, tx16_qparams qp,
                          int32_t* levels, void* stream);

/*
 * Inverse 2-D transform and reconstruction (Sec. 3.1: A_tilde = C_hat^t
 * B_tilde C_hat, blocks rearranged into the image).
 *   levels  device int32, block-major, for the n images of `out` in order;
 *           only the cells inside each image's Z_r are read.
 *   out     host array of n output descriptors (device sample buffers written)
 *   qp      host array of n quantisers (q and r of each image)
 * q > 0:  W = fl32(level * fl32(q s_u s_v)); X_tilde = T^t W T in binary32
 *         through the transposed factorisation, columns first.
 * q <= 0: 256 X_tilde = T^t (D' Y D') T exactly, D' = 16 S^2.
 * Sample = clip(round_half_away(X_tilde), 0, 2^bits - 1).
 */
tx16_status tx16_inverse(const int32_t* levels, const tx16_image* out, int32_t n,
                         const tx16_qparams* qp, void* stream);

/*
 * Fused codec: forward, quantise, inverse, reconstruction and squared-error
 * reduction of every block in one launch (Sec. 3.1 procedure; PSNR of
 * Sec. 3.1 from the returned SSE, see tx16_psnr).
 *   in      host array of n input descriptors
 *   out     host array of n output descriptors, or NULL (no samples written)
 *   qp      host array of n quantisers
 *   sse     device uint64[n] or NULL: sse[i] = sum (x - x_tilde)^2 over image
 *           i; zeroed by the call itself before accumulation
 *   levels  device int32, block-major, or NULL (levels not written)
 * Results are identical to tx16_forward + tx16_quantise + tx16_inverse.
 */
tx16_status tx16_codec_batch(const tx16_image* in, const tx16_image* out, int32_t n,
                             const tx16_qparams* qp, uint64_t* sse, int32_t* levels,
                             void* stream);

/*
 * Squared error between two sets of n images of equal shape (the separate
 * PSNR reduction of the unfused form).  sse: device uint64[n], zeroed by the
 * call before accumulation.
 */
tx16_status tx16_sse(const tx16_image* a, const tx16_image* b, int32_t n, uint64_t* sse,
                     void* stream);

/*
 * PSNR from squared error (host arithmetic, float64):
 * 10 log10((2^bits - 1)^2 W H / SSE), +inf for SSE = 0.
 *   sse   host array of n values; imgs: host descriptors (shape and bits);
 *   psnr  host array of n results.
 */
tx16_status tx16_psnr(const uint64_t* sse, const tx16_image* imgs, int32_t n, double* psnr);

/*
 * Zonal sweep: the paper's image experiment (Sec. 3.1, no quantiser; Fig. 2
 * plots PSNR per additive cost against r) for nr values of r at once.  Each
 * block is transformed forward once; for every r_list[j] the coefficients
 * outside Z_r are zeroed and the block is reconstructed exactly (256 X_tilde =
 * T^t (D' Y D') T over Z_r), rounded, clipped and compared with the input.
 *   imgs    host array of n input descriptors (any sample depth)
 *   r_list  host array of nr values in 1..256, 1 <= nr <= 16
 *   sse     device uint64[n * nr], sse[i * nr + j] = squared error of image i
 *           coded with r_list[j]; zeroed by the call
 * PSNR follows with tx16_psnr.  Nothing else is written.
 */
tx16_status tx16_zonal_sweep(const tx16_image* imgs, int32_t n, const int32_t* r_list, int32_t nr, uint64_t* sse,
                             void* stream);

/*
 * Codec of images of any size, and of colour images plane by plane.  The
 * paper codes images whose sides are multiples of 16 (Sec. 3.1: the image is
 * split into 16x16 blocks); it does not say what happens at a ragged edge.
 * Here the last row and the last column are repeated out to the next
 * multiple of 16 (edge replication), the padded blocks go through the
 * Sec. 3.1 codec exactly as in tx16_codec_batch, and only the image's own
 * width x height samples are written and counted in the squared error.  A
 * colour image is n = 3 (or more) descriptors, one per plane, each with its
 * own quantiser (Sec. 3.1 codes each channel separately).
 *   in      host array of n input descriptors: width, height >= 1 (not
 *           necessarily multiples of 16); data 16-byte aligned; pitch_bytes a
 *           multiple of 16 and >= width x sample size; bits 8..12
 *   out     host array of n output descriptors of the same widths, heights and
 *           bits (same rules), or NULL; only the width x height samples of
 *           each output are written, the pitch padding is left untouched
 *   qp      host array of n quantisers
 *   sse     device uint64[n] or NULL: squared error over the width x height
 *           samples of each image; zeroed by the call
 * Images whose sides are multiples of 16 give the results of
 * tx16_codec_batch.  PSNR follows with tx16_psnr, whose W x H is the
 * unpadded size.  Returns TX16_EINVAL (nothing launched) for a bad argument.
 */
tx16_status tx16_codec_any_size(const tx16_image* in, const tx16_image* out, int32_t n,
                                const tx16_qparams* qp, uint64_t* sse, void* stream);

/*
 * Mixed 8/16 tiling: the video experiment's second scenario (Sec. 3.2), where
 * the 8-point approximation T8 (14 additions, Sec. 2.1; the even rows of T on
 * the first 8 columns: the half of M2 M3 M4 that acts on the sums
 * x_i + x_{15-i}) codes blocks beside T.  Every 16x16 region of an image is
 * coded as one 16x16 block with T (quantiser q, zone Z_r16, as
 * tx16_codec_batch) and as four 8x8 blocks with T8 (the same q on
 * s8_u s8_v Y8[u][v], S8 = sqrt((T8 T8^t)^-1), zone = the first r8 cells of
 * the 8x8 zig-zag scan; without a quantiser the exact inverse
 * 64 X_tilde = T8^t (D8 Y8 D8) T8, D8 = 8 S8^2), and one of the two is kept:
 *   mode 0  the tiling with the smaller squared error of the region (ties:
 *           16x16) -- the paper leaves the choice to the encoder
 *   mode 1  always 16x16;   mode 2  always 8x8.
 *   in, out   as tx16_codec_batch (sides multiples of 16; out may be NULL)
 *   qp        host array of n tx16_mixed_qparams: q (<= 0: no quantiser),
 *             r16 in 1..256, r8 in 1..64, mode
 *   split     device uint8, one flag per 16x16 region (1 = four 8x8 blocks),
 *             regions in raster order, image after image; or NULL
 *   sse       device uint64[n] or NULL: squared error of the kept tiling;
 *             zeroed by the call
 * Returns TX16_EINVAL (nothing launched) for a bad argument.
 */
typedef struct {
  float q;
  int32_t r16;
  int32_t r8;
  int32_t mode;
} tx16_mixed_qparams;

tx16_status tx16_codec_mixed(const tx16_image* in, const tx16_image* out, int32_t n,
                             const tx16_mixed_qparams* qp, uint8_t* split, uint64_t* sse, void* stream);

/*
 * SSIM, the paper's second quality measure (Sec. 3.1: Fig. 2(b) plots SSIM per
 * additive cost, Fig. 3 quotes it per image).  The paper cites Wang, Bovik,
 * Sheikh and Simoncelli (2004) without fixing window or constants; this
 * library takes that article's: an 11 x 11 Gaussian window, standard
 * deviation 1.5, normalised to unit sum; C1 = (0.01 L)^2, C2 = (0.03 L)^2,
 * L = 2^bits - 1; local weighted statistics at every position where the window
 * lies inside the image (no padding, no downsampling); the index
 *   ((2 mu_a mu_b + C1)(2 s_ab + C2)) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2))
 * averaged over the (H - 10) x (W - 10) positions (MSSIM).
 *   a, b    host arrays of n descriptors of equal size and bits (typically the
 *           input and the reconstruction of tx16_codec_batch); width and
 *           height >= 11, any value; data 16-byte aligned; pitch a multiple of
 *           16 bytes and >= width x sample size
 *   mssim   device double[n]: the mean index of each pair; zeroed by the call
 *   map     device float array of sum_i (H_i - 10)(W_i - 10) elements, or
 *           NULL: image i's local indices, row-major, after those of images
 *           0 .. i-1
 * Arithmetic is binary32 with samples centred on 2^(bits-1); the difference
 * from the binary64 definition is bounded per position by the rounding of
 * the two 11-tap passes (see the tests).  Returns TX16_EINVAL for a bad
 * argument, nothing launched.
 */
tx16_status tx16_ssim(const tx16_image* a, const tx16_image* b, int32_t n, double* mssim, float* map,
                      void* stream);

/* ------------------------------------------------------------------------ */
/* Batch plans: uneven-size batches in one persistent launch per zonal class */
/* ------------------------------------------------------------------------ */

/* A plan holds a device-side work list for one batch: the per-image
 * descriptors of the codec (the same computation as tx16_codec_batch, Sec. 3.1
 * of the paper) in device memory, grouped by the extent of each image's zone
 * Z_r, plus one tile counter per group.  Running it launches one persistent
 * fused kernel per group whose CTAs claim tiles of 16 blocks from the counter,
 * so uneven image sizes and zones balance across the SMs.  The plan owns its
 * device memory (allocated once, at creation); the images' sample buffers
 * stay the caller's and must outlive the plan. */
typedef struct tx16_plan tx16_plan;

/* Build a plan for n images (host descriptor arrays, as for tx16_codec_batch;
 * out may be NULL).  Errors: TX16_EINVAL (arguments), TX16_ENOMEM (device
 * allocation), TX16_ECUDA.  Synchronous. */
tx16_status tx16_plan_create(const tx16_image* in, const tx16_image* out, int32_t n, const tx16_qparams* qp,
                             tx16_plan** plan);

/* Run the plan on `stream`.  sse: device uint64[n] (zeroed by the run) or
 * NULL; levels: device int32, block-major over the n images, or NULL.
 * Results equal tx16_codec_batch's on the same images.  Runs of one plan are
 * ordered by their stream; two runs of one plan must not overlap in time. */
tx16_status tx16_plan_run(tx16_plan* plan, uint64_t* sse, int32_t* levels, void* stream);

/* As tx16_plan_run, through a CUDA graph captured on first use (and again
 * when sse/levels change or after autotuning), replayed on `stream`. */
tx16_status tx16_plan_run_graph(tx16_plan* plan, uint64_t* sse, int32_t* levels, void* stream);

/* Time the schedule candidates of each group on the plan's own data and keep
 * the fastest.  The schedule tuned is that of the kernel a run without levels
 * uses.  For the fused groups (8-bit samples in the fused quantiser range) the
 * candidates are both mappings of blocks to lanes -- one 16x16 block per
 * thread (warps claiming 32-block tiles) in each of its compiled
 * configurations (warps per CTA, column pairs parked in shared memory, input
 * stages: see tx16_plan_variant), and the pair kernel (two blocks per pair of
 * binary32 lanes, CTAs claiming 16-block tiles) -- and, for each, the resident
 * CTAs per SM and the tiles per claim (for one block per thread also no
 * claims: a contiguous run of tiles per CTA).
 * cache_path: a text file of tuned schedules keyed by device, group and size
 * class (read and extended), or NULL.  Synchronous on `stream`; writes the
 * outputs. */
tx16_status tx16_plan_autotune(tx16_plan* plan, const char* cache_path, void* stream);

/* Introspection: number of groups and, for the first max_runs of them, the
 * zone class (0..5 for r <= 8, 16, 32, 64, 128, 256; -1 = general kernel),
 * tiles, CTAs per SM (0 = all that fit) and tiles per claim of the kernel a
 * run without levels uses.  Host arrays; any of them may be NULL. */
tx16_status tx16_plan_info(const tx16_plan* plan, int32_t* runs, int32_t* zone, int32_t* tiles,
                           int32_t* ctas_per_sm, int32_t* chunk, int32_t max_runs);

/* The mapping and configuration group `run` uses: the configuration index of
 * the one-block-per-thread kernel, or -1 for the pair kernel (and for the
 * general kernel's group), with its warps per CTA, column pairs parked in
 * shared memory and input stages (0 for -1).  Any output may be NULL.
 * TX16_EINVAL for a run index out of range. */
tx16_status tx16_plan_variant(const tx16_plan* plan, int32_t run, int32_t* variant, int32_t* warps_per_cta,
                              int32_t* parked_pairs, int32_t* stages);

/* Pin the schedule of group `run`: configuration index (as tx16_plan_variant
 * reports it: -1 selects the pair kernel), resident CTAs per SM (0 = all that
 * fit) and tiles per claim (>= 1; 0 for the one-block-per-thread kernel: no
 * claims, each CTA a contiguous run of tiles).  Results do not depend on the
 * schedule.
 * TX16_EINVAL for a run of the general kernel or out-of-range values. */
tx16_status tx16_plan_set_schedule(tx16_plan* plan, int32_t run, int32_t variant, int32_t ctas_per_sm,
                                   int32_t chunk);

/* Free the plan's device memory and graph.  NULL is ignored. */
void tx16_plan_destroy(tx16_plan* plan);

/* ------------------------------------------------------------------------ */
/* Serving loop                                                              */
/* ------------------------------------------------------------------------ */

/* A server codes requests (one image each, any size and bit depth accepted
 * by tx16_codec_batch, each with its own quantiser; Sec. 3.1 codec) as they
 * arrive.  A worker thread admits queued requests in arrival order while its
 * device arena has room for their planes, launches each admitted group as ONE
 * fused batch on one of several streams, and keeps admitting new requests
 * while earlier groups run: continuous batching, copies of one group
 * overlapping the kernel of another.  All device memory is allocated at
 * creation.  (The serving loop is a property of this library; the paper
 * codes images one at a time.) */
typedef struct tx16_server tx16_server;

/* json_cfg: NULL or a flat JSON object of numbers:
 *   "device_pool_mb"  device arena for request planes (default: a quarter of
 *                     the free HBM, at most 4096); fails with TX16_ENOMEM
 *                     when it exceeds the free HBM
 *   "streams"         groups in flight (default 6, 1..16)
 *   "max_batch"       requests per group (default 256)
 *   "max_queue"       queued requests before submit returns TX16_EBUSY
 *   "spin_us"         worker polling window, 0..1e6 (default 300): the
 *                     worker polls for submissions and finished groups while
 *                     a group is in flight and for this long after its last
 *                     progress, then blocks; 0 blocks at once when nothing
 *                     is in flight (no host core kept busy when idle, longer
 *                     hand-offs at low load)
 *   "wait_spin_us"    tx16_serve_wait polling window, 0..1e6 (default 2000):
 *                     the waiter polls this long, itself retiring the
 *                     request's group when its work has finished, before it
 *                     blocks; 0 blocks at once
 *   "band_mb"         a group of at most 16 requests holding a plane larger
 *                     than this (default 4; 0: never) is copied in, coded and
 *                     copied out in up to 8 bands of whole block rows, the
 *                     copies out of coded bands overlapping the copies in of
 *                     the next ones (lower latency at light load; larger
 *                     groups take one launch)
 * A request that arrives while nothing is queued or in flight is admitted and
 * launched by tx16_serve_submit on the caller's thread; otherwise the worker
 * admits it and the group's stream slot has its own thread issuing the
 * copies and the launch.  The server uses the device current at creation. */
tx16_status tx16_serve_create(const char* json_cfg, tx16_server** server);

/* Queue one request: host_pixels (w x h samples, uint8 for bits = 8, uint16
 * for 9..12, rows contiguous) must stay valid until the request is done;
 * host_recon (same size) receives the reconstruction, or NULL.  Pinned host
 * memory gives direct DMA.  *ticket identifies the request.
 * Errors: TX16_EINVAL (shape, bits, qp), TX16_ENOMEM (larger than the arena:
 * never admissible), TX16_EBUSY (queue full). */
tx16_status tx16_serve_submit(tx16_server* server, const void* host_pixels, int32_t w, int32_t h, int32_t bits,
                              tx16_qparams qp, void* host_recon, uint64_t* ticket);

/* Wait up to timeout_ms for a request; on success the ticket is released and
 * *psnr (dB, Sec. 3.1 PSNR) and *latency_us (submit to completion) are set
 * (either may be NULL).  TX16_ETIMEOUT leaves the ticket valid. */
tx16_status tx16_serve_wait(tx16_server* server, uint64_t ticket, int32_t timeout_ms, double* psnr,
                            double* latency_us);

/* Latency percentiles (microseconds, over a uniform reservoir of completed
 * requests) and coded Mblocks/s from the first submit to the last
 * completion since creation or the last reset. */
tx16_status tx16_serve_stats(tx16_server* server, double* p50_us, double* p99_us, double* p999_us,
                             double* mblocks_per_s);
tx16_status tx16_serve_reset_stats(tx16_server* server);

/* Hold (paused != 0) or resume admission; queued requests wait while held
 * (for draining or maintenance).  Requests already admitted finish. */
tx16_status tx16_serve_pause(tx16_server* server, int32_t paused);

/* Finish admitted and queued work, then free everything.  NULL is ignored. */
void tx16_serve_destroy(tx16_server* server);

/* ------------------------------------------------------------------------ */
/* The work-list codec for callers that cannot allocate device memory        */
/* ------------------------------------------------------------------------ */

/* Largest batch tx16_codec_batch_static accepts. */
#define TX16_STATIC_MAX_IMAGES 1024

/*
 * The same codec as tx16_codec_batch / tx16_plan_run (identical results), run
 * by the work-list kernel, but allocating nothing: no cudaMalloc, no cudaFree,
 * no allocating library call.  It is meant for callers that cannot allocate
 * device memory when they run the codec: a process whose device memory all
 * belongs to another allocator's pool, a latency-critical loop where an
 * allocation would synchronise the device, or a service whose memory budget is
 * fixed at start-up.  (This entry point is a property of this library; the
 * paper has no counterpart.)
 *
 * The work list (image descriptors and tile counters) lives in one fixed
 * device array inside the library, about 123 KB, which every GPU that loads
 * the library holds until the process exits.  The caller still passes all
 * inputs and outputs, with the arguments, layouts and errors of
 * tx16_codec_batch, except:
 *   - n may not exceed TX16_STATIC_MAX_IMAGES: larger batches return
 *     TX16_EINVAL and launch nothing;
 *   - every call uses the same array, which keeps the last call's contents:
 *     each call rewrites the descriptors and clears the counters itself, but
 *     two calls whose work overlaps on the GPU (different streams, or
 *     different host threads without ordering) race on the array.  Order such
 *     calls on one stream, or wait for one before issuing the next;
 *   - the descriptors reach the array through the parameters of small
 *     kernels launched on `stream` (up to 224 descriptors each), which also
 *     clear the tile counters and sse; the host copy of the list is not read
 *     after the call returns, and the call does not wait for earlier work on
 *     its stream;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and keeps it; make that
 *     first call before any stream capture.
 */
tx16_status tx16_codec_batch_static(const tx16_image* in, const tx16_image* out, int32_t n,
                                    const tx16_qparams* qp, uint64_t* sse, int32_t* levels, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TX16_H */
