/*
 * pocketgs.h — C ABI of libpocketgs.so, a GB300 (sm_103a) differentiable tile-based Gaussian
 * rasterizer: the training hot path of PocketGS (arXiv 2601.17354), operator T of Sec. III,
 *     T : (Theta_0, {I_t, T_t}) -> Theta*,
 * exposed as the three calls of one optimisation iteration: render (Sec. III-C, Eq. 7),
 * backward (Eq. 8 and the index-mapped scatter of Eq. 10) and step (Adam with moments aligned to
 * the canonical parameter buffer, Sec. III-C "Index-Mapped Gradient Scattering").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All tensor pointers are DEVICE pointers owned by the caller and borrowed for the call.
 *    Parameters are fp32, planar structure-of-arrays ("[k][n]" = k rows of n floats):
 *        means [3][n], log_scales [3][n], quats [4][n] (w, x, y, z; need not be unit),
 *        opacity_logits [n], sh [3][K][n] with K = (sh_degree + 1)^2 (channel-major).
 *    Rows need no particular alignment; 16-byte aligned rows with n % 4 == 0 take the
 *    vectorised path of pgs_step.
 *  - Images are [3][H][W] fp32 planar, row-major; pixel (x, y) covers [x, x+1) x [y, y+1).
 *  - Cameras are pinhole with OpenCV axes (x right, y down, z forward); viewmat is the
 *    row-major 3x4 world-to-camera matrix [R | t].
 *  - Every call enqueues work on the context's CUDA stream and returns without synchronising,
 *    except pgs_status, pgs_read_buffer and pgs_reserve (which may allocate).
 *  - A context is not thread-safe; use one context per host thread / stream.
 *  - Return value: PGS_OK (0) or a negative PGS_ERR_* code.  No C++ exception crosses the ABI.
 *    Errors detected on the device (pair capacity overflow, non-finite parameters) are recorded
 *    in the context's device status word and reported by the next pgs_status call.
 */
#ifndef POCKETGS_H
#define POCKETGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PGS_OK 0
#define PGS_ERR_INVALID_ARG (-1) /* null pointer, bad size, unsupported tile or degree */
#define PGS_ERR_NO_RENDER (-2)   /* pgs_backward without a preceding pgs_render */
#define PGS_ERR_CAPACITY (-3)    /* more (tile, Gaussian) pairs than pair_capacity */
#define PGS_ERR_NONFINITE (-4)   /* a parameter of a projected Gaussian was NaN or inf */
#define PGS_ERR_CUDA (-6)        /* a CUDA runtime call failed */
#define PGS_ERR_OOM (-7)         /* device allocation failed */
#define PGS_ERR_INTERNAL (-8)    /* a device-side consistency check failed (access skipped) */
#define PGS_ERR_TOO_LARGE (-9)   /* size beyond the fixed scratch of pgs_sort_pairs_static */
#define PGS_ERR_NOT_PD (-10)     /* bundle adjustment: damped reduced system not positive definite */
#define PGS_ERR_TIMEOUT (-11)    /* a bounded device-side wait ran out (the sort's look-back): results undefined */

typedef struct pgs_ctx pgs_ctx;

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12]; /* row-major 3x4 world -> camera [R | t] */
    float near_z;      /* Gaussians with camera depth z <= near_z are culled */
    float bg[3];       /* background colour composited behind the last Gaussian */
} pgs_camera;

typedef struct {
    int64_t n;
    int32_t sh_degree; /* 0..3 */
    int32_t pad_;
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logits;
    float* sh;
} pgs_gaussians;

typedef struct {
    int32_t tile;          /* screen tile edge T in pixels: 8, 16 or 32 (fixed for the context) */
    int32_t reserved_;
    int64_t pair_capacity; /* (tile, Gaussian) pairs the context holds; 0 = grow on demand */
    float adam_b1, adam_b2, adam_eps;
    /* learning rates of the parameter groups: means, log_scales, quats, opacity_logits,
       sh degree-0 coefficients, sh higher coefficients */
    float lr[6];
} pgs_config;

/* Create a context that enqueues on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
   The context owns all scratch memory (projected Gaussians, keys, tile ranges, per-pixel final
   transmittance and last-contributor index, screen-space gradients, status word).
   *out receives the context; on error *out is NULL. */
int pgs_create(pgs_ctx** out, const pgs_config* cfg, void* cuda_stream);

/* Free the context and its scratch.  Synchronises the context's stream first.  NULL is a no-op. */
void pgs_destroy(pgs_ctx* ctx);

/* Make sure the scratch covers n Gaussians, a width x height image and pair_capacity pairs,
   allocating if needed (this synchronises the device).  Calls whose sizes fit the reservation
   never allocate, so a sequence of them can be captured in a CUDA graph. */
int pgs_reserve(pgs_ctx* ctx, int64_t n, int32_t width, int32_t height, int64_t pair_capacity);

/* Forward pass, Eq. 7 front to back: project and cull every Gaussian (EWA projection, SH colour),
   emit (tile | depth, canonical index) pairs for the tiles of its footprint (the rectangle of the
   per-axis 3-sigma extents ceil(3 sqrt(Sigma_xx)), ceil(3 sqrt(Sigma_yy)), and of it the tiles
   whose pixel centres the 3-sigma ellipse reaches), sort them (the permutation pi of Eq. 10), find each
   tile's range, alpha-composite each pixel over its tile's depth-ordered list
   (alpha = min(0.99, o G); skip alpha < 1/255; stop before a Gaussian that would take the
   transmittance below 1e-4), and write image_out [3][H][W] = colour + T_final * bg.
   The context keeps, for pgs_backward, the projected Gaussians, the sorted pairs, the tile
   ranges, T_final [H][W] and last [H][W] (1 + list position of the last composited entry).
   The lists are built in two levels (Gaussians to super-tiles of 8 x 4 tiles, then to tiles), so
   besides the P pairs the pair buffers also hold the coarse stage's entries and counters; the
   capacity a render needs is max(P, its coarse entries, 32 counters per block of 256 of them),
   which is P on every scene but ones with very few pairs per super-tile.  If the capacity is too
   small the image is undefined and pgs_status reports PGS_ERR_CAPACITY with the capacity needed;
   with pair_capacity = 0 the context instead reads that back (one synchronisation) and grows
   before compositing. */
int pgs_render(pgs_ctx* ctx, const pgs_gaussians* params, const pgs_camera* cam, float* image_out);

/* L1 photometric loss of Sec. IV's training loop (the paper names no loss): for n = 3 H W values,
   dL_dimage[k] = sign(image[k] - target[k]) / n (sign(0) = 0) and, on the device,
   loss_out[0] = mean |image - target|, loss_out[1] = sum (image - target)^2 (for PSNR).
   loss_out is a device pointer to 2 floats. */
int pgs_loss_l1(pgs_ctx* ctx, const float* image, const float* target, int64_t n, float* dL_dimage,
                float* loss_out);
/* pgs_render (Eq. 7, Sec. III-C) followed by pgs_loss_l1 (the L1 loss of Sec. IV's training loop)
   on its image (n = 3 H W), in one pass: the compositing
   forward also reads target [3][H][W] (device), writes dL_dimage [3][H][W] (device) and adds its
   CTAs' sums into the loss, so no separate loss kernel reads the image back.  image_out, T_final,
   last and dL_dimage are bit for bit those of the two calls; loss_out (device, 2 floats) holds the
   same sums added in another order (per CTA, then in double), so they agree to rounding.  With the
   replay cache on, the recording forward is followed by the loss kernel instead.  Errors as
   pgs_render; PGS_ERR_INVALID_ARG for a null target, dL_dimage or loss_out. */
int pgs_render_l1(pgs_ctx* ctx, const pgs_gaussians* params, const pgs_camera* cam, const float* target,
                  float* image_out, float* dL_dimage, float* loss_out);
/* L1 + D-SSIM loss (the paper reports SSIM, Sec. IV, and names no training loss): per colour
   plane of [3][height][width] images, SSIM with the 11 x 11 Gaussian window (sigma 1.5, taps
   normalised to 1), zero padding, C1 = 0.01^2, C2 = 0.03^2; loss = (1 - lambda) mean|image -
   target| + lambda (1 - mean SSIM).  Writes dL_dimage (device [3][H][W]) and, on the device,
   loss_out[0] = the loss, loss_out[1] = mean SSIM (device pointer to 2 floats).  Context-owned
   scratch of 9 floats per pixel (grown with the image; growing synchronises).  lambda in [0, 1]. */
int pgs_loss_dssim(pgs_ctx* ctx, const float* image, const float* target, int32_t width, int32_t height,
                   float lambda, float* dL_dimage, float* loss_out);

/* Backward of the last pgs_render on this context for the upstream gradient dL_dimage [3][H][W]:
   per pixel, re-traverse its list back to front from `last`, rebuilding the transmittance from
   T_final (T_i = T_{i+1} / (1 - alpha_i)) and the colour behind each entry with Eq. 7, apply
   Eq. 8 for dL/dc and dL/dalpha, reduce over the pixels of a tile and scatter to the canonical
   index (Eq. 10); then chain to every parameter.  Gradients are ADDED to grads (same layout as
   the parameters; the caller zeroes them, pgs_step does so after reading them).  The parameter
   values must be those of the last render. */
int pgs_backward(pgs_ctx* ctx, const float* dL_dimage, pgs_gaussians* grads);

/* One Adam step over all parameter groups in one launch (Kingma & Ba 2015, bias-corrected, step
   number t >= 1, the context's b1, b2, eps and per-group learning rates):
   m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2; p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
   then g = 0.  params, grads, m and v share n and sh_degree. */
int pgs_step(pgs_ctx* ctx, pgs_gaussians* params, pgs_gaussians* grads, pgs_gaussians* m,
             pgs_gaussians* v, int64_t t);

/* pgs_backward followed by pgs_step for one view, fused: the compositing backward runs as in
   pgs_backward, then one kernel chains each Gaussian's screen-space gradient to its parameters
   and applies the Adam update of pgs_step directly (culled Gaussians with a zero gradient), so
   the parameter gradient is never written to memory.  Equivalent to pgs_backward into zeroed
   gradients followed by pgs_step; params must be those of the last render. */
int pgs_backward_step(pgs_ctx* ctx, const float* dL_dimage, pgs_gaussians* params,
                      pgs_gaussians* m, pgs_gaussians* v, int64_t t);

/* Synchronise the context's stream, return the first error recorded on the device since the
   last call (PGS_OK if none) and clear it.  *pairs_needed (optional) receives the pair count of
   the last render, or with PGS_ERR_CAPACITY the pair capacity it needs. */
int pgs_status(pgs_ctx* ctx, int64_t* pairs_needed);

/* The paper's replay cache (Sec. III-C, Eq. 9: the per-pixel record S of the forward, with its
   count reset every render) instead of the recompute backward.  k_max > 0: from the next render
   on, the forward records for every pixel its first k_max composited entries as 16-byte records
   {list position, alpha, transmittance in front} ([pixel][k_max], context-owned, allocated at
   that render; synchronises) and the backward replays them instead of re-evaluating alpha and
   dividing out the transmittance; pixels that composited more than k_max entries are recomputed
   (the paper's overflow case).  Compositing then runs one pixel per thread with 256 entries
   staged per batch (the variant setting is not used).  k_max = 0 (the default) returns to the
   recompute backward.  Changing the setting invalidates the last render (PGS_ERR_NO_RENDER until
   the next).  k_max at most 4096. */
int pgs_set_replay_cache(pgs_ctx* ctx, int32_t k_max);

/* Internal buffers of the last render/backward, copied to `dst` (host or device) for inspection.
   which: PGS_BUF_KEYS (uint64 [P], sorted keys (tile << 32) | depth bits, assembled on the host
   from the lists and the Gaussians' depths), PGS_BUF_VALUES (uint32 [P]), PGS_BUF_RANGES
   (uint32 [tiles][2]) -- these three in the order of the stable sort of the pairs by key (tiles
   row-major, an empty tile (0, 0)), whatever layout the render's buffers use --
   PGS_BUF_T_FINAL (float [H][W]), PGS_BUF_LAST (uint32 [H][W]), PGS_BUF_GRAD2D (float [9][n]: du, dv, d conic a, b, c, d opacity, d r, g, b),
   PGS_BUF_TILES_TOUCHED (uint32 [n]), PGS_BUF_NCOMP (uint32 [H][W], entries composited per
   pixel).  Copies min(max_bytes, size) bytes, stores the full size in
   *bytes, synchronises. */
#define PGS_BUF_KEYS 0
#define PGS_BUF_VALUES 1
#define PGS_BUF_RANGES 2
#define PGS_BUF_T_FINAL 3
#define PGS_BUF_LAST 4
#define PGS_BUF_GRAD2D 5
#define PGS_BUF_TILES_TOUCHED 6
#define PGS_BUF_NCOMP 7
int pgs_read_buffer(pgs_ctx* ctx, int which, void* dst, int64_t max_bytes, int64_t* bytes);

/* Decision trace of the last render (diagnostics and parity tests).  The compositing rules of Eq. 7
   decide per (pixel, entry) whether the entry is skipped (alpha < 1/255), composited, clamped at
   alpha = 0.99, or stops the pixel (the transmittance would fall below 1e-4); those integer
   outcomes are decided in fp32.  For each of npix pixels (x, y pairs, device int32 [npix][2])
   this walks the pixel's tile list front to back with the forward kernels' own arithmetic and
   writes, per evaluated entry (list order, at most max_entries recorded per pixel):
     og   [npix][max_entries] float: o G, the opacity times the Gaussian before the 0.99 clamp;
     code [npix][max_entries] uint8: 0 skipped, 1 composited, 2 composited clamped, 3 stop
          (not composited; the walk ends there);
   and per pixel: count [npix] int32 = entries evaluated (> max_entries: the rest not recorded;
   -1 for a pixel outside the image), T_final [npix] float, last [npix] uint32 and ncomp [npix]
   uint32, which equal the render's own T_final, last and composited count of the pixel.
   All pointers are device memory owned by the caller.  Asynchronous on the context's stream.
   PGS_ERR_NO_RENDER without a render on this context. */
int pgs_trace_pixels(pgs_ctx* ctx, const int32_t* pixels, int64_t npix, int32_t max_entries, float* og,
                     uint8_t* code, int32_t* count, float* T_final, uint32_t* last, uint32_t* ncomp);

/* Per-stage device time accounting.  pgs_profile(ctx, 1) makes every later call record CUDA
   events on the context's stream at its stage boundaries; pgs_stage_times synchronises, writes
   the total milliseconds and the number of timed executions of each stage since the previous
   read into ms[PGS_NUM_STAGES] and counts[PGS_NUM_STAGES], and resets the accumulators.
   Stages: projection (K1), binning = depth sort + pair count (K2), sort = coarse entries, their
   radix sort by super-tile and the tile lists + ranges (K3-K5), compositing forward (K6), loss (K7), compositing backward (K8), projection
   backward (K9), Adam (K10), fused projection backward + Adam (pgs_backward_step).
   pgs_profile(ctx, 0) stops recording. */
#define PGS_STAGE_PROJECT 0
#define PGS_STAGE_BIN 1
#define PGS_STAGE_SORT 2
#define PGS_STAGE_COMPOSITE_FWD 3
#define PGS_STAGE_LOSS 4
#define PGS_STAGE_COMPOSITE_BWD 5
#define PGS_STAGE_PROJECT_BWD 6
#define PGS_STAGE_ADAM 7
#define PGS_STAGE_PROJECT_BWD_ADAM 8
#define PGS_NUM_STAGES 9
int pgs_profile(pgs_ctx* ctx, int enable);
int pgs_stage_times(pgs_ctx* ctx, double* ms, int64_t* counts);

/* Number of kernels this context has launched since it was created (host-side count). */
int64_t pgs_launch_count(const pgs_ctx* ctx);

/* Allocation-free pair sort.  The paper has no counterpart: this entry point exists for callers
   that may not allocate device memory themselves, such as code whose device memory is owned by
   another allocator (a framework's caching pool or an arena reserved at start-up, where a direct
   cudaMalloc can fail or fragment the reservation) or latency-critical loops in which
   cudaMalloc / cudaFree would synchronise the device.  It runs the radix sort pgs_render uses for
   its depth keys and coarse entries (stable, least-significant-digit first, 8-bit digits, one
   launch per pass with decoupled look-back, the last digit masked) by the low key_bits
   bits of count (key, value) pairs (higher key bits never take part in the order; keys_out keeps
   them as they were): keys_in/vals_in (device, read only) -> keys_out/vals_out (device, caller
   owned, not overlapping the inputs).  It allocates nothing: its scratch is one file-scope device
   array of 3.8 MB, held by every GPU that loads the library until the process exits.
   count must be at most 262144 (PGS_ERR_TOO_LARGE otherwise); key_bits in 1..64.  The first call
   on a device looks the scratch address up (cudaGetSymbolAddress) with that device current; make
   that first call before any stream capture.  Every call shares the one scratch array, which
   keeps the previous call's contents (the call clears what must start at zero): calls that
   overlap on the GPU, on any streams, race and must be serialised by the caller.  Asynchronous on
   cuda_stream (NULL = legacy default stream). */
int pgs_sort_pairs_static(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                          uint32_t* vals_out, int64_t count, int32_t key_bits, void* cuda_stream);
/* The device-side check of pgs_sort_pairs_static (the sort's scatter checks every destination
   index against the pair count and skips an access that fails, recording it in a status word of the
   same static scratch, which stays set across sorts).  Synchronises cuda_stream, returns
   PGS_ERR_INTERNAL if a check failed since the previous call of this function (else PGS_OK) and
   clears the word.  No paper counterpart; allocates nothing. */
int pgs_sort_pairs_static_status(void* cuda_stream);

/* ---------------------------------------------------------------------------------------------
   Batched training: many views of many scenes (uneven Gaussian counts and resolutions) in one
   step.  All renders of a step share one projection launch, one depth sort, one binning (coarse
   entries of every render's super-tiles, one grouping sort, one fine stage), one
   persistent compositing launch forward and one backward (CTAs take tiles of every render,
   heaviest first, from a device work counter), one loss launch and one fused backward + Adam
   launch that sums each Gaussian's gradient over its scene's views.  The step can be captured
   in a CUDA graph and replayed; the Adam step counter lives on the device.
   --------------------------------------------------------------------------------------------- */
typedef struct pgs_batch pgs_batch;

typedef struct {
    int32_t scene; /* index into the scene arrays of pgs_batch_create */
    int32_t pad_;
    pgs_camera cam;
    float* image;        /* device [3][H][W]: the render */
    const float* target; /* device [3][H][W]: the view's ground truth */
    float* dL_dimage;    /* device [3][H][W]: written by the step's L1 loss */
} pgs_render_desc;

/* Plan a batch: n_scenes parameter sets with Adam moments m, v (same layout; all scenes share one
   sh_degree) and n_renders renders ordered scene by scene.  pair_capacity 0 = measure the pairs of
   the parameters as given and keep 25 % headroom (synchronises).  All buffers stay owned by the
   caller and must outlive the batch. */
int pgs_batch_create(pgs_batch** out, const pgs_config* cfg, int32_t n_scenes,
                     const pgs_gaussians* params, const pgs_gaussians* m, const pgs_gaussians* v,
                     int32_t n_renders, const pgs_render_desc* renders, int64_t pair_capacity,
                     void* cuda_stream);
void pgs_batch_destroy(pgs_batch* b);
/* One training step of every render (render, L1, backward, Adam with t = completed steps + 1):
   replays the captured graph if there is one, else enqueues the kernels.  A step whose pairs
   overflow the capacity changes no parameter, moment or step count (its Adam launch and its step
   count read the device's overflow flag), and neither do the steps after it until
   pgs_batch_status has reported PGS_ERR_CAPACITY (with the pairs needed) and cleared the flag;
   pgs_batch_reserve then grows the capacity. */
int pgs_batch_step(pgs_batch* b);
/* The two halves of a step as separate calls, for losses other than the built-in L1 (e.g. the
   L1 + D-SSIM of pgs_loss_dssim) or renders for evaluation.
   pgs_render_batch: the forward of every render (Eq. 7 front to back, as pgs_render: projection,
   one depth sort, pair emission and sort, one persistent compositing launch) into each render's
   image buffer; parameters, moments and the step count are not touched.  The batch keeps the
   projected Gaussians, pairs, T_final and last of every render for pgs_backward_batch.
   pgs_backward_batch: the backward of the last pgs_render_batch for the upstream gradients the
   caller has written into each render's dL_dimage buffer (device [3][H][W]): Eq. 8 per pixel back
   to front from `last`, scattered to the canonical indices (Eq. 10), chained to the parameters and
   summed over each scene's renders; ADDED to grads[scene] (host array of n_scenes descriptors of
   device buffers with the scene's n and sh_degree; the caller zeroes them).  PGS_ERR_NO_RENDER
   without a pgs_render_batch since the last pgs_batch_step (which changes the parameters).  An
   optimizer step on the gradients is the caller's (pgs_step per scene, with a context on the same
   stream).  Both are asynchronous on the batch's stream; a pair overflow is reported by
   pgs_batch_status and then the backward adds nothing. */
int pgs_render_batch(pgs_batch* b);
int pgs_backward_batch(pgs_batch* b, const pgs_gaussians* grads);
/* Capture one step into a CUDA graph (nothing runs during capture); later steps replay it. */
int pgs_batch_capture(pgs_batch* b);
/* Point every render at a new view before the next step (cameras[n_renders], targets[n_renders]
   device pointers): each render keeps its scene and image size (width and height must match);
   the render table is updated in device memory on the batch's stream, so a captured graph picks
   the new views up at its next replay. */
int pgs_batch_set_views(pgs_batch* b, const pgs_camera* cameras, const float* const* targets);
/* Grow the pair capacity to at least pair_capacity (synchronises; smaller values do nothing).  A
   captured graph is captured again over the new buffers. */
int pgs_batch_reserve(pgs_batch* b, int64_t pair_capacity);
/* Completed training steps: the device step counter (synchronises). */
int pgs_batch_steps(pgs_batch* b, int64_t* steps);
/* Per render: losses[2 r] = mean |image - target| and losses[2 r + 1] = sum of squared errors of
   the last step (host array of 2 n_renders doubles; synchronises). */
int pgs_batch_losses(pgs_batch* b, double* losses);
/* As pgs_status, for the batch (pairs = pairs of the last step). */
int pgs_batch_status(pgs_batch* b, int64_t* pairs);
int64_t pgs_batch_launch_count(const pgs_batch* b);

/* Compositing kernel variant (pixels per thread 1, 2, 4; entries staged per batch 64, 128, 256)
   of a context or a batch.  A tile of T x T pixels is one CTA of T * T / pixels_per_thread
   threads: T = 8 takes 1 or 2 pixels per thread, T = 16 takes 1, 2 or 4, T = 32 takes 2 or 4
   (PGS_ERR_INVALID_ARG otherwise).  Changing a batch's variant drops its captured graph. */
int pgs_set_variant(pgs_ctx* ctx, int32_t pixels_per_thread, int32_t depth);
int pgs_batch_set_variant(pgs_batch* b, int32_t pixels_per_thread, int32_t depth);
/* Autotuner measurement: runs the render part of a step once, then times the forward + backward
   compositing of every variant (reps repetitions, CUDA events on the batch's stream) and writes
   ms[9] in the order (1,64) (1,128) (1,256) (2,64) ... (4,256); a strip the tile edge does not
   take (4 pixels at T = 8, 1 pixel at T = 32) gets -1.  Parameters are not changed.
   The caller picks and sets the variant (the library's Python layer caches the choice per GPU
   and workload class). */
int pgs_batch_time_variants(pgs_batch* b, int32_t reps, float* ms);
/* Autotuner measurement of the render part of a step (projection, depth sort, key emission, pair
   sort, ranges, tile order: the part that depends on the tile edge besides the compositing):
   best of reps timed runs after one warm-up, *ms (host).  Parameters are not changed. */
int pgs_batch_time_render(pgs_batch* b, int32_t reps, float* ms);
/* The same measurement for a context, on its last render: the timed forwards write `image`
   ([3][H][W] scratch) and the backwards use dL_dimage [3][H][W]. */
int pgs_time_variants(pgs_ctx* ctx, float* image, const float* dL_dimage, int32_t reps, float* ms);
/* Separate compositing variants for the forward and the backward (pgs_set_variant sets both). */
int pgs_set_variants(pgs_ctx* ctx, int32_t fwd_pixels, int32_t fwd_depth, int32_t bwd_pixels, int32_t bwd_depth);
/* As pgs_time_variants, with the forward (ms_fwd [9]) and backward (ms_bwd [9]) times apart. */
int pgs_time_variants_split(pgs_ctx* ctx, float* image, const float* dL_dimage, int32_t reps, float* ms_fwd,
                            float* ms_bwd);

/* ---------------------------------------------------------------------------------------------
   Initialization (operator I of Sec. III-B) and its learned stand-in.
   --------------------------------------------------------------------------------------------- */
typedef struct pgs_init pgs_init;

/* A context for the initializer kernels on `cuda_stream`; owns the kNN grid scratch. */
int pgs_init_create(pgs_init** out, void* cuda_stream);
void pgs_init_destroy(pgs_init* ctx);

/* The k (3, 16 or 32) nearest other points of each of n points [3][n] (device fp32): nb [n][k]
   (device int32), ascending by squared distance d2 = fma(dx,dx, fma(dy,dy, dz*dz)) in fp32 with
   ties by index; exact (uniform grid, search widened until provably complete).  -1 pads when
   n - 1 < k.  Synchronises once (bounding box). */
int pgs_knn(pgs_init* ctx, const float* points, int64_t n, int32_t k, int32_t* nb);

/* From 32-neighbour lists nb [n][32]: the paper's initializer (Eq. 5 normal from 16 neighbours,
   Eq. 6 scale from 3, normal scale r_normal * s_t, z axis onto the normal, opacity logit(0.1),
   means = points, SH = 0) written into `init`; the 16 features of the learned initializer
   (eigenvalues / sum ascending, eigenvectors smallest first, mean offset / mean distance,
   -3 log mean distance) as features [n][16] fp32 and features_bf16 [n][16]; the eigenframe
   quaternion frame_q [4][n] (x largest, z smallest eigenvector).  All device pointers. */
int pgs_features_init(pgs_init* ctx, const float* points, int64_t n, const int32_t* nb32,
                      float r_normal, float* features, void* features_bf16, float* frame_q,
                      pgs_gaussians* init);

/* MLP 16-64-64-8 (GELU): master = FP32 parameters [W1 64x16 | b1 64 | W2 64x64 | b2 64 |
   W3 8x64 | b3 8] (row-major [out][in]), W1/W2/W3 = their BF16 copies used by the kernels. */
typedef struct {
    float* master;
    void* W1;
    void* W2;
    void* W3;
} pgs_mlp;
int pgs_mlp_param_count(void);
/* refresh the BF16 copies from the master parameters */
int pgs_mlp_pack(pgs_init* ctx, const pgs_mlp* w);
/* out [n][8] fp32 = MLP(x) for x [n][16] bf16 */
int pgs_mlp_forward(pgs_init* ctx, const pgs_mlp* w, const void* x_bf16, int64_t n, float* out);
/* adds d(loss)/d(parameters) to grad [param_count] and the summed per-point loss to *loss_sum
   (device double); loss = mean over points of |y0..2 - t0..2|^2 + (1 - <y3..6/|y3..6|, t3..6>^2)
   + (y7 - t7)^2, targets [n][8] fp32 with unit quaternions in t3..6 */
int pgs_mlp_grad(pgs_init* ctx, const pgs_mlp* w, const void* x_bf16, const float* targets,
                 int64_t n, float* grad, double* loss_sum);
/* Adam step t on the master parameters (b1 0.9, b2 0.999, eps 1e-8), BF16 copies refreshed,
   grad zeroed */
int pgs_mlp_adam(pgs_init* ctx, pgs_mlp* w, float* grad, float* m, float* v, float lr, int64_t t);

/* Learned initial parameters from MLP outputs y [n][8] (device), as corrections of the paper's
   initializer `pca` of the same point (operator I, Eq. 5-6): log-scales pca + y0..2, rotation
   normalise(pca q) (x) normalise(y3..6), opacity logit pca + y7, written into `out` (log_scales,
   quats, opacity_logits; means and SH are left to the caller).  Points whose output is not finite
   (or whose y3..6 is zero) keep the paper's initializer and are counted in *fallbacks (device
   uint32, added to). */
int pgs_apply_mlp(pgs_init* ctx, const float* y, const pgs_gaussians* pca, pgs_gaussians* out,
                  uint32_t* fallbacks);
/* Training targets t [n][8] (device fp32) of converged Gaussians relative to the paper's
   initializer `pca` of the same points: log-scale differences, conj(normalise(pca q)) (x)
   normalise(q), opacity-logit difference.  pca and converged have the same n. */
int pgs_make_targets(pgs_init* ctx, const pgs_gaussians* pca, const pgs_gaussians* converged, float* t);

/* ------------------------------------------------------------------------------------------
   Bundle adjustment of the geometry prior (Sec. III-A): Levenberg-Marquardt on the robust
   reprojection objective (Eq. 2), each step solved through the reduced camera system (Eq. 3):
   the point blocks are inverted independently (3 x 3 each), folded into a dense 6C x 6C camera
   system (Schur complement), which is solved by Cholesky (FP64), and the point steps follow by
   back-substitution.
     camera i: world-to-camera rotation R_i (row-major 3 x 3) and translation t_i, x = R_i P + t_i;
     observation o of point pt[o] in camera cam[o] at pixel uv[o]; intrinsics K = (fx, fy, cx, cy);
     residual r = pi(x) - uv, whitened norm e = |r| / sigma; Huber: rho = e^2 (e <= delta) or
     2 delta e - delta^2, solved by reweighting (weight 1 or delta / e);
     step: R_i <- exp([omega_i]x) R_i, t_i <- t_i + v_i, P_j <- P_j + d_j; damping
     H + lambda diag(H);
     gauge: camera 0 fixed, and of camera 1's translation the component along which its baseline
     to camera 0, in camera 1's frame, is largest (computed from the state at the call's start).
   Layout (all device, FP32 unless said): R [C][9], t [C][3], P [n][3], cam / pt [m] int32 with
   pt non-decreasing (observations grouped by point), uv [m][2]; K is a host array of 4 floats.
   Observations behind their camera (z <= 1e-6) carry no weight.  Errors: PGS_ERR_INVALID_ARG
   for a null pointer, bad size, a cam or pt index out of range or pt not sorted (checked on the
   device before any other work); PGS_ERR_NOT_PD when the damped reduced system is not positive
   definite.
   ------------------------------------------------------------------------------------------ */
typedef struct pgs_ba pgs_ba;
/* Buffers for C cameras (2..256), n points and m observations, work on `cuda_stream`. */
int pgs_ba_create(pgs_ba** out, int32_t n_cams, int64_t n_points, int64_t n_obs, void* cuda_stream);
void pgs_ba_destroy(pgs_ba* ba);
/* uv [count][2] and depth z [count] of the given (cam, pt) pairs (device); z is not checked, a
   pair with an index out of range gets NaN. */
int pgs_ba_project(pgs_ba* ba, const float* R, const float* t, const float* P, const int32_t* cam,
                   const int32_t* pt, int64_t count, const float* K, float* uv, float* z);
/* One damped step at `lambda` from the given state, not applied: dcam [C][6] (omega, v; zero for
   fixed parameters) and dP [n][3] (device), and the robust cost of the state (*cost, host). */
int pgs_ba_step(pgs_ba* ba, const float* R, const float* t, const float* P, const int32_t* cam,
                const int32_t* pt, const float* uv, const float* K, float sigma, float huber_delta,
                float lambda, float* dcam, float* dP, double* cost);
/* `iters` Levenberg-Marquardt trials from lambda0, R, t, P updated in place: a trial whose
   robust cost is lower is taken and lambda divided by 10, else lambda multiplied by 10 and the
   linearization reused.  costs [iters + 1] (host) receives the cost after each trial (costs[0]
   initial), *accepted (host) the number taken.  Synchronises once per trial. */
int pgs_ba_solve(pgs_ba* ba, float* R, float* t, float* P, const int32_t* cam, const int32_t* pt,
                 const float* uv, const float* K, float sigma, float huber_delta, int32_t iters,
                 float lambda0, double* costs, int32_t* accepted);

/* Device times (ms) of the stages of one iteration from the given state (nothing applied):
   ms[0] point linearization (H_pp, b_p, H_tp), ms[1] camera blocks (H_tt, b_t), ms[2] point
   inverses and E, ms[3] reduced-system blocks, ms[4] reduced-system solve, ms[5]
   back-substitution and candidate poses, ms[6] candidate cost.  Synchronises. */
int pgs_ba_stage_times(pgs_ba* ba, const float* R, const float* t, const float* P, const int32_t* cam,
                       const int32_t* pt, const float* uv, const float* K, float sigma, float huber_delta,
                       float lambda, float* ms);

/* ------------------------------------------------------------------------------------------
   Single-reference cost-volume MVS of the geometry prior (Sec. III-A): depth range of a target
   keyframe from the projected sparse points ([0.5 q.05, 1.5 q.95]), its reference keyframe by
   Eq. 4, census matching over a plane sweep, SGM aggregation, the 0.4 confidence filter, and
   fusion of the kept depths into world points.
     luma Y = 0.299 R + 0.587 G + 0.114 B; census: 7 x 7 window, 48 bits in raster order of the
     neighbours, set when the neighbour is darker, outside neighbours clear; D planes
     fronto-parallel in the target, uniform in inverse depth, plane 0 the farthest; cost = Hamming
     distance of the census codes at the target pixel and at the reference pixel its centre maps to
     through the plane (24 when behind the reference or outside it); SGM: 4 paths, P1 = 8,
     P2 = 32; a pixel is kept when its best plane is interior and 1 - S1 / S2 >= 0.4, S2 the best
     aggregated cost two or more planes away; depth refined by the parabola through the best plane
     and its neighbours, in inverse depth.  Eq. 4: b = distance of the camera centres, b_target =
     0.1 x the median sparse depth, sigma_b = 0.5 b_target, alpha = angle between the optical
     axes, alpha_min = 5 degrees; ties go to the lowest index.
   Images are device [3][H][W] FP32 of the context's size; cameras are pgs_camera (viewmat world ->
   camera) of that size.  A context holds one target's census codes (u64 [H][W] x 2), cost volume
   (u8 [H][W][D]) and aggregated cost (u16 [H][W][D]).
   ------------------------------------------------------------------------------------------ */
typedef struct pgs_mvs pgs_mvs;
#define PGS_MVS_CENSUS_TARGET 0    /* u64 [H][W] */
#define PGS_MVS_CENSUS_REFERENCE 1 /* u64 [H][W] */
#define PGS_MVS_COST 2             /* u8 [H][W][D] */
#define PGS_MVS_AGGREGATED 3       /* u16 [H][W][D] */
#define PGS_MVS_PLANE_MAPS 4       /* FP32 [D][9], row-major 3 x 3 per plane */
/* Buffers for width x height images and `planes` (3..128) depth hypotheses, work on cuda_stream. */
int pgs_mvs_create(pgs_mvs** out, int32_t width, int32_t height, int32_t planes, void* cuda_stream);
void pgs_mvs_destroy(pgs_mvs* mvs);
/* out[0..2] (host) = d_min, d_max, median sparse depth of the target, from the camera-z of the
   points [n][3] (device FP32) in front of it (z > 0.2) and inside its image; quantiles interpolate
   linearly between order statistics.  PGS_ERR_INVALID_ARG when no point qualifies.  Synchronises. */
int pgs_mvs_depth_range(pgs_mvs* mvs, const pgs_camera* target, const float* points, int64_t n, double* out);
/* The Eq. 4 reference of keyframe `target` among cams[0..count) (host array, count <= 1024):
   *ref (host), and the scores (host [count], optional; -inf for the target).  Synchronises. */
int pgs_mvs_select_reference(pgs_mvs* mvs, const pgs_camera* cams, int32_t count, int32_t target,
                             double median_depth, double* scores, int32_t* ref);
/* Depth map of the target (device [H][W] FP32 camera-z, NaN where not kept) between d_min and
   d_max; *kept (host, optional: synchronises when given) = kept pixels. */
int pgs_mvs_depth(pgs_mvs* mvs, const pgs_camera* target, const pgs_camera* reference, const float* image_t,
                  const float* image_r, double d_min, double d_max, float* depth, int64_t* kept);
/* pgs_mvs_depth with device times (ms): ms[0] census of both images, ms[1] plane maps and cost
   volume, ms[2] SGM, ms[3] selection.  Synchronises. */
int pgs_mvs_stage_times(pgs_mvs* mvs, const pgs_camera* target, const pgs_camera* reference, const float* image_t,
                        const float* image_r, double d_min, double d_max, float* depth, float* ms);
/* Copy an internal buffer of the last pgs_mvs_depth (PGS_MVS_*) to device memory dst. */
int pgs_mvs_read(pgs_mvs* mvs, int32_t what, void* dst, int64_t bytes);
/* World points (device [capacity][3] FP32) and row-major pixel indices (device int32) of the
   finite depths of a depth map, in pixel order; *count (host) = how many there are.
   PGS_ERR_CAPACITY when that exceeds capacity (the first `capacity` are written).  Synchronises. */
int pgs_mvs_fuse(pgs_mvs* mvs, const pgs_camera* target, const float* depth, float* points, int32_t* pixels,
                 int64_t capacity, int64_t* count);

/* Failure-detection self-test of the sort's bounded waits: one pass of the radix sort runs on the
   context's pair scratch with the first tile's look-back words never published, so the next tile's wait
   runs out (about a second), records the timeout in the device status word and abandons the pass
   without writing.  Synchronises; returns what pgs_status then reads (PGS_ERR_TIMEOUT when the
   detection works) and clears it.  The context stays usable; its last render is invalidated.
   No paper counterpart. */
int pgs_selftest_timeout(pgs_ctx* ctx);

/* Static description of an error code. */
const char* pgs_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* POCKETGS_H */
