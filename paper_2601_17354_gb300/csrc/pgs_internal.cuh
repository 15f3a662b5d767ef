// Internal declarations of libpocketgs: the context, its device scratch, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "pocketgs.h"

namespace pgs {

// Programmatic dependent launch between the short binning kernels. A kernel launched by
// launch_pdl may be scheduled while the kernel before it on the stream is finishing; it calls
// pdl_begin() first, which waits until that kernel has completed with its writes visible (a no-op
// for a plain launch) and then lets the kernel after it be scheduled early in turn. Nothing is
// read or written before the wait, so every kernel still sees all earlier kernels' results.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// screen tile edge T (pixels): 8, 16 (the default) or 32, one tile per compositing CTA
constexpr int kTileDefault = 16;
inline bool valid_tile(int T) { return T == 8 || T == 16 || T == 32; }
constexpr int kProjBlock = 256;      // threads per CTA of the per-Gaussian kernels
constexpr int kSortThreads = 256;    // threads per CTA of the radix-sort kernels
constexpr int kSortItems = 16;       // keys per thread in the radix-sort kernels of the pairs
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per sort CTA
// the coarse entries' sort: 512 threads x 8 keys, the pair sort's tile size
constexpr int kCoarseThreads = 512;
constexpr int kCoarseItems = 8;
static_assert(kCoarseThreads * kCoarseItems == kSortTile, "coarse sort CTAs cover kSortTile keys");
constexpr int kDepthThreads = 512;   // threads per CTA of the depth sort's passes (more warps per key)
constexpr int kDepthItems = 4;       // keys per thread in the depth sort (more, shorter CTAs)
constexpr int kDepthTile = kDepthThreads * kDepthItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 8;
// the digit totals of a sort are kept as this many partial copies (CTA b adds into copy b mod
// kTotalCopies), so no counter takes more than a few dozen CTAs' atomics
constexpr int kTotalCopies = 16;
constexpr int kTotalWords = kTotalCopies * kMaxPasses * kRadix;

// device status word bits
constexpr int32_t kStatusCapacity = 1;
constexpr int32_t kStatusNonfinite = 2;
constexpr int32_t kStatusInternal = 4;  // an index failed its bounds check; the access was skipped
constexpr int32_t kStatusTimeout = 8;   // a bounded wait on another CTA ran out; its work was abandoned
// words before the look-back region of a sort's scratch: an abort word and one ticket per pass
constexpr int kLookbackHead = 16;
// scratch words of a sort's look-back for `passes` passes over `tiles` CTA tiles
constexpr size_t lookback_words(int passes, int64_t tiles) { return kLookbackHead + (size_t)passes * 256 * tiles; }

// Two-level binning: screen tiles are grouped into super-tiles of kSuperW x kSuperH tiles (one bit
// each in a 32-bit mask); the pair lists are laid out super-tile by super-tile, tiles row-major
// inside a super-tile.  Coarse entries (one per Gaussian and super-tile its rectangle overlaps)
// are processed in blocks of kFineBlock.
constexpr int kSuperW = 8, kSuperH = 4;
constexpr int kFineBlock = 512;
inline int64_t super_tiles(int64_t TX, int64_t TY) {
    return ((TX + kSuperW - 1) / kSuperW) * ((TY + kSuperH - 1) / kSuperH);
}
// pair-buffer capacity the coarse stage needs besides the pairs themselves: its Ce entries, and 32
// counters per block of kFineBlock entries of a super-tile (at most floor(Ce / kFineBlock) + the
// non-empty super-tiles, at most min(S, Ce), blocks)
__host__ __device__ inline unsigned long long coarse_need(unsigned long long Ce, unsigned long long S) {
    const unsigned long long w = 32ull * (Ce / kFineBlock + (S < Ce ? S : Ce));
    return Ce > w ? Ce : w;
}

// Per-Gaussian projected record read by the compositing kernels (gathered by canonical index).
//   xyo   = (u, v, opacity, unused)   screen-space mean and opacity
//   conic = (a, b, c, unused)         inverse 2-D covariance; power = -(a dx^2 + c dy^2)/2 - b dx dy
//   rgb   = (r, g, b, unused)         view-dependent colour after the clamp at 0

struct Scratch {
    // per Gaussian
    float4* xyo = nullptr;
    float4* conic = nullptr;
    float4* rgb = nullptr;
    uint32_t* depth_bits = nullptr;
    uint2* rect = nullptr;  // (x0 | y0 << 16, x1 | y1 << 16), tiles, half-open
    uint32_t* hitmask = nullptr;  // rectangles of <= 32 tiles: bit k (row-major in the rectangle) = tile k reached
    uint4* smask = nullptr;       // > 32 tiles, super-tile rectangles of <= 2 x 2: mask per super-tile (smask_slot)
    uint32_t* touched = nullptr;
    uint32_t* block_sums = nullptr;
    unsigned long long* block_offsets = nullptr;
    // per super-tile: coarse entry range, first fine block (S + 1), pair count per tile (32 S),
    // pairs, first pair (S + 1)
    uint2* crange = nullptr;
    uint32_t* vbase = nullptr;
    uint32_t* stt = nullptr;
    uint32_t* ssum = nullptr;
    uint32_t* sbase = nullptr;
    float* grad2d = nullptr;  // [9][n]
    // per tile / pixel
    uint2* ranges = nullptr;
    uint32_t* tile_order = nullptr;  // tiles by decreasing list length (compositing schedule)
    float* T_final = nullptr;
    uint32_t* last = nullptr;
    uint32_t* ncomp = nullptr;  // entries composited per pixel
    // small words
    int32_t* status = nullptr;
    unsigned long long* pair_count = nullptr;
    unsigned long long* pair_need = nullptr;  // pair capacity the render needs (>= pair_count)
    unsigned long long* coarse_count = nullptr;
    uint32_t* bin_ticket = nullptr;  // [3] arrival counters of the binning's last-CTA steps (reset by it)
    uint32_t* tile_buckets = nullptr;  // [256] tile-order bucket counts (kept zero between renders), cursors
    uint32_t* sort_blocks = nullptr;  // sort CTAs with work in the current render
    uint32_t* digit_totals = nullptr; // [kTotalCopies][kMaxPasses][kRadix]
    float* loss_partials = nullptr;   // [2][kLossBlocks]
    uint32_t* loss_ticket = nullptr;
    double* l1_acc = nullptr;         // [3]: the fused L1's sums of |d| and d^2, then its CTA ticket
    // depth sort of the Gaussians: keys = depth bits (culled: all ones), values = canonical index;
    // its key count / CTA count words and histograms, separate from those of the coarse entries' sort
    unsigned long long* dkeys[2] = {nullptr, nullptr};
    uint32_t* dvals[2] = {nullptr, nullptr};
    uint32_t* dhist = nullptr;  // the depth sort's look-back
    uint32_t* dtotals = nullptr;
    unsigned long long* dcount = nullptr;
    uint32_t* dblocks = nullptr;
    // per pair (separate allocation, grows independently)
    unsigned long long* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* sort_hist = nullptr;  // the sort's look-back: head words, then [passes][tiles][kRadix]
    uint4* binfo = nullptr;         // fine blocks: super-tile, first entry, end entry, block of the
                                    // super-tile (pairs / 32 + 1 slots)
};

constexpr int kLossBlocks = 1024;

// One render of a batch (device table): its camera, its scene, where its projected Gaussians
// ("items"), tiles and pixels start in the batch-wide arrays, and its image buffers.
struct RenderDesc {
    pgs_camera cam;
    int32_t scene;
    int32_t TX, TY;
    int32_t tile;        // tile edge T
    int32_t SX;          // super-tiles per row
    int64_t item_base;   // first item: item j of the render = Gaussian j - item_base of the scene
    int64_t n;           // Gaussians of the scene
    int64_t tile_base;   // first batch-wide tile
    int64_t super_base;  // first batch-wide super-tile
    int64_t pixel_base;  // first pixel of the batch-wide per-pixel planes
    int64_t value_base;  // first value of the batch-wide image buffers (3 H W per render)
    float* image;        // [3][H][W]
    const float* target; // [3][H][W]
    float* dL;           // [3][H][W]
};

// One scene of a batch (device table): parameters and Adam moments, and its renders
// [first_render, first_render + n_renders) (renders are stored scene by scene).
struct SceneDesc {
    pgs_gaussians params, m, v;
    int32_t first_render, n_renders;
    int64_t gauss_base;  // first Gaussian of the scene in the batch-wide Gaussian numbering
};

// One Adam update (Kingma & Ba 2015) of parameter p with gradient g.  The bias corrections are
// folded into two per-step constants formed in double: lr_hat = lr / (1 - b1^t) and
// isb = 1 / sqrt(1 - b2^t), so p -= lr_hat m / (sqrt(v) isb + eps), which is algebraically the
// textbook lr m^ / (sqrt(v^) + eps).  The square root and the reciprocal use the approximate
// special-function instructions (relative error about 2^-22, far below the step's own scale);
// every other operation is an explicitly rounded fp32 multiply or fma, so the update is the same
// in every translation unit whatever its contraction flags.
__device__ __forceinline__ void adam_update(float& p, float& m, float& v, float g, float b1, float b2,
                                            float omb1, float omb2, float lr_hat, float isb, float eps) {
    m = __fmaf_rn(b1, m, __fmul_rn(omb1, g));
    v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(omb2, g), g));
    float s, r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(v));
    const float den = __fmaf_rn(s, isb, eps);
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(den));
    p = __fmaf_rn(-lr_hat, __fmul_rn(m, r), p);
}

// Compositing kernel variant: pixels per thread and entries staged per batch.
struct CompositeVariant {
    int pix, depth;
};
bool valid_variant(CompositeVariant v, int T);
CompositeVariant default_variant();

// ---------------------------------------------------------------------------------------------
// launchers (all asynchronous on `s`); each returns the number of kernels it launched
// ---------------------------------------------------------------------------------------------

// Word ranges of a render's scratch that must be zero before its binning (look-back words, digit
// totals, counters, tile and super-tile ranges).  The projection clears them on its way, so the
// binning launches no separate clears.
constexpr int kZeroRegions = 10;  // render_zero_plan adds at most 8
struct ZeroPlan {
    uint32_t* p[kZeroRegions];
    uint32_t words[kZeroRegions];
    int count;
};
// The ranges one render's depth sort, pair count and tile lists use (n Gaussians, `tiles` tiles
// in `supers` super-tiles, pair capacity `capacity`).
ZeroPlan render_zero_plan(const Scratch& sc, int64_t n, int64_t tiles, int64_t supers, int64_t capacity);
// The same clears as separate memsets (after the scratch moved, e.g. a grown pair arena).
void clear_zero_plan(const ZeroPlan& z, cudaStream_t s);

// K1: project + cull + SH colour; writes the projected record, depth bits, tile rectangle,
// tiles touched and the per-CTA sum of tiles touched, and zeroes the ranges of `zero`.
int launch_project_fwd(const pgs_gaussians& g, const pgs_camera& cam, int TX, int TY, int T,
                        const Scratch& sc, const ZeroPlan& zero, cudaStream_t s);
// K9: chain screen-space gradients (grad2d) to the parameters, added into grads.
int launch_project_bwd(const pgs_gaussians& g, const pgs_camera& cam, const Scratch& sc,
                        pgs_gaussians& grads, cudaStream_t s);

// Depth sort of the Gaussians (LSD radix over the 32 depth bits of dkeys[0] / dvals[0]); returns
// the kernels launched, *perm receives the buffer holding the depth-ordered canonical indices.
// cleared: its look-back words and digit totals are already zero (render_zero_plan).
int launch_depth_sort(int64_t n, const Scratch& sc, cudaStream_t s, const uint32_t** perm, bool cleared = false);
// K9 + K10 fused: chain the screen-space gradients to the parameters and apply one Adam step to
// every Gaussian (culled ones with a zero gradient) without storing the gradient.
int launch_project_bwd_adam(const pgs_gaussians& g, const pgs_camera& cam, const Scratch& sc,
                            pgs_gaussians& m, pgs_gaussians& v, const float lr[6], float b1,
                            float b2, float eps, int64_t t, cudaStream_t s);

// Batched variants (render / scene tables in device memory; see RenderDesc, SceneDesc).
int launch_project_fwd_batch(const RenderDesc* renders, int R, const SceneDesc* scenes, int deg,
                             int64_t items, const Scratch& sc, cudaStream_t s);
int launch_bwd_adam_batch(const RenderDesc* renders, const SceneDesc* scenes, int S, int deg,
                          int64_t gauss_total, int64_t items, const Scratch& sc, const float lr[6],
                          float b1, float b2, float eps, const int64_t* step, cudaStream_t s);
int launch_step_tick(int64_t* step, const int32_t* status, cudaStream_t s);
// The batched projection backward alone: each scene's parameter gradient, summed over its renders,
// added to grads[scene] (a device table of S pgs_gaussians).
int launch_bwd_batch(const RenderDesc* renders, const SceneDesc* scenes, int S, int deg, int64_t gauss_total,
                     int64_t items, const Scratch& sc, const pgs_gaussians* grads, cudaStream_t s);
int launch_loss_batch(const RenderDesc* renders, int R, int64_t values, double* losses, cudaStream_t s);

// Initializer path (K13 kNN, K14 features + paper initializer, K15 MLP).
size_t knn_scratch_bytes(int64_t n, int64_t cells);
int launch_bbox(int64_t n, const float* P, int* bbox_dev, cudaStream_t s);
void decode_bbox(const int* enc, float* out);
int launch_knn(int64_t n, const float* P, int k, int32_t* nb, void* scratch, size_t scratch_bytes,
               const float* host_bbox, cudaStream_t s);
int launch_features_init(int64_t n, const float* P, const int32_t* nb, float r_normal, float* feats,
                         void* feats_bf16, float* frame_q, pgs_gaussians& init, cudaStream_t s);
int launch_apply_mlp(int64_t n, const float* y, const pgs_gaussians& pca, pgs_gaussians& out,
                     uint32_t* fallbacks, cudaStream_t s);
int launch_make_targets(int64_t n, const pgs_gaussians& pca, const pgs_gaussians& conv, float* t,
                        cudaStream_t s);
int mlp_param_count();
int launch_mlp_forward(const void* x, int64_t n, const float* master, const void* W1, const void* W2,
                       const void* W3, float* out, cudaStream_t s);
int launch_mlp_train(const void* x, const float* target, int64_t n, const float* master, const void* W1,
                     const void* W2, const void* W3, float* grad, double* loss_sum, cudaStream_t s);
int launch_mlp_adam(float* master, float* grad, float* m, float* v, float lr, float b1, float b2,
                    float eps, int64_t t, void* W1, void* W2, void* W3, cudaStream_t s);
int launch_mlp_pack(const float* master, void* W1, void* W2, void* W3, cudaStream_t s);

// K2: pair count (the Gaussians' reached tiles, exact) and the coarse entries' per-CTA counts in
// depth order with their scan; writes pair_count, pair_need and coarse_count and raises the
// capacity status when pair_need exceeds `capacity`.  `supers` = super-tiles of the render (batch:
// of all renders).
// cleared: pair_count is already zero.
int launch_bin_count(int64_t n, int64_t supers, int64_t capacity, const uint32_t* perm, const Scratch& sc,
                     cudaStream_t s, bool cleared = false);
// K3-K5 after launch_bin_count: coarse entries in depth order, their stable sort by super-tile, the
// reached-tile masks and pair lists of every tile in depth order (values = canonical indices in
// vals[*out_buf], laid out super-tile by super-tile), and the tile ranges.  TX, TY: the tile grid
// of a single render (renders == nullptr); a batch reads each render's grid from `renders`.
// cleared: the ranges, the digit totals and the sort's look-back words are already zero.
int launch_bin_lists(int64_t n, int TX, int TY, int T, int64_t tiles, int64_t supers, int64_t capacity,
                     const uint32_t* perm, const Scratch& sc, cudaStream_t s, int* out_buf,
                     const RenderDesc* renders = nullptr, int R = 0, bool cleared = false);

// K4 alone over keys[0]/vals[0] with keys[1]/vals[1] as the other ping-pong buffer, sorting by the
// low key_bits bits only (higher bits never take part; the pair count is read from sc.pair_count,
// at most `capacity`); the digit totals must be zero on entry.
int launch_radix_sort_only(int64_t capacity, int key_bits, const Scratch& sc, cudaStream_t s,
                           int* out_buf);

// Failure-detection self-test: one sort pass whose first tile is never published (the next tile's
// bounded wait runs out and records kStatusTimeout); needs a pair capacity of three sort tiles.
int launch_timeout_selftest(int64_t capacity, const Scratch& sc, cudaStream_t s);

// Order the tiles by decreasing list length (quarter-octave buckets), so the compositing grids
// start the heaviest tiles first.
int launch_tile_order(int tiles, const Scratch& sc, cudaStream_t s);

// K6/K8: compositing forward and backward (sorted values in buffer `buf`).
// The L1 loss fused into the compositing forward (target == nullptr: off): with n = 3 H W values,
// dL[k] = sign(image[k] - target[k]) * inv_n; the CTAs add their sums of |d| and d^2 into acc[0],
// acc[1] (zero on entry) and the last CTA (ticket, zero on entry) writes out[0] = acc[0] / n,
// out[1] = acc[1].
struct L1Fused {
    const float* target = nullptr;
    float* dL = nullptr;
    float inv_n = 0.f;
    int64_t n = 0;
    double* acc = nullptr;
    uint32_t* ticket = nullptr;
    float* out = nullptr;
};
// zero_grad: also zero the first zero_grad floats of sc.grad2d (the coming backward's screen-space
// gradients), spread over the CTAs, in place of a separate clear.
int launch_composite_fwd(const pgs_camera& cam, int TX, int TY, int T, int buf, int64_t n,
                         const Scratch& sc, float* image, cudaStream_t s, CompositeVariant v,
                         int64_t zero_grad = 0, const L1Fused& l1f = L1Fused{});
int launch_composite_bwd(const pgs_camera& cam, int TX, int TY, int T, int buf, int64_t n,
                         const Scratch& sc, const float* dL_dimage, cudaStream_t s, CompositeVariant v);
// Replay-cache compositing (one pixel per thread): the forward records, per pixel, the first K
// composited entries as 16-byte records {position | clamp << 31, alpha, T in front, unused}
// into rec [pixels][K] and their count (K + 1 on overflow); the backward replays them
// (recomputing overflowed pixels).
int launch_composite_replay(const pgs_camera& cam, int TX, int TY, int T, int buf, int64_t n,
                            const Scratch& sc, float* image, const float* dL_dimage, float4* rec,
                            uint32_t* count, int K, bool backward, cudaStream_t s);
// Decision trace of listed pixels (x, y pairs) of the last render: per evaluated entry o G and the
// decision code, and per pixel the count, the fp32 transmittance, last and composited count.
int launch_trace_pixels(const pgs_camera& cam, int TX, int T, int buf, int64_t n, const Scratch& sc,
                        const int32_t* pix, int64_t npix, int max_entries, float* og, uint8_t* code,
                        int32_t* count, float* T_out, uint32_t* last, uint32_t* ncomp, cudaStream_t s);
// Batched compositing over every tile of every render in one persistent launch; `work` is a
// zeroed device counter.
int launch_composite_batch(const RenderDesc* renders, int R, int64_t total_tiles, int T, int buf,
                           int64_t n, const Scratch& sc, uint32_t* work, bool backward,
                           cudaStream_t s, CompositeVariant v);

// L1 + D-SSIM loss and gradient of [3][H][W] images; dm = 9 H W floats of scratch, sums = 2
// doubles of scratch, loss_out = device {loss, mean SSIM}.
int launch_loss_dssim(const float* image, const float* target, int W, int H, float lam, float* dm,
                      double* sums, float* grad, float* loss_out, cudaStream_t s);
// Does the 3-sigma ellipse {Q <= 9} of a projected Gaussian (screen position u, v; conic ca, cb,
// cc) reach the pixel-centre box of tile (tx, ty) of edge T?  The minimum of the convex Q over the
// box is at the clamped centre or on an edge at the clamped line minimum.  Part of the prescribed
// fp32 decision path (membership): every operation an explicit correctly rounded intrinsic, in
// the order of the oracle's definition.
__device__ __forceinline__ float hit_q(float X, float Y, float u, float v, float ca, float cb, float cc) {
    const float dx = __fadd_rn(X, -u), dy = __fadd_rn(Y, -v);
    return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(ca, dx), dx), __fmul_rn(__fmul_rn(__fadd_rn(cb, cb), dx), dy)),
                     __fmul_rn(__fmul_rn(cc, dy), dy));
}
// (sx, sy) = (cb / ca, cb / cc): the slopes of the line minima, per Gaussian; the test stops at the
// first candidate within the ellipse (min <= 9 exactly when some candidate is)
__device__ __forceinline__ bool tile_hit(float u, float v, float ca, float cb, float cc, float sx, float sy, int tx,
                                         int ty, int T) {
    const float xl = __fadd_rn((float)(tx * T), 0.5f), xh = __fadd_rn((float)(tx * T + T), -0.5f);
    const float yl = __fadd_rn((float)(ty * T), 0.5f), yh = __fadd_rn((float)(ty * T + T), -0.5f);
    if (hit_q(fminf(fmaxf(u, xl), xh), fminf(fmaxf(v, yl), yh), u, v, ca, cb, cc) <= 9.0f) return true;
    if (hit_q(xl, fminf(fmaxf(__fadd_rn(v, -__fmul_rn(sy, __fadd_rn(xl, -u))), yl), yh), u, v, ca, cb, cc) <= 9.0f)
        return true;
    if (hit_q(xh, fminf(fmaxf(__fadd_rn(v, -__fmul_rn(sy, __fadd_rn(xh, -u))), yl), yh), u, v, ca, cb, cc) <= 9.0f)
        return true;
    if (hit_q(fminf(fmaxf(__fadd_rn(u, -__fmul_rn(sx, __fadd_rn(yl, -v))), xl), xh), yl, u, v, ca, cb, cc) <= 9.0f)
        return true;
    return hit_q(fminf(fmaxf(__fadd_rn(u, -__fmul_rn(sx, __fadd_rn(yh, -v))), xl), xh), yh, u, v, ca, cb, cc) <= 9.0f;
}

// Reach masks of super-tiles (bit (ty mod kSuperH) kSuperW + tx mod kSuperW = tile (tx, ty)).
// A Gaussian of more than 32 tiles whose super-tile rectangle is at most 2 x 2 keeps its masks in
// one uint4, slot 2 (sy - sy0) + (sx - sx0) (x, y, z, w); smaller ones keep their reach bits in the
// rectangle's hitmask, larger ones have none (the binning computes theirs).
__device__ __forceinline__ bool small_super_rect(uint2 rect) {
    const uint32_t sx0 = (rect.x & 0xffffu) / kSuperW, sy0 = (rect.x >> 16) / kSuperH;
    const uint32_t sx1 = ((rect.y & 0xffffu) + kSuperW - 1) / kSuperW, sy1 = ((rect.y >> 16) + kSuperH - 1) / kSuperH;
    return sx1 - sx0 <= 2u && sy1 - sy0 <= 2u;
}
__device__ __forceinline__ uint32_t smask_slot(const uint4& m, uint32_t slot) {
    return slot == 0 ? m.x : slot == 1 ? m.y : slot == 2 ? m.z : m.w;
}
// add tile (tx, ty) to the masks of a Gaussian whose super-tile rectangle starts at (sx0, sy0)
__device__ __forceinline__ void smask_add(uint4& m, uint32_t tx, uint32_t ty, uint32_t sx0, uint32_t sy0) {
    const uint32_t slot = 2u * (ty / kSuperH - sy0) + (tx / kSuperW - sx0);
    const uint32_t bit = 1u << ((ty % kSuperH) * kSuperW + (tx % kSuperW));
    if (slot == 0) m.x |= bit;
    else if (slot == 1) m.y |= bit;
    else if (slot == 2) m.z |= bit;
    else m.w |= bit;
}
// Mask of super-tile (sx, sy), which overlaps the tile rectangle [x0, x1) x [y0, y1) of at most 32
// tiles, from the rectangle's reach bits `hits` (row-major in the rectangle).
__device__ __forceinline__ uint32_t super_mask_from_hits(uint32_t hits, uint32_t x0, uint32_t y0, uint32_t x1,
                                                         uint32_t y1, uint32_t sx, uint32_t sy) {
    const uint32_t bx = sx * kSuperW, by = sy * kSuperH;
    const uint32_t X0 = max(x0, bx), X1 = min(x1, bx + kSuperW), Y0 = max(y0, by), Y1 = min(y1, by + kSuperH);
    const uint32_t w = x1 - x0, row = (1u << (X1 - X0)) - 1u;
    uint32_t mask = 0;
    for (uint32_t ty = Y0; ty < Y1; ++ty)
        mask |= ((hits >> ((ty - y0) * w + (X0 - x0))) & row) << ((ty - by) * kSuperW + (X0 - bx));
    return mask;
}

// Bundle adjustment (Sec. III-A, Eq. 2-3): problem shape and chunking, index check, per-point
// offsets and camera masks, linearization, one Levenberg-Marquardt trial through the reduced
// camera system, robust cost, projection.
struct BaShape {
    int C = 0;             // cameras
    int64_t n = 0;         // points
    int64_t m = 0;         // observations
    int W = 0;             // 32-bit camera-mask words per point
    int N = 0;             // 6 C
    int pairs = 0;         // C (C + 1) / 2 camera pairs
    int chc = 1, chs = 1;  // chunks of a camera's observations in the camera-block and Schur launches
    bool blocked = false;  // blocked Cholesky of the full matrix in shared memory (6C <= 224)
    size_t solve_smem = 0; // shared memory of the solve (0: packed matrix in global scratch)
};
BaShape ba_shape(int C, int64_t n, int64_t m);
int ba_configure_solve();
int launch_ba_check(int64_t m, int64_t n, int C, const int32_t* cam, const int32_t* pt, int* flag, cudaStream_t s);
int launch_ba_index(const BaShape& sh, const int32_t* pt, const int32_t* cam, int64_t* start, uint32_t* mask,
                    int64_t* cam_count, int64_t* cam_start, int64_t* cam_obs, cudaStream_t s);
int launch_ba_linearize(const BaShape& sh, const float* R, const float* t, const float* P, const int32_t* cam,
                        const int32_t* pt, const float* uv, const int64_t* start, const int64_t* cam_start,
                        const int64_t* cam_obs, const float K[4], float sigma, float delta, float* Htp, double* Hpp,
                        double* bp, double* camp, double* cost, cudaStream_t s, cudaEvent_t* ev = nullptr);
int launch_ba_trial(const BaShape& sh, const int32_t* pt, const int64_t* start, const uint32_t* mask,
                    const int64_t* cam_start, const int64_t* cam_obs, const int32_t* cam, const float* Htp,
                    const double* Hpp, const double* bp, const double* camp, double lam, int fixed_axis, double* Hinv,
                    double* y, float* E, double* schp, double* rhsp, double* Sfull, double* rhs, float* Aglob,
                    double* dc, const float* R, const float* t, const float* P, float* Rn, float* tn, float* Pn,
                    float* dcam, float* dP, int* status, cudaStream_t s, cudaEvent_t* ev = nullptr);
int launch_ba_cost(const BaShape& sh, const float* R, const float* t, const float* P, const int32_t* cam,
                   const float* uv, const int64_t* start, const float K[4], float sigma, float delta, double* cost,
                   cudaStream_t s);
int launch_ba_project(int64_t m, int64_t n, int C, const float* R, const float* t, const float* P, const int32_t* cam,
                      const int32_t* pt, const float K[4], float* uv, float* z, cudaStream_t s);
// Single-reference MVS (Sec. III-A): census, plane maps + cost volume, SGM, selection, fusion,
// sparse-depth quantiles, Eq. 4 reference choice.
int launch_mvs_census(const float* rgb, int W, int H, uint64_t* code, cudaStream_t s);
int launch_mvs_cost(const pgs_camera& t, const pgs_camera& r, const uint64_t* cen_t, const uint64_t* cen_r, int W,
                    int H, int D, double inv_far, double step, float* maps, uint8_t* C, cudaStream_t s);
int launch_mvs_sgm(const uint8_t* C, uint8_t* L, int W, int H, int D, cudaStream_t s);
int launch_mvs_select(const uint8_t* L, uint16_t* S, int W, int H, int D, double inv_far, double step, float* depth,
                      uint8_t* kept, unsigned long long* count, cudaStream_t s);
int launch_mvs_fuse(const float* depth, int W, int H, const pgs_camera& cam, uint32_t* cta_scratch, int64_t* total,
                    int64_t capacity, float* points, int32_t* pix, cudaStream_t s);
int mvs_fuse_ctas(int W, int H);
int launch_mvs_range(const float* P, int64_t n, const pgs_camera& cam, double* zbuf, unsigned long long* count,
                     double* out, int* status, cudaStream_t s);
int launch_mvs_reference(const void* cams_f, int count, int target, double median, double* scores, int* best,
                         cudaStream_t s);
size_t mvs_camf_bytes();
void mvs_pack_cameras(const pgs_camera* cams, int count, void* host_out);
// K7: L1 loss; K10: fused Adam over all parameter groups.
int launch_loss_l1(const float* image, const float* target, int64_t n, float* grad,
                    float* loss_out, const Scratch& sc, cudaStream_t s);
int launch_adam(pgs_gaussians& p, pgs_gaussians& g, pgs_gaussians& m, pgs_gaussians& v,
                 const float lr[6], float b1, float b2, float eps, int64_t t, cudaStream_t s);

__host__ __device__ inline int sh_coeffs(int degree) { return (degree + 1) * (degree + 1); }
__host__ __device__ inline int param_rows(int degree) { return 11 + 3 * sh_coeffs(degree); }

}  // namespace pgs
