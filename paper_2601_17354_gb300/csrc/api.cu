// C ABI of libpocketgs: context, scratch arenas, and the render / loss / backward / step calls.
//
// Scratch lives in two device arenas owned by the context: one sized by (Gaussians, pixels,
// tiles) and one by the pair capacity, so growing the pair buffers never disturbs projected
// Gaussians of the render in flight.  Buffers are carved at 256-byte alignment.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pgs_internal.cuh"

using namespace pgs;

struct pgs_ctx {
    pgs_config cfg;
    cudaStream_t stream = nullptr;
    Scratch sc;
    void* arena_g = nullptr;
    void* arena_p = nullptr;
    int64_t cap_n = -1, cap_pixels = -1, cap_tiles = -1, cap_supers = -1, cap_pairs = 0;
    bool grow_pairs = false;
    // last render
    bool has_render = false;
    int64_t n = 0;
    int TX = 0, TY = 0, buf = 0;
    int tile = kTileDefault;  // tile edge T, fixed at creation
    // replay cache (pgs_set_replay_cache): K entries per pixel, off when 0
    int replay_k = 0;
    bool recorded = false;     // the last render recorded the cache
    bool grad_clean = false;   // grad2d is zero (cleared by the last forward), no backward since
    void* arena_c = nullptr;
    int64_t cap_c = 0;         // pixels x K the cache arena holds
    float4* c_rec = nullptr;
    uint32_t* c_count = nullptr;
    // D-SSIM scratch: 9 floats per pixel + 2 doubles
    void* arena_s = nullptr;
    int64_t cap_s = 0;
    pgs_camera cam{};
    pgs_gaussians params{};
    CompositeVariant variant = default_variant();       // forward compositing
    CompositeVariant variant_bwd = default_variant();   // backward compositing
    // instrumentation
    int64_t launches = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> events;       // pool, used in order
    size_t next_event = 0;
    struct Span { int stage; size_t a, b; };
    std::vector<Span> spans;
};

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += align256(sizeof(T) * (count ? count : 1));
        return p;
    }
};

// Layout of the (Gaussians, pixels, tiles) arena; with base == nullptr only measures.
size_t carve_g(Scratch& sc, char* base, int64_t n, int64_t pixels, int64_t tiles, int64_t supers) {
    Carver c{base};
    const int64_t nb = (n + kProjBlock - 1) / kProjBlock;
    sc.xyo = c.take<float4>(n);
    sc.conic = c.take<float4>(n);
    sc.rgb = c.take<float4>(n);
    sc.depth_bits = c.take<uint32_t>(n);
    sc.rect = c.take<uint2>(n);
    sc.hitmask = c.take<uint32_t>(n);
    sc.smask = c.take<uint4>(n);
    sc.touched = c.take<uint32_t>(n);
    sc.block_sums = c.take<uint32_t>(nb);
    sc.block_offsets = c.take<unsigned long long>(nb);
    sc.crange = c.take<uint2>(supers);
    sc.vbase = c.take<uint32_t>(supers + 1);
    sc.stt = c.take<uint32_t>(32 * supers);
    sc.ssum = c.take<uint32_t>(supers);
    sc.sbase = c.take<uint32_t>(supers + 1);
    sc.grad2d = c.take<float>(9 * n);
    sc.dkeys[0] = c.take<unsigned long long>(n);
    sc.dkeys[1] = c.take<unsigned long long>(n);
    sc.dvals[0] = c.take<uint32_t>(n);
    sc.dvals[1] = c.take<uint32_t>(n);
    sc.dhist = c.take<uint32_t>(lookback_words(32 / kRadixBits, (n + kDepthTile - 1) / kDepthTile));
    sc.dtotals = c.take<uint32_t>(kTotalWords);
    sc.dcount = c.take<unsigned long long>(1);
    sc.dblocks = c.take<uint32_t>(1);
    sc.ranges = c.take<uint2>(tiles);
    sc.tile_order = c.take<uint32_t>(tiles);
    sc.T_final = c.take<float>(pixels);
    sc.last = c.take<uint32_t>(pixels);
    sc.ncomp = c.take<uint32_t>(pixels);
    sc.status = c.take<int32_t>(1);
    sc.pair_count = c.take<unsigned long long>(1);
    sc.pair_need = c.take<unsigned long long>(1);
    sc.coarse_count = c.take<unsigned long long>(1);
    sc.bin_ticket = c.take<uint32_t>(3);
    sc.tile_buckets = c.take<uint32_t>(256);
    sc.sort_blocks = c.take<uint32_t>(1);
    sc.digit_totals = c.take<uint32_t>(kTotalWords);
    sc.loss_partials = c.take<float>(2 * kLossBlocks);
    sc.loss_ticket = c.take<uint32_t>(1);
    sc.l1_acc = c.take<double>(3);
    return c.off;
}

size_t carve_p(Scratch& sc, char* base, int64_t pairs) {
    Carver c{base};
    const int64_t sb = (pairs + kSortTile - 1) / kSortTile;
    sc.keys[0] = c.take<unsigned long long>(pairs);
    sc.keys[1] = c.take<unsigned long long>(pairs);
    sc.vals[0] = c.take<uint32_t>(pairs);
    sc.vals[1] = c.take<uint32_t>(pairs);
    sc.sort_hist = c.take<uint32_t>(lookback_words(32 / kRadixBits, sb ? sb : 1));  // 32-bit keys: at most 4 passes
    sc.binfo = c.take<uint4>(pairs / 32 + 1);
    return c.off;
}

constexpr size_t kEventPool = 8192;

// Record one event on the stream if profiling; returns its pool index or SIZE_MAX.
size_t mark(pgs_ctx* ctx) {
    if (!ctx->profiling) return SIZE_MAX;
    if (ctx->events.empty()) {
        ctx->events.resize(kEventPool);
        for (auto& e : ctx->events) cudaEventCreate(&e);
    }
    if (ctx->next_event >= ctx->events.size()) return SIZE_MAX;
    const size_t i = ctx->next_event++;
    cudaEventRecord(ctx->events[i], ctx->stream);
    return i;
}

void span(pgs_ctx* ctx, int stage, size_t a, size_t b) {
    if (a != SIZE_MAX && b != SIZE_MAX) ctx->spans.push_back({stage, a, b});
}

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return PGS_OK;
    if (e == cudaErrorMemoryAllocation) return PGS_ERR_OOM;
    return PGS_ERR_CUDA;
}

int reserve_g(pgs_ctx* ctx, int64_t n, int64_t pixels, int64_t tiles, int64_t supers) {
    if (n <= ctx->cap_n && pixels <= ctx->cap_pixels && tiles <= ctx->cap_tiles && supers <= ctx->cap_supers)
        return PGS_OK;
    n = n > ctx->cap_n ? n : ctx->cap_n;
    pixels = pixels > ctx->cap_pixels ? pixels : ctx->cap_pixels;
    tiles = tiles > ctx->cap_tiles ? tiles : ctx->cap_tiles;
    supers = supers > ctx->cap_supers ? supers : ctx->cap_supers;
    Scratch tmp = ctx->sc;
    const size_t bytes = carve_g(tmp, nullptr, n, pixels, tiles, supers);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(e);
    if (ctx->arena_g) cudaFree(ctx->arena_g);
    ctx->arena_g = nullptr;
    ctx->cap_n = ctx->cap_pixels = ctx->cap_tiles = ctx->cap_supers = -1;
    e = cudaMalloc(&ctx->arena_g, bytes);
    if (e != cudaSuccess) {
        ctx->arena_g = nullptr;
        return cuda_err(e);
    }
    carve_g(ctx->sc, static_cast<char*>(ctx->arena_g), n, pixels, tiles, supers);
    e = cudaMemsetAsync(ctx->arena_g, 0, bytes, ctx->stream);
    if (e != cudaSuccess) return cuda_err(e);
    ctx->cap_n = n;
    ctx->cap_pixels = pixels;
    ctx->cap_tiles = tiles;
    ctx->cap_supers = supers;
    ctx->has_render = false;
    return PGS_OK;
}

int reserve_p(pgs_ctx* ctx, int64_t pairs) {
    if (pairs <= ctx->cap_pairs) return PGS_OK;
    Scratch tmp = ctx->sc;
    const size_t bytes = carve_p(tmp, nullptr, pairs);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(e);
    if (ctx->arena_p) cudaFree(ctx->arena_p);
    ctx->arena_p = nullptr;
    ctx->cap_pairs = 0;
    e = cudaMalloc(&ctx->arena_p, bytes);
    if (e != cudaSuccess) {
        ctx->arena_p = nullptr;
        return cuda_err(e);
    }
    carve_p(ctx->sc, static_cast<char*>(ctx->arena_p), pairs);
    ctx->cap_pairs = pairs;
    ctx->has_render = false;
    return PGS_OK;
}

// replay cache arena for `pixels` pixels of K entries (16-byte records) plus a count per pixel
int reserve_c(pgs_ctx* ctx, int64_t pixels) {
    const int64_t K = ctx->replay_k;
    if (pixels * K <= ctx->cap_c && ctx->arena_c) return PGS_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(e);
    if (ctx->arena_c) cudaFree(ctx->arena_c);
    ctx->arena_c = nullptr;
    ctx->cap_c = 0;
    const size_t entries = (size_t)(pixels * K);
    const size_t bytes = align256(16 * entries) + align256(4 * (size_t)pixels);
    e = cudaMalloc(&ctx->arena_c, bytes);
    if (e != cudaSuccess) {
        ctx->arena_c = nullptr;
        return cuda_err(e);
    }
    Carver c{static_cast<char*>(ctx->arena_c)};
    ctx->c_rec = c.take<float4>(entries);
    ctx->c_count = c.take<uint32_t>((size_t)pixels);
    ctx->cap_c = pixels * K;
    return PGS_OK;
}

bool valid_gaussians(const pgs_gaussians* g) {
    if (!g || g->n < 0 || g->n >= (int64_t(1) << 32) || g->sh_degree < 0 || g->sh_degree > 3) return false;
    if (g->n == 0) return true;
    return g->means && g->log_scales && g->quats && g->opacity_logits && g->sh;
}

bool valid_camera(const pgs_camera* c) {
    if (!c || c->width <= 0 || c->height <= 0) return false;
    if (c->width > 65535 * 8 || c->height > 65535 * 8) return false;  // tile coordinates fit 16 bits
    return c->fx > 0.f && c->fy > 0.f && c->near_z > 0.f;
}

}  // namespace

extern "C" {

const char* pgs_strerror(int code) {
    switch (code) {
        case PGS_OK: return "ok";
        case PGS_ERR_INVALID_ARG: return "invalid argument";
        case PGS_ERR_NO_RENDER: return "backward without a preceding render on this context";
        case PGS_ERR_CAPACITY: return "more (tile, Gaussian) pairs than the pair capacity";
        case PGS_ERR_NONFINITE: return "non-finite parameter of a Gaussian";
        case PGS_ERR_CUDA: return "CUDA runtime error";
        case PGS_ERR_OOM: return "device allocation failed";
        case PGS_ERR_INTERNAL: return "device-side consistency check failed";
        case PGS_ERR_NOT_PD: return "bundle adjustment: damped reduced camera system not positive definite";
        case PGS_ERR_TOO_LARGE: return "size exceeds the fixed scratch of the allocation-free sort (262144 pairs)";
        case PGS_ERR_TIMEOUT: return "a bounded wait on the device ran out; the work it guarded was abandoned";
        default: return "unknown error";
    }
}

int pgs_create(pgs_ctx** out, const pgs_config* cfg, void* cuda_stream) {
    if (!out) return PGS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || !valid_tile(cfg->tile) || cfg->pair_capacity < 0) return PGS_ERR_INVALID_ARG;
    pgs_ctx* ctx = new (std::nothrow) pgs_ctx();
    if (!ctx) return PGS_ERR_OOM;
    ctx->cfg = *cfg;
    ctx->tile = cfg->tile;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->grow_pairs = cfg->pair_capacity == 0;
    int rc = reserve_g(ctx, 1, 1, 1, 1);
    if (rc == PGS_OK) rc = reserve_p(ctx, cfg->pair_capacity > 0 ? cfg->pair_capacity : (1 << 20));
    if (rc != PGS_OK) {
        pgs_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return PGS_OK;
}

void pgs_destroy(pgs_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& e : ctx->events) cudaEventDestroy(e);
    if (ctx->arena_g) cudaFree(ctx->arena_g);
    if (ctx->arena_p) cudaFree(ctx->arena_p);
    if (ctx->arena_c) cudaFree(ctx->arena_c);
    if (ctx->arena_s) cudaFree(ctx->arena_s);
    delete ctx;
}

int pgs_reserve(pgs_ctx* ctx, int64_t n, int32_t width, int32_t height, int64_t pair_capacity) {
    if (!ctx || n < 0 || width < 0 || height < 0 || pair_capacity < 0) return PGS_ERR_INVALID_ARG;
    const int64_t T = ctx->tile, TX = (width + T - 1) / T, TY = (height + T - 1) / T;
    int rc = reserve_g(ctx, n, (int64_t)width * height, TX * TY, super_tiles(TX, TY));
    if (rc == PGS_OK) rc = reserve_p(ctx, pair_capacity);
    return rc;
}

// pgs_render, and with target != nullptr pgs_render_l1 (the L1 loss in the compositing forward)
static int render_impl(pgs_ctx* ctx, const pgs_gaussians* params, const pgs_camera* cam, float* image_out,
                       const float* target, float* dL_dimage, float* loss_out) {
    if (!ctx || !valid_gaussians(params) || !valid_camera(cam) || !image_out) return PGS_ERR_INVALID_ARG;
    if (target && (!dL_dimage || !loss_out)) return PGS_ERR_INVALID_ARG;
    const int T = ctx->tile, TX = (cam->width + T - 1) / T, TY = (cam->height + T - 1) / T;
    const int64_t tiles = (int64_t)TX * TY, pixels = (int64_t)cam->width * cam->height;
    const int64_t supers = super_tiles(TX, TY);
    int rc = reserve_g(ctx, params->n, pixels, tiles, supers);
    if (rc != PGS_OK) return rc;
    cudaStream_t s = ctx->stream;
    ctx->has_render = false;
    ctx->grad_clean = false;
    const size_t e0 = mark(ctx);
    // the projection zeroes the binning's counters, look-back words and ranges on its way
    ctx->launches += launch_project_fwd(*params, *cam, TX, TY, T, ctx->sc,
                                        render_zero_plan(ctx->sc, params->n, tiles, supers, ctx->cap_pairs), s);
    const size_t e1 = mark(ctx);
    const uint32_t* perm = nullptr;
    if (params->n > 0) ctx->launches += launch_depth_sort(params->n, ctx->sc, s, &perm, true);
    ctx->launches += launch_bin_count(params->n, supers, ctx->cap_pairs, perm, ctx->sc, s, true);
    bool cleared = true;  // false once the pair arena has moved
    if (ctx->grow_pairs) {
        unsigned long long need = 0;
        cudaError_t e = cudaMemcpyAsync(&need, ctx->sc.pair_need, sizeof(need), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(e);
        if ((int64_t)need > ctx->cap_pairs) {
            // grow with headroom, clear the overflow flag, and count again (the coarse sort's CTA
            // count depends on the capacity)
            rc = reserve_p(ctx, (int64_t)(need + need / 4 + 1024));
            if (rc != PGS_OK) return rc;
            int32_t st = 0;
            e = cudaMemcpyAsync(&st, ctx->sc.status, sizeof(st), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_err(e);
            st &= ~kStatusCapacity;
            e = cudaMemcpyAsync(ctx->sc.status, &st, sizeof(st), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_err(e);
            ctx->launches += launch_bin_count(params->n, supers, ctx->cap_pairs, perm, ctx->sc, s);
            cleared = false;
        }
    }
    const size_t e2 = mark(ctx);
    ctx->launches += launch_bin_lists(params->n, TX, TY, T, tiles, supers, ctx->cap_pairs, perm, ctx->sc, s, &ctx->buf,
                                      nullptr, 0, cleared);
    ctx->launches += launch_tile_order((int)tiles, ctx->sc, s);
    const size_t e3 = mark(ctx);
    ctx->recorded = false;
    if (ctx->replay_k > 0) {
        rc = reserve_c(ctx, pixels);
        if (rc != PGS_OK) return rc;
        ctx->launches += launch_composite_replay(*cam, TX, TY, T, ctx->buf, params->n, ctx->sc, image_out, nullptr,
                                                 ctx->c_rec, ctx->c_count, ctx->replay_k, false, s);
        ctx->recorded = true;
    } else {
        // the forward also clears the screen-space gradients its backward accumulates
        L1Fused l1f;
        if (target) {
            l1f.target = target;
            l1f.dL = dL_dimage;
            l1f.n = 3 * pixels;
            l1f.inv_n = 1.0f / (float)l1f.n;
            l1f.acc = ctx->sc.l1_acc;  // zeroed by the projection
            l1f.ticket = reinterpret_cast<uint32_t*>(ctx->sc.l1_acc + 2);
            l1f.out = loss_out;
        }
        const int k = launch_composite_fwd(*cam, TX, TY, T, ctx->buf, params->n, ctx->sc, image_out, s, ctx->variant,
                                           9 * params->n, l1f);
        ctx->launches += k;
        ctx->grad_clean = k > 0;
    }
    const size_t e4 = mark(ctx);
    span(ctx, PGS_STAGE_PROJECT, e0, e1);
    span(ctx, PGS_STAGE_BIN, e1, e2);
    span(ctx, PGS_STAGE_SORT, e2, e3);
    span(ctx, PGS_STAGE_COMPOSITE_FWD, e3, e4);
    if (target && ctx->recorded) {  // the recording forward has no fused loss: the loss kernel
        const size_t e5 = mark(ctx);
        ctx->launches += launch_loss_l1(image_out, target, 3 * pixels, dL_dimage, loss_out, ctx->sc, s);
        span(ctx, PGS_STAGE_LOSS, e5, mark(ctx));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e);
    ctx->has_render = true;
    ctx->n = params->n;
    ctx->TX = TX;
    ctx->TY = TY;
    ctx->cam = *cam;
    ctx->params = *params;
    return PGS_OK;
}

int pgs_render(pgs_ctx* ctx, const pgs_gaussians* params, const pgs_camera* cam, float* image_out) {
    return render_impl(ctx, params, cam, image_out, nullptr, nullptr, nullptr);
}

int pgs_render_l1(pgs_ctx* ctx, const pgs_gaussians* params, const pgs_camera* cam, const float* target,
                  float* image_out, float* dL_dimage, float* loss_out) {
    if (!target) return PGS_ERR_INVALID_ARG;
    return render_impl(ctx, params, cam, image_out, target, dL_dimage, loss_out);
}

int pgs_loss_l1(pgs_ctx* ctx, const float* image, const float* target, int64_t n, float* dL_dimage,
                float* loss_out) {
    if (!ctx || !image || !target || !dL_dimage || !loss_out || n <= 0) return PGS_ERR_INVALID_ARG;
    const size_t e0 = mark(ctx);
    ctx->launches += launch_loss_l1(image, target, n, dL_dimage, loss_out, ctx->sc, ctx->stream);
    span(ctx, PGS_STAGE_LOSS, e0, mark(ctx));
    return cuda_err(cudaGetLastError());
}

// the backward compositing of the last render: replayed from the cache when it recorded one
static int composite_backward(pgs_ctx* ctx, const float* dL_dimage) {
    if (ctx->recorded)
        return launch_composite_replay(ctx->cam, ctx->TX, ctx->TY, ctx->tile, ctx->buf, ctx->n, ctx->sc, nullptr,
                                       dL_dimage, ctx->c_rec, ctx->c_count, ctx->replay_k, true, ctx->stream);
    return launch_composite_bwd(ctx->cam, ctx->TX, ctx->TY, ctx->tile, ctx->buf, ctx->n, ctx->sc, dL_dimage,
                                ctx->stream, ctx->variant_bwd);
}

int pgs_set_replay_cache(pgs_ctx* ctx, int32_t k_max) {
    if (!ctx || k_max < 0 || k_max > 4096) return PGS_ERR_INVALID_ARG;
    if (k_max != ctx->replay_k) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_err(e);
        if (ctx->arena_c) cudaFree(ctx->arena_c);
        ctx->arena_c = nullptr;
        ctx->cap_c = 0;
        ctx->replay_k = k_max;
        ctx->recorded = false;
        ctx->has_render = false;  // the next backward needs a render made with this setting
    }
    return PGS_OK;
}

int pgs_loss_dssim(pgs_ctx* ctx, const float* image, const float* target, int32_t width, int32_t height,
                   float lambda, float* dL_dimage, float* loss_out) {
    if (!ctx || !image || !target || !dL_dimage || !loss_out || width <= 0 || height <= 0 ||
        !(lambda >= 0.f && lambda <= 1.f))
        return PGS_ERR_INVALID_ARG;
    const int64_t pixels = (int64_t)width * height;
    if (pixels > ctx->cap_s) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_err(e);
        if (ctx->arena_s) cudaFree(ctx->arena_s);
        ctx->arena_s = nullptr;
        ctx->cap_s = 0;
        e = cudaMalloc(&ctx->arena_s, 256 + align256(sizeof(float) * 9 * (size_t)pixels));
        if (e != cudaSuccess) {
            ctx->arena_s = nullptr;
            return cuda_err(e);
        }
        ctx->cap_s = pixels;
    }
    double* sums = static_cast<double*>(ctx->arena_s);
    float* dm = reinterpret_cast<float*>(static_cast<char*>(ctx->arena_s) + 256);
    const size_t e0 = mark(ctx);
    ctx->launches += launch_loss_dssim(image, target, width, height, lambda, dm, sums, dL_dimage, loss_out,
                                       ctx->stream);
    span(ctx, PGS_STAGE_LOSS, e0, mark(ctx));
    return cuda_err(cudaGetLastError());
}

int pgs_backward(pgs_ctx* ctx, const float* dL_dimage, pgs_gaussians* grads) {
    if (!ctx || !dL_dimage || !valid_gaussians(grads)) return PGS_ERR_INVALID_ARG;
    if (!ctx->has_render) return PGS_ERR_NO_RENDER;
    if (grads->n != ctx->n || grads->sh_degree != ctx->params.sh_degree) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = ctx->stream;
    if (ctx->n > 0 && !ctx->grad_clean) cudaMemsetAsync(ctx->sc.grad2d, 0, sizeof(float) * 9 * (size_t)ctx->n, s);
    ctx->grad_clean = false;
    const size_t e0 = mark(ctx);
    ctx->launches += composite_backward(ctx, dL_dimage);
    const size_t e1 = mark(ctx);
    ctx->launches += launch_project_bwd(ctx->params, ctx->cam, ctx->sc, *grads, s);
    const size_t e2 = mark(ctx);
    span(ctx, PGS_STAGE_COMPOSITE_BWD, e0, e1);
    span(ctx, PGS_STAGE_PROJECT_BWD, e1, e2);
    return cuda_err(cudaGetLastError());
}

int pgs_step(pgs_ctx* ctx, pgs_gaussians* params, pgs_gaussians* grads, pgs_gaussians* m,
             pgs_gaussians* v, int64_t t) {
    if (!ctx || !valid_gaussians(params) || !valid_gaussians(grads) || !valid_gaussians(m) ||
        !valid_gaussians(v) || t < 1)
        return PGS_ERR_INVALID_ARG;
    const pgs_gaussians* all[3] = {grads, m, v};
    for (auto* q : all)
        if (q->n != params->n || q->sh_degree != params->sh_degree) return PGS_ERR_INVALID_ARG;
    if (params->n == 0) return PGS_OK;
    const size_t e0 = mark(ctx);
    ctx->launches += launch_adam(*params, *grads, *m, *v, ctx->cfg.lr, ctx->cfg.adam_b1,
                                 ctx->cfg.adam_b2, ctx->cfg.adam_eps, t, ctx->stream);
    span(ctx, PGS_STAGE_ADAM, e0, mark(ctx));
    return cuda_err(cudaGetLastError());
}

int pgs_backward_step(pgs_ctx* ctx, const float* dL_dimage, pgs_gaussians* params,
                      pgs_gaussians* m, pgs_gaussians* v, int64_t t) {
    if (!ctx || !dL_dimage || !valid_gaussians(params) || !valid_gaussians(m) ||
        !valid_gaussians(v) || t < 1)
        return PGS_ERR_INVALID_ARG;
    if (!ctx->has_render) return PGS_ERR_NO_RENDER;
    const pgs_gaussians* all[3] = {params, m, v};
    for (auto* q : all)
        if (q->n != ctx->n || q->sh_degree != ctx->params.sh_degree) return PGS_ERR_INVALID_ARG;
    if (params->means != ctx->params.means) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = ctx->stream;
    if (ctx->n > 0 && !ctx->grad_clean) cudaMemsetAsync(ctx->sc.grad2d, 0, sizeof(float) * 9 * (size_t)ctx->n, s);
    ctx->grad_clean = false;
    const size_t e0 = mark(ctx);
    ctx->launches += composite_backward(ctx, dL_dimage);
    const size_t e1 = mark(ctx);
    ctx->launches += launch_project_bwd_adam(*params, ctx->cam, ctx->sc, *m, *v, ctx->cfg.lr,
                                             ctx->cfg.adam_b1, ctx->cfg.adam_b2, ctx->cfg.adam_eps, t, s);
    const size_t e2 = mark(ctx);
    span(ctx, PGS_STAGE_COMPOSITE_BWD, e0, e1);
    span(ctx, PGS_STAGE_PROJECT_BWD_ADAM, e1, e2);
    return cuda_err(cudaGetLastError());
}

int pgs_status(pgs_ctx* ctx, int64_t* pairs_needed) {
    if (!ctx) return PGS_ERR_INVALID_ARG;
    int32_t st = 0;
    unsigned long long P = 0;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(&st, ctx->sc.status, sizeof(st), cudaMemcpyDeviceToHost, s);
    unsigned long long need = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&P, ctx->sc.pair_count, sizeof(P), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&need, ctx->sc.pair_need, sizeof(need), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->sc.status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    if (st & kStatusCapacity) P = need;  // the capacity to grow to (the pairs, or more for the coarse stage)
    if (pairs_needed) *pairs_needed = (int64_t)P;
    if (st & kStatusInternal) return PGS_ERR_INTERNAL;
    if (st & kStatusTimeout) return PGS_ERR_TIMEOUT;
    if (st & kStatusCapacity) return PGS_ERR_CAPACITY;
    if (st & kStatusNonfinite) return PGS_ERR_NONFINITE;
    return PGS_OK;
}

int pgs_trace_pixels(pgs_ctx* ctx, const int32_t* pixels, int64_t npix, int32_t max_entries, float* og,
                     uint8_t* code, int32_t* count, float* T_final, uint32_t* last, uint32_t* ncomp) {
    if (!ctx || npix < 0 || max_entries < 0 || (npix > 0 && (!pixels || !count || !T_final || !last || !ncomp)) ||
        (max_entries > 0 && npix > 0 && (!og || !code)))
        return PGS_ERR_INVALID_ARG;
    if (!ctx->has_render) return PGS_ERR_NO_RENDER;
    ctx->launches += launch_trace_pixels(ctx->cam, ctx->TX, ctx->tile, ctx->buf, ctx->n, ctx->sc, pixels, npix,
                                         max_entries, og, code, count, T_final, last, ncomp, ctx->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_selftest_timeout(pgs_ctx* ctx) {
    if (!ctx) return PGS_ERR_INVALID_ARG;
    int rc = reserve_p(ctx, 3 * (int64_t)kSortTile > ctx->cap_pairs ? 3 * (int64_t)kSortTile : ctx->cap_pairs);
    if (rc != PGS_OK) return rc;
    ctx->has_render = false;
    ctx->launches += launch_timeout_selftest(ctx->cap_pairs, ctx->sc, ctx->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e);
    return pgs_status(ctx, nullptr);
}

int pgs_profile(pgs_ctx* ctx, int enable) {
    if (!ctx) return PGS_ERR_INVALID_ARG;
    ctx->profiling = enable != 0;
    return PGS_OK;
}

int pgs_stage_times(pgs_ctx* ctx, double* ms, int64_t* counts) {
    if (!ctx || !ms || !counts) return PGS_ERR_INVALID_ARG;
    for (int k = 0; k < PGS_NUM_STAGES; ++k) {
        ms[k] = 0.0;
        counts[k] = 0;
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(e);
    for (const auto& sp : ctx->spans) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ctx->events[sp.a], ctx->events[sp.b]);
        if (e != cudaSuccess) return cuda_err(e);
        ms[sp.stage] += t;
        counts[sp.stage] += 1;
    }
    ctx->spans.clear();
    ctx->next_event = 0;
    return PGS_OK;
}

int64_t pgs_launch_count(const pgs_ctx* ctx) { return ctx ? ctx->launches : 0; }

int pgs_set_variant(pgs_ctx* ctx, int32_t pixels_per_thread, int32_t depth) {
    const CompositeVariant v{pixels_per_thread, depth};
    if (!ctx || !valid_variant(v, ctx->tile)) return PGS_ERR_INVALID_ARG;
    ctx->variant = v;
    ctx->variant_bwd = v;
    return PGS_OK;
}

int pgs_set_variants(pgs_ctx* ctx, int32_t fwd_pixels, int32_t fwd_depth, int32_t bwd_pixels, int32_t bwd_depth) {
    const CompositeVariant f{fwd_pixels, fwd_depth}, b{bwd_pixels, bwd_depth};
    if (!ctx || !valid_variant(f, ctx->tile) || !valid_variant(b, ctx->tile)) return PGS_ERR_INVALID_ARG;
    ctx->variant = f;
    ctx->variant_bwd = b;
    return PGS_OK;
}

int pgs_time_variants_split(pgs_ctx* ctx, float* image, const float* dL_dimage, int32_t reps, float* ms_fwd,
                            float* ms_bwd) {
    if (!ctx || !image || !dL_dimage || !ms_fwd || !ms_bwd || reps < 1) return PGS_ERR_INVALID_ARG;
    if (!ctx->has_render) return PGS_ERR_NO_RENDER;
    cudaStream_t s = ctx->stream;
    cudaEvent_t ev[3];
    for (auto& e : ev) cudaEventCreate(&e);
    const int P[3] = {1, 2, 4}, D[3] = {64, 128, 256};
    int idx = 0;
    cudaError_t err = cudaSuccess;
    for (int pi = 0; pi < 3 && err == cudaSuccess; ++pi)
        for (int di = 0; di < 3 && err == cudaSuccess; ++di, ++idx) {
            const CompositeVariant v{P[pi], D[di]};
            if (!valid_variant(v, ctx->tile)) {  // no such strip for this tile edge
                ms_fwd[idx] = ms_bwd[idx] = -1.0f;
                continue;
            }
            float bf = 1e30f, bb = 1e30f;
            for (int rep = 0; rep < reps + 1; ++rep) {
                cudaEventRecord(ev[0], s);
                launch_composite_fwd(ctx->cam, ctx->TX, ctx->TY, ctx->tile, ctx->buf, ctx->n, ctx->sc, image, s, v);
                cudaEventRecord(ev[1], s);
                launch_composite_bwd(ctx->cam, ctx->TX, ctx->TY, ctx->tile, ctx->buf, ctx->n, ctx->sc, dL_dimage, s, v);
                cudaEventRecord(ev[2], s);
                err = cudaEventSynchronize(ev[2]);
                if (err != cudaSuccess) break;
                float tf = 0.f, tb = 0.f;
                cudaEventElapsedTime(&tf, ev[0], ev[1]);
                cudaEventElapsedTime(&tb, ev[1], ev[2]);
                if (rep > 0) {
                    bf = tf < bf ? tf : bf;
                    bb = tb < bb ? tb : bb;
                }
            }
            ms_fwd[idx] = bf;
            ms_bwd[idx] = bb;
        }
    for (auto& e : ev) cudaEventDestroy(e);
    // the timing overwrote the screen-space gradients: the next backward clears and recomputes them
    ctx->grad_clean = false;
    return err == cudaSuccess ? PGS_OK : cuda_err(err);
}

int pgs_time_variants(pgs_ctx* ctx, float* image, const float* dL_dimage, int32_t reps, float* ms) {
    if (!ctx || !image || !dL_dimage || !ms || reps < 1) return PGS_ERR_INVALID_ARG;
    if (!ctx->has_render) return PGS_ERR_NO_RENDER;
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int P[3] = {1, 2, 4}, D[3] = {64, 128, 256};
    int idx = 0;
    cudaError_t err = cudaSuccess;
    for (int pi = 0; pi < 3; ++pi)
        for (int di = 0; di < 3; ++di, ++idx) {
            const CompositeVariant v{P[pi], D[di]};
            if (!valid_variant(v, ctx->tile)) {  // no such strip for this tile edge
                ms[idx] = -1.0f;
                continue;
            }
            float best = 1e30f;
            for (int rep = 0; rep < reps + 1; ++rep) {
                cudaEventRecord(e0, s);
                launch_composite_fwd(ctx->cam, ctx->TX, ctx->TY, ctx->tile, ctx->buf, ctx->n, ctx->sc, image, s, v);
                launch_composite_bwd(ctx->cam, ctx->TX, ctx->TY, ctx->tile, ctx->buf, ctx->n, ctx->sc, dL_dimage, s, v);
                cudaEventRecord(e1, s);
                err = cudaEventSynchronize(e1);
                if (err != cudaSuccess) break;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < best) best = t;
            }
            ms[idx] = best;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timing overwrote the screen-space gradients: the next backward clears and recomputes them
    ctx->grad_clean = false;
    return err == cudaSuccess ? PGS_OK : cuda_err(err);
}

int pgs_read_buffer(pgs_ctx* ctx, int which, void* dst, int64_t max_bytes, int64_t* bytes) {
    if (!ctx || max_bytes < 0) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = ctx->stream;
    unsigned long long P = 0;
    cudaError_t e = cudaMemcpyAsync(&P, ctx->sc.pair_count, sizeof(P), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    const int64_t kept = (int64_t)P < ctx->cap_pairs ? (int64_t)P : ctx->cap_pairs;
    const int64_t pixels = (int64_t)ctx->cam.width * ctx->cam.height;
    const int64_t tiles = (int64_t)ctx->TX * ctx->TY;
    const void* src = nullptr;
    int64_t size = 0;
    switch (which) {
        case PGS_BUF_KEYS: size = 8 * kept; break;
        case PGS_BUF_VALUES: size = 4 * kept; break;
        case PGS_BUF_RANGES: size = 8 * tiles; break;
        case PGS_BUF_T_FINAL: src = ctx->sc.T_final; size = 4 * pixels; break;
        case PGS_BUF_LAST: src = ctx->sc.last; size = 4 * pixels; break;
        case PGS_BUF_GRAD2D: src = ctx->sc.grad2d; size = 36 * ctx->n; break;
        case PGS_BUF_TILES_TOUCHED: src = ctx->sc.touched; size = 4 * ctx->n; break;
        case PGS_BUF_NCOMP: src = ctx->sc.ncomp; size = 4 * pixels; break;
        default: return PGS_ERR_INVALID_ARG;
    }
    if (!ctx->has_render) return PGS_ERR_NO_RENDER;
    if (bytes) *bytes = size;
    const int64_t cp = size < max_bytes ? size : max_bytes;
    if (cp <= 0 || !dst) return PGS_OK;
    if (src) {
        e = cudaMemcpyAsync(dst, src, (size_t)cp, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? PGS_OK : cuda_err(e);
    }
    // Pair lists, ranges and keys in the order of the stable sort of (tile << 32 | depth bits)
    // pairs: tiles row-major, each tile's list as the render holds it (the render lays the lists
    // out super-tile by super-tile; this read-back only reorders whole lists).
    std::vector<uint2> rng((size_t)tiles);
    std::vector<uint32_t> vals((size_t)kept);
    e = cudaMemcpyAsync(rng.data(), ctx->sc.ranges, sizeof(uint2) * (size_t)tiles, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && kept > 0)
        e = cudaMemcpyAsync(vals.data(), ctx->sc.vals[ctx->buf], 4 * (size_t)kept, cudaMemcpyDeviceToHost, s);
    std::vector<uint32_t> depth;
    if (which == PGS_BUF_KEYS && ctx->n > 0) {
        depth.resize((size_t)ctx->n);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(depth.data(), ctx->sc.depth_bits, 4 * (size_t)ctx->n, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    if (which == PGS_BUF_RANGES) {
        std::vector<uint2> out((size_t)tiles);
        uint32_t at = 0;
        for (int64_t t = 0; t < tiles; ++t) {
            const uint32_t len = rng[t].y - rng[t].x;
            out[t] = len ? make_uint2(at, at + len) : make_uint2(0u, 0u);  // an empty tile reads (0, 0)
            at += len;
        }
        std::memcpy(dst, out.data(), (size_t)cp);
        return PGS_OK;
    }
    std::vector<uint64_t> out;
    out.reserve((size_t)kept);
    for (int64_t t = 0; t < tiles; ++t)
        for (uint32_t k = rng[t].x; k < rng[t].y && (int64_t)k < kept; ++k) {
            const uint32_t g = vals[k];
            if (which == PGS_BUF_VALUES) out.push_back(g);
            else out.push_back(((uint64_t)t << 32) | (g < depth.size() ? depth[g] : 0xffffffffu));
        }
    if (which == PGS_BUF_VALUES) {
        std::vector<uint32_t> v32(out.begin(), out.end());
        std::memcpy(dst, v32.data(), (size_t)std::min<int64_t>(cp, 4 * (int64_t)v32.size()));
    } else {
        std::memcpy(dst, out.data(), (size_t)std::min<int64_t>(cp, 8 * (int64_t)out.size()));
    }
    return PGS_OK;
}

}  // extern "C"

// ================================================================================================
// batch
// ================================================================================================
struct pgs_batch {
    pgs_config cfg;
    cudaStream_t stream = nullptr;
    int S = 0, R = 0, deg = 0;
    std::vector<SceneDesc> scenes;
    std::vector<RenderDesc> renders;
    int64_t items = 0, gauss = 0, tiles = 0, supers = 0, pixels = 0, values = 0, cap_pairs = 0;
    Scratch sc;
    void* arena_g = nullptr;
    void* arena_p = nullptr;
    void* arena_t = nullptr;  // tables, losses, counters
    SceneDesc* d_scenes = nullptr;
    RenderDesc* d_renders = nullptr;
    double* d_losses = nullptr;
    uint32_t* d_work = nullptr;  // forward and backward work counters
    int64_t* d_step = nullptr;
    pgs_gaussians* d_grads = nullptr;  // gradient buffers of pgs_backward_batch, one per scene
    bool rendered = false;             // pgs_render_batch ran since the last parameter change
    int buf = 0;
    CompositeVariant variant = default_variant();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    int64_t launches_per_step = 0;  // kernels in the captured graph
};

namespace {

void drop_graph(pgs_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// the render part of a step: projection .. tile order (returns kernels launched)
int64_t enqueue_render(pgs_batch* b) {
    cudaStream_t s = b->stream;
    int64_t k = 0;
    k += launch_project_fwd_batch(b->d_renders, b->R, b->d_scenes, b->deg, b->items, b->sc, s);
    const uint32_t* perm = nullptr;
    if (b->items > 0) k += launch_depth_sort(b->items, b->sc, s, &perm);
    k += launch_bin_count(b->items, b->supers, b->cap_pairs, perm, b->sc, s);
    k += launch_bin_lists(b->items, 0, 0, b->cfg.tile, b->tiles, b->supers, b->cap_pairs, perm, b->sc, s, &b->buf,
                          b->d_renders, b->R);
    k += launch_tile_order((int)b->tiles, b->sc, s);
    return k;
}

int64_t enqueue_step(pgs_batch* b) {
    cudaStream_t s = b->stream;
    int64_t k = enqueue_render(b);
    cudaMemsetAsync(b->d_work, 0, 2 * sizeof(uint32_t), s);
    k += launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc, b->d_work,
                                false, s, b->variant);
    cudaMemsetAsync(b->d_losses, 0, sizeof(double) * 2 * b->R, s);
    k += launch_loss_batch(b->d_renders, b->R, b->values, b->d_losses, s);
    cudaMemsetAsync(b->sc.grad2d, 0, sizeof(float) * 9 * (size_t)b->items, s);
    k += launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc, b->d_work + 1,
                                true, s, b->variant);
    k += launch_bwd_adam_batch(b->d_renders, b->d_scenes, b->S, b->deg, b->gauss, b->items, b->sc,
                               b->cfg.lr, b->cfg.adam_b1, b->cfg.adam_b2, b->cfg.adam_eps, b->d_step, s);
    k += launch_step_tick(b->d_step, b->sc.status, s);
    return k;
}

}  // namespace

extern "C" {

int pgs_batch_create(pgs_batch** out, const pgs_config* cfg, int32_t n_scenes,
                     const pgs_gaussians* params, const pgs_gaussians* m, const pgs_gaussians* v,
                     int32_t n_renders, const pgs_render_desc* renders, int64_t pair_capacity,
                     void* cuda_stream) {
    if (!out) return PGS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || !valid_tile(cfg->tile) || n_scenes < 1 || n_renders < 1 || !params || !m || !v ||
        !renders || pair_capacity < 0)
        return PGS_ERR_INVALID_ARG;
    const int deg = params[0].sh_degree;
    for (int k = 0; k < n_scenes; ++k) {
        if (!valid_gaussians(&params[k]) || !valid_gaussians(&m[k]) || !valid_gaussians(&v[k]))
            return PGS_ERR_INVALID_ARG;
        if (params[k].sh_degree != deg || m[k].n != params[k].n || v[k].n != params[k].n ||
            m[k].sh_degree != deg || v[k].sh_degree != deg)
            return PGS_ERR_INVALID_ARG;
    }
    for (int r = 0; r < n_renders; ++r) {
        const pgs_render_desc& d = renders[r];
        if (d.scene < 0 || d.scene >= n_scenes || !valid_camera(&d.cam) || !d.image || !d.target ||
            !d.dL_dimage)
            return PGS_ERR_INVALID_ARG;
        if (r > 0 && d.scene < renders[r - 1].scene) return PGS_ERR_INVALID_ARG;  // scene by scene
    }
    pgs_batch* b = new (std::nothrow) pgs_batch();
    if (!b) return PGS_ERR_OOM;
    b->cfg = *cfg;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->S = n_scenes;
    b->R = n_renders;
    b->deg = deg;
    b->scenes.resize(n_scenes);
    for (int k = 0; k < n_scenes; ++k) {
        SceneDesc& sd = b->scenes[k];
        sd.params = params[k];
        sd.m = m[k];
        sd.v = v[k];
        sd.first_render = 0;
        sd.n_renders = 0;
        sd.gauss_base = b->gauss;
        b->gauss += params[k].n;
    }
    b->renders.resize(n_renders);
    for (int r = 0; r < n_renders; ++r) {
        const pgs_render_desc& d = renders[r];
        RenderDesc& rd = b->renders[r];
        std::memset(&rd, 0, sizeof(rd));
        rd.cam = d.cam;
        rd.scene = d.scene;
        rd.tile = cfg->tile;
        rd.TX = (d.cam.width + cfg->tile - 1) / cfg->tile;
        rd.TY = (d.cam.height + cfg->tile - 1) / cfg->tile;
        rd.item_base = b->items;
        rd.n = params[d.scene].n;
        rd.tile_base = b->tiles;
        rd.SX = (rd.TX + kSuperW - 1) / kSuperW;
        rd.super_base = b->supers;
        rd.pixel_base = b->pixels;
        rd.value_base = b->values;
        rd.image = d.image;
        rd.target = d.target;
        rd.dL = d.dL_dimage;
        b->items += rd.n;
        b->tiles += (int64_t)rd.TX * rd.TY;
        b->supers += super_tiles(rd.TX, rd.TY);
        b->pixels += (int64_t)d.cam.width * d.cam.height;
        b->values += 3ll * d.cam.width * d.cam.height;
        SceneDesc& sd = b->scenes[d.scene];
        if (sd.n_renders == 0) sd.first_render = r;
        sd.n_renders++;
    }
    auto fail = [&](int rc) {
        pgs_batch_destroy(b);
        return rc;
    };
    if (b->items >= (int64_t(1) << 32) || b->tiles >= (int64_t(1) << 32)) return fail(PGS_ERR_INVALID_ARG);
    // arenas
    Scratch tmp;
    const size_t gbytes = carve_g(tmp, nullptr, b->items, b->pixels, b->tiles, b->supers);
    cudaError_t e = cudaMalloc(&b->arena_g, gbytes);
    if (e != cudaSuccess) return fail(cuda_err(e));
    carve_g(b->sc, static_cast<char*>(b->arena_g), b->items, b->pixels, b->tiles, b->supers);
    const size_t tbytes = align256(sizeof(SceneDesc) * n_scenes) + align256(sizeof(RenderDesc) * n_renders) +
                          align256(sizeof(double) * 2 * n_renders) + 256 + 256 +
                          align256(sizeof(pgs_gaussians) * n_scenes);
    e = cudaMalloc(&b->arena_t, tbytes);
    if (e != cudaSuccess) return fail(cuda_err(e));
    {
        Carver c{static_cast<char*>(b->arena_t)};
        b->d_scenes = c.take<SceneDesc>(n_scenes);
        b->d_renders = c.take<RenderDesc>(n_renders);
        b->d_losses = c.take<double>(2 * n_renders);
        b->d_work = c.take<uint32_t>(2);
        b->d_step = c.take<int64_t>(1);
        b->d_grads = c.take<pgs_gaussians>(n_scenes);
    }
    cudaStream_t s = b->stream;
    e = cudaMemsetAsync(b->arena_g, 0, gbytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena_t, 0, tbytes, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_scenes, b->scenes.data(), sizeof(SceneDesc) * n_scenes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_renders, b->renders.data(), sizeof(RenderDesc) * n_renders, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_err(e));
    // pair capacity: measured on the parameters as given when not specified
    int64_t cap = pair_capacity;
    if (cap == 0) {
        launch_project_fwd_batch(b->d_renders, b->R, b->d_scenes, b->deg, b->items, b->sc, s);
        const uint32_t* perm = nullptr;
        launch_depth_sort(b->items, b->sc, s, &perm);
        launch_bin_count(b->items, b->supers, 0, perm, b->sc, s);
        unsigned long long P = 0;
        int32_t zero = 0;
        e = cudaMemcpyAsync(&P, b->sc.pair_need, sizeof(P), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->sc.status, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(cuda_err(e));
        cap = (int64_t)(P + P / 4 + 4096);
    }
    const size_t pbytes = carve_p(tmp, nullptr, cap);
    e = cudaMalloc(&b->arena_p, pbytes);
    if (e != cudaSuccess) return fail(cuda_err(e));
    carve_p(b->sc, static_cast<char*>(b->arena_p), cap);
    b->cap_pairs = cap;
    *out = b;
    return PGS_OK;
}

void pgs_batch_destroy(pgs_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->arena_g) cudaFree(b->arena_g);
    if (b->arena_p) cudaFree(b->arena_p);
    if (b->arena_t) cudaFree(b->arena_t);
    delete b;
}

int pgs_render_batch(pgs_batch* b) {
    if (!b) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = b->stream;
    b->launches += enqueue_render(b);
    cudaMemsetAsync(b->d_work, 0, sizeof(uint32_t), s);
    b->launches += launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc,
                                          b->d_work, false, s, b->variant);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e);
    b->rendered = true;
    return PGS_OK;
}

int pgs_backward_batch(pgs_batch* b, const pgs_gaussians* grads) {
    if (!b || !grads) return PGS_ERR_INVALID_ARG;
    for (int k = 0; k < b->S; ++k) {
        const pgs_gaussians& p = b->scenes[k].params;
        if (!valid_gaussians(&grads[k]) || grads[k].n != p.n || grads[k].sh_degree != p.sh_degree)
            return PGS_ERR_INVALID_ARG;
    }
    if (!b->rendered) return PGS_ERR_NO_RENDER;
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemcpyAsync(b->d_grads, grads, sizeof(pgs_gaussians) * b->S, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->sc.grad2d, 0, sizeof(float) * 9 * (size_t)b->items, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_work + 1, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_err(e);
    b->launches += launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc,
                                          b->d_work + 1, true, s, b->variant);
    b->launches += launch_bwd_batch(b->d_renders, b->d_scenes, b->S, b->deg, b->gauss, b->items, b->sc, b->d_grads, s);
    return cuda_err(cudaGetLastError());
}

int pgs_batch_step(pgs_batch* b) {
    if (!b) return PGS_ERR_INVALID_ARG;
    b->rendered = false;  // the step changes the parameters
    if (b->exec) {
        const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return cuda_err(e);
        b->launches += b->launches_per_step;
        return PGS_OK;
    }
    b->launches += enqueue_step(b);
    return cuda_err(cudaGetLastError());
}

int pgs_batch_set_views(pgs_batch* b, const pgs_camera* cameras, const float* const* targets) {
    if (!b || !cameras || !targets) return PGS_ERR_INVALID_ARG;
    for (int r = 0; r < b->R; ++r) {
        const RenderDesc& rd = b->renders[r];
        if (!valid_camera(&cameras[r]) || cameras[r].width != rd.cam.width ||
            cameras[r].height != rd.cam.height || !targets[r])
            return PGS_ERR_INVALID_ARG;
    }
    for (int r = 0; r < b->R; ++r) {
        b->renders[r].cam = cameras[r];
        b->renders[r].target = targets[r];
    }
    const cudaError_t e = cudaMemcpyAsync(b->d_renders, b->renders.data(), sizeof(RenderDesc) * b->R,
                                          cudaMemcpyHostToDevice, b->stream);
    return cuda_err(e);
}

int pgs_batch_capture(pgs_batch* b) {
    if (!b) return PGS_ERR_INVALID_ARG;
    drop_graph(b);
    // relaxed: one-time launch-configuration queries of the kernels may run during the capture
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaGetLastError();  // do not leave the failure for an unrelated later check
        return cuda_err(e);
    }
    b->launches_per_step = enqueue_step(b);
    e = cudaStreamEndCapture(b->stream, &b->graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        return cuda_err(e);
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        drop_graph(b);
        return cuda_err(e);
    }
    return PGS_OK;
}

int pgs_batch_reserve(pgs_batch* b, int64_t pair_capacity) {
    if (!b || pair_capacity < 0) return PGS_ERR_INVALID_ARG;
    if (pair_capacity <= b->cap_pairs) return PGS_OK;
    const bool recapture = b->exec != nullptr;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e);
    drop_graph(b);  // the graph holds the old pair buffers
    Scratch tmp;
    const size_t bytes = carve_p(tmp, nullptr, pair_capacity);
    if (b->arena_p) cudaFree(b->arena_p);
    b->arena_p = nullptr;
    b->cap_pairs = 0;
    e = cudaMalloc(&b->arena_p, bytes);
    if (e != cudaSuccess) {
        b->arena_p = nullptr;
        return cuda_err(e);
    }
    carve_p(b->sc, static_cast<char*>(b->arena_p), pair_capacity);
    b->cap_pairs = pair_capacity;
    return recapture ? pgs_batch_capture(b) : PGS_OK;
}

int pgs_batch_steps(pgs_batch* b, int64_t* steps) {
    if (!b || !steps) return PGS_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(steps, b->d_step, sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return cuda_err(e);
}

int pgs_batch_losses(pgs_batch* b, double* losses) {
    if (!b || !losses) return PGS_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(losses, b->d_losses, sizeof(double) * 2 * b->R, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e);
    for (int r = 0; r < b->R; ++r)
        losses[2 * r] /= 3.0 * b->renders[r].cam.width * b->renders[r].cam.height;
    return PGS_OK;
}

int pgs_batch_status(pgs_batch* b, int64_t* pairs) {
    if (!b) return PGS_ERR_INVALID_ARG;
    int32_t st = 0;
    unsigned long long P = 0;
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemcpyAsync(&st, b->sc.status, sizeof(st), cudaMemcpyDeviceToHost, s);
    unsigned long long need = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&P, b->sc.pair_count, sizeof(P), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&need, b->sc.pair_need, sizeof(need), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->sc.status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    if (st & kStatusCapacity) P = need;  // the capacity to grow to (the pairs, or more for the coarse stage)
    if (pairs) *pairs = (int64_t)P;
    if (st & kStatusInternal) return PGS_ERR_INTERNAL;
    if (st & kStatusTimeout) return PGS_ERR_TIMEOUT;
    if (st & kStatusCapacity) return PGS_ERR_CAPACITY;
    if (st & kStatusNonfinite) return PGS_ERR_NONFINITE;
    return PGS_OK;
}

int64_t pgs_batch_launch_count(const pgs_batch* b) { return b ? b->launches : 0; }

int pgs_batch_set_variant(pgs_batch* b, int32_t pixels_per_thread, int32_t depth) {
    const CompositeVariant v{pixels_per_thread, depth};
    if (!b || !valid_variant(v, b->cfg.tile)) return PGS_ERR_INVALID_ARG;
    if (v.pix != b->variant.pix || v.depth != b->variant.depth) drop_graph(b);
    b->variant = v;
    return PGS_OK;
}

int pgs_batch_time_render(pgs_batch* b, int32_t reps, float* ms) {
    if (!b || !ms || reps < 1) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = b->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < reps + 1; ++rep) {  // first repetition warms up
        cudaEventRecord(e0, s);
        enqueue_render(b);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return err == cudaSuccess ? PGS_OK : cuda_err(err);
}

int pgs_batch_time_variants(pgs_batch* b, int32_t reps, float* ms) {
    if (!b || !ms || reps < 1) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = b->stream;
    enqueue_render(b);
    // a render's forward composite also writes the images the loss needs: run one of each
    cudaMemsetAsync(b->d_work, 0, 2 * sizeof(uint32_t), s);
    launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc, b->d_work, false, s, b->variant);
    cudaMemsetAsync(b->d_losses, 0, sizeof(double) * 2 * b->R, s);
    launch_loss_batch(b->d_renders, b->R, b->values, b->d_losses, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int P[3] = {1, 2, 4}, D[3] = {64, 128, 256};
    int idx = 0;
    cudaError_t err = cudaSuccess;
    for (int pi = 0; pi < 3; ++pi)
        for (int di = 0; di < 3; ++di, ++idx) {
            const CompositeVariant v{P[pi], D[di]};
            if (!valid_variant(v, b->cfg.tile)) {  // no such strip for this tile edge
                ms[idx] = -1.0f;
                continue;
            }
            float best = 1e30f;
            for (int rep = 0; rep < reps + 1; ++rep) {  // first repetition warms up
                cudaEventRecord(e0, s);
                cudaMemsetAsync(b->d_work, 0, 2 * sizeof(uint32_t), s);
                launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc, b->d_work, false, s, v);
                cudaMemsetAsync(b->sc.grad2d, 0, sizeof(float) * 9 * (size_t)b->items, s);
                launch_composite_batch(b->d_renders, b->R, b->tiles, b->cfg.tile, b->buf, b->items, b->sc, b->d_work + 1, true, s, v);
                cudaEventRecord(e1, s);
                err = cudaEventSynchronize(e1);
                if (err != cudaSuccess) break;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < best) best = t;
            }
            ms[idx] = best;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err == cudaSuccess ? PGS_OK : cuda_err(err);
}

}  // extern "C"

// ================================================================================================
// initializer
// ================================================================================================
struct pgs_init {
    cudaStream_t stream = nullptr;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int* bbox = nullptr;
};

extern "C" {

int pgs_init_create(pgs_init** out, void* cuda_stream) {
    if (!out) return PGS_ERR_INVALID_ARG;
    *out = nullptr;
    pgs_init* c = new (std::nothrow) pgs_init();
    if (!c) return PGS_ERR_OOM;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e = cudaMalloc(&c->bbox, 6 * sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return cuda_err(e);
    }
    *out = c;
    return PGS_OK;
}

void pgs_init_destroy(pgs_init* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->scratch) cudaFree(c->scratch);
    if (c->bbox) cudaFree(c->bbox);
    delete c;
}

int pgs_knn(pgs_init* c, const float* points, int64_t n, int32_t k, int32_t* nb) {
    if (!c || !points || !nb || n < 0 || n >= (int64_t(1) << 31) || (k != 3 && k != 16 && k != 32))
        return PGS_ERR_INVALID_ARG;
    if (n == 0) return PGS_OK;
    cudaStream_t s = c->stream;
    launch_bbox(n, points, c->bbox, s);
    int enc[6];
    cudaError_t e = cudaMemcpyAsync(enc, c->bbox, sizeof(enc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    float bb[6];
    decode_bbox(enc, bb);
    // scratch for up to 4 cells per point (the grid coarsens to fit)
    const size_t want = knn_scratch_bytes(n, 4 * n + 1024);
    if (c->scratch_bytes < want) {
        e = cudaStreamSynchronize(s);
        if (c->scratch) cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
        e = cudaMalloc(&c->scratch, want);
        if (e != cudaSuccess) return cuda_err(e);
        c->scratch_bytes = want;
    }
    launch_knn(n, points, k, nb, c->scratch, c->scratch_bytes, bb, s);
    return cuda_err(cudaGetLastError());
}

int pgs_features_init(pgs_init* c, const float* points, int64_t n, const int32_t* nb32, float r_normal,
                      float* features, void* features_bf16, float* frame_q, pgs_gaussians* init) {
    if (!c || !points || !nb32 || !features || !features_bf16 || !frame_q || !valid_gaussians(init) ||
        init->n != n || n < 33)
        return PGS_ERR_INVALID_ARG;
    launch_features_init(n, points, nb32, r_normal, features, features_bf16, frame_q, *init, c->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_mlp_param_count(void) { return mlp_param_count(); }

int pgs_mlp_pack(pgs_init* c, const pgs_mlp* w) {
    if (!c || !w || !w->master || !w->W1 || !w->W2 || !w->W3) return PGS_ERR_INVALID_ARG;
    launch_mlp_pack(w->master, w->W1, w->W2, w->W3, c->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_mlp_forward(pgs_init* c, const pgs_mlp* w, const void* x, int64_t n, float* out) {
    if (!c || !w || !w->master || !x || !out || n < 0) return PGS_ERR_INVALID_ARG;
    launch_mlp_forward(x, n, w->master, w->W1, w->W2, w->W3, out, c->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_mlp_grad(pgs_init* c, const pgs_mlp* w, const void* x, const float* targets, int64_t n,
                 float* grad, double* loss_sum) {
    if (!c || !w || !w->master || !x || !targets || !grad || !loss_sum || n < 0) return PGS_ERR_INVALID_ARG;
    launch_mlp_train(x, targets, n, w->master, w->W1, w->W2, w->W3, grad, loss_sum, c->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_mlp_adam(pgs_init* c, pgs_mlp* w, float* grad, float* m, float* v, float lr, int64_t t) {
    if (!c || !w || !w->master || !grad || !m || !v || t < 1) return PGS_ERR_INVALID_ARG;
    launch_mlp_adam(w->master, grad, m, v, lr, 0.9f, 0.999f, 1e-8f, t, w->W1, w->W2, w->W3, c->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_apply_mlp(pgs_init* c, const float* y, const pgs_gaussians* pca, pgs_gaussians* out,
                  uint32_t* fallbacks) {
    if (!c || !y || !valid_gaussians(pca) || !valid_gaussians(out) || !fallbacks || pca->n != out->n)
        return PGS_ERR_INVALID_ARG;
    launch_apply_mlp(out->n, y, *pca, *out, fallbacks, c->stream);
    return cuda_err(cudaGetLastError());
}

int pgs_make_targets(pgs_init* c, const pgs_gaussians* pca, const pgs_gaussians* conv, float* t) {
    if (!c || !valid_gaussians(pca) || !valid_gaussians(conv) || !t || pca->n != conv->n)
        return PGS_ERR_INVALID_ARG;
    launch_make_targets(conv->n, *pca, *conv, t, c->stream);
    return cuda_err(cudaGetLastError());
}

}  // extern "C"
