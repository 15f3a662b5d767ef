// C ABI of the single-reference MVS (kernels in mvs.cu, contract in include/pocketgs.h).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pgs_internal.cuh"

using namespace pgs;

struct pgs_mvs {
    cudaStream_t stream = nullptr;
    int W = 0, H = 0, D = 0;
    void* arena = nullptr;
    uint64_t *cen_t = nullptr, *cen_r = nullptr;
    float* maps = nullptr;
    uint8_t* C = nullptr;
    uint8_t* L = nullptr;  // [4][H][W][D], one SGM path each
    uint16_t* S = nullptr;
    uint8_t* kept = nullptr;
    unsigned long long* count = nullptr;  // [0] kept pixels, [1] sparse depths
    double* range = nullptr;              // d_min, d_max, median
    int* status = nullptr;                // [0] no sparse point visible, [1] reference index
    void* cams = nullptr;                 // 1024 packed cameras
    double* scores = nullptr;             // 1024
    uint32_t* cta = nullptr;
    int64_t* total = nullptr;
    double* zbuf = nullptr;  // sparse depths, grown on demand
    int64_t zcap = 0;
};

namespace {

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

int err(cudaError_t e) {
    if (e == cudaSuccess) return PGS_OK;
    return e == cudaErrorMemoryAllocation ? PGS_ERR_OOM : PGS_ERR_CUDA;
}

bool same_size(const pgs_mvs* m, const pgs_camera* c) { return c && c->width == m->W && c->height == m->H; }

bool finite_camera(const pgs_camera* c) {
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !std::isfinite(c->cx) || !std::isfinite(c->cy)) return false;
    for (float v : c->viewmat)
        if (!std::isfinite(v)) return false;
    return true;
}

}  // namespace

extern "C" {

int pgs_mvs_create(pgs_mvs** out, int32_t width, int32_t height, int32_t planes, void* cuda_stream) {
    if (!out) return PGS_ERR_INVALID_ARG;
    *out = nullptr;
    if (width < 1 || height < 1 || (int64_t)width * height > (int64_t(1) << 28) || planes < 3 || planes > 128)
        return PGS_ERR_INVALID_ARG;
    pgs_mvs* m = new (std::nothrow) pgs_mvs();
    if (!m) return PGS_ERR_OOM;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    m->W = width;
    m->H = height;
    m->D = planes;
    const size_t px = (size_t)width * height, D = planes;
    const size_t sizes[] = {8 * px, 8 * px, 4 * 9 * D, px * D, 4 * px * D, 2 * px * D, px, 16, 24, 8,
                            1024 * mvs_camf_bytes(), 8 * 1024, 4 * (size_t)mvs_fuse_ctas(width, height), 8};
    void** slots[] = {(void**)&m->cen_t, (void**)&m->cen_r, (void**)&m->maps, (void**)&m->C, (void**)&m->L, (void**)&m->S,
                      (void**)&m->kept, (void**)&m->count, (void**)&m->range, (void**)&m->status, &m->cams,
                      (void**)&m->scores, (void**)&m->cta, (void**)&m->total};
    constexpr int kSlots = sizeof(sizes) / sizeof(sizes[0]);
    static_assert(kSlots == sizeof(slots) / sizeof(slots[0]), "one size per buffer");
    size_t total = 0;
    for (size_t z : sizes) total += a256(z);
    cudaError_t e = cudaMalloc(&m->arena, total);
    if (e != cudaSuccess) {
        delete m;
        return err(e);
    }
    char* p = static_cast<char*>(m->arena);
    for (int k = 0; k < kSlots; ++k) {
        *slots[k] = p;
        p += a256(sizes[k]);
    }
    e = cudaMemsetAsync(m->arena, 0, total, m->stream);
    if (e != cudaSuccess) {
        cudaFree(m->arena);
        delete m;
        return err(e);
    }
    *out = m;
    return PGS_OK;
}

void pgs_mvs_destroy(pgs_mvs* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    if (m->zbuf) cudaFree(m->zbuf);
    if (m->arena) cudaFree(m->arena);
    delete m;
}

int pgs_mvs_depth_range(pgs_mvs* m, const pgs_camera* target, const float* points, int64_t n, double* out) {
    if (!m || !same_size(m, target) || !finite_camera(target) || (!points && n > 0) || n < 0 || !out)
        return PGS_ERR_INVALID_ARG;
    if (n > m->zcap) {
        cudaStreamSynchronize(m->stream);
        if (m->zbuf) cudaFree(m->zbuf);
        m->zbuf = nullptr;
        m->zcap = 0;
        cudaError_t e = cudaMalloc(&m->zbuf, sizeof(double) * n);
        if (e != cudaSuccess) return err(e);
        m->zcap = n;
    }
    cudaMemsetAsync(m->status, 0, sizeof(int), m->stream);
    launch_mvs_range(points, n, *target, m->zbuf, m->count + 1, m->range, m->status, m->stream);
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(out, m->range, 3 * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return err(e);
    return st ? PGS_ERR_INVALID_ARG : PGS_OK;
}

int pgs_mvs_select_reference(pgs_mvs* m, const pgs_camera* cams, int32_t count, int32_t target,
                             double median_depth, double* scores, int32_t* ref) {
    if (!m || !cams || count < 2 || count > 1024 || target < 0 || target >= count || !ref || !(median_depth > 0.0))
        return PGS_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!finite_camera(&cams[i])) return PGS_ERR_INVALID_ARG;
    std::vector<char> packed(mvs_camf_bytes() * count);
    mvs_pack_cameras(cams, count, packed.data());
    cudaError_t e = cudaMemcpyAsync(m->cams, packed.data(), packed.size(), cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return err(e);
    launch_mvs_reference(m->cams, count, target, median_depth, m->scores, m->status + 1, m->stream);
    int best = -1;
    e = cudaMemcpyAsync(&best, m->status + 1, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess && scores)
        e = cudaMemcpyAsync(scores, m->scores, sizeof(double) * count, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return err(e);
    *ref = best;
    return PGS_OK;
}

int pgs_mvs_depth(pgs_mvs* m, const pgs_camera* target, const pgs_camera* reference, const float* image_t,
                  const float* image_r, double d_min, double d_max, float* depth, int64_t* kept) {
    if (!m || !same_size(m, target) || !same_size(m, reference) || !finite_camera(target) ||
        !finite_camera(reference) || !image_t || !image_r || !depth || !(d_min > 0.0) || !(d_max > d_min) ||
        !std::isfinite(d_max))
        return PGS_ERR_INVALID_ARG;
    cudaStream_t s = m->stream;
    const double inv_far = 1.0 / d_max;
    const double step = (1.0 / d_min - inv_far) / (m->D - 1);
    launch_mvs_census(image_t, m->W, m->H, m->cen_t, s);
    launch_mvs_census(image_r, m->W, m->H, m->cen_r, s);
    launch_mvs_cost(*target, *reference, m->cen_t, m->cen_r, m->W, m->H, m->D, inv_far, step, m->maps, m->C, s);
    launch_mvs_sgm(m->C, m->L, m->W, m->H, m->D, s);
    launch_mvs_select(m->L, m->S, m->W, m->H, m->D, inv_far, step, depth, m->kept, m->count, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(e);
    if (kept) {
        unsigned long long c = 0;
        e = cudaMemcpyAsync(&c, m->count, sizeof(c), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return err(e);
        *kept = (int64_t)c;
    }
    return PGS_OK;
}

int pgs_mvs_stage_times(pgs_mvs* m, const pgs_camera* target, const pgs_camera* reference, const float* image_t,
                        const float* image_r, double d_min, double d_max, float* depth, float* ms) {
    if (!m || !same_size(m, target) || !same_size(m, reference) || !finite_camera(target) ||
        !finite_camera(reference) || !image_t || !image_r || !depth || !ms || !(d_min > 0.0) || !(d_max > d_min) ||
        !std::isfinite(d_max))
        return PGS_ERR_INVALID_ARG;
    cudaStream_t s = m->stream;
    const double inv_far = 1.0 / d_max;
    const double step = (1.0 / d_min - inv_far) / (m->D - 1);
    cudaEvent_t ev[5];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 5; ++made) {
        e = cudaEventCreate(&ev[made]);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) {
        cudaEventRecord(ev[0], s);
        launch_mvs_census(image_t, m->W, m->H, m->cen_t, s);
        launch_mvs_census(image_r, m->W, m->H, m->cen_r, s);
        cudaEventRecord(ev[1], s);
        launch_mvs_cost(*target, *reference, m->cen_t, m->cen_r, m->W, m->H, m->D, inv_far, step, m->maps, m->C, s);
        cudaEventRecord(ev[2], s);
        launch_mvs_sgm(m->C, m->L, m->W, m->H, m->D, s);
        cudaEventRecord(ev[3], s);
        launch_mvs_select(m->L, m->S, m->W, m->H, m->D, inv_far, step, depth, m->kept, m->count, s);
        cudaEventRecord(ev[4], s);
        e = cudaEventSynchronize(ev[4]);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    return err(e);
}

int pgs_mvs_read(pgs_mvs* m, int32_t what, void* dst, int64_t bytes) {
    if (!m || !dst) return PGS_ERR_INVALID_ARG;
    const size_t px = (size_t)m->W * m->H;
    const void* src = nullptr;
    size_t need = 0;
    switch (what) {
        case PGS_MVS_CENSUS_TARGET: src = m->cen_t; need = 8 * px; break;
        case PGS_MVS_CENSUS_REFERENCE: src = m->cen_r; need = 8 * px; break;
        case PGS_MVS_COST: src = m->C; need = px * m->D; break;
        case PGS_MVS_AGGREGATED: src = m->S; need = 2 * px * m->D; break;
        case PGS_MVS_PLANE_MAPS: src = m->maps; need = 36 * (size_t)m->D; break;
        default: return PGS_ERR_INVALID_ARG;
    }
    if (bytes < (int64_t)need) return PGS_ERR_INVALID_ARG;
    return err(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, m->stream));
}

int pgs_mvs_fuse(pgs_mvs* m, const pgs_camera* target, const float* depth, float* points, int32_t* pixels,
                 int64_t capacity, int64_t* count) {
    if (!m || !same_size(m, target) || !finite_camera(target) || !depth || capacity < 0 ||
        (capacity > 0 && (!points || !pixels)) || !count)
        return PGS_ERR_INVALID_ARG;
    launch_mvs_fuse(depth, m->W, m->H, *target, m->cta, m->total, capacity, points, pixels, m->stream);
    int64_t n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, m->total, sizeof(n), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return err(e);
    *count = n;
    return n > capacity ? PGS_ERR_CAPACITY : PGS_OK;
}

}  // extern "C"
