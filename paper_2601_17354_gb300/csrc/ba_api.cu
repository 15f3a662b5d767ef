// C ABI of the bundle adjustment (kernels in ba.cu, contract in include/pocketgs.h).
#include <cmath>
#include <new>

#include "pgs_internal.cuh"

using namespace pgs;

struct pgs_ba {
    cudaStream_t stream = nullptr;
    BaShape sh;
    int64_t m = 0;
    void* arena = nullptr;
    int64_t* start = nullptr;
    uint32_t* mask = nullptr;
    int64_t *cam_count = nullptr, *cam_start = nullptr, *cam_obs = nullptr;
    float *Htp = nullptr, *E = nullptr;
    double *Hpp = nullptr, *bp = nullptr, *Hinv = nullptr, *y = nullptr;
    double *camp = nullptr, *schp = nullptr, *rhsp = nullptr, *Sfull = nullptr, *rhs = nullptr, *dc = nullptr,
           *cost = nullptr;
    float* Aglob = nullptr;
    float *Rn = nullptr, *tn = nullptr, *Pn = nullptr;
    int* status = nullptr;  // [0] reduced system not positive definite, [1] index check
};

namespace {

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

int err(cudaError_t e) {
    if (e == cudaSuccess) return PGS_OK;
    return e == cudaErrorMemoryAllocation ? PGS_ERR_OOM : PGS_ERR_CUDA;
}

// the fixed translation component of camera 1: largest component of its baseline to camera 0 in
// its own frame (centres c = -R^T t), from host copies of the first two cameras
int gauge_axis(const float* R, const float* t) {
    double c[2][3];
    for (int i = 0; i < 2; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            for (int q = 0; q < 3; ++q) v -= (double)R[9 * i + 3 * q + a] * t[3 * i + q];
            c[i][a] = v;
        }
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        for (int q = 0; q < 3; ++q) v += (double)R[9 + 3 * a + q] * (c[1][q] - c[0][q]);
        if (fabs(v) > bv) {
            bv = fabs(v);
            best = a;
        }
    }
    return best;
}

bool valid(const pgs_ba* b, const float* R, const float* t, const float* P, const int32_t* cam, const int32_t* pt,
           const float* uv, const float* K, float sigma, float delta) {
    return b && R && t && P && cam && pt && uv && K && sigma > 0.f && delta > 0.f;
}

// index check, status reset, gauge axis, point offsets and camera masks; one synchronisation
int begin(pgs_ba* b, const float* R, const float* t, const int32_t* cam, const int32_t* pt, int* axis) {
    cudaStream_t s = b->stream;
    cudaMemsetAsync(b->status, 0, sizeof(int), s);
    launch_ba_check(b->m, b->sh.n, b->sh.C, cam, pt, b->status + 1, s);
    float host[24];
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(host, R, sizeof(float) * 18, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host + 18, t, sizeof(float) * 6, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, b->status + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(e);
    if (flag) return PGS_ERR_INVALID_ARG;
    *axis = gauge_axis(host, host + 18);
    launch_ba_index(b->sh, pt, cam, b->start, b->mask, b->cam_count, b->cam_start, b->cam_obs, s);
    return err(cudaGetLastError());
}

int linearize(pgs_ba* b, const float* R, const float* t, const float* P, const int32_t* cam, const int32_t* pt,
              const float* uv, const float* K, float sigma, float delta, cudaEvent_t* ev = nullptr) {
    launch_ba_linearize(b->sh, R, t, P, cam, pt, uv, b->start, b->cam_start, b->cam_obs, K, sigma, delta, b->Htp,
                        b->Hpp, b->bp, b->camp, b->cost, b->stream, ev);
    return err(cudaGetLastError());
}

void trial(pgs_ba* b, const float* R, const float* t, const float* P, const int32_t* cam, const int32_t* pt, double lam,
           int axis, float* dcam, float* dP, cudaEvent_t* ev = nullptr) {
    launch_ba_trial(b->sh, pt, b->start, b->mask, b->cam_start, b->cam_obs, cam, b->Htp, b->Hpp, b->bp, b->camp, lam,
                    axis, b->Hinv, b->y, b->E, b->schp, b->rhsp, b->Sfull, b->rhs, b->Aglob, b->dc, R, t, P, b->Rn, b->tn, b->Pn, dcam,
                    dP, b->status, b->stream, ev);
}

int finish(pgs_ba* b) {
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return err(e);
    return st ? PGS_ERR_NOT_PD : PGS_OK;
}

}  // namespace

extern "C" {

int pgs_ba_create(pgs_ba** out, int32_t n_cams, int64_t n_points, int64_t n_obs, void* cuda_stream) {
    if (!out) return PGS_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_cams < 2 || n_cams > 256 || n_points < 0 || n_obs < 0 || n_points >= (int64_t(1) << 31) ||
        n_obs >= (int64_t(1) << 40))
        return PGS_ERR_INVALID_ARG;
    pgs_ba* b = new (std::nothrow) pgs_ba();
    if (!b) return PGS_ERR_OOM;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->sh = ba_shape(n_cams, n_points, n_obs);
    b->m = n_obs;
    const BaShape& sh = b->sh;
    const size_t C = n_cams, n = n_points, m = n_obs, N = sh.N;
    const size_t packed = sh.solve_smem ? 1 : N * (N + 1) / 2;
    const size_t sizes[] = {8 * (n + 1), 4 * sh.W * n, 8 * C, 8 * (C + 1), 8 * m, 4 * 18 * m, 4 * 18 * m,
                            8 * 6 * n, 8 * 3 * n, 8 * 6 * n, 8 * 3 * n, 8 * 27 * C * sh.chc,
                            8 * 36 * (size_t)sh.pairs * sh.chs, 8 * 6 * C * sh.chs, 8 * N * N, 8 * N, 4 * packed,
                            8 * N, 16, 4 * 9 * C, 4 * 3 * C, 4 * 3 * n, 256};
    void** slots[] = {(void**)&b->start, (void**)&b->mask, (void**)&b->cam_count, (void**)&b->cam_start,
                      (void**)&b->cam_obs, (void**)&b->Htp, (void**)&b->E, (void**)&b->Hpp,
                      (void**)&b->bp, (void**)&b->Hinv, (void**)&b->y, (void**)&b->camp, (void**)&b->schp,
                      (void**)&b->rhsp, (void**)&b->Sfull, (void**)&b->rhs, (void**)&b->Aglob, (void**)&b->dc, (void**)&b->cost, (void**)&b->Rn,
                      (void**)&b->tn, (void**)&b->Pn, (void**)&b->status};
    constexpr int kSlots = sizeof(sizes) / sizeof(sizes[0]);
    static_assert(kSlots == sizeof(slots) / sizeof(slots[0]), "one size per buffer");
    size_t total = 0;
    for (size_t z : sizes) total += a256(z);
    if (ba_configure_solve() != 0) {
        delete b;
        return PGS_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc(&b->arena, total);
    if (e != cudaSuccess) {
        delete b;
        return err(e);
    }
    char* p = static_cast<char*>(b->arena);
    for (int k = 0; k < kSlots; ++k) {
        *slots[k] = p;
        p += a256(sizes[k]);
    }
    e = cudaMemsetAsync(b->arena, 0, total, b->stream);
    if (e != cudaSuccess) {
        cudaFree(b->arena);
        delete b;
        return err(e);
    }
    *out = b;
    return PGS_OK;
}

void pgs_ba_destroy(pgs_ba* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->arena) cudaFree(b->arena);
    delete b;
}

int pgs_ba_project(pgs_ba* b, const float* R, const float* t, const float* P, const int32_t* cam,
                   const int32_t* pt, int64_t count, const float* K, float* uv, float* z) {
    if (!b || !R || !t || !P || !cam || !pt || !K || !uv || !z || count < 0) return PGS_ERR_INVALID_ARG;
    launch_ba_project(count, b->sh.n, b->sh.C, R, t, P, cam, pt, K, uv, z, b->stream);
    return err(cudaGetLastError());
}

int pgs_ba_step(pgs_ba* b, const float* R, const float* t, const float* P, const int32_t* cam, const int32_t* pt,
                const float* uv, const float* K, float sigma, float huber_delta, float lambda, float* dcam,
                float* dP, double* cost) {
    if (!valid(b, R, t, P, cam, pt, uv, K, sigma, huber_delta) || !dcam || !dP || !cost || !(lambda >= 0.f))
        return PGS_ERR_INVALID_ARG;
    int axis = 0;
    int rc = begin(b, R, t, cam, pt, &axis);
    if (rc == PGS_OK) rc = linearize(b, R, t, P, cam, pt, uv, K, sigma, huber_delta);
    if (rc != PGS_OK) return rc;
    trial(b, R, t, P, cam, pt, lambda, axis, dcam, dP);
    cudaError_t e = cudaMemcpyAsync(cost, b->cost, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return err(e);
    return finish(b);
}

int pgs_ba_solve(pgs_ba* b, float* R, float* t, float* P, const int32_t* cam, const int32_t* pt, const float* uv,
                 const float* K, float sigma, float huber_delta, int32_t iters, float lambda0, double* costs,
                 int32_t* accepted) {
    if (!valid(b, R, t, P, cam, pt, uv, K, sigma, huber_delta) || iters < 0 || !(lambda0 > 0.f) || !costs ||
        !accepted)
        return PGS_ERR_INVALID_ARG;
    cudaStream_t s = b->stream;
    int axis = 0;
    int rc = begin(b, R, t, cam, pt, &axis);
    if (rc == PGS_OK) rc = linearize(b, R, t, P, cam, pt, uv, K, sigma, huber_delta);
    if (rc != PGS_OK) return rc;
    double cur = 0.0;
    cudaError_t e = cudaMemcpyAsync(&cur, b->cost, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(e);
    costs[0] = cur;
    double lam = lambda0;
    int acc = 0;
    for (int it = 0; it < iters; ++it) {
        trial(b, R, t, P, cam, pt, lam, axis, nullptr, nullptr);
        launch_ba_cost(b->sh, b->Rn, b->tn, b->Pn, cam, uv, b->start, K, sigma, huber_delta, b->cost + 1, s);
        double cand = 0.0;
        int st = 0;
        e = cudaMemcpyAsync(&cand, b->cost + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return err(e);
        if (st) return PGS_ERR_NOT_PD;
        if (cand < cur) {  // take the candidate and relinearize there
            cudaMemcpyAsync(R, b->Rn, sizeof(float) * 9 * b->sh.C, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(t, b->tn, sizeof(float) * 3 * b->sh.C, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(P, b->Pn, sizeof(float) * 3 * b->sh.n, cudaMemcpyDeviceToDevice, s);
            cur = cand;
            lam /= 10.0;
            ++acc;
            rc = linearize(b, R, t, P, cam, pt, uv, K, sigma, huber_delta);
            if (rc != PGS_OK) return rc;
        } else {
            lam *= 10.0;
        }
        costs[it + 1] = cur;
    }
    *accepted = acc;
    return finish(b);
}

int pgs_ba_stage_times(pgs_ba* b, const float* R, const float* t, const float* P, const int32_t* cam,
                       const int32_t* pt, const float* uv, const float* K, float sigma, float huber_delta,
                       float lambda, float* ms) {
    if (!valid(b, R, t, P, cam, pt, uv, K, sigma, huber_delta) || !ms || !(lambda >= 0.f)) return PGS_ERR_INVALID_ARG;
    cudaStream_t s = b->stream;
    int axis = 0;
    int rc = begin(b, R, t, cam, pt, &axis);
    if (rc != PGS_OK) return rc;
    cudaEvent_t ev[8];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 8; ++made) {
        e = cudaEventCreate(&ev[made]);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) {
        linearize(b, R, t, P, cam, pt, uv, K, sigma, huber_delta, ev);
        trial(b, R, t, P, cam, pt, lambda, axis, nullptr, nullptr, ev + 3);
        launch_ba_cost(b->sh, b->Rn, b->tn, b->Pn, cam, uv, b->start, K, sigma, huber_delta, b->cost + 1, s);
        cudaEventRecord(ev[7], s);
        e = cudaEventSynchronize(ev[7]);
        for (int k = 0; k < 7 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return err(e);
    return finish(b);
}

}  // extern "C"
