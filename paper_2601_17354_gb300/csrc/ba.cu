// Bundle adjustment of the geometry prior (Sec. III-A): Levenberg-Marquardt on the robust
// reprojection objective of Eq. 2, each step solved through the reduced camera system of Eq. 3.
//
//   camera i: world-to-camera R_i (row-major 3 x 3), t_i; point P_j; pinhole (fx, fy, cx, cy);
//   r = pi(R_i P_j + t_i) - p_ij, whitened by sigma; Huber weight w = 1 (e <= delta) or delta / e
//   on the whitened norm e; camera update R <- exp([omega]x) R, t <- t + v; point update P <- P + d;
//   gauge: camera 0 fixed, and camera 1's translation component along the axis of its largest
//   initial baseline component (in its own frame) fixed.
//
// Observations are grouped by point with cameras increasing inside a group; every point carries a
// bit mask of the cameras that see it (the observation of camera a at point j is start[j] + the
// mask bits below a), and every camera a list of its observations in point order.  No kernel adds
// floating point with atomics except the scalar cost; every block of the normal equations has one
// owner:
//   linearize  thread per point: residual (FP64: pixel coordinates ~1e3, residuals ~1), Jacobians
//              (FP32), H_pp and b_p, H_tp of every observation (6 x 3, FP32), robust cost;
//   camblocks  CTA per (camera, chunk of its observations): H_tt block (21) and b_t (6), Jacobians
//              recomputed from the state (cheaper than storing them);
//   points     thread per point, per trial: (H_pp + lam diag)^-1, y = H_pp^-1 b_p and
//              E = H_tp H_pp^-1 per observation (the independent 3 x 3 inverses of Eq. 3);
//   schur      CTA per (camera pair a <= b, chunk of a's observations): sum over the points seen
//              by both of E_a H_tp,b^T (6 x 6) and, for a == b, of H_tp,a y (the reduced rhs);
//   assemble   thread per entry: the damped reduced system from the chunk sums (FP64);
//   solve      one CTA: gauge and unobserved rows fixed, scaled to a unit diagonal (Jacobi; this takes its condition
//              number from ~1e8 to ~1e3 on ring-camera problems, so FP32 factorization keeps a
//              backward error ~1e-8 while GB300's FP64 rate is 1/64 of its FP32 rate), then
//              blocked Cholesky in shared memory (6C <= 224) or, for more cameras, symmetric
//              elimination of the packed upper triangle with the rhs carried along;
//   backsub    thread per point: Delta_p = H_pp^-1 (b_p - sum H_tp^T Delta_t), candidate points;
//   cameras    candidate poses; cost of the candidate.
// The host accepts the candidate when the robust cost drops (lam / 10) or keeps the current state
// and retries with lam * 10 (the linearization is reused).
#include <cmath>

#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int kBaThreads = 256;
constexpr int kPointThreads = 64;  // per-point kernels: ~80 CTAs per 20k points would leave SMs idle
constexpr int kSolveThreads = 1024;
constexpr int kBlockedThreads = 512;  // 128 registers a thread: the 32-float rows stay in registers
constexpr int kMaxN = 6 * 256;
constexpr int kMaxBlockedN = 224;  // (224 x 225) FP32 = 197 KB of shared memory
constexpr size_t kMaxSolveSmem = 200 * 1024;  // + 13 KB static: within the 227 KB a CTA may use

struct Intr {
    float fx, fy, cx, cy;
};

// x = R_i P + t_i in double (the products of FP32 inputs are exact)
__device__ __forceinline__ void cam_point(const float* __restrict__ R, const float* __restrict__ t, int i,
                                          double px, double py, double pz, double X[3]) {
    const float* r = R + 9 * i;
    X[0] = fma((double)r[0], px, fma((double)r[1], py, fma((double)r[2], pz, (double)t[3 * i + 0])));
    X[1] = fma((double)r[3], px, fma((double)r[4], py, fma((double)r[5], pz, (double)t[3 * i + 1])));
    X[2] = fma((double)r[6], px, fma((double)r[7], py, fma((double)r[8], pz, (double)t[3 * i + 2])));
}

// residual (double: the pixel coordinates are ~1e3 and the residuals ~1), IRLS weight over sigma^2
// and robust cost of one observation; false when behind the camera
__device__ __forceinline__ bool residual(const double X[3], Intr K, float u, float v, float sigma, float delta,
                                         double r[2], double& Wm, double& rho) {
    if (!(X[2] > 1e-6)) return false;
    const double iz = 1.0 / X[2];
    r[0] = fma((double)K.fx * X[0], iz, (double)K.cx - u);
    r[1] = fma((double)K.fy * X[1], iz, (double)K.cy - v);
    const double e = sqrt(r[0] * r[0] + r[1] * r[1]) / sigma;
    const double w = e <= delta ? 1.0 : delta / e;
    Wm = w / ((double)sigma * sigma);
    rho = e <= delta ? e * e : 2.0 * delta * e - (double)delta * delta;
    return true;
}

// d pi / d(omega, v) and d pi / dP at camera-frame point X of camera i (FP32: their rounding is
// that of the stored H_tp)
__device__ __forceinline__ void jacobians(const float* __restrict__ R, const float* __restrict__ t, int i,
                                          const double X[3], Intr K, float Jc[2][6], float Jp[2][3]) {
    const float iz = (float)(1.0 / X[2]);
    const float x0 = (float)X[0], x1 = (float)X[1];
    // d pi / dx = [[a0, 0, a2], [0, b1, b2]]
    const float a0 = K.fx * iz, a2 = -K.fx * x0 * iz * iz;
    const float b1 = K.fy * iz, b2 = -K.fy * x1 * iz * iz;
    // q = R P = x - t; d x / d omega = -[q]x = [[0, q2, -q1], [-q2, 0, q0], [q1, -q0, 0]]
    const float q0 = (float)(X[0] - t[3 * i]), q1 = (float)(X[1] - t[3 * i + 1]), q2 = (float)(X[2] - t[3 * i + 2]);
    Jc[0][0] = a2 * q1;
    Jc[0][1] = a0 * q2 - a2 * q0;
    Jc[0][2] = -a0 * q1;
    Jc[0][3] = a0;
    Jc[0][4] = 0.f;
    Jc[0][5] = a2;
    Jc[1][0] = -b1 * q2 + b2 * q1;
    Jc[1][1] = -b2 * q0;
    Jc[1][2] = b1 * q0;
    Jc[1][3] = 0.f;
    Jc[1][4] = b1;
    Jc[1][5] = b2;
    const float* rr = R + 9 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Jp[0][c] = a0 * rr[c] + a2 * rr[6 + c];
        Jp[1][c] = b1 * rr[3 + c] + b2 * rr[6 + c];
    }
}

// observation of camera a at point j (the bit is set); W mask words per point
__device__ __forceinline__ int64_t obs_of(const int64_t* __restrict__ start, const uint32_t* __restrict__ mask,
                                          int W, int64_t j, int a) {
    int64_t o = start[j];
    const uint32_t* mk = mask + (size_t)j * W;
    for (int w = 0; w < (a >> 5); ++w) o += __popc(mk[w]);
    return o + __popc(mk[a >> 5] & ((1u << (a & 31)) - 1u));
}

__device__ __forceinline__ bool sees(const uint32_t* __restrict__ mask, int W, int64_t j, int a) {
    return (mask[(size_t)j * W + (a >> 5)] >> (a & 31)) & 1u;
}

// sum of v over the CTA (kBaThreads) in FP32 (FP64 adds run at 1/64 of the FP32 rate here):
// returns the sum of element t in thread t < kN
template <int kN>
__device__ __forceinline__ float block_sum(float (&v)[kN], float (*s_red)[kN]) {
#pragma unroll
    for (int q = 0; q < kN; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < kN; ++q) s_red[threadIdx.x >> 5][q] = v[q];
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < kN)
        for (int w = 0; w < kBaThreads / 32; ++w) t += s_red[w][threadIdx.x];
    return t;
}

template <int kThreads>
__device__ __forceinline__ void block_add_double(double v, double* s_red, double* dst) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
        atomicAdd(dst, t);
    }
}

// observation indices in range, grouped by point, cameras increasing inside a group; flag 1 otherwise
__global__ void k_ba_check(int64_t m, int64_t n, int C, const int32_t* __restrict__ cam,
                           const int32_t* __restrict__ pt, int* __restrict__ flag) {
    const int64_t o = (int64_t)blockIdx.x * kBaThreads + threadIdx.x;
    if (o >= m) return;
    const int32_t i = cam[o], j = pt[o];
    bool bad = i < 0 || i >= C || j < 0 || j >= n;
    if (o > 0) {
        const int32_t jp = pt[o - 1], ip = cam[o - 1];
        bad = bad || jp > j || (jp == j && ip >= i);
    }
    if (bad) atomicOr(flag, 1);
}

// the lower bound of point j in the point-ordered observations
__global__ void k_ba_offsets(int64_t n, int64_t m, const int32_t* __restrict__ pt, int64_t* __restrict__ start) {
    const int64_t j = (int64_t)blockIdx.x * kBaThreads + threadIdx.x;
    if (j > n) return;
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pt[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    start[j] = lo;
}

__global__ void k_ba_masks(int64_t n, int W, const int64_t* __restrict__ start, const int32_t* __restrict__ cam,
                           uint32_t* __restrict__ mask) {
    const int64_t j = (int64_t)blockIdx.x * kBaThreads + threadIdx.x;
    if (j >= n) return;
    uint32_t* mk = mask + (size_t)j * W;
    for (int w = 0; w < W; ++w) mk[w] = 0u;
    for (int64_t o = start[j]; o < start[j + 1]; ++o) mk[cam[o] >> 5] |= 1u << (cam[o] & 31);
}

__global__ void k_ba_cam_count(int64_t m, const int32_t* __restrict__ cam, int64_t* __restrict__ count) {
    const int64_t o = (int64_t)blockIdx.x * kBaThreads + threadIdx.x;
    if (o < m) atomicAdd(reinterpret_cast<unsigned long long*>(&count[cam[o]]), 1ull);
}

// CTA per camera a: its observations in point order (a stable compaction of the observation list),
// written from cam_start[a] = sum of the counts of cameras before a
__global__ void __launch_bounds__(1024)
k_ba_cam_fill(int64_t m, int C, const int32_t* __restrict__ cam, const int64_t* __restrict__ count,
              int64_t* __restrict__ cam_start, int64_t* __restrict__ cam_obs) {
    __shared__ int s_warp[32];
    __shared__ int64_t s_base;
    const int a = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int64_t b = 0;
        for (int c = 0; c < a; ++c) b += count[c];
        s_base = b;
        cam_start[a] = b;
        if (a == C - 1) cam_start[C] = b + count[a];
    }
    __syncthreads();
    int64_t base = s_base;
    for (int64_t o0 = 0; o0 < m; o0 += 1024) {
        const int64_t o = o0 + threadIdx.x;
        const bool mine = o < m && cam[o] == a;
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 32; ++w) {
            const int c = s_warp[w];
            before += w < warp ? c : 0;
            total += c;
        }
        if (mine) cam_obs[base + before + __popc(bal & ((1u << lane) - 1u))] = o;
        base += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kPointThreads)
k_ba_linearize(int64_t n, const float* __restrict__ R, const float* __restrict__ t, const float* __restrict__ P,
               const int32_t* __restrict__ cam, const float* __restrict__ uv, const int64_t* __restrict__ start,
               Intr K, float sigma, float delta, float* __restrict__ Htp, double* __restrict__ Hpp,
               double* __restrict__ bp, double* __restrict__ cost) {
    __shared__ double s_red[kPointThreads / 32];
    const int64_t j = (int64_t)blockIdx.x * kPointThreads + threadIdx.x;
    double rho_sum = 0.0;
    if (j < n) {
        const double px = P[3 * j], py = P[3 * j + 1], pz = P[3 * j + 2];
        double hp[6] = {0, 0, 0, 0, 0, 0}, gp[3] = {0, 0, 0};
        for (int64_t o = start[j]; o < start[j + 1]; ++o) {
            const int i = cam[o];
            double X[3], r[2], Wm, rho;
            cam_point(R, t, i, px, py, pz, X);
            float* __restrict__ H = Htp + 18 * o;
            if (!residual(X, K, uv[2 * o], uv[2 * o + 1], sigma, delta, r, Wm, rho)) {
                for (int q = 0; q < 18; ++q) H[q] = 0.f;
                continue;
            }
            rho_sum += rho;
            float Jc[2][6], Jp[2][3];
            jacobians(R, t, i, X, K, Jc, Jp);
            const float w = (float)Wm, r0 = (float)r[0], r1 = (float)r[1];
#pragma unroll
            for (int a = 0; a < 6; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) H[3 * a + c] = w * (Jc[0][a] * Jp[0][c] + Jc[1][a] * Jp[1][c]);
            // point block (upper: xx xy xz yy yz zz) and gradient
            int u = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = a; c < 3; ++c) hp[u++] += (double)(w * (Jp[0][a] * Jp[0][c] + Jp[1][a] * Jp[1][c]));
#pragma unroll
            for (int a = 0; a < 3; ++a) gp[a] -= (double)(w * (Jp[0][a] * r0 + Jp[1][a] * r1));
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) Hpp[6 * j + q] = hp[q];
#pragma unroll
        for (int q = 0; q < 3; ++q) bp[3 * j + q] = gp[q];
    }
    block_add_double<kPointThreads>(rho_sum, s_red, cost);
}

// items [q0, q1) of chunk c of `chunks` over `len` items
__device__ __forceinline__ void chunk_of(int64_t len, int c, int chunks, int64_t& q0, int64_t& q1) {
    q0 = len * c / chunks;
    q1 = len * (c + 1) / chunks;
}

// camera a's H_tt block (upper 21) and b_t (6) over one chunk of its observations
__global__ void __launch_bounds__(kBaThreads)
k_ba_camblocks(int C, const float* __restrict__ R, const float* __restrict__ t, const float* __restrict__ P,
               const int32_t* __restrict__ pt, const float* __restrict__ uv, const int64_t* __restrict__ cam_start,
               const int64_t* __restrict__ cam_obs, Intr K, float sigma, float delta, double* __restrict__ camp) {
    __shared__ float s_red[kBaThreads / 32][27];
    const int a = blockIdx.x, c = blockIdx.y;
    int64_t q0, q1;
    chunk_of(cam_start[a + 1] - cam_start[a], c, gridDim.y, q0, q1);
    const int64_t* __restrict__ list = cam_obs + cam_start[a];
    float acc[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) acc[q] = 0.f;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += kBaThreads) {
        const int64_t o = list[q], j = pt[o];
        double X[3], r[2], Wm, rho;
        cam_point(R, t, a, P[3 * j], P[3 * j + 1], P[3 * j + 2], X);
        if (!residual(X, K, uv[2 * o], uv[2 * o + 1], sigma, delta, r, Wm, rho)) continue;
        float Jc[2][6], Jp[2][3];
        jacobians(R, t, a, X, K, Jc, Jp);
        const float w = (float)Wm, r0 = (float)r[0], r1 = (float)r[1];
        int u = 0;
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
            for (int s2 = p; s2 < 6; ++s2) acc[u++] += w * (Jc[0][p] * Jc[0][s2] + Jc[1][p] * Jc[1][s2]);
#pragma unroll
        for (int p = 0; p < 6; ++p) acc[21 + p] -= w * (Jc[0][p] * r0 + Jc[1][p] * r1);
    }
    const float tot = block_sum<27>(acc, s_red);
    if (threadIdx.x < 27) camp[((size_t)c * C + a) * 27 + threadIdx.x] = tot;
}

// (H_pp + lam diag)^-1, y = H^-1 b_p, E = H_tp H^-1 for the point's observations
__global__ void __launch_bounds__(kPointThreads)
k_ba_points(int64_t n, const int64_t* __restrict__ start, const double* __restrict__ Hpp, const double* __restrict__ bp,
            const float* __restrict__ Htp, double lam, double* __restrict__ Hinv, double* __restrict__ y,
            float* __restrict__ E) {
    const int64_t j = (int64_t)blockIdx.x * kPointThreads + threadIdx.x;
    if (j >= n) return;
    const double* h = Hpp + 6 * j;
    const double a = h[0] * (1 + lam), b = h[1], c = h[2], d = h[3] * (1 + lam), e = h[4], f = h[5] * (1 + lam);
    // symmetric [[a b c] [b d e] [c e f]]: inverse by cofactors
    const double A = d * f - e * e, B = c * e - b * f, Cc = b * e - c * d;
    const double det = a * A + b * B + c * Cc;
    double inv[6] = {0, 0, 0, 0, 0, 0};
    if (h[0] > 0.0 && det > 0.0) {  // a point no observation weighs keeps a zero step
        const double id = 1.0 / det;
        inv[0] = A * id;
        inv[1] = B * id;
        inv[2] = Cc * id;
        inv[3] = (a * f - c * c) * id;
        inv[4] = (b * c - a * e) * id;
        inv[5] = (a * d - b * b) * id;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) Hinv[6 * j + q] = inv[q];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int q0 = r == 0 ? 0 : (r == 1 ? 1 : 2), q1 = r == 0 ? 1 : (r == 1 ? 3 : 4), q2 = r == 0 ? 2 : (r == 1 ? 4 : 5);
        y[3 * j + r] = inv[q0] * bp[3 * j] + inv[q1] * bp[3 * j + 1] + inv[q2] * bp[3 * j + 2];
    }
    const float M[3][3] = {{(float)inv[0], (float)inv[1], (float)inv[2]},
                           {(float)inv[1], (float)inv[3], (float)inv[4]},
                           {(float)inv[2], (float)inv[4], (float)inv[5]}};
    for (int64_t o = start[j]; o < start[j + 1]; ++o) {
        const float* H = Htp + 18 * o;
        float* __restrict__ Eo = E + 18 * o;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const float h0 = H[3 * r], h1 = H[3 * r + 1], h2 = H[3 * r + 2];
#pragma unroll
            for (int c2 = 0; c2 < 3; ++c2) Eo[3 * r + c2] = h0 * M[0][c2] + h1 * M[1][c2] + h2 * M[2][c2];
        }
    }
}

__device__ __forceinline__ void load18(const float* __restrict__ src, float (&v)[18]) {
    const float2* s2 = reinterpret_cast<const float2*>(src);  // 72-byte records: 8-byte aligned
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float2 u = __ldg(s2 + q);
        v[2 * q] = u.x;
        v[2 * q + 1] = u.y;
    }
}

// camera pair p = (a, b), a <= b, in row-major order of the upper triangle of C x C
__device__ __forceinline__ void pair_of(int p, int C, int& a, int& b) {
    a = 0;
    while (p >= C - a) {
        p -= C - a;
        ++a;
    }
    b = a + p;
}

// over one chunk of camera a's observations, the points also seen by b: sum of E_a H_tp,b^T; for
// a == b also of H_tp,a y
__global__ void __launch_bounds__(kBaThreads, 3)
k_ba_schur(int C, int W, const int32_t* __restrict__ pt, const int64_t* __restrict__ start,
           const uint32_t* __restrict__ mask, const int64_t* __restrict__ cam_start, const int64_t* __restrict__ cam_obs,
           const float* __restrict__ Htp, const float* __restrict__ E, const double* __restrict__ y,
           double* __restrict__ schp, double* __restrict__ rhsp) {
    __shared__ float s_red[kBaThreads / 32][42];
    const int p = blockIdx.x, c = blockIdx.y, P = gridDim.x;
    int a, b;
    pair_of(p, C, a, b);
    int64_t q0, q1;
    chunk_of(cam_start[a + 1] - cam_start[a], c, gridDim.y, q0, q1);
    const int64_t* __restrict__ list = cam_obs + cam_start[a];
    float acc[36];
#pragma unroll
    for (int q = 0; q < 36; ++q) acc[q] = 0.f;
    float ry[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t q = q0 + threadIdx.x; q < q1; q += kBaThreads) {
        const int64_t oa = list[q], j = pt[oa];
        int64_t ob = oa;
        if (a != b) {
            if (!sees(mask, W, j, b)) continue;
            ob = obs_of(start, mask, W, j, b);
        }
        float Ea[18], Hb[18];
        load18(E + 18 * oa, Ea);
        load18(Htp + 18 * ob, Hb);
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int s2 = 0; s2 < 6; ++s2)
                acc[6 * r + s2] = fmaf(Ea[3 * r], Hb[3 * s2],
                                       fmaf(Ea[3 * r + 1], Hb[3 * s2 + 1], fmaf(Ea[3 * r + 2], Hb[3 * s2 + 2], acc[6 * r + s2])));
        if (a == b) {
            const float y0 = (float)y[3 * j], y1 = (float)y[3 * j + 1], y2 = (float)y[3 * j + 2];
#pragma unroll
            for (int r = 0; r < 6; ++r) ry[r] = fmaf(Hb[3 * r], y0, fmaf(Hb[3 * r + 1], y1, fmaf(Hb[3 * r + 2], y2, ry[r])));
        }
    }
    float v[42];
#pragma unroll
    for (int q = 0; q < 36; ++q) v[q] = acc[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[36 + q] = ry[q];
    const float tot = block_sum<42>(v, s_red);
    if (threadIdx.x < 36) schp[((size_t)c * P + p) * 36 + threadIdx.x] = tot;
    else if (a == b && threadIdx.x < 42) rhsp[((size_t)c * C + a) * 6 + threadIdx.x - 36] = tot;
}

__device__ __forceinline__ int64_t row_off(int i, int N) { return (int64_t)i * N - (int64_t)i * (i - 1) / 2; }

// entry (i, j), i <= j, of the damped reduced matrix from the chunk sums (FP64)
__device__ __forceinline__ double reduced_entry(int i, int j, int C, int chc, int chs, const double* __restrict__ camp,
                                                const double* __restrict__ schp, double lam) {
    const int a = i / 6, r = i % 6, b = j / 6, q = j % 6, P = C * (C + 1) / 2;
    const int p = a * C - a * (a - 1) / 2 + (b - a);
    double v = 0.0;
    for (int k = 0; k < chs; ++k) v -= schp[((size_t)k * P + p) * 36 + 6 * r + q];
    if (a == b) {  // camera block, upper index of (r, q), r <= q
        const int u = r * 6 - r * (r - 1) / 2 + (q - r);
        double h = 0.0;
        for (int k = 0; k < chc; ++k) h += camp[((size_t)k * C + a) * 27 + u];
        v += r == q ? h * (1.0 + lam) : h;
    }
    return v;
}

// the damped reduced matrix S [N][N] (both triangles) and rhs [N] from the chunk sums, FP64,
// thread per entry (many CTAs: the sums are FP64, whose rate on one SM would make this serial)
__global__ void __launch_bounds__(kBaThreads)
k_ba_assemble(int C, int chc, int chs, const double* __restrict__ camp, const double* __restrict__ schp,
              const double* __restrict__ rhsp, double lam, double* __restrict__ S, double* __restrict__ rhs) {
    const int N = 6 * C;
    const int64_t e = (int64_t)blockIdx.x * kBaThreads + threadIdx.x;
    if (e >= (int64_t)N * N) return;
    const int i = (int)(e / N), j = (int)(e % N);
    S[e] = reduced_entry(i < j ? i : j, i < j ? j : i, C, chc, chs, camp, schp, lam);
    if (e < N) {
        const int a = (int)e / 6, r = (int)e % 6;
        double g = 0.0;
        for (int k = 0; k < chc; ++k) g += camp[((size_t)k * C + a) * 27 + 21 + r];
        for (int k = 0; k < chs; ++k) g -= rhsp[((size_t)k * C + a) * 6 + r];
        rhs[e] = g;
    }
}

// fixed rows (gauge, unobserved) and the Jacobi scale: s_id[i] = 1 / sqrt(S_ii), 0 for a fixed row;
// s_rhs[i] = rhs_i / sqrt(S_ii) (FP32: the scaled system is what gets factored)
template <int kThreads>
__device__ __forceinline__ void scale_rows(int N, int NP, int fixed_axis, const double* __restrict__ S,
                                           const double* __restrict__ rhs, float* s_id, float* s_rhs) {
    for (int i = threadIdx.x; i < NP; i += kThreads) {
        if (i >= N) {
            s_id[i] = 0.f;
            s_rhs[i] = 0.f;
            continue;
        }
        const double dg = S[(int64_t)i * N + i];
        const bool fixed = i < 6 || i == 9 + fixed_axis || !(dg > 0.0);
        const float id = fixed ? 0.f : rsqrtf((float)dg);
        s_id[i] = id;
        s_rhs[i] = fixed ? 0.f : (float)rhs[i] * id;
    }
}

__device__ __forceinline__ float scaled_entry(const double* __restrict__ S, int N, int i, int j, const float* s_id) {
    if (i == j) return 1.f;
    const float a = s_id[i], b = s_id[j];
    return (a == 0.f || b == 0.f) ? 0.f : (float)S[(int64_t)i * N + j] * a * b;
}

// One CTA: the Jacobi-scaled reduced system in packed upper storage A (FP32; shared memory when it
// fits, else global scratch), eliminated with the rhs carried along, then back-substituted.
__global__ void __launch_bounds__(kSolveThreads)
k_ba_solve(int C, const double* __restrict__ S, const double* __restrict__ rhs, int fixed_axis,
           float* __restrict__ Aglob, double* __restrict__ dc, int* __restrict__ status) {
    extern __shared__ float s_dyn[];
    __shared__ float s_rhs[kMaxN];
    __shared__ float s_d[kMaxN];  // 1 / sqrt of the diagonal; 0 marks a fixed row
    const int N = 6 * C;
    float* A = Aglob ? Aglob : s_dyn;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = kSolveThreads / 32;
    scale_rows<kSolveThreads>(N, N, fixed_axis, S, rhs, s_d, s_rhs);
    __syncthreads();
    for (int i = warp; i < N; i += warps) {
        const int64_t oi = row_off(i, N);
        for (int j = i + lane; j < N; j += 32) A[oi + (j - i)] = scaled_entry(S, N, i, j, s_d);
    }
    __syncthreads();
    // symmetric elimination: row i -= (A_ki / A_kk) row k for i > k, upper part and rhs
    for (int k = 0; k < N - 1; ++k) {
        const int64_t ok = row_off(k, N);
        const float d = A[ok];
        const float inv = d > 0.f ? 1.0f / d : 0.f;
        if (threadIdx.x == 0 && !(d > 0.f)) atomicOr(status, 1);
        const float rk = s_rhs[k];
        for (int i = k + 1 + warp; i < N; i += warps) {
            const float f = A[ok + (i - k)] * inv;
            if (f == 0.f) continue;
            const int64_t oi = row_off(i, N);
            for (int j = i + lane; j < N; j += 32) A[oi + (j - i)] = fmaf(-f, A[ok + (j - k)], A[oi + (j - i)]);
            if (lane == 0) s_rhs[i] = fmaf(-f, rk, s_rhs[i]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && !(A[row_off(N - 1, N)] > 0.f)) atomicOr(status, 1);
    // back substitution by one warp, column-oriented: x_k = rhs_k / A_kk, rhs_i -= A_ik x_k (i < k)
    if (warp == 0) {
        for (int k = N - 1; k >= 0; --k) {
            const float dk = A[row_off(k, N)];
            const float x = dk > 0.f ? s_rhs[k] / dk : 0.f;
            for (int i = lane; i < k; i += 32) s_rhs[i] = fmaf(-A[row_off(i, N) + (k - i)], x, s_rhs[i]);
            if (lane == 0) dc[k] = (double)x * s_d[k];
            __syncwarp();
        }
    }
}

// ---- blocked solve (N padded to NP, a multiple of 32, NP <= 224): full lower triangle in shared
// memory, row stride NP + 1 (column walks hit distinct banks), Cholesky right-looking by 8-column
// panels (one warp factors the diagonal block in registers, a thread per
// row solves the rows below it, 4 x 4 register micro-tiles update the trailing lower triangle; one
// barrier per column step, whatever its form, cost ~1k cycles here, so the column steps are kept
// inside a warp), then forward and back substitution by 32-row panels.

constexpr int kPanel = 8;  // factorization panel width: 3 barriers a panel, 8 short column steps in registers

// warp: Cholesky of the kPanel x kPanel diagonal block at B (row stride ld), lane r < kPanel
// holding row r in registers; rdiag[k] = 1 / L_kk.  The pivot goes through the hardware
// reciprocal square root (2 ulp): the correctly rounded sqrt and division are multi-instruction
// sequences, and they sit on the dependent chain of every column.
__device__ __forceinline__ void factor_diag_block(float* B, int ld, int lane, float* rdiag, int* status) {
    float a[kPanel];
#pragma unroll
    for (int c = 0; c < kPanel; ++c) a[c] = (lane < kPanel && c <= lane) ? B[lane * ld + c] : 0.f;
#pragma unroll
    for (int k = 0; k < kPanel; ++k) {
        float d = __shfl_sync(0xffffffffu, a[k], k);
        if (!(d > 0.f)) {
            if (lane == 0) atomicOr(status, 1);
            d = 1.f;
        }
        const float rs = rsqrtf(d);
        if (lane == 0) rdiag[k] = rs;
        a[k] = lane == k ? d * rs : (lane > k ? a[k] * rs : a[k]);
#pragma unroll
        for (int c = k + 1; c < kPanel; ++c) {
            const float lck = __shfl_sync(0xffffffffu, a[k], c);
            if (lane >= c) a[c] = fmaf(-a[k], lck, a[c]);
        }
    }
    if (lane < kPanel)
#pragma unroll
        for (int c = 0; c < kPanel; ++c)
            if (c <= lane) B[lane * ld + c] = a[c];
}

__global__ void __launch_bounds__(kBlockedThreads)
k_ba_solve_blocked(int C, const double* __restrict__ S, const double* __restrict__ rhs, int fixed_axis,
                   double* __restrict__ dc, int* __restrict__ status) {
    extern __shared__ float A[];
    __shared__ float s_rhs[kMaxBlockedN];
    __shared__ float s_id[kMaxBlockedN];  // 1 / sqrt of the diagonal; 0 marks a fixed (or padding) row
    __shared__ float s_rdiag[kMaxBlockedN];  // 1 / L_kk
    const int N = 6 * C, NP = (N + 31) & ~31, ld = NP + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = kBlockedThreads / 32;
    scale_rows<kBlockedThreads>(N, NP, fixed_axis, S, rhs, s_id, s_rhs);
    __syncthreads();
    for (int r = warp; r < NP; r += warps)
#pragma unroll 4
        for (int c = lane; c <= r; c += 32)
            A[r * ld + c] = r < N ? scaled_entry(S, N, r, c, s_id) : (r == c ? 1.f : 0.f);
    __syncthreads();
    for (int c0 = 0; c0 < NP; c0 += kPanel) {
        if (warp == 0) factor_diag_block(A + c0 * ld + c0, ld, lane, s_rdiag + c0, status);
        __syncthreads();
        // rows below the panel, thread per row: x L_pp^T = a by forward substitution
        const int t0 = c0 + kPanel;
        for (int r = t0 + threadIdx.x; r < NP; r += kBlockedThreads) {
            float x[kPanel];
#pragma unroll
            for (int q = 0; q < kPanel; ++q) x[q] = A[r * ld + c0 + q];
#pragma unroll
            for (int k = 0; k < kPanel; ++k) {
                const float* Lk = A + (c0 + k) * ld + c0;
                float v = x[k];
#pragma unroll
                for (int q = 0; q < k; ++q) v = fmaf(-Lk[q], x[q], v);
                x[k] = v * s_rdiag[c0 + k];
            }
#pragma unroll
            for (int q = 0; q < kPanel; ++q) A[r * ld + c0 + q] = x[q];
        }
        __syncthreads();
        // trailing lower triangle in 4 x 4 micro-tiles: A_rc -= sum_q L_rq L_cq over the panel
        const int mt = (NP - t0) >> 2;
        for (int mi = warp; mi < mt; mi += warps)
            for (int mj = lane; mj <= mi; mj += 32) {
                const float* Lr = A + (t0 + 4 * mi) * ld + c0;
                const float* Lc = A + (t0 + 4 * mj) * ld + c0;
                float acc[4][4] = {};
#pragma unroll
                for (int q = 0; q < kPanel; ++q) {
                    float lr[4], lc[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        lr[u] = Lr[u * ld + q];
                        lc[u] = Lc[u * ld + q];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(lr[u], lc[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (mi > mj || v <= u) A[(t0 + 4 * mi + u) * ld + t0 + 4 * mj + v] -= acc[u][v];
            }
        __syncthreads();
    }
    // L z = rhs
    for (int c0 = 0; c0 < NP; c0 += 32) {
        if (warp == 0) {
            const float rd = s_rdiag[c0 + lane];
            float z = s_rhs[c0 + lane];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                if (lane == k) z *= rd;
                const float zk = __shfl_sync(0xffffffffu, z, k);
                if (lane > k) z = fmaf(-A[(c0 + lane) * ld + c0 + k], zk, z);
            }
            s_rhs[c0 + lane] = z;
        }
        __syncthreads();
        for (int r = c0 + 32 + warp; r < NP; r += warps) {
            float part = A[r * ld + c0 + lane] * s_rhs[c0 + lane];
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) s_rhs[r] -= part;
        }
        __syncthreads();
    }
    // L^T x = z, panels from the last
    for (int c0 = NP - 32; c0 >= 0; c0 -= 32) {
        if (warp == 0) {
            const float rd = s_rdiag[c0 + lane];
            float x = s_rhs[c0 + lane];
#pragma unroll
            for (int k = 31; k >= 0; --k) {
                if (lane == k) x *= rd;
                const float xk = __shfl_sync(0xffffffffu, x, k);
                if (lane < k) x = fmaf(-A[(c0 + k) * ld + c0 + lane], xk, x);
            }
            s_rhs[c0 + lane] = x;
        }
        __syncthreads();
        for (int r = warp; r < c0; r += warps) {
            float part = A[(c0 + lane) * ld + r] * s_rhs[c0 + lane];
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) s_rhs[r] -= part;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += kBlockedThreads) dc[i] = (double)s_rhs[i] * s_id[i];
}

// Delta_p = H^-1 (b_p - sum H_tp^T Delta_t); candidate points
__global__ void __launch_bounds__(kPointThreads)
k_ba_backsub(int64_t n, const int64_t* __restrict__ start, const int32_t* __restrict__ cam, const float* __restrict__ Htp,
             const double* __restrict__ Hinv, const double* __restrict__ bp, const double* __restrict__ dc,
             const float* __restrict__ P, float* __restrict__ Pn, float* __restrict__ dP) {
    const int64_t j = (int64_t)blockIdx.x * kPointThreads + threadIdx.x;
    if (j >= n) return;
    double g[3] = {bp[3 * j], bp[3 * j + 1], bp[3 * j + 2]};
    for (int64_t o = start[j]; o < start[j + 1]; ++o) {
        const int i = cam[o];
        const float* H = Htp + 18 * o;
        float dci[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) dci[r] = (float)dc[6 * i + r];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = 0.f;
#pragma unroll
            for (int r = 0; r < 6; ++r) v = fmaf(H[3 * r + c], dci[r], v);
            g[c] -= v;
        }
    }
    const double* h = Hinv + 6 * j;
    const double d0 = h[0] * g[0] + h[1] * g[1] + h[2] * g[2];
    const double d1 = h[1] * g[0] + h[3] * g[1] + h[4] * g[2];
    const double d2 = h[2] * g[0] + h[4] * g[1] + h[5] * g[2];
    if (dP) {
        dP[3 * j] = (float)d0;
        dP[3 * j + 1] = (float)d1;
        dP[3 * j + 2] = (float)d2;
    }
    Pn[3 * j] = (float)(P[3 * j] + d0);
    Pn[3 * j + 1] = (float)(P[3 * j + 1] + d1);
    Pn[3 * j + 2] = (float)(P[3 * j + 2] + d2);
}

// candidate poses: R <- exp([omega]x) R (Rodrigues, double), t <- t + v
__global__ void k_ba_cameras(int C, const double* __restrict__ dc, const float* __restrict__ R, const float* __restrict__ t,
                             float* __restrict__ Rn, float* __restrict__ tn, float* __restrict__ dcam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const double w0 = dc[6 * i], w1 = dc[6 * i + 1], w2 = dc[6 * i + 2];
    const double th = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
    double Ex[3][3];
    const double Kx[3][3] = {{0, -w2, w1}, {w2, 0, -w0}, {-w1, w0, 0}};
    const double s = th > 1e-12 ? sin(th) / th : 1.0, c = th > 1e-12 ? (1.0 - cos(th)) / (th * th) : 0.5;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double kk = 0.0;
            for (int q = 0; q < 3; ++q) kk += Kx[a][q] * Kx[q][b];
            Ex[a][b] = (a == b ? 1.0 : 0.0) + s * Kx[a][b] + c * kk;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0.0;
            for (int q = 0; q < 3; ++q) v += Ex[a][q] * (double)R[9 * i + 3 * q + b];
            Rn[9 * i + 3 * a + b] = (float)v;
        }
    for (int a = 0; a < 3; ++a) tn[3 * i + a] = (float)((double)t[3 * i + a] + dc[6 * i + 3 + a]);
    if (dcam)
        for (int a = 0; a < 6; ++a) dcam[6 * i + a] = (float)dc[6 * i + a];
}

// robust cost of (R, t, P) over all observations (thread per point); behind a camera: 1e30
__global__ void __launch_bounds__(kPointThreads)
k_ba_cost(int64_t n, const float* __restrict__ R, const float* __restrict__ t, const float* __restrict__ P,
          const int32_t* __restrict__ cam, const float* __restrict__ uv, const int64_t* __restrict__ start, Intr K,
          float sigma, float delta, double* __restrict__ cost) {
    __shared__ double s_red[kPointThreads / 32];
    const int64_t j = (int64_t)blockIdx.x * kPointThreads + threadIdx.x;
    double rho_sum = 0.0;
    if (j < n) {
        for (int64_t o = start[j]; o < start[j + 1]; ++o) {
            double X[3], r[2], Wm, rho;
            cam_point(R, t, cam[o], P[3 * j], P[3 * j + 1], P[3 * j + 2], X);
            if (residual(X, K, uv[2 * o], uv[2 * o + 1], sigma, delta, r, Wm, rho)) rho_sum += rho;
            else rho_sum += 1e30;
        }
    }
    block_add_double<kPointThreads>(rho_sum, s_red, cost);
}

__global__ void k_ba_project(int64_t m, int64_t n, int C, const float* __restrict__ R, const float* __restrict__ t,
                             const float* __restrict__ P, const int32_t* __restrict__ cam,
                             const int32_t* __restrict__ pt, Intr K, float* __restrict__ uv, float* __restrict__ z) {
    const int64_t o = (int64_t)blockIdx.x * kBaThreads + threadIdx.x;
    if (o >= m) return;
    const int64_t j = pt[o];
    const int i = cam[o];
    if (i < 0 || i >= C || j < 0 || j >= n) {  // out of range: NaN, no access
        z[o] = uv[2 * o] = uv[2 * o + 1] = __int_as_float(0x7fc00000);
        return;
    }
    double X[3];
    cam_point(R, t, i, P[3 * j], P[3 * j + 1], P[3 * j + 2], X);
    z[o] = (float)X[2];
    const double iz = 1.0 / X[2];
    uv[2 * o] = (float)fma((double)K.fx * X[0], iz, (double)K.cx);
    uv[2 * o + 1] = (float)fma((double)K.fy * X[1], iz, (double)K.cy);
}

unsigned blocks_for(int64_t k) { return (unsigned)((k + kBaThreads - 1) / kBaThreads); }
unsigned points_blocks(int64_t k) { return (unsigned)((k + kPointThreads - 1) / kPointThreads); }

Intr intr(const float K[4]) { return Intr{K[0], K[1], K[2], K[3]}; }

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
BaShape ba_shape(int C, int64_t n, int64_t m) {
    BaShape sh;
    sh.C = C;
    sh.n = n;
    sh.m = m;
    sh.W = (C + 31) / 32;
    sh.N = 6 * C;
    sh.pairs = C * (C + 1) / 2;
    // chunks of a camera's observation list: enough CTAs to fill the SMs, at least ~4 items a thread
    const int64_t per_cam = C > 0 ? m / C : 0;
    const int64_t max_chunks = per_cam / 1024 > 1 ? per_cam / 1024 : 1;
    auto chunks = [&](int64_t ctas, int64_t target) {
        int64_t k = (target + ctas - 1) / ctas;
        return (int)(k < 1 ? 1 : (k > max_chunks ? max_chunks : k));
    };
    sh.chc = chunks(C, 2 * 152);
    sh.chs = chunks(sh.pairs, 6 * 152);  // three resident CTAs per SM, two waves
    const size_t NP = ((size_t)sh.N + 31) & ~(size_t)31;
    const size_t full = NP * (NP + 1) * sizeof(float), packed = (size_t)sh.N * (sh.N + 1) / 2 * sizeof(float);
    sh.blocked = NP <= (size_t)kMaxBlockedN;
    sh.solve_smem = sh.blocked ? full : (packed <= kMaxSolveSmem ? packed : 0);
    return sh;
}

int ba_configure_solve() {
    // one bound for every problem size, so contexts of different sizes can coexist
    const bool ok =
        cudaFuncSetAttribute(k_ba_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSolveSmem) == cudaSuccess &&
        cudaFuncSetAttribute(k_ba_solve_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSolveSmem) ==
            cudaSuccess;
    return ok ? 0 : -1;
}

int launch_ba_check(int64_t m, int64_t n, int C, const int32_t* cam, const int32_t* pt, int* flag, cudaStream_t s) {
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (m > 0) k_ba_check<<<blocks_for(m), kBaThreads, 0, s>>>(m, n, C, cam, pt, flag);
    return m > 0 ? 1 : 0;
}

int launch_ba_index(const BaShape& sh, const int32_t* pt, const int32_t* cam, int64_t* start, uint32_t* mask,
                    int64_t* cam_count, int64_t* cam_start, int64_t* cam_obs, cudaStream_t s) {
    k_ba_offsets<<<blocks_for(sh.n + 1), kBaThreads, 0, s>>>(sh.n, sh.m, pt, start);
    if (sh.n > 0) k_ba_masks<<<blocks_for(sh.n), kBaThreads, 0, s>>>(sh.n, sh.W, start, cam, mask);
    cudaMemsetAsync(cam_count, 0, sizeof(int64_t) * sh.C, s);
    if (sh.m > 0) k_ba_cam_count<<<blocks_for(sh.m), kBaThreads, 0, s>>>(sh.m, cam, cam_count);
    k_ba_cam_fill<<<sh.C, 1024, 0, s>>>(sh.m, sh.C, cam, cam_count, cam_start, cam_obs);
    return 4;
}

int launch_ba_linearize(const BaShape& sh, const float* R, const float* t, const float* P, const int32_t* cam,
                        const int32_t* pt, const float* uv, const int64_t* start, const int64_t* cam_start,
                        const int64_t* cam_obs, const float K[4], float sigma, float delta, float* Htp, double* Hpp,
                        double* bp, double* camp, double* cost, cudaStream_t s, cudaEvent_t* ev) {
    cudaMemsetAsync(cost, 0, sizeof(double), s);
    if (ev) cudaEventRecord(ev[0], s);
    if (sh.n > 0)
        k_ba_linearize<<<points_blocks(sh.n), kPointThreads, 0, s>>>(sh.n, R, t, P, cam, uv, start, intr(K), sigma,
                                                                       delta, Htp, Hpp, bp, cost);
    if (ev) cudaEventRecord(ev[1], s);
    k_ba_camblocks<<<dim3(sh.C, sh.chc), kBaThreads, 0, s>>>(sh.C, R, t, P, pt, uv, cam_start, cam_obs, intr(K), sigma,
                                                              delta, camp);
    if (ev) cudaEventRecord(ev[2], s);
    return sh.n > 0 ? 2 : 1;
}

int launch_ba_trial(const BaShape& sh, const int32_t* pt, const int64_t* start, const uint32_t* mask,
                    const int64_t* cam_start, const int64_t* cam_obs, const int32_t* cam, const float* Htp,
                    const double* Hpp, const double* bp, const double* camp, double lam, int fixed_axis, double* Hinv,
                    double* y, float* E, double* schp, double* rhsp, double* Sfull, double* rhs, float* Aglob,
                    double* dc, const float* R, const float* t, const float* P, float* Rn, float* tn, float* Pn,
                    float* dcam, float* dP, int* status, cudaStream_t s, cudaEvent_t* ev) {
    int launches = 1;
    if (sh.n > 0) {
        k_ba_points<<<points_blocks(sh.n), kPointThreads, 0, s>>>(sh.n, start, Hpp, bp, Htp, lam, Hinv, y, E);
        ++launches;
    }
    if (ev) cudaEventRecord(ev[0], s);
    k_ba_schur<<<dim3(sh.pairs, sh.chs), kBaThreads, 0, s>>>(sh.C, sh.W, pt, start, mask, cam_start, cam_obs, Htp, E,
                                                              y, schp, rhsp);
    if (ev) cudaEventRecord(ev[1], s);
    k_ba_assemble<<<(unsigned)(((int64_t)sh.N * sh.N + kBaThreads - 1) / kBaThreads), kBaThreads, 0, s>>>(
        sh.C, sh.chc, sh.chs, camp, schp, rhsp, lam, Sfull, rhs);
    if (sh.blocked)
        k_ba_solve_blocked<<<1, kBlockedThreads, sh.solve_smem, s>>>(sh.C, Sfull, rhs, fixed_axis, dc, status);
    else
        k_ba_solve<<<1, kSolveThreads, sh.solve_smem, s>>>(sh.C, Sfull, rhs, fixed_axis,
                                                           sh.solve_smem ? nullptr : Aglob, dc, status);
    if (ev) cudaEventRecord(ev[2], s);
    if (sh.n > 0) {
        k_ba_backsub<<<points_blocks(sh.n), kPointThreads, 0, s>>>(sh.n, start, cam, Htp, Hinv, bp, dc, P, Pn, dP);
        ++launches;
    }
    k_ba_cameras<<<(sh.C + 63) / 64, 64, 0, s>>>(sh.C, dc, R, t, Rn, tn, dcam);
    if (ev) cudaEventRecord(ev[3], s);
    return launches + 3;
}

int launch_ba_cost(const BaShape& sh, const float* R, const float* t, const float* P, const int32_t* cam,
                   const float* uv, const int64_t* start, const float K[4], float sigma, float delta, double* cost,
                   cudaStream_t s) {
    cudaMemsetAsync(cost, 0, sizeof(double), s);
    if (sh.n <= 0) return 0;
    k_ba_cost<<<points_blocks(sh.n), kPointThreads, 0, s>>>(sh.n, R, t, P, cam, uv, start, intr(K), sigma, delta, cost);
    return 1;
}

int launch_ba_project(int64_t m, int64_t n, int C, const float* R, const float* t, const float* P, const int32_t* cam,
                      const int32_t* pt, const float K[4], float* uv, float* z, cudaStream_t s) {
    if (m <= 0) return 0;
    k_ba_project<<<blocks_for(m), kBaThreads, 0, s>>>(m, n, C, R, t, P, cam, pt, intr(K), uv, z);
    return 1;
}

}  // namespace pgs
