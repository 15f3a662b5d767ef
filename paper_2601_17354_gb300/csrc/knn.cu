// K13 knn_grid and K14 features / PCA initializer (operator I of PocketGS, Sec. III-B).
//
// kNN: points are counting-sorted into a uniform grid; each query scans the cells within
// Chebyshev distance rho of its own cell, keeping a sorted list of its k best (squared distance,
// index) pairs, and widens rho until the k-th distance is below rho times the cell size, which
// guarantees that no unscanned point can be closer: the result is the exact k nearest other
// points.  Squared distances use the fp32 sequence d2 = fma(dx, dx, fma(dy, dy, dz * dz)) with
// dx = p_j - p_i, ties broken by index, so the neighbour lists are reproducible bit for bit.
//
// Features and the paper's initializer are computed per point in FP64 (a few hundred operations
// per point): Eq. 5 covariance of the K_n = 16 nearest neighbours about their centroid, its
// smallest-eigenvalue eigenvector as the normal (cyclic Jacobi, eigenvectors canonicalised so the
// largest-magnitude component is positive), Eq. 6 tangential scale from the K_s = 3 nearest
// neighbours, normal scale r_normal s_t, z axis rotated onto the normal, opacity logit(0.1); and
// the 16 features of the learned initializer from the 32 nearest neighbours.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int kThreads = 256;

// Order-preserving integer image of a float (and its own inverse): non-negative floats keep their
// bits, negative ones flip all but the sign bit, so signed integer order = float order.
__device__ __host__ __forceinline__ int ordered(int bits) { return bits >= 0 ? bits : bits ^ 0x7fffffff; }

__global__ void k_bbox(int64_t n, const float* __restrict__ P, int* bbox) {
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fminf(lo[d], P[d * n + i]);
            hi[d] = fmaxf(hi[d], P[d * n + i]);
        }
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(bbox + d, ordered(__float_as_int(lo[d])));
            atomicMax(bbox + 3 + d, ordered(__float_as_int(hi[d])));
        }
    }
}

struct Grid {
    float lo[3];
    float h;
    int dim[3];
};

__device__ __forceinline__ int cell_coord(float x, float lo, float h, int dim) {
    return min(max((int)floorf((x - lo) / h), 0), dim - 1);
}

__global__ void k_cell_count(int64_t n, const float* __restrict__ P, Grid g, uint32_t* __restrict__ cell_of,
                             uint32_t* __restrict__ counts) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const int cx = cell_coord(P[i], g.lo[0], g.h, g.dim[0]);
    const int cy = cell_coord(P[n + i], g.lo[1], g.h, g.dim[1]);
    const int cz = cell_coord(P[2 * n + i], g.lo[2], g.h, g.dim[2]);
    const uint32_t c = ((uint32_t)cz * g.dim[1] + cy) * g.dim[0] + cx;
    cell_of[i] = c;
    atomicAdd(&counts[c], 1u);
}

// exclusive scan of counts[0..m) into start[0..m], start[m] = total (one CTA, chunked)
__global__ void __launch_bounds__(1024) k_scan_cells(int64_t m, const uint32_t* __restrict__ counts,
                                                     uint32_t* __restrict__ start) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < m; base += 1024) {
        const int64_t idx = base + threadIdx.x;
        const uint32_t v = idx < m ? counts[idx] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_warp[lane];
            uint32_t wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            s_warp[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t carry = s_carry;
        if (idx < m) start[idx] = carry + s_warp[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + s_warp[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[m] = s_carry;
}

// points in cell order: their indices and a copy of their positions ([3][n]), so the queries read
// each cell's candidates contiguously
__global__ void k_cell_scatter(int64_t n, const float* __restrict__ P, const uint32_t* __restrict__ cell_of,
                               uint32_t* __restrict__ cursor, uint32_t* __restrict__ sorted,
                               float* __restrict__ Ps) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t s = atomicAdd(&cursor[cell_of[i]], 1u);
    sorted[s] = (uint32_t)i;
    Ps[s] = P[i];
    Ps[n + s] = P[n + i];
    Ps[2 * n + s] = P[2 * n + i];
}

template <int K>
__global__ void __launch_bounds__(128)
k_knn_query(int64_t n, const float* __restrict__ P, Grid g, const uint32_t* __restrict__ start,
            const uint32_t* __restrict__ sorted, const float* __restrict__ Ps, int32_t* __restrict__ nb) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= n) return;
    const float qx = P[i], qy = P[n + i], qz = P[2 * n + i];
    const int cx = cell_coord(qx, g.lo[0], g.h, g.dim[0]);
    const int cy = cell_coord(qy, g.lo[1], g.h, g.dim[1]);
    const int cz = cell_coord(qz, g.lo[2], g.h, g.dim[2]);
    float bd[K];
    int32_t bi[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
        bd[a] = 3.4e38f;
        bi[a] = 0x7fffffff;
    }
    const int maxr = max(g.dim[0], max(g.dim[1], g.dim[2]));
    for (int rho = 0; rho <= maxr; ++rho) {
        for (int dz = -rho; dz <= rho; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.dim[2]) continue;
            for (int dy = -rho; dy <= rho; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.dim[1]) continue;
                const bool face = abs(dz) == rho || abs(dy) == rho;
                for (int dx = -rho; dx <= rho; dx += (face ? 1 : 2 * max(rho, 1))) {
                    const int x = cx + dx;
                    if (x < 0 || x >= g.dim[0]) continue;
                    const uint32_t c = ((uint32_t)z * g.dim[1] + y) * g.dim[0] + x;
                    for (uint32_t s = start[c]; s < start[c + 1]; ++s) {
                        const int32_t j = (int32_t)sorted[s];
                        if (j == i) continue;
                        const float ex = Ps[s] - qx, ey = Ps[n + s] - qy, ez = Ps[2 * n + s] - qz;
                        const float d2 = __fmaf_rn(ex, ex, __fmaf_rn(ey, ey, __fmul_rn(ez, ez)));
                        if (d2 < bd[K - 1] || (d2 == bd[K - 1] && j < bi[K - 1])) {
                            // insertion by a fixed pass of compare-and-swap (static indices keep the
                            // list in registers): the candidate trades places with every entry it
                            // precedes, and the last entry falls off
                            float cd = d2;
                            int32_t cj = j;
#pragma unroll
                            for (int a = 0; a < K; ++a) {
                                const bool before = cd < bd[a] || (cd == bd[a] && cj < bi[a]);
                                const float td = bd[a];
                                const int32_t tj = bi[a];
                                bd[a] = before ? cd : td;
                                bi[a] = before ? cj : tj;
                                cd = before ? td : cd;
                                cj = before ? tj : cj;
                            }
                        }
                    }
                }
            }
        }
        // every point within rho * h of the query lies in the scanned block
        const float reach = (float)rho * g.h;
        if (bi[K - 1] != 0x7fffffff && bd[K - 1] < reach * reach * 0.9999f) break;
    }
#pragma unroll
    for (int a = 0; a < K; ++a) nb[i * K + a] = bi[a] == 0x7fffffff ? -1 : bi[a];
}

// ---------------------------------------------------------------------------------------------
// features and the paper's initializer (FP64)
// ---------------------------------------------------------------------------------------------

__device__ void jacobi3(double A[3][3], double w[3], double V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    // ascending eigenvalues (three-element sorting network)
    if (A[idx[1]][idx[1]] < A[idx[0]][idx[0]]) { int t = idx[0]; idx[0] = idx[1]; idx[1] = t; }
    if (A[idx[2]][idx[2]] < A[idx[1]][idx[1]]) { int t = idx[1]; idx[1] = idx[2]; idx[2] = t; }
    if (A[idx[1]][idx[1]] < A[idx[0]][idx[0]]) { int t = idx[0]; idx[0] = idx[1]; idx[1] = t; }
    double W[3][3];
    for (int k = 0; k < 3; ++k) {
        w[k] = A[idx[k]][idx[k]];
        int big = 0;
        for (int r = 1; r < 3; ++r)
            if (fabs(V[r][idx[k]]) > fabs(V[big][idx[k]])) big = r;
        const double sg = V[big][idx[k]] < 0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) W[r][k] = sg * V[r][idx[k]];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) V[a][b] = W[a][b];
}

__device__ void neighbour_cov(const float* __restrict__ P, int64_t n, const int32_t* nb, int k, double C[3][3]) {
    double c[3] = {0, 0, 0};
    for (int a = 0; a < k; ++a)
        for (int d = 0; d < 3; ++d) c[d] += P[d * n + nb[a]];
    for (int d = 0; d < 3; ++d) c[d] /= k;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a][b] = 0.0;
    for (int j = 0; j < k; ++j) {
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = P[d * n + nb[j]] - c[d];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[a][b] += v[a] * v[b];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a][b] /= k;
}

__device__ double pdist(const float* __restrict__ P, int64_t n, int64_t i, int64_t j) {
    double s = 0;
    for (int d = 0; d < 3; ++d) {
        const double v = (double)P[d * n + j] - (double)P[d * n + i];
        s += v * v;
    }
    return sqrt(s);
}

__device__ void mat_to_quat(const double R[3][3], double q[4]) {
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr > 0) {
        const double s = sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * s;
        q[1] = (R[2][1] - R[1][2]) / s;
        q[2] = (R[0][2] - R[2][0]) / s;
        q[3] = (R[1][0] - R[0][1]) / s;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        const double s = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2;
        q[0] = (R[2][1] - R[1][2]) / s;
        q[1] = 0.25 * s;
        q[2] = (R[0][1] + R[1][0]) / s;
        q[3] = (R[0][2] + R[2][0]) / s;
    } else if (R[1][1] > R[2][2]) {
        const double s = sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2;
        q[0] = (R[0][2] - R[2][0]) / s;
        q[1] = (R[0][1] + R[1][0]) / s;
        q[2] = 0.25 * s;
        q[3] = (R[1][2] + R[2][1]) / s;
    } else {
        const double s = sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2;
        q[0] = (R[1][0] - R[0][1]) / s;
        q[1] = (R[0][2] + R[2][0]) / s;
        q[2] = (R[1][2] + R[2][1]) / s;
        q[3] = 0.25 * s;
    }
}

// One thread per point: nb [n][32] ascending.  Writes features (fp32 [n][16] and bf16 [n][16]),
// the eigenframe quaternion frame_q [4][n], and the paper's initializer into init (log-scales,
// quaternions, opacity logits; means = the points; SH zero).
__global__ void __launch_bounds__(128)
k_features_init(int64_t n, const float* __restrict__ P, const int32_t* __restrict__ nb, float r_normal,
                float* __restrict__ feats, __nv_bfloat16* __restrict__ feats_bf16, float* __restrict__ frame_q,
                pgs_gaussians init) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= n) return;
    const int32_t* nbi = nb + i * 32;
    double C[3][3], w[3], V[3][3];
    // features from the 32 nearest neighbours
    neighbour_cov(P, n, nbi, 32, C);
    jacobi3(C, w, V);
    float f[16];
    const double sum = w[0] + w[1] + w[2];
    for (int a = 0; a < 3; ++a) f[a] = (float)(sum > 0 ? w[a] / sum : 1.0 / 3.0);
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) f[3 + 3 * k + d] = (float)V[d][k];
    double md = 0, off[3] = {0, 0, 0};
    for (int a = 0; a < 32; ++a) {
        md += pdist(P, n, i, nbi[a]);
        for (int d = 0; d < 3; ++d) off[d] += (double)P[d * n + nbi[a]] - P[d * n + i];
    }
    md /= 32.0;
    for (int d = 0; d < 3; ++d) f[12 + d] = (float)(off[d] / 32.0 / md);
    f[15] = (float)(-3.0 * log(md));
    for (int a = 0; a < 16; ++a) {
        feats[i * 16 + a] = f[a];
        feats_bf16[i * 16 + a] = __float2bfloat16_rn(f[a]);
    }
    double R[3][3];
    for (int d = 0; d < 3; ++d) {
        R[d][0] = V[d][2];
        R[d][1] = V[d][1];
        R[d][2] = V[d][0];
    }
    const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                       R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                       R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
    if (det < 0)
        for (int d = 0; d < 3; ++d) R[d][0] = -R[d][0];
    double q[4];
    mat_to_quat(R, q);
    for (int a = 0; a < 4; ++a) frame_q[a * n + i] = (float)q[a];

    // the paper's initializer: normal from 16 neighbours (Eq. 5), scale from 3 (Eq. 6)
    neighbour_cov(P, n, nbi, 16, C);
    jacobi3(C, w, V);
    const double nx = V[0][0], ny = V[1][0], nz = V[2][0];
    double st = 0;
    for (int a = 0; a < 3; ++a) st += pdist(P, n, i, nbi[a]);
    st /= 3.0;
    init.log_scales[i] = (float)log(st);
    init.log_scales[n + i] = (float)log(st);
    init.log_scales[2 * n + i] = (float)log((double)r_normal * st);
    double qw, qx, qy, qz;
    if (nz < -1.0 + 1e-12) {
        qw = 0; qx = 1; qy = 0; qz = 0;
    } else {
        qw = sqrt(0.5 * (1.0 + nz));
        const double s = 1.0 / (2.0 * qw);
        qx = -ny * s;
        qy = nx * s;
        qz = 0.0;
    }
    init.quats[i] = (float)qw;
    init.quats[n + i] = (float)qx;
    init.quats[2 * n + i] = (float)qy;
    init.quats[3 * n + i] = (float)qz;
    init.opacity_logits[i] = (float)log(0.1 / 0.9);
    for (int d = 0; d < 3; ++d) init.means[d * n + i] = P[d * n + i];
    const int K = (init.sh_degree + 1) * (init.sh_degree + 1);
    for (int c = 0; c < 3 * K; ++c) init.sh[(int64_t)c * n + i] = 0.f;
}

// Hamilton product of (w, x, y, z) quaternions
__device__ __forceinline__ void qmul(const float a[4], const float b[4], float o[4]) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Learned parameters from MLP outputs y [n][8], as corrections of the paper's initializer `pca`
// of the same point: log-scales pca + y0..2, rotation normalise(pca q) (x) normalise(y3..6),
// logit pca + y7.  A point whose outputs are not finite (or whose quaternion is zero) keeps the
// paper's initializer and is counted in *fallbacks.
__global__ void k_apply_mlp(int64_t n, const float* __restrict__ y, pgs_gaussians pca, pgs_gaussians out,
                            uint32_t* fallbacks) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float* yi = y + i * 8;
    bool ok = true;
    for (int k = 0; k < 8; ++k) ok = ok && isfinite(yi[k]);
    const float qn = sqrtf(yi[3] * yi[3] + yi[4] * yi[4] + yi[5] * yi[5] + yi[6] * yi[6]);
    ok = ok && qn > 1e-12f;
    if (ok) {
        const float ql[4] = {yi[3] / qn, yi[4] / qn, yi[5] / qn, yi[6] / qn};
        float qb[4] = {pca.quats[i], pca.quats[n + i], pca.quats[2 * n + i], pca.quats[3 * n + i]};
        const float bn = sqrtf(qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3]);
        for (int k = 0; k < 4; ++k) qb[k] /= bn;
        float q[4];
        qmul(qb, ql, q);
        for (int k = 0; k < 3; ++k) out.log_scales[k * n + i] = pca.log_scales[k * n + i] + yi[k];
        for (int k = 0; k < 4; ++k) out.quats[k * n + i] = q[k];
        out.opacity_logits[i] = pca.opacity_logits[i] + yi[7];
    } else {
        for (int k = 0; k < 3; ++k) out.log_scales[k * n + i] = pca.log_scales[k * n + i];
        for (int k = 0; k < 4; ++k) out.quats[k * n + i] = pca.quats[k * n + i];
        out.opacity_logits[i] = pca.opacity_logits[i];
        atomicAdd(fallbacks, 1u);
    }
}

// Training targets [n][8] of converged Gaussians relative to the paper's initializer `pca` of the
// same point: log-scale differences, conj(normalise(pca q)) (x) normalise(q), logit difference.
__global__ void k_make_targets(int64_t n, pgs_gaussians pca, pgs_gaussians conv, float* __restrict__ t) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    float q[4] = {conv.quats[i], conv.quats[n + i], conv.quats[2 * n + i], conv.quats[3 * n + i]};
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) q[k] /= qn;
    float qb[4] = {pca.quats[i], pca.quats[n + i], pca.quats[2 * n + i], pca.quats[3 * n + i]};
    const float bn = sqrtf(qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3]);
    const float qc[4] = {qb[0] / bn, -qb[1] / bn, -qb[2] / bn, -qb[3] / bn};
    float ql[4];
    qmul(qc, q, ql);
    for (int k = 0; k < 3; ++k) t[i * 8 + k] = conv.log_scales[k * n + i] - pca.log_scales[k * n + i];
    for (int k = 0; k < 4; ++k) t[i * 8 + 3 + k] = ql[k];
    t[i * 8 + 7] = conv.opacity_logits[i] - pca.opacity_logits[i];
}

}  // namespace

int launch_apply_mlp(int64_t n, const float* y, const pgs_gaussians& pca, pgs_gaussians& out,
                     uint32_t* fallbacks, cudaStream_t s) {
    if (n <= 0) return 0;
    k_apply_mlp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, y, pca, out, fallbacks);
    return 1;
}

int launch_make_targets(int64_t n, const pgs_gaussians& pca, const pgs_gaussians& conv, float* t,
                        cudaStream_t s) {
    if (n <= 0) return 0;
    k_make_targets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pca, conv, t);
    return 1;
}

// Scratch of the kNN: bbox (6 floats), cell of each point (n), counts / cursors (cells + 1),
// starts (cells + 1), sorted indices (n).  Returns the bytes needed for n points and `cells` cells.
size_t knn_scratch_bytes(int64_t n, int64_t cells) {
    return 256 + 4 * (size_t)n + 2 * 4 * (size_t)(cells + 1) + 4 * (size_t)n + 12 * (size_t)n + 5 * 256;
}

int launch_knn(int64_t n, const float* P, int k, int32_t* nb, void* scratch, size_t scratch_bytes,
               const float* host_bbox, cudaStream_t s) {
    if (n <= 0) return 0;
    // grid: cell edge from the bounding box volume per point (the ring search keeps it exact
    // whatever the density)
    const float ex = fmaxf(host_bbox[3] - host_bbox[0], 1e-6f), ey = fmaxf(host_bbox[4] - host_bbox[1], 1e-6f),
                ez = fmaxf(host_bbox[5] - host_bbox[2], 1e-6f);
    // a fine grid (about 2.4 cells per point over the bounding box): surface points fill few
    // cells densely, and fewer candidates per cell beat fewer, fuller cells
    float h = 0.75f * cbrtf(ex * ey * ez / (float)n);
    Grid g;
    for (int d = 0; d < 3; ++d) g.lo[d] = host_bbox[d];
    int64_t cells = 0;
    for (;;) {
        g.h = h;
        g.dim[0] = (int)fminf(1024.f, floorf(ex / h) + 1);
        g.dim[1] = (int)fminf(1024.f, floorf(ey / h) + 1);
        g.dim[2] = (int)fminf(1024.f, floorf(ez / h) + 1);
        cells = (int64_t)g.dim[0] * g.dim[1] * g.dim[2];
        if (knn_scratch_bytes(n, cells) <= scratch_bytes) break;
        h *= 1.25f;
    }
    char* base = static_cast<char*>(scratch);
    uint32_t* cell_of = reinterpret_cast<uint32_t*>(base + 256);
    uint32_t* counts = cell_of + n;
    uint32_t* start = counts + (cells + 1);
    uint32_t* sorted = start + (cells + 1);
    float* Ps = reinterpret_cast<float*>(base + ((256 + 4 * (size_t)n + 2 * 4 * (size_t)(cells + 1) +
                                                   4 * (size_t)n + 255) & ~(size_t)255));
    cudaMemsetAsync(counts, 0, 4 * (size_t)(cells + 1), s);
    const unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
    k_cell_count<<<blocks, kThreads, 0, s>>>(n, P, g, cell_of, counts);
    k_scan_cells<<<1, 1024, 0, s>>>(cells, counts, start);
    cudaMemcpyAsync(counts, start, 4 * (size_t)cells, cudaMemcpyDeviceToDevice, s);
    k_cell_scatter<<<blocks, kThreads, 0, s>>>(n, P, cell_of, counts, sorted, Ps);
    const unsigned qb = (unsigned)((n + 127) / 128);
    switch (k) {
        case 3: k_knn_query<3><<<qb, 128, 0, s>>>(n, P, g, start, sorted, Ps, nb); break;
        case 16: k_knn_query<16><<<qb, 128, 0, s>>>(n, P, g, start, sorted, Ps, nb); break;
        default: k_knn_query<32><<<qb, 128, 0, s>>>(n, P, g, start, sorted, Ps, nb); break;
    }
    return 4;
}

int launch_bbox(int64_t n, const float* P, int* bbox_dev, cudaStream_t s) {
    int enc[6];
    const float inf = 3.4e38f, ninf = -3.4e38f;
    int bi, bn;
    memcpy(&bi, &inf, 4);
    memcpy(&bn, &ninf, 4);
    for (int d = 0; d < 3; ++d) {
        enc[d] = ordered(bi);
        enc[3 + d] = ordered(bn);
    }
    cudaMemcpyAsync(bbox_dev, enc, sizeof(enc), cudaMemcpyHostToDevice, s);
    const int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, 1024);
    if (blocks > 0) k_bbox<<<(unsigned)blocks, kThreads, 0, s>>>(n, P, bbox_dev);
    return 1;
}

void decode_bbox(const int* enc, float* out) {
    for (int d = 0; d < 6; ++d) {
        const int b = ordered(enc[d]);
        memcpy(&out[d], &b, 4);
    }
}

int launch_features_init(int64_t n, const float* P, const int32_t* nb, float r_normal, float* feats,
                         void* feats_bf16, float* frame_q, pgs_gaussians& init, cudaStream_t s) {
    if (n <= 0) return 0;
    k_features_init<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
        n, P, nb, r_normal, feats, static_cast<__nv_bfloat16*>(feats_bf16), frame_q, init);
    return 1;
}

}  // namespace pgs
