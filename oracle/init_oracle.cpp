// Plain CPU oracle of the initializer path — TEST INFRASTRUCTURE ONLY (see pgs_oracle.cpp).
//
// Operator I of PocketGS (Sec. III-B, "Prior-Conditioned Gaussian Parameterization"):
//   * local surface statistics (Eq. 5): covariance of the K_n = 16 nearest neighbours about their
//     centroid; its smallest-eigenvalue eigenvector is the normal;
//   * disc-like seeding (Eq. 6): tangential scale s_t = mean distance to the K_s = 3 nearest
//     neighbours, normal scale r_normal s_t (r_normal = 0.1, a reading), z axis along the normal,
//     opacity logit(0.1);
// and the learned stand-in for it: 16 neighbourhood features from the 32 nearest neighbours and a
// 16-64-64-8 GELU MLP (BF16 weights and activations, FP32 accumulation), trained on converged
// Gaussians with loss |ls - t|^2 + (1 - <q, t_q>^2) + (logit - t)^2.
//
// Precision: neighbour decisions use squared distances in fp32 with a prescribed order
// (d2 = fma(dx, dx, fma(dy, dy, dz * dz)), dx = q - p in fp32), ties by index, so neighbour
// indices are reproducible bit for bit; statistics are FP64; the MLP is FP32 with BF16
// round-to-nearest-even wherever the GPU stores BF16 (inputs, weights, activations, and the
// gradients fed to the tensor-core products).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

float d2f(const float* P, int64_t n, int64_t i, int64_t j) {
    const float dx = P[j] - P[i];
    const float dy = P[n + j] - P[n + i];
    const float dz = P[2 * n + j] - P[2 * n + i];
    return std::fma(dx, dx, std::fma(dy, dy, dz * dz));
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (FP64).  Eigenvalues ascending;
// eigenvector columns V[:, k]; each eigenvector's largest-magnitude component made positive.
void jacobi3(const double A_in[3][3], double w[3], double V[3][3]) {
    double A[3][3];
    std::memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {  // A = J^T A J
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
    std::sort(idx, idx + 3, [&](int a, int b) { return A[a][a] < A[b][b]; });
    double W[3][3];
    for (int k = 0; k < 3; ++k) {
        w[k] = A[idx[k]][idx[k]];
        int big = 0;
        for (int r = 1; r < 3; ++r)
            if (std::fabs(V[r][idx[k]]) > std::fabs(V[big][idx[k]])) big = r;
        const double sg = V[big][idx[k]] < 0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) W[r][k] = sg * V[r][idx[k]];
    }
    std::memcpy(V, W, sizeof(W));
}

// covariance of the first k neighbours about their centroid (Eq. 5), FP64
void neighbour_cov(const float* P, int64_t n, int64_t i, const int32_t* nb, int k, double C[3][3],
                   double centroid[3]) {
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
    for (int d = 0; d < 3; ++d) centroid[d] = c[d];
}

double dist(const float* P, int64_t n, int64_t i, int64_t j) {
    double s = 0;
    for (int d = 0; d < 3; ++d) {
        const double v = (double)P[d * n + j] - (double)P[d * n + i];
        s += v * v;
    }
    return std::sqrt(s);
}

// quaternion (w, x, y, z) of a proper rotation matrix with columns = the rotated axes
void mat_to_quat(const double R[3][3], double q[4]) {
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr > 0) {
        const double s = std::sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * s;
        q[1] = (R[2][1] - R[1][2]) / s;
        q[2] = (R[0][2] - R[2][0]) / s;
        q[3] = (R[1][0] - R[0][1]) / s;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        const double s = std::sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2;
        q[0] = (R[2][1] - R[1][2]) / s;
        q[1] = 0.25 * s;
        q[2] = (R[0][1] + R[1][0]) / s;
        q[3] = (R[0][2] + R[2][0]) / s;
    } else if (R[1][1] > R[2][2]) {
        const double s = std::sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2;
        q[0] = (R[0][2] - R[2][0]) / s;
        q[1] = (R[0][1] + R[1][0]) / s;
        q[2] = 0.25 * s;
        q[3] = (R[1][2] + R[2][1]) / s;
    } else {
        const double s = std::sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2;
        q[0] = (R[1][0] - R[0][1]) / s;
        q[1] = (R[0][2] + R[2][0]) / s;
        q[2] = (R[1][2] + R[2][1]) / s;
        q[3] = 0.25 * s;
    }
}

float bf16(float x) {  // round to nearest even bfloat16, returned as float
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

constexpr int kIn = 16, kHid = 64, kOut = 8;

double gelu(double x) { return 0.5 * x * (1.0 + std::erf(x / std::sqrt(2.0))); }
double gelu_d(double x) {
    return 0.5 * (1.0 + std::erf(x / std::sqrt(2.0))) + x * std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
}

}  // namespace

extern "C" {

// k nearest neighbours of every point among the other points (brute force, fp32 prescribed
// squared distance, ties by index): nb [n][k] ascending by (distance, index).
void oracle_knn(int64_t n, const float* P, int k, int32_t* nb) {
    std::vector<std::pair<float, int32_t>> cand(n > 0 ? n - 1 : 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) cand[c++] = {d2f(P, n, i, j), (int32_t)j};
        const int kk = (int)std::min<int64_t>(k, c);
        std::partial_sort(cand.begin(), cand.begin() + kk, cand.begin() + c);
        for (int a = 0; a < k; ++a) nb[i * k + a] = a < kk ? cand[a].second : -1;
    }
}

// Jacobi eigen-decomposition of one symmetric 3x3 matrix (row-major A[9]): w[3] ascending,
// V[9] row-major with eigenvector columns.
void oracle_eig3(const double* A, double* w, double* V) {
    double M[3][3], VV[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = A[3 * a + b];
    jacobi3(M, w, VV);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) V[3 * a + b] = VV[a][b];
}

// Paper initializer (Eq. 5, Eq. 6) from 32-neighbour lists nb [n][32] (ascending): normal from
// the first 16, tangential scale from the first 3.  Outputs per point: log_scales [3][n]
// (log s_t, log s_t, log(r_normal s_t)), quats [4][n] (z axis -> normal, minimal rotation;
// 180 degrees about x if the normal is -z), logits [n] = logit(0.1).
void oracle_pca_init(int64_t n, const float* P, const int32_t* nb, int knb, double r_normal,
                     double* log_scales, double* quats, double* logits) {
    for (int64_t i = 0; i < n; ++i) {
        double C[3][3], cen[3], w[3], V[3][3];
        neighbour_cov(P, n, i, nb + i * knb, 16, C, cen);
        jacobi3(C, w, V);
        const double nrm[3] = {V[0][0], V[1][0], V[2][0]};
        double st = 0;
        for (int a = 0; a < 3; ++a) st += dist(P, n, i, nb[i * knb + a]);
        st /= 3.0;
        log_scales[i] = std::log(st);
        log_scales[n + i] = std::log(st);
        log_scales[2 * n + i] = std::log(r_normal * st);
        double q[4];
        const double c = nrm[2];  // cos of the angle between +z and n
        if (c < -1.0 + 1e-12) {
            q[0] = 0; q[1] = 1; q[2] = 0; q[3] = 0;
        } else {
            // rotation axis z x n = (-n_y, n_x, 0), half-angle form
            q[0] = std::sqrt(0.5 * (1.0 + c));
            const double s = 1.0 / (2.0 * q[0]);
            q[1] = -nrm[1] * s;
            q[2] = nrm[0] * s;
            q[3] = 0.0;
        }
        for (int a = 0; a < 4; ++a) quats[a * n + i] = q[a];
        logits[i] = std::log(0.1 / 0.9);
    }
}

// 16 features per point from its 32 nearest neighbours: eigenvalues of the centred covariance
// ascending and divided by their sum (3); the three canonicalised eigenvectors, smallest first,
// each (x, y, z) (9); mean of the offsets p_k - p_i divided by the mean neighbour distance (3);
// -3 log(mean neighbour distance) (1).  Also the quaternion of the eigenframe (columns largest,
// middle, smallest eigenvector, made proper) in frame_q [4][n].  feats [n][16].
void oracle_features(int64_t n, const float* P, const int32_t* nb, int knb, double* feats,
                     double* frame_q) {
    for (int64_t i = 0; i < n; ++i) {
        double C[3][3], cen[3], w[3], V[3][3];
        neighbour_cov(P, n, i, nb + i * knb, 32, C, cen);
        jacobi3(C, w, V);
        double* f = feats + i * 16;
        const double sum = w[0] + w[1] + w[2];
        for (int a = 0; a < 3; ++a) f[a] = sum > 0 ? w[a] / sum : 1.0 / 3.0;
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) f[3 + 3 * k + d] = V[d][k];
        double md = 0, off[3] = {0, 0, 0};
        for (int a = 0; a < 32; ++a) {
            md += dist(P, n, i, nb[i * knb + a]);
            for (int d = 0; d < 3; ++d) off[d] += (double)P[d * n + nb[i * knb + a]] - P[d * n + i];
        }
        md /= 32.0;
        for (int d = 0; d < 3; ++d) f[12 + d] = off[d] / 32.0 / md;
        f[15] = -3.0 * std::log(md);
        // eigenframe: x = largest, y = middle, z = smallest (normal); flip x to make it proper
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
        for (int a = 0; a < 4; ++a) frame_q[a * n + i] = q[a];
    }
}

// MLP 16-64-64-8, exact GELU, y = W3 g(W2 g(W1 x + b1) + b2) + b3; weights row-major [out][in].
// mode 1: FP32 with BF16 rounding of x, weights, hidden activations (the GPU's storage);
// mode 0: FP64 without rounding (for finite differences).  out [n][8].
void oracle_mlp_forward(int64_t n, const float* x, const float* W1, const float* b1, const float* W2,
                        const float* b2, const float* W3, const float* b3, int mode, double* out) {
    auto r = [&](double v) { return mode ? (double)bf16((float)v) : v; };
    for (int64_t p = 0; p < n; ++p) {
        double h1[kHid], h2[kHid];
        for (int o = 0; o < kHid; ++o) {
            double acc = 0;
            for (int k = 0; k < kIn; ++k) acc += r(W1[o * kIn + k]) * r(x[p * kIn + k]);
            h1[o] = r(gelu(mode ? (double)(float)(acc + b1[o]) : acc + b1[o]));
        }
        for (int o = 0; o < kHid; ++o) {
            double acc = 0;
            for (int k = 0; k < kHid; ++k) acc += r(W2[o * kHid + k]) * h1[k];
            h2[o] = r(gelu(mode ? (double)(float)(acc + b2[o]) : acc + b2[o]));
        }
        for (int o = 0; o < kOut; ++o) {
            double acc = 0;
            for (int k = 0; k < kHid; ++k) acc += r(W3[o * kHid + k]) * h2[k];
            out[p * kOut + o] = acc + b3[o];
        }
    }
}

// Loss of the initializer (summed over points, divided by n): |y[0:3] - t[0:3]|^2
// + (1 - <y[3:7]/|y[3:7]|, t[3:7]>^2) + (y[7] - t[7])^2, targets t [n][8] (unit quaternions).
// dy [n][8] receives dLoss/dy.  Returns the loss.
double oracle_init_loss(int64_t n, const double* y, const float* t, double* dy) {
    double L = 0;
    for (int64_t p = 0; p < n; ++p) {
        const double* a = y + p * 8;
        const float* b = t + p * 8;
        double* g = dy + p * 8;
        for (int k = 0; k < 3; ++k) {
            const double d = a[k] - b[k];
            L += d * d;
            g[k] = 2 * d / n;
        }
        const double qn = std::sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5] + a[6] * a[6]);
        double f = 0;
        for (int k = 0; k < 4; ++k) f += a[3 + k] / qn * b[3 + k];
        L += 1 - f * f;
        double dqh[4], dot = 0;
        for (int k = 0; k < 4; ++k) {
            dqh[k] = -2 * f * b[3 + k];
            dot += dqh[k] * a[3 + k] / qn;
        }
        for (int k = 0; k < 4; ++k) g[3 + k] = (dqh[k] - a[3 + k] / qn * dot) / qn / n;
        const double d = a[7] - b[7];
        L += d * d;
        g[7] = 2 * d / n;
    }
    return L / n;
}

// Backward of the MLP for upstream dy [n][8]; weight gradients (same layouts) overwritten.
// mode as in oracle_mlp_forward; in mode 1 the upstream gradient and the hidden-layer gradients
// are rounded to BF16 where the GPU feeds them to the tensor-core products (the bias gradients
// and the GELU derivative use the unrounded FP32 values).
void oracle_mlp_backward(int64_t n, const float* x, const float* W1, const float* b1, const float* W2,
                         const float* b2, const float* W3, const float* b3, const double* dy, int mode,
                         double* dW1, double* db1, double* dW2, double* db2, double* dW3, double* db3) {
    (void)b3;  // the output bias does not enter any gradient
    auto r = [&](double v) { return mode ? (double)bf16((float)v) : v; };
    std::fill(dW1, dW1 + kHid * kIn, 0.0);
    std::fill(dW2, dW2 + kHid * kHid, 0.0);
    std::fill(dW3, dW3 + kOut * kHid, 0.0);
    std::fill(db1, db1 + kHid, 0.0);
    std::fill(db2, db2 + kHid, 0.0);
    std::fill(db3, db3 + kOut, 0.0);
    for (int64_t p = 0; p < n; ++p) {
        double xi[kIn], z1[kHid], h1[kHid], z2[kHid], h2[kHid];
        for (int k = 0; k < kIn; ++k) xi[k] = r(x[p * kIn + k]);
        for (int o = 0; o < kHid; ++o) {
            double acc = 0;
            for (int k = 0; k < kIn; ++k) acc += r(W1[o * kIn + k]) * xi[k];
            z1[o] = mode ? (double)(float)(acc + b1[o]) : acc + b1[o];
            h1[o] = r(gelu(z1[o]));
        }
        for (int o = 0; o < kHid; ++o) {
            double acc = 0;
            for (int k = 0; k < kHid; ++k) acc += r(W2[o * kHid + k]) * h1[k];
            z2[o] = mode ? (double)(float)(acc + b2[o]) : acc + b2[o];
            h2[o] = r(gelu(z2[o]));
        }
        double g3[kOut], g3r[kOut];
        for (int o = 0; o < kOut; ++o) {
            g3[o] = dy[p * kOut + o];
            g3r[o] = r(g3[o]);
            db3[o] += g3[o];
            for (int k = 0; k < kHid; ++k) dW3[o * kHid + k] += g3r[o] * h2[k];
        }
        double dz2[kHid], dz2r[kHid];
        for (int k = 0; k < kHid; ++k) {
            double acc = 0;
            for (int o = 0; o < kOut; ++o) acc += g3r[o] * r(W3[o * kHid + k]);
            dz2[k] = acc * gelu_d(z2[k]);
            dz2r[k] = r(dz2[k]);
            db2[k] += dz2[k];
            for (int j = 0; j < kHid; ++j) dW2[k * kHid + j] += dz2r[k] * h1[j];
        }
        for (int j = 0; j < kHid; ++j) {
            double acc = 0;
            for (int k = 0; k < kHid; ++k) acc += dz2r[k] * r(W2[k * kHid + j]);
            const double dz1 = acc * gelu_d(z1[j]);
            db1[j] += dz1;
            const double dz1r = r(dz1);
            for (int k = 0; k < kIn; ++k) dW1[j * kIn + k] += dz1r * xi[k];
        }
    }
}

static void qmul(const double a[4], const double b[4], double o[4]) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Learned parameters from MLP outputs y [n][8], as corrections of the paper's initializer of the
// same point (base: log-scales [3][n], quaternions [4][n], logits [n]): log-scales base + y0..2,
// rotation normalise(base q) (x) normalise(y3..6), logit base + y7.
void oracle_apply_mlp(int64_t n, const double* y, const double* base_ls, const double* base_q,
                      const double* base_logit, double* log_scales, double* quats, double* logits) {
    for (int64_t i = 0; i < n; ++i) {
        const double* a = y + i * 8;
        const double qn = std::sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5] + a[6] * a[6]);
        const double ql[4] = {a[3] / qn, a[4] / qn, a[5] / qn, a[6] / qn};
        double qb[4] = {base_q[i], base_q[n + i], base_q[2 * n + i], base_q[3 * n + i]};
        const double bn = std::sqrt(qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3]);
        for (int k = 0; k < 4; ++k) qb[k] /= bn;
        double q[4];
        qmul(qb, ql, q);
        for (int k = 0; k < 3; ++k) log_scales[k * n + i] = base_ls[k * n + i] + a[k];
        for (int k = 0; k < 4; ++k) quats[k * n + i] = q[k];
        logits[i] = base_logit[i] + a[7];
    }
}

// Targets [n][8] of converged Gaussians relative to the paper's initializer of the same point:
// log-scale differences, conj(normalise(base q)) (x) normalise(q), logit difference.
void oracle_make_targets(int64_t n, const double* base_ls, const double* base_q, const double* base_logit,
                         const double* log_scales, const double* quats, const double* logits, double* t) {
    for (int64_t i = 0; i < n; ++i) {
        double q[4] = {quats[i], quats[n + i], quats[2 * n + i], quats[3 * n + i]};
        const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int k = 0; k < 4; ++k) q[k] /= qn;
        double qb[4] = {base_q[i], base_q[n + i], base_q[2 * n + i], base_q[3 * n + i]};
        const double bn = std::sqrt(qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3]);
        const double qc[4] = {qb[0] / bn, -qb[1] / bn, -qb[2] / bn, -qb[3] / bn};
        double ql[4];
        qmul(qc, q, ql);
        for (int k = 0; k < 3; ++k) t[i * 8 + k] = log_scales[k * n + i] - base_ls[k * n + i];
        for (int k = 0; k < 4; ++k) t[i * 8 + 3 + k] = ql[k];
        t[i * 8 + 7] = logits[i] - base_logit[i];
    }
}

}  // extern "C"
