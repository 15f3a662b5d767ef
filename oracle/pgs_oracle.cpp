// Plain, slow CPU oracle for the differentiable tile-based Gaussian rasterizer.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file; only the tests,
// the smoke check and the benchmark's CPU-baseline leg load it.  It shares no code, header or
// constant table with the CUDA library: every formula below is written out again from the paper
// and from the numerics readings that fix what the paper leaves open.
//
// What it computes (PocketGS, Sec. III-C "Hardware-Aligned Differentiable Splatting"):
//   * per Gaussian: the projection of the canonical parameters (mu, Sigma, c, alpha) [Fig. 2,
//     Sec. III-C] to a screen-space ellipse, its tile rectangle and its depth;
//   * per pixel: the depth-ordered alpha composite of the Gaussians whose tile rectangle holds the
//     pixel's tile, i.e. the recurrence of Eq. 7 (C_out = C_in (1 - a) + a c) evaluated front to
//     back with transmittance T, plus a back-to-front Eq. 7 form as a cross-check;
//   * the (tile | depth) keys and per-tile ranges that a GPU sort produces (the permutation pi of
//     Eq. 10), by enumeration and std::stable_sort;
//   * the analytic backward: Eq. 8 (dL/dC_in, dL/dc, dL/dalpha) and a second, independent direct
//     differentiation of the front-to-back sum, scattered to canonical indices (Eq. 10), then
//     chained to the parameters;
//   * the textbook Adam update (Kingma & Ba 2015) that keeps moments aligned with the canonical
//     parameters (Sec. III-C, gradient scattering paragraph);
//   * the L1 image loss and its gradient (the paper names no loss).
//
// Precision: decision quantities (depth, screen position, 2-D covariance, radii, tile rectangle)
// are computed in fp32 with a prescribed operation order (each +, -, *, / and sqrt correctly
// rounded, fma fused, compiled with -ffp-contract=off), so that keys are reproducible bit for bit
// by any IEEE implementation of the same sequence.  Everything else is FP64.
//
// Readings of points the paper leaves open (all listed in the design notes):
//   projection model = pinhole + first-order (EWA) covariance projection with 0.3 px^2 dilation;
//   near cull z <= near; Jacobian at x/z, y/z clamped to +-1.3 tan(half FoV) with zero gradient
//   through the clamp; pixel i covers [i, i+1), centre i + 0.5; tile rectangle from the radii
//   ceil(3 sqrt(Sigma_xx)), ceil(3 sqrt(Sigma_yy)) (the box of the 3-sigma ellipse), and of its
//   tiles those whose pixel-centre box the 3-sigma ellipse reaches;
//   alpha = min(0.99, o exp(power)), skip if alpha < 1/255, stop before compositing when
//   T (1 - alpha) < 1e-4; colour = real orthonormal SH (no Condon-Shortley phase) + 0.5, clamped
//   at 0; ties in depth broken by canonical index.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <omp.h>
#include <unordered_map>
#include <vector>

extern "C" {

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float view[12];  // row-major 3x4 world -> camera [R | t], OpenCV axes
    float near_z;
    float bg[3];
} ocam_t;

typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t pad_;
    const float* means;       // [3][n]
    const float* log_scales;  // [3][n]
    const float* quats;       // [4][n]  (w, x, y, z), unnormalised
    const float* logits;      // [n]
    const float* sh;          // [3][K][n], K = (sh_degree + 1)^2
} ogauss_t;

}  // extern "C"

namespace {

// ------------------------------------------------------------------------------------------------
// fp32 decision path
// ------------------------------------------------------------------------------------------------

// exp in fp32 by Cody-Waite range reduction and a degree-7 Taylor polynomial:
//   k = rint(x * log2 e);  r = x - k ln2 (ln2 split hi + lo, each step one fma);
//   p(r) = sum_{i<=7} r^i / i!  (Horner, fma);  exp(x) = p(r) * 2^k  (exact power-of-two scaling).
// Every step is a correctly rounded IEEE operation, so the result is reproducible bit for bit.
float det_expf(float x) {
    if (x != x) return x;
    if (x < -87.0f) x = -87.0f;
    if (x > 88.0f) x = 88.0f;
    const float k = std::rint(x * 0x1.715476p+0f);
    float r = std::fma(-k, 0x1.62e4p-1f, x);
    r = std::fma(-k, 0x1.7f7d1cp-20f, r);
    float p = 0x1.a01a02p-13f;           // 1/7!
    p = std::fma(p, r, 0x1.6c16c2p-10f);  // 1/6!
    p = std::fma(p, r, 0x1.111112p-7f);   // 1/5!
    p = std::fma(p, r, 0x1.555556p-5f);   // 1/4!
    p = std::fma(p, r, 0x1.555556p-3f);   // 1/3!
    p = std::fma(p, r, 0.5f);
    p = std::fma(p, r, 1.0f);
    p = std::fma(p, r, 1.0f);
    const int32_t ki = (int32_t)k;
    const uint32_t bits = (uint32_t)(ki + 127) << 23;
    float scale;
    std::memcpy(&scale, &bits, 4);
    return p * scale;
}

struct Decision {
    bool visible = false;
    float xc = 0, yc = 0, zc = 0;
    float u = 0, v = 0;
    float cov_a = 0, cov_b = 0, cov_c = 0, det = 0;
    int32_t radius_x = 0, radius_y = 0;
    int32_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    float ca = 0, cb = 0, cc = 0;  // conic (inverse 2-D covariance), fp32 decision path
    int32_t hits = 0;              // tiles of the rectangle the 3-sigma ellipse reaches
};

inline float fclampf(float x, float lo, float hi) { return std::fmin(std::fmax(x, lo), hi); }

// Does the 3-sigma ellipse {Q <= 9}, Q(X, Y) = (X - u, Y - v) conic (X - u, Y - v)^T, reach a pixel
// centre box of tile (tx, ty)?  The minimum of the convex Q over the box is at the clamped centre
// or on an edge at the clamped line minimum; fp32 in this order, every operation rounded.
inline bool tile_hit(const Decision& d, int tx, int ty, int tile) {
    const float xl = (float)(tx * tile) + 0.5f, xh = (float)(tx * tile + tile) - 0.5f;
    const float yl = (float)(ty * tile) + 0.5f, yh = (float)(ty * tile + tile) - 0.5f;
    auto Q = [&](float X, float Y) {
        const float dx = X - d.u, dy = Y - d.v;
        return (((d.ca * dx) * dx) + (((d.cb + d.cb) * dx) * dy)) + ((d.cc * dy) * dy);
    };
    const float sy = d.cb / d.cc, sx = d.cb / d.ca;
    float best = Q(fclampf(d.u, xl, xh), fclampf(d.v, yl, yh));
    best = std::fmin(best, Q(xl, fclampf(d.v - sy * (xl - d.u), yl, yh)));
    best = std::fmin(best, Q(xh, fclampf(d.v - sy * (xh - d.u), yl, yh)));
    best = std::fmin(best, Q(fclampf(d.u - sx * (yl - d.v), xl, xh), yl));
    best = std::fmin(best, Q(fclampf(d.u - sx * (yh - d.v), xl, xh), yh));
    return best <= 9.0f;
}

// The prescribed fp32 sequence for every quantity that decides membership and order.
Decision decide(const ogauss_t& G, const ocam_t& cam, int tile, int64_t i) {
    Decision d;
    const int64_t n = G.n;
    const float mx = G.means[i], my = G.means[n + i], mz = G.means[2 * n + i];
    const float* V = cam.view;
    // camera coordinates: x_c = r00 mx + r01 my + r02 mz + t0, innermost term first
    d.xc = std::fma(V[0], mx, std::fma(V[1], my, std::fma(V[2], mz, V[3])));
    d.yc = std::fma(V[4], mx, std::fma(V[5], my, std::fma(V[6], mz, V[7])));
    d.zc = std::fma(V[8], mx, std::fma(V[9], my, std::fma(V[10], mz, V[11])));
    if (!(d.zc > cam.near_z)) return d;
    const float tx = d.xc / d.zc, ty = d.yc / d.zc;
    d.u = std::fma(cam.fx, tx, cam.cx);
    d.v = std::fma(cam.fy, ty, cam.cy);
    if (!std::isfinite(d.u) || !std::isfinite(d.v)) return d;

    // rotation from the normalised quaternion
    const float qw = G.quats[i], qx = G.quats[n + i], qy = G.quats[2 * n + i], qz = G.quats[3 * n + i];
    const float n2 = std::fma(qw, qw, std::fma(qx, qx, std::fma(qy, qy, qz * qz)));
    if (!(n2 > 0.0f) || !std::isfinite(n2)) return d;
    const float qn = std::sqrt(n2);
    const float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    const float s[3] = {det_expf(G.log_scales[i]), det_expf(G.log_scales[n + i]),
                        det_expf(G.log_scales[2 * n + i])};
    float M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) M[a][k] = R[a][k] * s[k];
    float S[3][3];  // Sigma = M M^T
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) {
            S[a][b] = std::fma(M[a][0], M[b][0], std::fma(M[a][1], M[b][1], M[a][2] * M[b][2]));
            S[b][a] = S[a][b];
        }
    // Jacobian of the pinhole at the clamped normalised coordinates
    const float limx = 1.3f * ((0.5f * (float)cam.width) / cam.fx);
    const float limy = 1.3f * ((0.5f * (float)cam.height) / cam.fy);
    const float cxh = fclampf(tx, -limx, limx), cyh = fclampf(ty, -limy, limy);
    const float j00 = cam.fx / d.zc;
    const float j02 = -((cam.fx * cxh) / d.zc);
    const float j11 = cam.fy / d.zc;
    const float j12 = -((cam.fy * cyh) / d.zc);
    float T[2][3];  // T = J W, W = world-to-camera rotation
    for (int k = 0; k < 3; ++k) {
        T[0][k] = std::fma(j00, V[k], j02 * V[8 + k]);
        T[1][k] = std::fma(j11, V[4 + k], j12 * V[8 + k]);
    }
    float A[2][3];  // A = T Sigma
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k)
            A[a][k] = std::fma(T[a][0], S[0][k], std::fma(T[a][1], S[1][k], T[a][2] * S[2][k]));
    d.cov_a = std::fma(A[0][0], T[0][0], std::fma(A[0][1], T[0][1], A[0][2] * T[0][2])) + 0.3f;
    d.cov_b = std::fma(A[0][0], T[1][0], std::fma(A[0][1], T[1][1], A[0][2] * T[1][2]));
    d.cov_c = std::fma(A[1][0], T[1][0], std::fma(A[1][1], T[1][1], A[1][2] * T[1][2])) + 0.3f;
    d.det = (d.cov_a * d.cov_c) - (d.cov_b * d.cov_b);
    if (!(d.det > 0.0f) || !std::isfinite(d.det)) return d;
    // per-axis 3-sigma extents: the bounding box of the 3-sigma ellipse of the 2-D covariance
    const float rx = std::ceil(3.0f * std::sqrt(d.cov_a));
    const float ry = std::ceil(3.0f * std::sqrt(d.cov_c));
    if (!std::isfinite(rx) || !std::isfinite(ry)) return d;
    const float tf = (float)tile;
    const int32_t TX = (cam.width + tile - 1) / tile, TY = (cam.height + tile - 1) / tile;
    d.x0 = (int32_t)fclampf(std::floor((d.u - rx) / tf), 0.0f, (float)TX);
    d.x1 = (int32_t)fclampf(std::floor((d.u + rx) / tf) + 1.0f, 0.0f, (float)TX);
    d.y0 = (int32_t)fclampf(std::floor((d.v - ry) / tf), 0.0f, (float)TY);
    d.y1 = (int32_t)fclampf(std::floor((d.v + ry) / tf) + 1.0f, 0.0f, (float)TY);
    d.radius_x = (int32_t)rx;
    d.radius_y = (int32_t)ry;
    const float inv = 1.0f / d.det;
    d.ca = d.cov_c * inv;
    d.cb = -d.cov_b * inv;
    d.cc = d.cov_a * inv;
    for (int ty = d.y0; ty < d.y1; ++ty)
        for (int tx = d.x0; tx < d.x1; ++tx) d.hits += tile_hit(d, tx, ty, tile);
    d.visible = d.hits > 0;
    return d;
}

inline uint32_t fbits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

// ------------------------------------------------------------------------------------------------
// FP64 value path
// ------------------------------------------------------------------------------------------------

// Real orthonormal spherical harmonics up to degree 3 as polynomials in the unit direction
// (x, y, z); index k = l^2 + l + m, m = -l..l, no Condon-Shortley phase.  Constants from the
// closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) with the usual real-form factors.
void sh_basis(const double d[3], double Y[16], double dY[16][3]) {
    const double pi = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    const double k0 = 0.5 / std::sqrt(pi);
    const double k1 = std::sqrt(3.0 / (4.0 * pi));
    const double k2a = 0.5 * std::sqrt(15.0 / pi);
    const double k2b = 0.25 * std::sqrt(5.0 / pi);
    const double k2c = 0.25 * std::sqrt(15.0 / pi);
    const double k3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * std::sqrt(105.0 / pi);
    const double k3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * std::sqrt(7.0 / pi);
    const double k3e = 0.25 * std::sqrt(105.0 / pi);
    const double val[16] = {
        k0,
        k1 * y, k1 * z, k1 * x,
        k2a * x * y, k2a * y * z, k2b * (3 * z * z - 1), k2a * x * z, k2c * (x * x - y * y),
        k3a * y * (3 * x * x - y * y), k3b * x * y * z, k3c * y * (5 * z * z - 1),
        k3d * z * (5 * z * z - 3), k3c * x * (5 * z * z - 1), k3e * z * (x * x - y * y),
        k3a * x * (x * x - 3 * y * y)};
    const double grad[16][3] = {
        {0, 0, 0},
        {0, k1, 0}, {0, 0, k1}, {k1, 0, 0},
        {k2a * y, k2a * x, 0}, {0, k2a * z, k2a * y}, {0, 0, k2b * 6 * z}, {k2a * z, 0, k2a * x},
        {k2c * 2 * x, -k2c * 2 * y, 0},
        {k3a * 6 * x * y, k3a * (3 * x * x - 3 * y * y), 0},
        {k3b * y * z, k3b * x * z, k3b * x * y},
        {0, k3c * (5 * z * z - 1), k3c * 10 * y * z},
        {0, 0, k3d * (15 * z * z - 3)},
        {k3c * (5 * z * z - 1), 0, k3c * 10 * x * z},
        {k3e * 2 * x * z, -k3e * 2 * y * z, k3e * (x * x - y * y)},
        {k3a * (3 * x * x - 3 * y * y), -k3a * 6 * x * y, 0}};
    for (int k = 0; k < 16; ++k) {
        Y[k] = val[k];
        if (dY)
            for (int c = 0; c < 3; ++c) dY[k][c] = grad[k][c];
    }
}

struct Value {
    // camera-space point, normalised quaternion, rotation, scales, covariances
    double pc[3];
    double qn, qh[4];
    double R[3][3], s[3], M[3][3], Sig[3][3];
    double tx, ty, cxh, cyh;
    bool xclamped, yclamped;
    double J00, J02, J11, J12;
    double T[2][3];
    double A, B, C, D;  // 2-D covariance [[A, B], [B, C]] and its determinant
    double u, v;
    double conic[3];  // (a, b, c) with power = -1/2 (a dx^2 + c dy^2) - b dx dy
    double opacity;
    double dir[3], dist;
    double raw[3], rgb[3];
    bool clamped[3];
    double Y[16], dY[16][3];
};

Value evaluate(const ogauss_t& G, const ocam_t& cam, int64_t i) {
    Value q;
    const int64_t n = G.n;
    const double mu[3] = {G.means[i], G.means[n + i], G.means[2 * n + i]};
    double W[3][3], t[3];
    for (int a = 0; a < 3; ++a) {
        for (int k = 0; k < 3; ++k) W[a][k] = cam.view[4 * a + k];
        t[a] = cam.view[4 * a + 3];
    }
    for (int a = 0; a < 3; ++a) q.pc[a] = W[a][0] * mu[0] + W[a][1] * mu[1] + W[a][2] * mu[2] + t[a];
    const double z = q.pc[2];
    q.tx = q.pc[0] / z;
    q.ty = q.pc[1] / z;
    q.u = (double)cam.fx * q.tx + (double)cam.cx;
    q.v = (double)cam.fy * q.ty + (double)cam.cy;

    const double qr[4] = {G.quats[i], G.quats[n + i], G.quats[2 * n + i], G.quats[3 * n + i]};
    q.qn = std::sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    for (int k = 0; k < 4; ++k) q.qh[k] = qr[k] / q.qn;
    const double w = q.qh[0], x = q.qh[1], y = q.qh[2], zq = q.qh[3];
    q.R[0][0] = 1 - 2 * (y * y + zq * zq);
    q.R[0][1] = 2 * (x * y - w * zq);
    q.R[0][2] = 2 * (x * zq + w * y);
    q.R[1][0] = 2 * (x * y + w * zq);
    q.R[1][1] = 1 - 2 * (x * x + zq * zq);
    q.R[1][2] = 2 * (y * zq - w * x);
    q.R[2][0] = 2 * (x * zq - w * y);
    q.R[2][1] = 2 * (y * zq + w * x);
    q.R[2][2] = 1 - 2 * (x * x + y * y);
    for (int k = 0; k < 3; ++k) q.s[k] = std::exp((double)G.log_scales[k * n + i]);
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) q.M[a][k] = q.R[a][k] * q.s[k];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            q.Sig[a][b] = q.M[a][0] * q.M[b][0] + q.M[a][1] * q.M[b][1] + q.M[a][2] * q.M[b][2];

    const double limx = 1.3 * (0.5 * cam.width / (double)cam.fx);
    const double limy = 1.3 * (0.5 * cam.height / (double)cam.fy);
    q.xclamped = q.tx < -limx || q.tx > limx;
    q.yclamped = q.ty < -limy || q.ty > limy;
    q.cxh = std::min(std::max(q.tx, -limx), limx);
    q.cyh = std::min(std::max(q.ty, -limy), limy);
    q.J00 = cam.fx / z;
    q.J02 = -cam.fx * q.cxh / z;
    q.J11 = cam.fy / z;
    q.J12 = -cam.fy * q.cyh / z;
    for (int k = 0; k < 3; ++k) {
        q.T[0][k] = q.J00 * W[0][k] + q.J02 * W[2][k];
        q.T[1][k] = q.J11 * W[1][k] + q.J12 * W[2][k];
    }
    double A = 0, B = 0, C = 0;
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k) {
            A += q.T[0][m] * q.Sig[m][k] * q.T[0][k];
            B += q.T[0][m] * q.Sig[m][k] * q.T[1][k];
            C += q.T[1][m] * q.Sig[m][k] * q.T[1][k];
        }
    q.A = A + 0.3;
    q.B = B;
    q.C = C + 0.3;
    q.D = q.A * q.C - q.B * q.B;
    q.conic[0] = q.C / q.D;
    q.conic[1] = -q.B / q.D;
    q.conic[2] = q.A / q.D;
    q.opacity = 1.0 / (1.0 + std::exp(-(double)G.logits[i]));

    // colour: direction from the camera centre c = -W^T t to the mean
    double cc[3];
    for (int k = 0; k < 3; ++k) cc[k] = -(W[0][k] * t[0] + W[1][k] * t[1] + W[2][k] * t[2]);
    double dv[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    q.dist = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int k = 0; k < 3; ++k) q.dir[k] = dv[k] / q.dist;
    sh_basis(q.dir, q.Y, q.dY);
    const int K = (G.sh_degree + 1) * (G.sh_degree + 1);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += (double)G.sh[((int64_t)c * K + k) * n + i] * q.Y[k];
        q.raw[c] = acc;
        q.clamped[c] = acc < 0.0;
        q.rgb[c] = q.clamped[c] ? 0.0 : acc;
    }
    return q;
}

// ------------------------------------------------------------------------------------------------
// per-tile lists and per-pixel compositing
// ------------------------------------------------------------------------------------------------

struct Scene {
    const ogauss_t& G;
    const ocam_t& cam;
    int tile;
    int TX, TY;
    std::vector<Decision> dec;
    std::vector<Value> val;
    std::vector<std::vector<int64_t>> lists;  // per tile, sorted by (depth bits, canonical id)
    Scene(const ogauss_t& g, const ocam_t& c, int t) : G(g), cam(c), tile(t) {
        TX = (cam.width + tile - 1) / tile;
        TY = (cam.height + tile - 1) / tile;
        dec.resize(G.n);
        val.resize(G.n);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < G.n; ++i) {
            dec[i] = decide(G, cam, tile, i);
            if (dec[i].visible) val[i] = evaluate(G, cam, i);
        }
        // membership: Gaussian i belongs to the list of every tile of its rectangle that its
        // 3-sigma ellipse reaches
        lists.assign((size_t)TX * TY, {});
        for (int64_t i = 0; i < G.n; ++i) {
            if (!dec[i].visible) continue;
            for (int ty = dec[i].y0; ty < dec[i].y1; ++ty)
                for (int tx = dec[i].x0; tx < dec[i].x1; ++tx)
                    if (tile_hit(dec[i], tx, ty, tile)) lists[(size_t)ty * TX + tx].push_back(i);
        }
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = 0; t < (int64_t)lists.size(); ++t)
            std::sort(lists[t].begin(), lists[t].end(), [&](int64_t a, int64_t b) {
                const uint32_t da = fbits(dec[a].zc), db = fbits(dec[b].zc);
                return da != db ? da < db : a < b;
            });
    }
    const std::vector<int64_t>& list_of(int px, int py) const {
        return lists[(size_t)(py / tile) * TX + (px / tile)];
    }
};

// Compositing decisions.  Whether an entry is skipped (alpha < 1/255), clamped (o G > 0.99) or
// stops the pixel (T (1 - alpha) < 1e-4) is an integer outcome decided in floating point, so the
// oracle takes it in the kernel's precision, fp32, from the fp32 quantities of the decision path
// (screen position u, v and conic of decide()), in the compositing kernels' evaluation order:
//   dx = fl(x + 1/2 - u), dy = fl(y + 1/2 - v);
//   exponent base 2: A = fl(-log2(e)/2 a), B = fl(-log2(e) b), C = fl(-log2(e)/2 c) (log2(e) in
//   fp32), p = fma(C, fl(dy dy), fma(B, fl(dx dy), fl(A fl(dx dx))));
//   og = o 2^p,  alpha = min(0.99f, og),  skip alpha < fl(1/255),  T' = fl(T fl(1 - alpha)),
//   stop when T' < 1e-4f.
// Two steps of the kernel are not reproducible bit for bit: its 2^p is a hardware approximation
// and its opacity goes through the library exp.  The oracle evaluates og from the exact 2^p and
// the FP64 opacity and carries the kernel's possible deviation as a bound: |og_k / og - 1| <=
// EPS_OG, and a running relative bound on its fp32 transmittance chain.  A decision whose
// threshold lies inside that bound is ambiguous: the pixel is flagged (FLAG_*), and a test can
// replay the kernel's own decisions for it (composite with forced decisions), each forced
// decision that differs from the oracle's being checked to be an ambiguous one.
// Values (the composited alpha, colour and transmittance) stay FP64, from the value path.
enum { FLAG_SKIP = 1, FLAG_STOP = 2, FLAG_CLAMP = 4 };
constexpr double ALPHA_MIN = (double)(1.0f / 255.0f), ALPHA_MAX = (double)0.99f, T_MIN = (double)1e-4f;
constexpr double U32 = 0x1p-24;                  // unit roundoff of fp32
constexpr double EPS_EX2 = 0x1p-21;              // hardware 2^x approximation, relative
constexpr double EPS_OPACITY = 4.0 * 0x1p-23;    // fp32 logistic 1 / (1 + exp(-x)) via the library exp
constexpr double EPS_OG = EPS_EX2 + EPS_OPACITY + U32;  // the kernel's o G against o 2^p
constexpr float LOG2E_F = 1.4426950408889634f;

// decision codes of one evaluated list entry (as a kernel trace reports them)
enum { CODE_SKIP = 0, CODE_COMPOSITE = 1, CODE_CLAMPED = 2, CODE_STOP = 3 };

struct Entry {
    int64_t g;
    double alpha, G, T;  // T = transmittance in front of the entry
    double dx, dy;
    bool clamped;
};

struct PixelResult {
    double C[3];
    double T;
    int32_t last;  // 1 + list position of the last composited entry, 0 if none
    uint8_t flag;
    int64_t evals;   // list entries evaluated (up to and including the stopping one)
    int32_t ncomp;   // entries composited
    int32_t nclamp;  // composited entries clamped at 0.99
    int32_t flips;   // forced decisions that differ from the oracle's own
    int32_t illegal; // ... of which the oracle's own decision was not ambiguous
    std::vector<Entry> used;
};

// The fp32 exponent p (base 2) of Gaussian g at pixel (px, py), in the kernels' order.
inline float decision_exponent(const Decision& d, int px, int py) {
    const float A = (-0.5f * LOG2E_F) * d.ca, B = -LOG2E_F * d.cb, Cc = (-0.5f * LOG2E_F) * d.cc;
    const float dx = ((float)px + 0.5f) - d.u, dy = ((float)py + 0.5f) - d.v;
    const float adx2 = A * (dx * dx);
    return std::fma(Cc, dy * dy, std::fma(B, dx * dy, adx2));
}

// Composite pixel (px, py) front to back.  keep: record the composited entries (for the
// backward).  forced / nforced: the decision codes of the first nforced evaluated entries
// (CODE_*), followed instead of the oracle's own decisions; nullptr = the oracle decides.
// dtrace (optional): receives (decision-side o 2^p, the code taken) of every evaluated entry.
PixelResult composite(const Scene& sc, int px, int py, bool keep, const uint8_t* forced = nullptr,
                      int64_t nforced = 0, std::vector<std::pair<double, uint8_t>>* dtrace = nullptr) {
    PixelResult r{};
    r.C[0] = r.C[1] = r.C[2] = 0.0;
    double T = 1.0;      // FP64 value transmittance
    float T32 = 1.0f;    // fp32 decision transmittance
    double dT = 0.0;     // relative bound on |T32 - the kernel's fp32 transmittance| / T32
    const auto& L = sc.list_of(px, py);
    const double cx = px + 0.5, cy = py + 0.5;
    for (size_t k = 0; k < L.size(); ++k) {
        const Value& q = sc.val[L[k]];
        const Decision& d = sc.dec[L[k]];
        r.evals++;
        // decision side (fp32 exponent, exact 2^p and FP64 opacity, bounded deviation)
        const double og_d = q.opacity * std::exp2((double)decision_exponent(d, px, py));
        const double a_d = std::min(ALPHA_MAX, og_d);
        const bool skip_o = a_d < ALPHA_MIN;
        const bool skip_amb = std::fabs(og_d - ALPHA_MIN) <= EPS_OG * og_d;
        const bool clamp_o = og_d > ALPHA_MAX;
        const bool clamp_amb = std::fabs(og_d - ALPHA_MAX) <= EPS_OG * og_d;
        // the kernel's alpha differs from a32 by at most (EPS_OG + U32) alpha (0 when both clamp)
        const float a32 = (float)a_d;
        const float Tn32 = T32 * (1.0f - a32);
        const double e_a = (clamp_o && !clamp_amb) ? 0.0 : (EPS_OG + U32) * a_d / (1.0 - a_d);
        const double dTn = (1.0 + dT) * (1.0 + e_a) * (1.0 + 4.0 * U32) - 1.0;
        const bool stop_o = Tn32 < (float)T_MIN;
        const bool stop_amb = std::fabs((double)Tn32 - T_MIN) <= dTn * (double)Tn32;
        if (skip_amb) r.flag |= FLAG_SKIP;
        if (!skip_o && clamp_amb) r.flag |= FLAG_CLAMP;
        if (!skip_o && stop_amb) r.flag |= FLAG_STOP;
        const int own = skip_o ? CODE_SKIP : (stop_o ? CODE_STOP : (clamp_o ? CODE_CLAMPED : CODE_COMPOSITE));
        int code = own;
        if (forced) {
            if ((int64_t)k >= nforced) {  // the kernel ended here without a stop: only if the list did
                r.illegal++;
                break;
            }
            code = forced[k];
            if (code != own) {
                r.flips++;
                const bool skip_f = code == CODE_SKIP, stop_f = code == CODE_STOP, clamp_f = code == CODE_CLAMPED;
                bool ok = skip_f == skip_o || skip_amb;
                if (!skip_f) ok = ok && (stop_f == stop_o || stop_amb);
                if (!skip_f && !stop_f) ok = ok && (clamp_f == clamp_o || clamp_amb);
                if (!ok) r.illegal++;
            }
        }
        if (dtrace) dtrace->emplace_back(og_d, (uint8_t)code);
        if (code == CODE_SKIP) continue;
        if (code == CODE_STOP) break;
        // composited: FP64 value of the entry on the decided branch
        const double dx = cx - q.u, dy = cy - q.v;
        const double power = -0.5 * (q.conic[0] * dx * dx + q.conic[2] * dy * dy) - q.conic[1] * dx * dy;
        const double Gv = std::exp(power);
        const bool clamped = code == CODE_CLAMPED;
        const double alpha = clamped ? 0.99 : q.opacity * Gv;  // the clamp's value is 0.99 itself
        for (int c = 0; c < 3; ++c) r.C[c] += q.rgb[c] * alpha * T;
        if (keep) r.used.push_back(Entry{L[k], alpha, Gv, T, dx, dy, clamped});
        r.ncomp++;
        r.nclamp += clamped;
        T *= 1.0 - alpha;
        T32 = clamped ? T32 * (1.0f - 0.99f) : Tn32;
        dT = dTn;
        r.last = (int32_t)(k + 1);
    }
    if (forced && r.evals < nforced) r.illegal++;  // the kernel evaluated entries the list lacks
    for (int c = 0; c < 3; ++c) r.C[c] += T * (double)sc.cam.bg[c];
    r.T = T;
    return r;
}

// What a perturbation must leave unchanged for a pixel's value to be a smooth function of it.
inline int64_t signature(const PixelResult& r) {
    return ((int64_t)r.last << 40) ^ ((int64_t)r.ncomp << 20) ^ ((int64_t)r.nclamp << 52) ^ r.evals;
}

// Forced decisions of some pixels (a kernel's own decisions for them): pixel (x, y) -> its codes.
struct Forced {
    std::unordered_map<int64_t, std::pair<const uint8_t*, int64_t>> by_pixel;
    int W = 0;
    Forced() = default;
    Forced(int width, int64_t npix, const int32_t* pix, const int64_t* off, const uint8_t* codes) : W(width) {
        for (int64_t k = 0; k < npix; ++k)
            by_pixel[(int64_t)pix[2 * k + 1] * W + pix[2 * k]] = {codes + off[k], off[k + 1] - off[k]};
    }
    PixelResult composite_at(const Scene& sc, int px, int py, bool keep) const {
        if (!by_pixel.empty()) {
            const auto it = by_pixel.find((int64_t)py * W + px);
            if (it != by_pixel.end()) return composite(sc, px, py, keep, it->second.first, it->second.second);
        }
        return composite(sc, px, py, keep);
    }
};

// Per-Gaussian screen-space gradient: du, dv, da, db, dc (conic), d opacity, d r, d g, d b.
struct G2 {
    double v[9];
};

// Backward of one pixel.  mode 0: direct differentiation of C = sum_i c_i a_i T_i + T_N bg,
// dC/da_i = c_i T_i - (sum_{j>i} c_j a_j T_j + T_N bg) / (1 - a_i).  mode 1: the paper's Eq. 7
// recurrence run back to front (C_in starts at bg) with Eq. 8 applied per entry and
// dL/dC_out of entry i = T_i dL/dC.
void pixel_backward(const Scene& sc, const PixelResult& r, int px, int py, const double dLdC[3],
                    int mode, std::vector<G2>& g2, const int64_t* only = nullptr) {
    const size_t N = r.used.size();
    double S[3], B[3];
    for (int c = 0; c < 3; ++c) {
        S[c] = r.T * sc.cam.bg[c];
        B[c] = sc.cam.bg[c];
    }
    (void)px;
    (void)py;
    for (size_t ii = N; ii-- > 0;) {
        const Entry& e = r.used[ii];
        const Value& q = sc.val[e.g];
        double dalpha = 0.0, dc[3];
        if (mode == 0) {
            for (int c = 0; c < 3; ++c) {
                const double dCda = q.rgb[c] * e.T - S[c] / (1.0 - e.alpha);
                dalpha += dLdC[c] * dCda;
                dc[c] = e.alpha * e.T * dLdC[c];
                S[c] += q.rgb[c] * e.alpha * e.T;
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                const double dCout = e.T * dLdC[c];
                dc[c] = e.alpha * dCout;              // dL/dc = alpha dL/dC_out
                dalpha += dCout * (q.rgb[c] - B[c]);  // dL/dalpha = <dL/dC_out, c - C_in>
                B[c] = B[c] * (1.0 - e.alpha) + e.alpha * q.rgb[c];
            }
        }
        if (only && e.g != *only) continue;
        G2& o = g2[only ? 0 : e.g];
        for (int c = 0; c < 3; ++c) o.v[6 + c] += dc[c];
        if (e.clamped) continue;  // alpha = 0.99 is constant in (o, G)
        o.v[5] += dalpha * e.G;
        const double dpow = dalpha * e.alpha;
        const double a = q.conic[0], b = q.conic[1], cc = q.conic[2];
        o.v[0] += dpow * (a * e.dx + b * e.dy);
        o.v[1] += dpow * (cc * e.dy + b * e.dx);
        o.v[2] += -0.5 * dpow * e.dx * e.dx;
        o.v[3] += -dpow * e.dx * e.dy;
        o.v[4] += -0.5 * dpow * e.dy * e.dy;
    }
}

// Chain the screen-space gradient of Gaussian i to its parameters.  out layout per Gaussian:
// d mean (3), d log-scale (3), d quat (4), d logit (1), d sh [3][K] (channel-major).
void chain_to_params(const Scene& sc, int64_t i, const G2& g, double* out) {
    const ogauss_t& G = sc.G;
    const ocam_t& cam = sc.cam;
    const Value& q = sc.val[i];
    const int64_t n = G.n;
    const int K = (G.sh_degree + 1) * (G.sh_degree + 1);
    double W[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) W[a][k] = cam.view[4 * a + k];
    double dmu[3] = {0, 0, 0};

    // colour -> SH coefficients and the view direction
    double ddir[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        const double gc = q.clamped[c] ? 0.0 : g.v[6 + c];
        for (int k = 0; k < K; ++k) {
            out[11 + c * K + k] = gc * q.Y[k];
            const double coef = (double)G.sh[((int64_t)c * K + k) * n + i];
            for (int a = 0; a < 3; ++a) ddir[a] += gc * coef * q.dY[k][a];
        }
    }
    const double dd = ddir[0] * q.dir[0] + ddir[1] * q.dir[1] + ddir[2] * q.dir[2];
    for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - q.dir[a] * dd) / q.dist;

    // opacity logit
    out[10] = g.v[5] * q.opacity * (1.0 - q.opacity);

    // conic (a, b, c) = (C/D, -B/D, A/D) -> 2-D covariance (A, B, C), D = A C - B^2
    const double A = q.A, B = q.B, C = q.C, D = q.D, D2 = D * D;
    const double ga = g.v[2], gb = g.v[3], gcn = g.v[4];
    const double dA = ga * (-C * C / D2) + gb * (B * C / D2) + gcn * (1.0 / D - A * C / D2);
    const double dB = ga * (2.0 * B * C / D2) + gb * (-1.0 / D - 2.0 * B * B / D2) + gcn * (2.0 * A * B / D2);
    const double dC = ga * (1.0 / D - C * A / D2) + gb * (B * A / D2) + gcn * (-A * A / D2);

    // A = T0 Sig T0^T, B = T0 Sig T1^T, C = T1 Sig T1^T (the 0.3 dilation is constant)
    double Gs[3][3];
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k)
            Gs[m][k] = dA * q.T[0][m] * q.T[0][k] + dB * q.T[0][m] * q.T[1][k] + dC * q.T[1][m] * q.T[1][k];
    double ST0[3], ST1[3];
    for (int m = 0; m < 3; ++m) {
        ST0[m] = q.Sig[m][0] * q.T[0][0] + q.Sig[m][1] * q.T[0][1] + q.Sig[m][2] * q.T[0][2];
        ST1[m] = q.Sig[m][0] * q.T[1][0] + q.Sig[m][1] * q.T[1][1] + q.Sig[m][2] * q.T[1][2];
    }
    double dT[2][3];
    for (int m = 0; m < 3; ++m) {
        dT[0][m] = 2.0 * dA * ST0[m] + dB * ST1[m];
        dT[1][m] = dB * ST0[m] + 2.0 * dC * ST1[m];
    }
    // T = J W
    double dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
    for (int m = 0; m < 3; ++m) {
        dJ00 += dT[0][m] * W[0][m];
        dJ02 += dT[0][m] * W[2][m];
        dJ11 += dT[1][m] * W[1][m];
        dJ12 += dT[1][m] * W[2][m];
    }
    const double z = q.pc[2], x = q.pc[0], y = q.pc[1];
    const double fx = cam.fx, fy = cam.fy;
    double dpc[3] = {0, 0, 0};
    dpc[2] += dJ00 * (-fx / (z * z)) + dJ02 * (fx * q.cxh / (z * z)) + dJ11 * (-fy / (z * z)) +
              dJ12 * (fy * q.cyh / (z * z));
    const double dcxh = dJ02 * (-fx / z), dcyh = dJ12 * (-fy / z);
    if (!q.xclamped) {
        dpc[0] += dcxh / z;
        dpc[2] += dcxh * (-x / (z * z));
    }
    if (!q.yclamped) {
        dpc[1] += dcyh / z;
        dpc[2] += dcyh * (-y / (z * z));
    }
    // screen position u = fx x / z + cx, v = fy y / z + cy
    dpc[0] += g.v[0] * fx / z;
    dpc[2] += g.v[0] * (-fx * x / (z * z));
    dpc[1] += g.v[1] * fy / z;
    dpc[2] += g.v[1] * (-fy * y / (z * z));
    for (int k = 0; k < 3; ++k) dmu[k] += dpc[0] * W[0][k] + dpc[1] * W[1][k] + dpc[2] * W[2][k];

    // Sig = M M^T with M = R diag(s): dL/dM = (Gs + Gs^T) M
    double dM[3][3];
    for (int p = 0; p < 3; ++p)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += (Gs[p][m] + Gs[m][p]) * q.M[m][k];
            dM[p][k] = acc;
        }
    double dR[3][3];
    for (int k = 0; k < 3; ++k) {
        double ds = 0;
        for (int p = 0; p < 3; ++p) {
            dR[p][k] = dM[p][k] * q.s[k];
            ds += dM[p][k] * q.R[p][k];
        }
        out[3 + k] = ds * q.s[k];
    }
    // rotation entries as functions of the unit quaternion (w, x, y, z)
    const double w = q.qh[0], qx = q.qh[1], qy = q.qh[2], qz = q.qh[3];
    double dq[4] = {0, 0, 0, 0};
    // R00 = 1 - 2(y^2 + z^2)
    dq[2] += dR[0][0] * (-4 * qy);
    dq[3] += dR[0][0] * (-4 * qz);
    // R01 = 2(xy - wz)
    dq[0] += dR[0][1] * (-2 * qz); dq[1] += dR[0][1] * (2 * qy); dq[2] += dR[0][1] * (2 * qx); dq[3] += dR[0][1] * (-2 * w);
    // R02 = 2(xz + wy)
    dq[0] += dR[0][2] * (2 * qy); dq[1] += dR[0][2] * (2 * qz); dq[2] += dR[0][2] * (2 * w); dq[3] += dR[0][2] * (2 * qx);
    // R10 = 2(xy + wz)
    dq[0] += dR[1][0] * (2 * qz); dq[1] += dR[1][0] * (2 * qy); dq[2] += dR[1][0] * (2 * qx); dq[3] += dR[1][0] * (2 * w);
    // R11 = 1 - 2(x^2 + z^2)
    dq[1] += dR[1][1] * (-4 * qx);
    dq[3] += dR[1][1] * (-4 * qz);
    // R12 = 2(yz - wx)
    dq[0] += dR[1][2] * (-2 * qx); dq[1] += dR[1][2] * (-2 * w); dq[2] += dR[1][2] * (2 * qz); dq[3] += dR[1][2] * (2 * qy);
    // R20 = 2(xz - wy)
    dq[0] += dR[2][0] * (-2 * qy); dq[1] += dR[2][0] * (2 * qz); dq[2] += dR[2][0] * (-2 * w); dq[3] += dR[2][0] * (2 * qx);
    // R21 = 2(yz + wx)
    dq[0] += dR[2][1] * (2 * qx); dq[1] += dR[2][1] * (2 * w); dq[2] += dR[2][1] * (2 * qz); dq[3] += dR[2][1] * (2 * qy);
    // R22 = 1 - 2(x^2 + y^2)
    dq[1] += dR[2][2] * (-4 * qx);
    dq[2] += dR[2][2] * (-4 * qy);
    // normalisation q_hat = q / |q|
    const double dot = dq[0] * w + dq[1] * qx + dq[2] * qy + dq[3] * qz;
    for (int k = 0; k < 4; ++k) out[6 + k] = (dq[k] - q.qh[k] * dot) / q.qn;
    for (int k = 0; k < 3; ++k) out[k] = dmu[k];
}

int param_count(int sh_degree) { return 11 + 3 * (sh_degree + 1) * (sh_degree + 1); }

// scatter a per-Gaussian parameter gradient (layout of chain_to_params) into the planar layout
void scatter_planar(const ogauss_t& G, int64_t i, const double* p, double* out) {
    const int64_t n = G.n;
    const int K = (G.sh_degree + 1) * (G.sh_degree + 1);
    double* means = out;
    double* ls = out + 3 * n;
    double* qs = out + 6 * n;
    double* lg = out + 10 * n;
    double* sh = out + 11 * n;
    for (int k = 0; k < 3; ++k) means[k * n + i] += p[k];
    for (int k = 0; k < 3; ++k) ls[k * n + i] += p[3 + k];
    for (int k = 0; k < 4; ++k) qs[k * n + i] += p[6 + k];
    lg[i] += p[10];
    for (int k = 0; k < 3 * K; ++k) sh[(int64_t)k * n + i] += p[11 + k];
}

}  // namespace

// ================================================================================================
// C ABI of the oracle
// ================================================================================================
extern "C" {

float oracle_det_expf(float x) { return det_expf(x); }

// Threads of the parallel loops (pixel rows, pixels, Gaussians); n <= 0 leaves the default (all
// cores).  Returns the count now in effect.
int oracle_set_threads(int n) {
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

// The bound EPS_OG on the kernel's o G relative to the oracle's decision-side o 2^p.
double oracle_decision_bound(void) { return EPS_OG; }

void oracle_sh_basis(const double* dir, double* out_y, double* out_dy) {
    double Y[16], dY[16][3];
    sh_basis(dir, Y, dY);
    for (int k = 0; k < 16; ++k) {
        out_y[k] = Y[k];
        if (out_dy)
            for (int c = 0; c < 3; ++c) out_dy[3 * k + c] = dY[k][c];
    }
}

int oracle_param_count(int sh_degree) { return param_count(sh_degree); }

// Per-Gaussian projection.  Decision outputs (fp32 path): visible, radii [N][2] (x, y), rect [N][4]
// (x0, y0, x1, y1 in tiles, half-open), depth, uv [N][2], cov2d [N][3].  Value outputs (FP64):
// mean2d [N][2], conic [N][3], opacity [N], rgb [N][3].  Any output pointer may be null.
void oracle_project(const ogauss_t* G, const ocam_t* cam, int tile, int32_t* visible,
                    int32_t* radius, int32_t* rect, float* depth, float* uv, float* cov2d,
                    double* mean2d, double* conic, double* opacity, double* rgb) {
    for (int64_t i = 0; i < G->n; ++i) {
        const Decision d = decide(*G, *cam, tile, i);
        if (visible) visible[i] = d.visible ? 1 : 0;
        if (radius) {
            radius[2 * i] = d.visible ? d.radius_x : 0;
            radius[2 * i + 1] = d.visible ? d.radius_y : 0;
        }
        if (rect) {
            rect[4 * i + 0] = d.visible ? d.x0 : 0;
            rect[4 * i + 1] = d.visible ? d.y0 : 0;
            rect[4 * i + 2] = d.visible ? d.x1 : 0;
            rect[4 * i + 3] = d.visible ? d.y1 : 0;
        }
        if (depth) depth[i] = d.zc;
        if (uv) {
            uv[2 * i] = d.u;
            uv[2 * i + 1] = d.v;
        }
        if (cov2d) {
            cov2d[3 * i] = d.cov_a;
            cov2d[3 * i + 1] = d.cov_b;
            cov2d[3 * i + 2] = d.cov_c;
        }
        if (!d.visible) continue;
        const Value q = evaluate(*G, *cam, i);
        if (mean2d) {
            mean2d[2 * i] = q.u;
            mean2d[2 * i + 1] = q.v;
        }
        if (conic)
            for (int k = 0; k < 3; ++k) conic[3 * i + k] = q.conic[k];
        if (opacity) opacity[i] = q.opacity;
        if (rgb)
            for (int k = 0; k < 3; ++k) rgb[3 * i + k] = q.rgb[k];
    }
}

// Keys of every (tile, Gaussian) pair: Gaussians in canonical order, tiles row-major inside each
// rectangle (those the 3-sigma ellipse reaches); key = (tile << 32) | float bits of the depth; value = canonical index.  Stable sort
// by key; ranges[2 t], ranges[2 t + 1] = [first, last + 1) of tile t, [0, 0) if empty.
// Writes at most `capacity` pairs and returns the total pair count.
int64_t oracle_keys(const ogauss_t* G, const ocam_t* cam, int tile, int64_t capacity,
                    uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
    const int TX = (cam->width + tile - 1) / tile, TY = (cam->height + tile - 1) / tile;
    std::vector<std::pair<uint64_t, uint32_t>> pairs;
    for (int64_t i = 0; i < G->n; ++i) {
        const Decision d = decide(*G, *cam, tile, i);
        if (!d.visible) continue;
        for (int ty = d.y0; ty < d.y1; ++ty)
            for (int tx = d.x0; tx < d.x1; ++tx) {
                if (!tile_hit(d, tx, ty, tile)) continue;
                const uint64_t t = (uint64_t)ty * TX + tx;
                pairs.emplace_back((t << 32) | fbits(d.zc), (uint32_t)i);
            }
    }
    std::stable_sort(pairs.begin(), pairs.end(),
                     [](const auto& a, const auto& b) { return a.first < b.first; });
    const int64_t P = (int64_t)pairs.size();
    for (int64_t k = 0; k < P && k < capacity; ++k) {
        if (keys) keys[k] = pairs[k].first;
        if (vals) vals[k] = pairs[k].second;
    }
    if (ranges) {
        std::memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)TX * TY);
        for (int64_t k = 0; k < P; ++k) {
            const uint64_t t = pairs[k].first >> 32;
            if (k == 0 || (pairs[k - 1].first >> 32) != t) ranges[2 * t] = (uint32_t)k;
            if (k == P - 1 || (pairs[k + 1].first >> 32) != t) ranges[2 * t + 1] = (uint32_t)(k + 1);
        }
    }
    return P;
}

// Render every pixel.  image [3][H][W], T_final [H][W], last [H][W], flag [H][W], evals [H][W],
// ncomp [H][W] (entries composited); any output may be null.
void oracle_render(const ogauss_t* G, const ocam_t* cam, int tile, double* image, double* T_final,
                   int32_t* last, uint8_t* flag, int64_t* evals, int32_t* ncomp) {
    Scene sc(*G, *cam, tile);
    const int W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const PixelResult r = composite(sc, px, py, false);
            const size_t p = (size_t)py * W + px;
            if (image)
                for (int c = 0; c < 3; ++c) image[(size_t)c * W * H + p] = r.C[c];
            if (T_final) T_final[p] = r.T;
            if (last) last[p] = r.last;
            if (flag) flag[p] = r.flag;
            if (evals) evals[p] = r.evals;
            if (ncomp) ncomp[p] = r.ncomp;
        }
}

// Render a list of pixels (x, y pairs).  rgb [npix][3], T [npix], last [npix], flag [npix].
void oracle_render_pixels(const ogauss_t* G, const ocam_t* cam, int tile, int64_t npix,
                          const int32_t* pix, double* rgb, double* T_final, int32_t* last,
                          uint8_t* flag) {
    Scene sc(*G, *cam, tile);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < npix; ++k) {
        const PixelResult r = composite(sc, pix[2 * k], pix[2 * k + 1], false);
        if (rgb)
            for (int c = 0; c < 3; ++c) rgb[3 * k + c] = r.C[c];
        if (T_final) T_final[k] = r.T;
        if (last) last[k] = r.last;
        if (flag) flag[k] = r.flag;
    }
}

// Render a list of pixels (x, y pairs) following given decisions: pixel k's evaluated entries take
// the codes codes[off[k] .. off[k + 1]) (0 skipped, 1 composited, 2 composited clamped at 0.99,
// 3 stop), values stay FP64.  rgb [npix][3], T [npix], last [npix], ncomp [npix]; flips [npix]
// counts the codes that differ from the oracle's own decisions and illegal [npix] those of them
// whose own decision was not within the error bound of its threshold (or codes that end before
// the list without a stop, or run past it).
void oracle_render_forced(const ogauss_t* G, const ocam_t* cam, int tile, int64_t npix,
                          const int32_t* pix, const int64_t* off, const uint8_t* codes, double* rgb,
                          double* T_final, int32_t* last, int32_t* ncomp, int32_t* flips, int32_t* illegal) {
    Scene sc(*G, *cam, tile);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < npix; ++k) {
        const PixelResult r = composite(sc, pix[2 * k], pix[2 * k + 1], false, codes + off[k], off[k + 1] - off[k]);
        for (int c = 0; c < 3; ++c) rgb[3 * k + c] = r.C[c];
        T_final[k] = r.T;
        last[k] = r.last;
        ncomp[k] = r.ncomp;
        flips[k] = r.flips;
        illegal[k] = r.illegal;
    }
}

// The oracle's own decisions for a list of pixels: for each evaluated entry (at most max_entries
// per pixel) its decision-side o 2^p (FP64 opacity, exact 2^p of the fp32 exponent) into
// og [npix][max_entries] and its code (as in oracle_render_forced) into code [npix][max_entries];
// count [npix] = entries evaluated (-1 when more than max_entries).
void oracle_decisions(const ogauss_t* G, const ocam_t* cam, int tile, int64_t npix, const int32_t* pix,
                      int64_t max_entries, double* og, uint8_t* code, int64_t* count) {
    Scene sc(*G, *cam, tile);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < npix; ++k) {
        const int px = pix[2 * k], py = pix[2 * k + 1];
        std::vector<std::pair<double, uint8_t>> dt;
        const PixelResult r = composite(sc, px, py, false, nullptr, 0, &dt);
        count[k] = r.evals <= max_entries ? r.evals : -1;
        for (int64_t e = 0; e < (int64_t)dt.size() && e < max_entries; ++e) {
            og[k * max_entries + e] = dt[e].first;
            code[k * max_entries + e] = dt[e].second;
        }
    }
}

// The same image through Eq. 7 itself: per pixel, take the composited entries in depth order and
// run C_out = C_in (1 - alpha) + alpha c from the back (C_in = bg) to the front.
void oracle_render_eq7(const ogauss_t* G, const ocam_t* cam, int tile, double* image) {
    Scene sc(*G, *cam, tile);
    const int W = cam->width, H = cam->height;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const PixelResult r = composite(sc, px, py, true);
            double C[3] = {cam->bg[0], cam->bg[1], cam->bg[2]};
            for (size_t i = r.used.size(); i-- > 0;) {
                const Value& q = sc.val[r.used[i].g];
                const double a = r.used[i].alpha;
                for (int c = 0; c < 3; ++c) C[c] = C[c] * (1.0 - a) + a * q.rgb[c];
            }
            const size_t p = (size_t)py * W + px;
            for (int c = 0; c < 3; ++c) image[(size_t)c * W * H + p] = C[c];
        }
}


// Backward of the whole image for an upstream gradient dL/dimage [3][H][W].
// grad2d [N][9] (du, dv, d conic a, b, c, d opacity, d rgb) and grads in the planar parameter
// layout (means [3][N], log_scales [3][N], quats [4][N], logits [N], sh [3][K][N]); both are
// overwritten.  mode 0 / 1 select the two derivations of dL/d(alpha, c).
// Pixels listed in (nf, fpix, foff, fcodes) follow those decisions (as in oracle_render_forced).
void oracle_backward_forced(const ogauss_t* G, const ocam_t* cam, int tile, const double* dL_dimage,
                            int mode, int64_t nf, const int32_t* fpix, const int64_t* foff,
                            const uint8_t* fcodes, double* grad2d, double* grads) {
    Scene sc(*G, *cam, tile);
    const Forced F(cam->width, nf, fpix, foff, fcodes);
    const int W = cam->width, H = cam->height;
    // pixel rows split into one contiguous band per thread; each band sums into its own copy of the
    // screen-space gradients, and the copies are added in band order
    const int nt = omp_get_max_threads();
    std::vector<std::vector<G2>> part((size_t)nt);
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), nth = omp_get_num_threads();
        std::vector<G2>& g2t = part[(size_t)t];
        g2t.resize((size_t)G->n);
        for (auto& e : g2t) std::fill(e.v, e.v + 9, 0.0);
        const int y0 = (int)((int64_t)H * t / nth), y1 = (int)((int64_t)H * (t + 1) / nth);
        for (int py = y0; py < y1; ++py)
            for (int px = 0; px < W; ++px) {
                const size_t p = (size_t)py * W + px;
                const double dLdC[3] = {dL_dimage[p], dL_dimage[(size_t)W * H + p],
                                        dL_dimage[2 * (size_t)W * H + p]};
                const PixelResult r = F.composite_at(sc, px, py, true);
                pixel_backward(sc, r, px, py, dLdC, mode, g2t);
            }
    }
    std::vector<G2> g2((size_t)G->n);
    for (auto& e : g2) std::fill(e.v, e.v + 9, 0.0);
    for (const auto& g2t : part)
        for (size_t i = 0; i < g2t.size(); ++i)
            for (int k = 0; k < 9; ++k) g2[i].v[k] += g2t[i].v[k];
    const int PC = param_count(G->sh_degree);
    if (grads) std::fill(grads, grads + (size_t)PC * G->n, 0.0);
#pragma omp parallel
    {
        std::vector<double> tmp(PC);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < G->n; ++i) {
            if (grad2d)
                for (int k = 0; k < 9; ++k) grad2d[9 * i + k] = g2[i].v[k];
            if (!grads || !sc.dec[i].visible) continue;
            std::fill(tmp.begin(), tmp.end(), 0.0);
            chain_to_params(sc, i, g2[i], tmp.data());
            scatter_planar(*G, i, tmp.data(), grads);
        }
    }
}

void oracle_backward(const ogauss_t* G, const ocam_t* cam, int tile, const double* dL_dimage,
                     int mode, double* grad2d, double* grads) {
    oracle_backward_forced(G, cam, tile, dL_dimage, mode, 0, nullptr, nullptr, nullptr, grad2d, grads);
}

// Parameter gradients of selected Gaussians only, for images too large to differentiate whole:
// for each selected Gaussian, every pixel of its tile rectangle is composited and the direct
// derivative (mode 0) of that pixel with respect to the selected Gaussian is accumulated.
// grad2d [nsel][9]; grads [nsel][P] with P = 11 + 3K in the per-Gaussian layout
// (mean 3, log-scale 3, quat 4, logit 1, sh [3][K]).
// Pixels listed in (nf, fpix, foff, fcodes) follow those decisions (as in oracle_render_forced).
void oracle_backward_subset_forced(const ogauss_t* G, const ocam_t* cam, int tile,
                                   const double* dL_dimage, int64_t nsel, const int64_t* sel, int64_t nf,
                                   const int32_t* fpix, const int64_t* foff, const uint8_t* fcodes,
                                   double* grad2d, double* grads) {
    Scene sc(*G, *cam, tile);
    const Forced F(cam->width, nf, fpix, foff, fcodes);
    const int W = cam->width, H = cam->height;
    const int PC = param_count(G->sh_degree);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < nsel; ++s) {
        const int64_t gi = sel[s];
        std::vector<G2> one(1);
        std::fill(one[0].v, one[0].v + 9, 0.0);
        const Decision& d = sc.dec[gi];
        if (d.visible) {
            for (int py = d.y0 * tile; py < std::min(H, d.y1 * tile); ++py)
                for (int px = d.x0 * tile; px < std::min(W, d.x1 * tile); ++px) {
                    const size_t p = (size_t)py * W + px;
                    const double dLdC[3] = {dL_dimage[p], dL_dimage[(size_t)W * H + p],
                                            dL_dimage[2 * (size_t)W * H + p]};
                    const PixelResult r = F.composite_at(sc, px, py, true);
                    pixel_backward(sc, r, px, py, dLdC, 0, one, &gi);
                }
        }
        if (grad2d)
            for (int k = 0; k < 9; ++k) grad2d[9 * s + k] = one[0].v[k];
        if (grads) {
            std::fill(grads + s * PC, grads + (s + 1) * PC, 0.0);
            if (d.visible) chain_to_params(sc, gi, one[0], grads + s * PC);
        }
    }
}

void oracle_backward_subset(const ogauss_t* G, const ocam_t* cam, int tile,
                            const double* dL_dimage, int64_t nsel, const int64_t* sel,
                            double* grad2d, double* grads) {
    oracle_backward_subset_forced(G, cam, tile, dL_dimage, nsel, sel, 0, nullptr, nullptr, nullptr, grad2d, grads);
}

// FP64 central finite differences of L = sum_p <w_p, C_p> (w = dL_dimage [3][H][W]) with respect
// to every parameter of the selected Gaussians.  Each perturbed evaluation changes one parameter
// of one Gaussian by +-h (h = h_rel * max(1, |theta|), applied to the fp32 parameter), recomputes
// that Gaussian alone, and re-composites the pixels of its tile rectangle (no other pixel
// depends on it).  A coordinate whose perturbation changes a decision - the rectangle, the depth
// order inside a tile, or any pixel's (last, composited count, evaluated count) - is reported as
// NaN.  out [nsel][11 + 3K] in the per-Gaussian layout of oracle_backward_subset.
// Pixels listed in (nf, fpix, foff, fcodes) keep those decisions in every evaluation.
void oracle_fd_subset_forced(const ogauss_t* G, const ocam_t* cam, int tile, const double* dL_dimage,
                             int64_t nsel, const int64_t* sel, double h_rel, int64_t nf, const int32_t* fpix,
                             const int64_t* foff, const uint8_t* fcodes, double* out) {
    Scene sc(*G, *cam, tile);
    const Forced F(cam->width, nf, fpix, foff, fcodes);
    const int W = cam->width, H = cam->height;
    const int K = (G->sh_degree + 1) * (G->sh_degree + 1);
    const int PC = param_count(G->sh_degree);
    const int64_t n = G->n;
    for (int64_t s = 0; s < nsel; ++s) {
        const int64_t gi = sel[s];
        const Decision d0 = sc.dec[gi];
        const Value v0 = sc.val[gi];
        // one-Gaussian parameter copy
        float prm[59];
        for (int k = 0; k < 3; ++k) prm[k] = G->means[k * n + gi];
        for (int k = 0; k < 3; ++k) prm[3 + k] = G->log_scales[k * n + gi];
        for (int k = 0; k < 4; ++k) prm[6 + k] = G->quats[k * n + gi];
        prm[10] = G->logits[gi];
        for (int k = 0; k < 3 * K; ++k) prm[11 + k] = G->sh[(int64_t)k * n + gi];
        auto one = [&](const float* q) {
            ogauss_t g1;
            g1.n = 1;
            g1.sh_degree = G->sh_degree;
            g1.pad_ = 0;
            static thread_local float buf[59];
            for (int k = 0; k < PC; ++k) buf[k] = q[k];
            g1.means = buf;
            g1.log_scales = buf + 3;
            g1.quats = buf + 6;
            g1.logits = buf + 10;
            g1.sh = buf + 11;
            // planar [k][1] layout of a single Gaussian is the packed vector itself
            return g1;
        };
        // pixels of the rectangle (clipped to the image), with their base signatures
        std::vector<std::pair<int, int>> pix;
        if (d0.visible)
            for (int py = d0.y0 * tile; py < std::min(H, d0.y1 * tile); ++py)
                for (int px = d0.x0 * tile; px < std::min(W, d0.x1 * tile); ++px) pix.emplace_back(px, py);
        std::vector<int64_t> sig0;
        for (auto& pp : pix) {
            const PixelResult r = F.composite_at(sc, pp.first, pp.second, false);
            sig0.push_back(signature(r));
        }
        auto loss_with = [&](const float* q, bool& ok) {
            ogauss_t g1 = one(q);
            const Decision d = decide(g1, *cam, tile, 0);
            ok = d.visible == d0.visible && d.x0 == d0.x0 && d.x1 == d0.x1 && d.y0 == d0.y0 && d.y1 == d0.y1;
            for (int ty = d.y0; ty < d.y1 && ok; ++ty)  // the same tiles of the rectangle reached
                for (int tx = d.x0; tx < d.x1 && ok; ++tx) ok = tile_hit(d, tx, ty, tile) == tile_hit(d0, tx, ty, tile);
            if (!ok) return 0.0;
            // depth order inside every tile of the rectangle must be unchanged
            const uint32_t b0 = fbits(d0.zc), b1 = fbits(d.zc);
            if (b0 != b1)
                for (int ty = d.y0; ty < d.y1 && ok; ++ty)
                    for (int tx = d.x0; tx < d.x1 && ok; ++tx)
                        for (int64_t o : sc.lists[(size_t)ty * sc.TX + tx]) {
                            if (o == gi) continue;
                            const uint32_t bo = fbits(sc.dec[o].zc);
                            const uint32_t lo = std::min(b0, b1), hi = std::max(b0, b1);
                            if (bo >= lo && bo <= hi) {
                                ok = false;
                                break;
                            }
                        }
            if (!ok) return 0.0;
            sc.dec[gi] = d;
            sc.val[gi] = evaluate(g1, *cam, 0);
            double L = 0.0;
            for (size_t k = 0; k < pix.size() && ok; ++k) {
                const int px = pix[k].first, py = pix[k].second;
                const PixelResult r = F.composite_at(sc, px, py, false);
                if (signature(r) != sig0[k] || r.illegal) ok = false;
                const size_t p = (size_t)py * W + px;
                for (int c = 0; c < 3; ++c) L += dL_dimage[(size_t)c * W * H + p] * r.C[c];
            }
            sc.dec[gi] = d0;
            sc.val[gi] = v0;
            return L;
        };
        for (int k = 0; k < PC; ++k) {
            double& o = out[s * PC + k];
            if (!d0.visible) {
                o = 0.0;
                continue;
            }
            const float x = prm[k];
            const double h = h_rel * std::max(1.0, std::fabs((double)x));
            float qp[59], qm[59];
            std::memcpy(qp, prm, sizeof(float) * PC);
            std::memcpy(qm, prm, sizeof(float) * PC);
            qp[k] = (float)((double)x + h);
            qm[k] = (float)((double)x - h);
            bool okp = false, okm = false;
            const double Lp = loss_with(qp, okp);
            const double Lm = loss_with(qm, okm);
            o = (okp && okm) ? (Lp - Lm) / ((double)qp[k] - (double)qm[k]) : std::nan("");
        }
    }
}

void oracle_fd_subset(const ogauss_t* G, const ocam_t* cam, int tile, const double* dL_dimage,
                      int64_t nsel, const int64_t* sel, double h_rel, double* out) {
    oracle_fd_subset_forced(G, cam, tile, dL_dimage, nsel, sel, h_rel, 0, nullptr, nullptr, nullptr, out);
}

// Chain given screen-space gradients grad2d [N][9] to parameters (planar layout, overwritten).
void oracle_chain(const ogauss_t* G, const ocam_t* cam, int tile, const double* grad2d,
                  double* grads) {
    Scene sc(*G, *cam, tile);
    const int PC = param_count(G->sh_degree);
    std::fill(grads, grads + (size_t)PC * G->n, 0.0);
    std::vector<double> tmp(PC);
    for (int64_t i = 0; i < G->n; ++i) {
        if (!sc.dec[i].visible) continue;
        G2 g;
        for (int k = 0; k < 9; ++k) g.v[k] = grad2d[9 * i + k];
        std::fill(tmp.begin(), tmp.end(), 0.0);
        chain_to_params(sc, i, g, tmp.data());
        scatter_planar(*G, i, tmp.data(), grads);
    }
}

// Per-Gaussian flags for decisions of the value path that switch a gradient on or off:
// bit 0 a colour channel within 1e-5 of the clamp at 0; bit 1 x/z or y/z within relative 1e-5
// of the Jacobian clamp.
void oracle_gaussian_flags(const ogauss_t* G, const ocam_t* cam, int tile, uint8_t* flags) {
    for (int64_t i = 0; i < G->n; ++i) {
        flags[i] = 0;
        const Decision d = decide(*G, *cam, tile, i);
        if (!d.visible) continue;
        const Value q = evaluate(*G, *cam, i);
        for (int c = 0; c < 3; ++c)
            if (std::fabs(q.raw[c]) < 1e-5) flags[i] |= 1;
        const double limx = 1.3 * (0.5 * cam->width / (double)cam->fx);
        const double limy = 1.3 * (0.5 * cam->height / (double)cam->fy);
        if (std::fabs(std::fabs(q.tx) - limx) < 1e-5 * limx) flags[i] |= 2;
        if (std::fabs(std::fabs(q.ty) - limy) < 1e-5 * limy) flags[i] |= 2;
    }
}

// L1 loss over n values: loss = mean |img - gt|, grad = sign(img - gt) / n with sign(0) = 0,
// sse = sum (img - gt)^2.
void oracle_l1(int64_t n, const double* img, const double* gt, double* grad, double* loss,
               double* sse) {
    double l = 0, s = 0;
    for (int64_t k = 0; k < n; ++k) {
        const double d = img[k] - gt[k];
        l += std::fabs(d);
        s += d * d;
        if (grad) grad[k] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)n;
    }
    if (loss) *loss = l / (double)n;
    if (sse) *sse = s;
}

// Adam (Kingma & Ba 2015) with bias correction, one step t >= 1 over n values with one
// learning rate: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
void oracle_adam(int64_t n, double* p, const double* g, double* m, double* v, double lr,
                 double b1, double b2, double eps, int64_t t) {
    const double bc1 = 1.0 - std::pow(b1, (double)t), bc2 = 1.0 - std::pow(b2, (double)t);
    for (int64_t k = 0; k < n; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        const double mh = m[k] / bc1, vh = v[k] / bc2;
        p[k] -= lr * mh / (std::sqrt(vh) + eps);
    }
}

}  // extern "C"
