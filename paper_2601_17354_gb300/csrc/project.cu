// K1 project_fwd and K9 project_bwd: one thread per Gaussian over the planar SoA parameters.
//
// The canonical parameter buffer (mu, Sigma, c, alpha) of Fig. 2 / Sec. III-C is read in place;
// nothing is reordered (the sorted view exists only as the key/value pairs, Eq. 10).
//
// Decision quantities (camera depth, screen position, 2-D covariance, radii, tile rectangle)
// follow a prescribed fp32 operation order with every operation an explicit correctly rounded
// intrinsic, and this file is compiled with --fmad=false, so the keys are reproducible bit for
// bit by any IEEE implementation of the same sequence.  Value quantities (conic, opacity,
// colour) and the backward use ordinary fp32 arithmetic.
//
// Readings of what the paper leaves open: pinhole + first-order (EWA) projection of the 3-D
// covariance with a 0.3 px^2 dilation; cull at z <= near; Jacobian evaluated at x/z, y/z clamped
// to +-1.3 tan(half field of view) with zero gradient through the clamp; per-axis radii
// ceil(3 sqrt(Sigma_xx)), ceil(3 sqrt(Sigma_yy)) (the box of the 3-sigma ellipse); colour from
// real orthonormal spherical harmonics (no Condon-Shortley phase) of the direction camera ->
// mean, + 0.5, clamped at 0.
#include "pgs_internal.cuh"

namespace pgs {
namespace {

// exp in fp32 by Cody-Waite reduction + degree-7 Taylor polynomial (Horner with fma) and an
// exact power-of-two scale: k = rint(x log2 e), r = x - k ln2 (ln2 as hi + lo), exp = p(r) 2^k.
// Bit-reproducible (every step is a correctly rounded IEEE operation); within 2 ulp of exp.
__device__ __forceinline__ float det_expf(float x) {
    if (x != x) return x;
    x = fminf(fmaxf(x, -87.0f), 88.0f);
    const float k = rintf(__fmul_rn(x, 0x1.715476p+0f));
    float r = __fmaf_rn(-k, 0x1.62e4p-1f, x);
    r = __fmaf_rn(-k, 0x1.7f7d1cp-20f, r);
    float p = 0x1.a01a02p-13f;
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
    p = __fmaf_rn(p, r, 0x1.111112p-7f);
    p = __fmaf_rn(p, r, 0x1.555556p-5f);
    p = __fmaf_rn(p, r, 0x1.555556p-3f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const float scale = __int_as_float(((int)k + 127) << 23);
    return __fmul_rn(p, scale);
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
    return fminf(fmaxf(x, lo), hi);
}

// fp32 state shared by the forward and the backward of one Gaussian.
struct Geo {
    float xc, yc, zc, tx, ty;
    float u, v;
    float qn, w, x, y, z;  // quaternion norm and unit quaternion
    float R[3][3], s[3], M[3][3], Sig[3][3];
    float cxh, cyh;
    bool xclamp, yclamp;
    float j00, j02, j11, j12;
    float T[2][3];
    float cov_a, cov_b, cov_c, det;
};

// The prescribed decision sequence.  Returns false if the Gaussian is culled before a rectangle
// exists (behind the near plane, degenerate quaternion or covariance, non-finite position).
__device__ __forceinline__ bool geometry(const float mu[3], const float ls[3], const float q[4],
                                         const pgs_camera& cam, Geo& G) {
    const float* V = cam.viewmat;
    G.xc = __fmaf_rn(V[0], mu[0], __fmaf_rn(V[1], mu[1], __fmaf_rn(V[2], mu[2], V[3])));
    G.yc = __fmaf_rn(V[4], mu[0], __fmaf_rn(V[5], mu[1], __fmaf_rn(V[6], mu[2], V[7])));
    G.zc = __fmaf_rn(V[8], mu[0], __fmaf_rn(V[9], mu[1], __fmaf_rn(V[10], mu[2], V[11])));
    if (!(G.zc > cam.near_z)) return false;
    G.tx = __fdiv_rn(G.xc, G.zc);
    G.ty = __fdiv_rn(G.yc, G.zc);
    G.u = __fmaf_rn(cam.fx, G.tx, cam.cx);
    G.v = __fmaf_rn(cam.fy, G.ty, cam.cy);
    if (!isfinite(G.u) || !isfinite(G.v)) return false;

    const float n2 = __fmaf_rn(q[0], q[0], __fmaf_rn(q[1], q[1], __fmaf_rn(q[2], q[2], __fmul_rn(q[3], q[3]))));
    if (!(n2 > 0.0f) || !isfinite(n2)) return false;
    G.qn = __fsqrt_rn(n2);
    G.w = __fdiv_rn(q[0], G.qn);
    G.x = __fdiv_rn(q[1], G.qn);
    G.y = __fdiv_rn(q[2], G.qn);
    G.z = __fdiv_rn(q[3], G.qn);
    const float xx = __fmul_rn(G.x, G.x), yy = __fmul_rn(G.y, G.y), zz = __fmul_rn(G.z, G.z);
    const float xy = __fmul_rn(G.x, G.y), xz = __fmul_rn(G.x, G.z), yz = __fmul_rn(G.y, G.z);
    const float wx = __fmul_rn(G.w, G.x), wy = __fmul_rn(G.w, G.y), wz = __fmul_rn(G.w, G.z);
    G.R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    G.R[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    G.R[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    G.R[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    G.R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    G.R[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    G.R[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    G.R[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    G.R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
#pragma unroll
    for (int k = 0; k < 3; ++k) G.s[k] = det_expf(ls[k]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) G.M[a][k] = __fmul_rn(G.R[a][k], G.s[k]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            G.Sig[a][b] = __fmaf_rn(G.M[a][0], G.M[b][0],
                                    __fmaf_rn(G.M[a][1], G.M[b][1], __fmul_rn(G.M[a][2], G.M[b][2])));
            G.Sig[b][a] = G.Sig[a][b];
        }
    const float limx = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)cam.width), cam.fx));
    const float limy = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)cam.height), cam.fy));
    G.xclamp = G.tx < -limx || G.tx > limx;
    G.yclamp = G.ty < -limy || G.ty > limy;
    G.cxh = clampf(G.tx, -limx, limx);
    G.cyh = clampf(G.ty, -limy, limy);
    G.j00 = __fdiv_rn(cam.fx, G.zc);
    G.j02 = -__fdiv_rn(__fmul_rn(cam.fx, G.cxh), G.zc);
    G.j11 = __fdiv_rn(cam.fy, G.zc);
    G.j12 = -__fdiv_rn(__fmul_rn(cam.fy, G.cyh), G.zc);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        G.T[0][k] = __fmaf_rn(G.j00, V[k], __fmul_rn(G.j02, V[8 + k]));
        G.T[1][k] = __fmaf_rn(G.j11, V[4 + k], __fmul_rn(G.j12, V[8 + k]));
    }
    float A[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            A[a][k] = __fmaf_rn(G.T[a][0], G.Sig[0][k],
                                __fmaf_rn(G.T[a][1], G.Sig[1][k], __fmul_rn(G.T[a][2], G.Sig[2][k])));
    G.cov_a = __fadd_rn(__fmaf_rn(A[0][0], G.T[0][0], __fmaf_rn(A[0][1], G.T[0][1], __fmul_rn(A[0][2], G.T[0][2]))), 0.3f);
    G.cov_b = __fmaf_rn(A[0][0], G.T[1][0], __fmaf_rn(A[0][1], G.T[1][1], __fmul_rn(A[0][2], G.T[1][2])));
    G.cov_c = __fadd_rn(__fmaf_rn(A[1][0], G.T[1][0], __fmaf_rn(A[1][1], G.T[1][1], __fmul_rn(A[1][2], G.T[1][2]))), 0.3f);
    G.det = __fsub_rn(__fmul_rn(G.cov_a, G.cov_c), __fmul_rn(G.cov_b, G.cov_b));
    if (!(G.det > 0.0f) || !isfinite(G.det)) return false;
    return true;
}

// Real orthonormal SH, k = l^2 + l + m.  Constants: 1/(2 sqrt(pi)), sqrt(3/(4 pi)),
// sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4, sqrt(35/(2 pi))/4, sqrt(105/pi)/2,
// sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float K0 = 0.28209479177387814f;
constexpr float K1 = 0.4886025119029199f;
constexpr float K2A = 1.0925484305920792f;
constexpr float K2B = 0.31539156525252005f;
constexpr float K2C = 0.5462742152960396f;
constexpr float K3A = 0.5900435899266435f;
constexpr float K3B = 2.890611442640554f;
constexpr float K3C = 0.4570457994644658f;
constexpr float K3D = 0.3731763325901154f;
constexpr float K3E = 1.445305721320277f;

__device__ __forceinline__ void sh_eval(int K, float x, float y, float z, float Y[16]) {
    Y[0] = K0;
    if (K > 1) {
        Y[1] = K1 * y;
        Y[2] = K1 * z;
        Y[3] = K1 * x;
    }
    if (K > 4) {
        Y[4] = K2A * x * y;
        Y[5] = K2A * y * z;
        Y[6] = K2B * (3.0f * z * z - 1.0f);
        Y[7] = K2A * x * z;
        Y[8] = K2C * (x * x - y * y);
    }
    if (K > 9) {
        Y[9] = K3A * y * (3.0f * x * x - y * y);
        Y[10] = K3B * x * y * z;
        Y[11] = K3C * y * (5.0f * z * z - 1.0f);
        Y[12] = K3D * z * (5.0f * z * z - 3.0f);
        Y[13] = K3C * x * (5.0f * z * z - 1.0f);
        Y[14] = K3E * z * (x * x - y * y);
        Y[15] = K3A * x * (x * x - 3.0f * y * y);
    }
}

// d/d(x, y, z) of sum_k w_k Y_k (Cartesian polynomial forms above).
__device__ __forceinline__ void sh_grad(int K, float x, float y, float z, const float w[16],
                                        float d[3]) {
    d[0] = d[1] = d[2] = 0.0f;
    if (K > 1) {
        d[0] += K1 * w[3];
        d[1] += K1 * w[1];
        d[2] += K1 * w[2];
    }
    if (K > 4) {
        d[0] += K2A * (w[4] * y + w[7] * z) + K2C * w[8] * 2.0f * x;
        d[1] += K2A * (w[4] * x + w[5] * z) - K2C * w[8] * 2.0f * y;
        d[2] += K2A * (w[5] * y + w[7] * x) + K2B * w[6] * 6.0f * z;
    }
    if (K > 9) {
        const float a = 5.0f * z * z - 1.0f;
        d[0] += K3A * w[9] * 6.0f * x * y + K3B * w[10] * y * z + K3C * w[13] * a +
                K3E * w[14] * 2.0f * x * z + K3A * w[15] * 3.0f * (x * x - y * y);
        d[1] += K3A * w[9] * 3.0f * (x * x - y * y) + K3B * w[10] * x * z + K3C * w[11] * a -
                K3E * w[14] * 2.0f * y * z - K3A * w[15] * 6.0f * x * y;
        d[2] += K3B * w[10] * x * y + K3C * w[11] * 10.0f * y * z + K3D * w[12] * (15.0f * z * z - 3.0f) +
                K3C * w[13] * 10.0f * x * z + K3E * w[14] * (x * x - y * y);
    }
}

__device__ __forceinline__ void camera_centre(const pgs_camera& cam, float c[3]) {
    const float* V = cam.viewmat;
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = -(V[k] * V[3] + V[4 + k] * V[7] + V[8 + k] * V[11]);
}

// The reach tests of a warp's rectangles, load-balanced: the candidate tiles of the 32 lanes'
// rectangles are numbered in lane order (row-major inside each rectangle) and evaluated 32 per
// round, candidate k by lane k mod 32 with its owner's parameters (found by a binary search over
// the lanes' inclusive counts); a lane's count and bit mask of reached tiles (rectangles of <= 32
// tiles) come from the round ballots over its own candidates.  Every lane of the warp calls it;
// the warp's rectangles hold at most 32 x 1024 candidates.  For a lane with `super` set (a rectangle
// of more than 32 tiles whose super-tile rectangle starts at (sx0, sy0) and spans at most 2 x 2)
// the lane that evaluates a reached candidate also sets its bit in the owner's super-tile masks,
// s_sm[4 owner + slot] (the warp's 32 x 4 words of shared memory, cleared by the owners before).
__device__ __forceinline__ void warp_reach(uint32_t area, uint32_t w, uint32_t x0, uint32_t y0, float u, float v,
                                           float ca, float cb, float cc, float sx, float sy, int T, uint32_t& count,
                                           uint32_t& hits, bool super, uint32_t sx0, uint32_t sy0,
                                           uint32_t* s_sm) {
    constexpr unsigned kAll = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t incl = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kAll, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t total = __shfl_sync(kAll, incl, 31);
    const uint32_t first = incl - area;  // this lane's first candidate
    count = 0;
    hits = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t k = base + lane;
        int lo = 0, hi = 31;  // owner of candidate k: the first lane whose inclusive count exceeds k
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            const uint32_t im = __shfl_sync(kAll, incl, mid);
            if (lo < hi) {
                if (im > k) hi = mid;
                else lo = mid + 1;
            }
        }
        const uint32_t ofirst = __shfl_sync(kAll, first, lo), ow = __shfl_sync(kAll, w, lo);
        const uint32_t ox0 = __shfl_sync(kAll, x0, lo), oy0 = __shfl_sync(kAll, y0, lo);
        const float ou = __shfl_sync(kAll, u, lo), ov = __shfl_sync(kAll, v, lo);
        const float oca = __shfl_sync(kAll, ca, lo), ocb = __shfl_sync(kAll, cb, lo), occ = __shfl_sync(kAll, cc, lo);
        const float osx = __shfl_sync(kAll, sx, lo), osy = __shfl_sync(kAll, sy, lo);
        const int oT = __shfl_sync(kAll, T, lo);
        const bool osuper = __shfl_sync(kAll, super, lo);
        const uint32_t osx0 = __shfl_sync(kAll, sx0, lo), osy0 = __shfl_sync(kAll, sy0, lo);
        bool h = false;
        if (k < total) {  // then the owner's rectangle is not empty (ow >= 1)
            const uint32_t local = k - ofirst;
            const uint32_t dy = local / ow, dx = local - dy * ow;
            const uint32_t tx = ox0 + dx, ty = oy0 + dy;
            h = tile_hit(ou, ov, oca, ocb, occ, osx, osy, (int)tx, (int)ty, oT);
            if (h && osuper)
                atomicOr(&s_sm[4 * lo + 2u * (ty / kSuperH - osy0) + (tx / kSuperW - osx0)],
                         1u << ((ty % kSuperH) * kSuperW + (tx % kSuperW)));
        }
        const uint32_t hb = __ballot_sync(kAll, h);
        // this lane's candidates in the round: [s0, s1), at lanes s0 - base ..
        const uint32_t s0 = max(first, base), s1 = min(incl, base + 32u);
        if (s1 > s0) {
            const uint32_t nb = s1 - s0;
            const uint32_t mine = (hb >> (s0 - base)) & (nb == 32u ? kAll : (1u << nb) - 1u);
            count += __popc(mine);
            if (area <= 32u) hits |= mine << (s0 - first);
        }
    }
}

// Project Gaussian i of g through cam (tiles of T x T pixels, grid TX x TY) and write its record at
// item j.  Every lane of the warp calls it (the reach tests are warp-collective); lanes with
// active == false only take part in them.
template <int DEG>
__device__ __forceinline__ uint32_t project_item(const pgs_gaussians& g, int64_t i, const pgs_camera& cam,
                                                 int TX, int TY, int T, int64_t j, const Scratch& sc, bool active,
                                                 uint32_t* s_sm) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int64_t n = g.n;
    uint32_t count = 0;
    float mu[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f}, logit = 0.f;
    if (active) {
        mu[0] = g.means[i];
        mu[1] = g.means[n + i];
        mu[2] = g.means[2 * n + i];
        ls[0] = g.log_scales[i];
        ls[1] = g.log_scales[n + i];
        ls[2] = g.log_scales[2 * n + i];
        q[0] = g.quats[i];
        q[1] = g.quats[n + i];
        q[2] = g.quats[2 * n + i];
        q[3] = g.quats[3 * n + i];
        logit = g.opacity_logits[i];
    }
    bool finite = isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(ls[0]) &&
                  isfinite(ls[1]) && isfinite(ls[2]) && isfinite(q[0]) && isfinite(q[1]) &&
                  isfinite(q[2]) && isfinite(q[3]) && isfinite(logit);
    Geo G;
    bool vis = active && finite && geometry(mu, ls, q, cam, G);
    uint32_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    float con_a = 0.f, con_b = 0.f, con_c = 0.f;  // conic, decision path
    float sx = 0.f, sy = 0.f;                      // slopes of the reach test's line minima
    uint32_t hits = 0;                             // reached tiles of a rectangle of <= 32
    if (vis) {
        // per-axis 3-sigma extents: the bounding box of the 3-sigma ellipse of the 2-D covariance
        const float rx = ceilf(__fmul_rn(3.0f, __fsqrt_rn(G.cov_a)));
        const float ry = ceilf(__fmul_rn(3.0f, __fsqrt_rn(G.cov_c)));
        vis = isfinite(rx) && isfinite(ry);
        if (vis) {
            const float tf = (float)T;  // a power of two: the division is an exact scaling
            x0 = (uint32_t)clampf(floorf(__fdiv_rn(__fsub_rn(G.u, rx), tf)), 0.0f, (float)TX);
            x1 = (uint32_t)clampf(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(G.u, rx), tf)), 1.0f), 0.0f, (float)TX);
            y0 = (uint32_t)clampf(floorf(__fdiv_rn(__fsub_rn(G.v, ry), tf)), 0.0f, (float)TY);
            y1 = (uint32_t)clampf(__fadd_rn(floorf(__fdiv_rn(__fadd_rn(G.v, ry), tf)), 1.0f), 0.0f, (float)TY);
            const float inv = __fdiv_rn(1.0f, G.det);
            con_a = __fmul_rn(G.cov_c, inv);
            con_b = __fmul_rn(-G.cov_b, inv);
            con_c = __fmul_rn(G.cov_a, inv);
            sx = __fdiv_rn(con_b, con_a);
            sy = __fdiv_rn(con_b, con_c);
        }
    }
    // of the rectangle's tiles, those whose pixel centres the 3-sigma ellipse reaches
    const uint32_t rw = vis ? x1 - x0 : 0u, area = vis ? rw * (y1 - y0) : 0u;  // at most 65535^2
    // super-tile masks of rectangles of more than 32 tiles whose super-tile rectangle spans at most
    // 2 x 2 (smaller rectangles keep their reach bits in hitmask)
    const uint2 rect = make_uint2(x0 | (y0 << 16), x1 | (y1 << 16));
    const bool super = area > 0u && small_super_rect(rect);
    const uint32_t sx0 = x0 / kSuperW, sy0 = y0 / kSuperH;
    uint4 sm = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t lane = threadIdx.x & 31;
    uint32_t* const warp_sm = s_sm + 128 * (threadIdx.x >> 5);  // 32 lanes x 4 slots
#pragma unroll
    for (int k = 0; k < 4; ++k) warp_sm[4 * lane + k] = 0u;
    __syncwarp();
    if (__any_sync(0xffffffffu, area > 1024u)) {
        // a large rectangle in the warp: each lane walks its own
        uint32_t k = 0;
        for (uint32_t ty = y0; ty < y1 && vis; ++ty)
            for (uint32_t tx = x0; tx < x1; ++tx, ++k) {
                const bool h = tile_hit(G.u, G.v, con_a, con_b, con_c, sx, sy, (int)tx, (int)ty, T);
                count += h;
                if (area <= 32u && h) hits |= 1u << k;
                if (super && area > 32u && h) smask_add(sm, tx, ty, sx0, sy0);
            }
    } else {
        warp_reach(area, rw, x0, y0, vis ? G.u : 0.f, vis ? G.v : 0.f, con_a, con_b, con_c, sx, sy, T, count, hits,
                   super && area > 32u, sx0, sy0, warp_sm);
        __syncwarp();
        if (super && area > 32u)
            sm = make_uint4(warp_sm[4 * lane], warp_sm[4 * lane + 1], warp_sm[4 * lane + 2], warp_sm[4 * lane + 3]);
    }
    if (!active) return 0xffffffffu;
    if (count > 0) {
        // value path: opacity, colour (the conic is the decision path's)
        const float opacity = 1.0f / (1.0f + expf(-logit));
        float cc[3];
        camera_centre(cam, cc);
        float d[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
        const float inv_len = 1.0f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] *= inv_len;
        d[1] *= inv_len;
        d[2] *= inv_len;
        float Y[16];
        sh_eval(K, d[0], d[1], d[2], Y);
        float rgb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += g.sh[((int64_t)c * K + k) * n + i] * Y[k];
            rgb[c] = fmaxf(acc, 0.0f);
        }
        if (!isfinite(rgb[0]) || !isfinite(rgb[1]) || !isfinite(rgb[2])) {
            count = 0;
            finite = false;
        } else {
            sc.xyo[j] = make_float4(G.u, G.v, opacity, 0.0f);
            sc.conic[j] = make_float4(con_a, con_b, con_c, 0.0f);
            sc.rgb[j] = make_float4(rgb[0], rgb[1], rgb[2], 0.0f);
            sc.depth_bits[j] = __float_as_uint(G.zc);
            sc.rect[j] = rect;
            sc.hitmask[j] = hits;
            if (super && area > 32u) sc.smask[j] = sm;
        }
    }
    if (!finite) atomicOr(sc.status, kStatusNonfinite);
    sc.touched[j] = count;
    // depth-sort input: visible Gaussians by depth bits, culled ones last
    const uint32_t key = count > 0 ? sc.depth_bits[j] : 0xffffffffu;
    reinterpret_cast<uint32_t*>(sc.dkeys[0])[j] = key;
    sc.dvals[0][j] = (uint32_t)j;
    return key;
}

template <int DEG>
__global__ void __launch_bounds__(kProjBlock)
k_project_fwd(pgs_gaussians g, pgs_camera cam, int TX, int TY, int T, Scratch sc, ZeroPlan zero) {
    const int64_t n = g.n;
    const int64_t i = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    __shared__ uint32_t s_sm[4 * kProjBlock];
    project_item<DEG>(g, i < n ? i : 0, cam, TX, TY, T, i, sc, i < n, s_sm);
    if (i == 0) {
        *sc.dcount = (unsigned long long)n;
        *sc.dblocks = (uint32_t)((n + kDepthTile - 1) / kDepthTile);
    }
    // the binning's scratch, grid-stride (a few MB against the projection's reads)
    const uint64_t stride = (uint64_t)gridDim.x * kProjBlock;
#pragma unroll
    for (int r = 0; r < kZeroRegions; ++r) {
        if (r >= zero.count) break;
        uint32_t* const dst = zero.p[r];
        for (uint64_t w = (uint64_t)i; w < zero.words[r]; w += stride) dst[w] = 0u;
    }
}

// last render whose first item is <= j
__device__ __forceinline__ int render_of_item(const RenderDesc* __restrict__ renders, int R, int64_t j) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (renders[mid].item_base <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched projection: item j = (render r, Gaussian j - item_base of r's scene).
template <int DEG>
__global__ void __launch_bounds__(kProjBlock)
k_project_fwd_batch(const RenderDesc* __restrict__ renders, int R, const SceneDesc* __restrict__ scenes,
                    int64_t items, Scratch sc) {
    const int64_t j = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    const bool active = j < items;
    const RenderDesc& rd = renders[active ? render_of_item(renders, R, j) : 0];
    __shared__ uint32_t s_sm[4 * kProjBlock];
    project_item<DEG>(scenes[rd.scene].params, active ? j - rd.item_base : 0, rd.cam, rd.TX, rd.TY, rd.tile, j, sc,
                      active, s_sm);
    if (j == 0) {
        *sc.dcount = (unsigned long long)items;
        *sc.dblocks = (uint32_t)((items + kDepthTile - 1) / kDepthTile);
    }
}

// Backward of one Gaussian: screen-space gradient (du, dv, d conic, d opacity, d rgb) ->
// parameters.  Matrix form: H = -Q Gq Q (Q the conic matrix, Gq its gradient with the
// off-diagonal halved), dSigma = T^T H T, dT = 2 H T Sigma, dM = 2 dSigma M.
struct GradParts {
    float dmu[3], dls[3], dq[4], dlogit;
    float gc[3];  // colour gradient after the clamp; d sh[c][k] = gc[c] Y[k]
    float Y[16];
};

template <int DEG>
__device__ __forceinline__ void chain(const pgs_gaussians& g, const pgs_camera& cam,
                                      const float* __restrict__ grad2d, int64_t gstride, int64_t gidx,
                                      int64_t i, GradParts& out) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int64_t n = g.n;
    const float mu[3] = {g.means[i], g.means[n + i], g.means[2 * n + i]};
    const float ls[3] = {g.log_scales[i], g.log_scales[n + i], g.log_scales[2 * n + i]};
    const float q[4] = {g.quats[i], g.quats[n + i], g.quats[2 * n + i], g.quats[3 * n + i]};
    Geo G;
    geometry(mu, ls, q, cam, G);
    float gr[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) gr[k] = grad2d[k * gstride + gidx];
    const float* V = cam.viewmat;

    // colour -> SH coefficients and view direction
    float cc[3];
    camera_centre(cam, cc);
    float d[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    const float dist = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float inv_len = 1.0f / dist;
    d[0] *= inv_len;
    d[1] *= inv_len;
    d[2] *= inv_len;
    float* Y = out.Y;
    sh_eval(K, d[0], d[1], d[2], Y);
    float wsum[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) wsum[k] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.5f;
        float coef[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            coef[k] = g.sh[((int64_t)c * K + k) * n + i];
            acc += coef[k] * Y[k];
        }
        const float gc = acc < 0.0f ? 0.0f : gr[6 + c];  // zero gradient through the clamp
        out.gc[c] = gc;
#pragma unroll
        for (int k = 0; k < K; ++k) wsum[k] += gc * coef[k];
    }
    float ddir[3];
    sh_grad(K, d[0], d[1], d[2], wsum, ddir);
    const float dd = ddir[0] * d[0] + ddir[1] * d[1] + ddir[2] * d[2];
    float dmu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] = (ddir[k] - d[k] * dd) * inv_len;

    // opacity logit
    const float o = 1.0f / (1.0f + expf(-g.opacity_logits[i]));
    out.dlogit = gr[5] * o * (1.0f - o);

    // conic -> 2-D covariance
    const float inv_det = 1.0f / G.det;
    const float qa = G.cov_c * inv_det, qb = -G.cov_b * inv_det, qc = G.cov_a * inv_det;
    const float ga = gr[2], gb = 0.5f * gr[3], gcn = gr[4];
    const float P00 = qa * ga + qb * gb, P01 = qa * gb + qb * gcn;
    const float P10 = qb * ga + qc * gb, P11 = qb * gb + qc * gcn;
    const float H00 = -(P00 * qa + P01 * qb);
    const float H01 = -0.5f * ((P00 * qb + P01 * qc) + (P10 * qa + P11 * qb));
    const float H11 = -(P10 * qb + P11 * qc);
    const float H[2][2] = {{H00, H01}, {H01, H11}};

    // dSigma = T^T H T ; dT = 2 H T Sigma
    float HT[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) HT[a][k] = H[a][0] * G.T[0][k] + H[a][1] * G.T[1][k];
    float dSig[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) dSig[m][k] = G.T[0][m] * HT[0][k] + G.T[1][m] * HT[1][k];
    float dT[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dT[a][k] = 2.0f * (HT[a][0] * G.Sig[0][k] + HT[a][1] * G.Sig[1][k] + HT[a][2] * G.Sig[2][k]);
    // T = J W
    float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dJ00 += dT[0][k] * V[k];
        dJ02 += dT[0][k] * V[8 + k];
        dJ11 += dT[1][k] * V[4 + k];
        dJ12 += dT[1][k] * V[8 + k];
    }
    const float z = G.zc, iz = 1.0f / z, iz2 = iz * iz;
    float dpc[3] = {0.f, 0.f, 0.f};
    dpc[2] += -cam.fx * iz2 * dJ00 + cam.fx * G.cxh * iz2 * dJ02 - cam.fy * iz2 * dJ11 +
              cam.fy * G.cyh * iz2 * dJ12;
    const float dcxh = -cam.fx * iz * dJ02, dcyh = -cam.fy * iz * dJ12;
    if (!G.xclamp) {
        dpc[0] += dcxh * iz;
        dpc[2] -= dcxh * G.xc * iz2;
    }
    if (!G.yclamp) {
        dpc[1] += dcyh * iz;
        dpc[2] -= dcyh * G.yc * iz2;
    }
    dpc[0] += gr[0] * cam.fx * iz;
    dpc[2] -= gr[0] * cam.fx * G.xc * iz2;
    dpc[1] += gr[1] * cam.fy * iz;
    dpc[2] -= gr[1] * cam.fy * G.yc * iz2;
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] += dpc[0] * V[k] + dpc[1] * V[4 + k] + dpc[2] * V[8 + k];

    // Sigma = M M^T, M = R diag(s)
    float dR[3][3], dls[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ds = 0.f;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float dM = 2.0f * (dSig[p][0] * G.M[0][k] + dSig[p][1] * G.M[1][k] + dSig[p][2] * G.M[2][k]);
            dR[p][k] = dM * G.s[k];
            ds += dM * G.R[p][k];
        }
        dls[k] = ds * G.s[k];
    }
    const float w = G.w, x = G.x, y = G.y, zq = G.z;
    const float dw = 2.f * (-zq * dR[0][1] + y * dR[0][2] + zq * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    const float dx = 2.f * (y * dR[0][1] + zq * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                            zq * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    const float dy = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + zq * dR[1][2] -
                            w * dR[2][0] + zq * dR[2][1] - 2.f * y * dR[2][2]);
    const float dz = 2.f * (-2.f * zq * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] -
                            2.f * zq * dR[1][1] + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float dot = dw * w + dx * x + dy * y + dz * zq;
    const float iq = 1.0f / G.qn;
    out.dq[0] = (dw - w * dot) * iq;
    out.dq[1] = (dx - x * dot) * iq;
    out.dq[2] = (dy - y * dot) * iq;
    out.dq[3] = (dz - zq * dot) * iq;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        out.dls[k] = dls[k];
        out.dmu[k] = dmu[k];
    }
}

// Parameter row r of the (11 + 3K) x n matrix: its group (0 means, 1 log-scales, 2 quaternions,
// 3 opacity logits, 4 SH) and its row inside the group.
__device__ __forceinline__ constexpr int row_group(int r) {
    return r < 3 ? 0 : (r < 6 ? 1 : (r < 10 ? 2 : (r == 10 ? 3 : 4)));
}
__device__ __forceinline__ constexpr int row_sub(int r) {
    return r < 3 ? r : (r < 6 ? r - 3 : (r < 10 ? r - 6 : (r == 10 ? 0 : r - 11)));
}

struct Rows {
    float* __restrict__ g[5];
};

__device__ __forceinline__ Rows rows_of(const pgs_gaussians& q) {
    return Rows{{q.means, q.log_scales, q.quats, q.opacity_logits, q.sh}};
}

// gradient of parameter row r of one Gaussian (rows 11.. are SH coefficients: gc[c] Y[k])
template <int DEG>
__device__ __forceinline__ float grad_row(const GradParts& gp, int r) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    if (r < 3) return gp.dmu[r];
    if (r < 6) return gp.dls[r - 3];
    if (r < 10) return gp.dq[r - 6];
    if (r == 10) return gp.dlogit;
    return gp.gc[(r - 11) / K] * gp.Y[(r - 11) % K];
}

__device__ __forceinline__ void zero_parts(GradParts& gp) {
#pragma unroll
    for (int k = 0; k < 3; ++k) gp.dmu[k] = gp.dls[k] = gp.gc[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) gp.dq[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) gp.Y[k] = 0.f;
    gp.dlogit = 0.f;
}

constexpr int kChunk = 8;  // parameter rows whose loads are issued together

__device__ __forceinline__ void prefetch_l2(const float* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Start the DRAM reads of one Gaussian's Adam moments (rows of m and v) into L2, so that they
// overlap the gradient chain instead of following it (the kernel's register use leaves 16 warps
// per SM, too few to cover the moments' latency by themselves).
template <int ROWS>
__device__ __forceinline__ void prefetch_moments(const Rows& Mm, const Rows& Vv, int64_t n, int64_t i) {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int64_t idx = (int64_t)row_sub(r) * n + i;
        prefetch_l2(Mm.g[row_group(r)] + idx);
        prefetch_l2(Vv.g[row_group(r)] + idx);
    }
}

template <int DEG>
__global__ void __launch_bounds__(kProjBlock, 2)
k_project_bwd(pgs_gaussians g, pgs_camera cam, Scratch sc, pgs_gaussians out) {
    constexpr int ROWS = 11 + 3 * (DEG + 1) * (DEG + 1);
    const int64_t n = g.n;
    const int64_t i = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    if (i >= n || sc.touched[i] == 0) return;
    GradParts gp;
    chain<DEG>(g, cam, sc.grad2d, n, i, i, gp);
    const Rows O = rows_of(out);
#pragma unroll
    for (int r0 = 0; r0 < ROWS; r0 += kChunk) {
        float acc[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
            if (r0 + j < ROWS) acc[j] = O.g[row_group(r0 + j)][(int64_t)row_sub(r0 + j) * n + i];
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
            if (r0 + j < ROWS)
                O.g[row_group(r0 + j)][(int64_t)row_sub(r0 + j) * n + i] = acc[j] + grad_row<DEG>(gp, r0 + j);
    }
}

// Fused projection backward + Adam for one training step on one view: the parameter gradient of
// each Gaussian (zero for culled ones) is consumed in registers by the Adam update of its 11 + 3K
// parameters, so it never round-trips through memory.
struct AdamStep {
    float lr[6];  // learning rates already divided by 1 - b1^t
    float b1, b2, omb1, omb2, eps, isb;  // isb = 1 / sqrt(1 - b2^t)
};

template <int DEG>
__global__ void __launch_bounds__(kProjBlock, 2)
k_project_bwd_adam(pgs_gaussians g, pgs_camera cam, Scratch sc, pgs_gaussians m, pgs_gaussians v,
                   AdamStep a) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int ROWS = 11 + 3 * K;
    const int64_t n = g.n;
    const int64_t i = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    if (i >= n) return;
    const Rows Pp = rows_of(g), Mm = rows_of(m), Vv = rows_of(v);
    prefetch_moments<ROWS>(Mm, Vv, n, i);
    GradParts gp;
    if (sc.touched[i] != 0) chain<DEG>(g, cam, sc.grad2d, n, i, i, gp);
    else zero_parts(gp);
#pragma unroll
    for (int r0 = 0; r0 < ROWS; r0 += kChunk) {
        float pp[kChunk], mm[kChunk], vv[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            if (r0 + j < ROWS) {
                const int gi = row_group(r0 + j);
                const int64_t idx = (int64_t)row_sub(r0 + j) * n + i;
                pp[j] = Pp.g[gi][idx];
                mm[j] = Mm.g[gi][idx];
                vv[j] = Vv.g[gi][idx];
            }
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int r = r0 + j;
            if (r < ROWS) {
                const int gi = row_group(r);
                const float lr = gi < 4 ? a.lr[gi] : (row_sub(r) % K == 0 ? a.lr[4] : a.lr[5]);
                adam_update(pp[j], mm[j], vv[j], grad_row<DEG>(gp, r), a.b1, a.b2, a.omb1, a.omb2, lr,
                            a.isb, a.eps);
                const int64_t idx = (int64_t)row_sub(r) * n + i;
                Pp.g[gi][idx] = pp[j];
                Mm.g[gi][idx] = mm[j];
                Vv.g[gi][idx] = vv[j];
            }
        }
    }
}

// Adam bias corrections for step t read from the device (so a captured step graph advances it).
struct AdamDev {
    float lr[6];
    float b1, b2, omb1, omb2, eps;
};

// Counts a completed step; a step whose pairs overflowed the capacity did no Adam update and is
// not counted.
__global__ void k_step_tick(int64_t* step, const int32_t* status) {
    if ((*status & kStatusCapacity) == 0) *step += 1;
}

__device__ __forceinline__ int scene_of(const SceneDesc* __restrict__ scenes, int S, int64_t k) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (scenes[mid].gauss_base <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched backward + Adam: one thread per Gaussian of every scene.  The Gaussian's parameter
// gradient is summed over the scene's renders (views) in shared memory, row by row, and then
// consumed by the Adam update (step t = completed steps + 1) of the scene's parameters.  When the
// step's pairs overflowed the capacity (the renders are incomplete) nothing is written.
template <int DEG>
__global__ void __launch_bounds__(kProjBlock, 2)
k_bwd_adam_batch(const RenderDesc* __restrict__ renders, const SceneDesc* __restrict__ scenes, int S,
                 int64_t gauss_total, int64_t items, Scratch sc, AdamDev a, const int64_t* __restrict__ step) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int ROWS = 11 + 3 * K;
    extern __shared__ float s_acc[];  // [ROWS][kProjBlock]
    __shared__ float s_lr[6], s_isb;
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        const double t = (double)(*step + 1);
        const double bc1 = 1.0 - pow((double)a.b1, t), bc2 = 1.0 - pow((double)a.b2, t);
        for (int q = 0; q < 6; ++q) s_lr[q] = (float)((double)a.lr[q] / bc1);
        s_isb = (float)(1.0 / sqrt(bc2));
        s_skip = (*sc.status & kStatusCapacity) != 0;
    }
    const int64_t k = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    float* acc = s_acc + threadIdx.x;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r * kProjBlock] = 0.f;
    __syncthreads();
    const float isb = s_isb;
    if (k >= gauss_total || s_skip) return;
    const SceneDesc& sd = scenes[scene_of(scenes, S, k)];
    const int64_t i = k - sd.gauss_base;
    const int64_t n = sd.params.n;
    prefetch_moments<ROWS>(rows_of(sd.m), rows_of(sd.v), n, i);
    for (int rr = 0; rr < sd.n_renders; ++rr) {
        const RenderDesc& rd = renders[sd.first_render + rr];
        const int64_t j = rd.item_base + i;
        if (sc.touched[j] == 0) continue;
        GradParts gp;
        chain<DEG>(sd.params, rd.cam, sc.grad2d, items, j, i, gp);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) acc[r * kProjBlock] += grad_row<DEG>(gp, r);
    }
    const Rows Pp = rows_of(sd.params), Mm = rows_of(sd.m), Vv = rows_of(sd.v);
#pragma unroll
    for (int r0 = 0; r0 < ROWS; r0 += kChunk) {
        float pp[kChunk], mm[kChunk], vv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (r0 + q < ROWS) {
                const int gi = row_group(r0 + q);
                const int64_t idx = (int64_t)row_sub(r0 + q) * n + i;
                pp[q] = Pp.g[gi][idx];
                mm[q] = Mm.g[gi][idx];
                vv[q] = Vv.g[gi][idx];
            }
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int r = r0 + q;
            if (r < ROWS) {
                const int gi = row_group(r);
                const float lr = gi < 4 ? s_lr[gi] : (row_sub(r) % K == 0 ? s_lr[4] : s_lr[5]);
                adam_update(pp[q], mm[q], vv[q], acc[r * kProjBlock], a.b1, a.b2, a.omb1, a.omb2, lr, isb,
                            a.eps);
                const int64_t idx = (int64_t)row_sub(r) * n + i;
                Pp.g[gi][idx] = pp[q];
                Mm.g[gi][idx] = mm[q];
                Vv.g[gi][idx] = vv[q];
            }
        }
    }
}

// Batched projection backward without Adam: one thread per Gaussian of every scene; the
// Gaussian's parameter gradient is summed over the scene's renders (views) in shared memory, row
// by row, and added to the scene's gradient buffer grads[scene] (Eq. 10's scatter of every view
// into the canonical parameter buffer).  Nothing is written when the pairs overflowed the capacity.
template <int DEG>
__global__ void __launch_bounds__(kProjBlock, 2)
k_bwd_batch(const RenderDesc* __restrict__ renders, const SceneDesc* __restrict__ scenes, int S,
            int64_t gauss_total, int64_t items, Scratch sc, const pgs_gaussians* __restrict__ grads) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int ROWS = 11 + 3 * K;
    extern __shared__ float s_acc[];  // [ROWS][kProjBlock]
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (*sc.status & kStatusCapacity) != 0;
    const int64_t k = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    float* acc = s_acc + threadIdx.x;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r * kProjBlock] = 0.f;
    __syncthreads();
    if (k >= gauss_total || s_skip) return;
    const int si = scene_of(scenes, S, k);
    const SceneDesc& sd = scenes[si];
    const int64_t i = k - sd.gauss_base;
    const int64_t n = sd.params.n;
    bool any = false;
    for (int rr = 0; rr < sd.n_renders; ++rr) {
        const RenderDesc& rd = renders[sd.first_render + rr];
        const int64_t j = rd.item_base + i;
        if (sc.touched[j] == 0) continue;
        any = true;
        GradParts gp;
        chain<DEG>(sd.params, rd.cam, sc.grad2d, items, j, i, gp);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) acc[r * kProjBlock] += grad_row<DEG>(gp, r);
    }
    if (!any) return;
    const Rows Gg = rows_of(grads[si]);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int64_t idx = (int64_t)row_sub(r) * n + i;
        Gg.g[row_group(r)][idx] += acc[r * kProjBlock];
    }
}

}  // namespace

int launch_project_fwd(const pgs_gaussians& g, const pgs_camera& cam, int TX, int TY, int T,
                       const Scratch& sc, const ZeroPlan& zero, cudaStream_t s) {
    const int64_t blocks = (g.n + kProjBlock - 1) / kProjBlock;
    if (blocks == 0) {
        clear_zero_plan(zero, s);
        return 0;
    }
    switch (g.sh_degree) {
        case 0: k_project_fwd<0><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, TX, TY, T, sc, zero); break;
        case 1: k_project_fwd<1><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, TX, TY, T, sc, zero); break;
        case 2: k_project_fwd<2><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, TX, TY, T, sc, zero); break;
        default: k_project_fwd<3><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, TX, TY, T, sc, zero); break;
    }
    return 1;
}

int launch_project_bwd(const pgs_gaussians& g, const pgs_camera& cam, const Scratch& sc,
                       pgs_gaussians& grads, cudaStream_t s) {
    const int64_t blocks = (g.n + kProjBlock - 1) / kProjBlock;
    if (blocks == 0) return 0;
    switch (g.sh_degree) {
        case 0: k_project_bwd<0><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, grads); break;
        case 1: k_project_bwd<1><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, grads); break;
        case 2: k_project_bwd<2><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, grads); break;
        default: k_project_bwd<3><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, grads); break;
    }
    return 1;
}

int launch_project_bwd_adam(const pgs_gaussians& g, const pgs_camera& cam, const Scratch& sc,
                            pgs_gaussians& m, pgs_gaussians& v, const float lr[6], float b1,
                            float b2, float eps, int64_t t, cudaStream_t s) {
    const int64_t blocks = (g.n + kProjBlock - 1) / kProjBlock;
    if (blocks == 0) return 0;
    AdamStep a;
    const double bc1 = 1.0 - pow((double)b1, (double)t), bc2 = 1.0 - pow((double)b2, (double)t);
    for (int k = 0; k < 6; ++k) a.lr[k] = (float)((double)lr[k] / bc1);
    a.b1 = b1;
    a.b2 = b2;
    a.omb1 = (float)(1.0 - (double)b1);
    a.omb2 = (float)(1.0 - (double)b2);
    a.eps = eps;
    a.isb = (float)(1.0 / sqrt(bc2));
    switch (g.sh_degree) {
        case 0: k_project_bwd_adam<0><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, m, v, a); break;
        case 1: k_project_bwd_adam<1><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, m, v, a); break;
        case 2: k_project_bwd_adam<2><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, m, v, a); break;
        default: k_project_bwd_adam<3><<<(unsigned)blocks, kProjBlock, 0, s>>>(g, cam, sc, m, v, a); break;
    }
    return 1;
}

int launch_project_fwd_batch(const RenderDesc* renders, int R, const SceneDesc* scenes, int deg,
                             int64_t items, const Scratch& sc, cudaStream_t s) {
    const int64_t blocks = (items + kProjBlock - 1) / kProjBlock;
    if (blocks == 0) return 0;
    switch (deg) {
        case 0: k_project_fwd_batch<0><<<(unsigned)blocks, kProjBlock, 0, s>>>(renders, R, scenes, items, sc); break;
        case 1: k_project_fwd_batch<1><<<(unsigned)blocks, kProjBlock, 0, s>>>(renders, R, scenes, items, sc); break;
        case 2: k_project_fwd_batch<2><<<(unsigned)blocks, kProjBlock, 0, s>>>(renders, R, scenes, items, sc); break;
        default: k_project_fwd_batch<3><<<(unsigned)blocks, kProjBlock, 0, s>>>(renders, R, scenes, items, sc); break;
    }
    return 1;
}

int launch_step_tick(int64_t* step, const int32_t* status, cudaStream_t s) {
    k_step_tick<<<1, 1, 0, s>>>(step, status);
    return 1;
}

template <int DEG>
static int launch_bwd_adam_batch_deg(const RenderDesc* renders, const SceneDesc* scenes, int S,
                                     int64_t gauss_total, int64_t items, const Scratch& sc,
                                     const AdamDev& a, const int64_t* step, cudaStream_t s) {
    constexpr int ROWS = 11 + 3 * (DEG + 1) * (DEG + 1);
    const size_t smem = sizeof(float) * ROWS * kProjBlock;
    static bool attr = [&] {
        cudaFuncSetAttribute(k_bwd_adam_batch<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return true;
    }();
    (void)attr;
    const int64_t blocks = (gauss_total + kProjBlock - 1) / kProjBlock;
    k_bwd_adam_batch<DEG><<<(unsigned)blocks, kProjBlock, smem, s>>>(renders, scenes, S, gauss_total,
                                                                     items, sc, a, step);
    return 1;
}

int launch_bwd_adam_batch(const RenderDesc* renders, const SceneDesc* scenes, int S, int deg,
                          int64_t gauss_total, int64_t items, const Scratch& sc, const float lr[6],
                          float b1, float b2, float eps, const int64_t* step, cudaStream_t s) {
    if (gauss_total == 0) return 0;
    AdamDev a;
    for (int k = 0; k < 6; ++k) a.lr[k] = lr[k];
    a.b1 = b1;
    a.b2 = b2;
    a.omb1 = (float)(1.0 - (double)b1);
    a.omb2 = (float)(1.0 - (double)b2);
    a.eps = eps;
    switch (deg) {
        case 0: return launch_bwd_adam_batch_deg<0>(renders, scenes, S, gauss_total, items, sc, a, step, s);
        case 1: return launch_bwd_adam_batch_deg<1>(renders, scenes, S, gauss_total, items, sc, a, step, s);
        case 2: return launch_bwd_adam_batch_deg<2>(renders, scenes, S, gauss_total, items, sc, a, step, s);
        default: return launch_bwd_adam_batch_deg<3>(renders, scenes, S, gauss_total, items, sc, a, step, s);
    }
}

}  // namespace pgs

namespace pgs {

template <int DEG>
static int launch_bwd_batch_deg(const RenderDesc* renders, const SceneDesc* scenes, int S, int64_t gauss_total,
                                int64_t items, const Scratch& sc, const pgs_gaussians* grads, cudaStream_t s) {
    constexpr int ROWS = 11 + 3 * (DEG + 1) * (DEG + 1);
    const size_t smem = sizeof(float) * ROWS * kProjBlock;
    static bool attr = [&] {
        cudaFuncSetAttribute(k_bwd_batch<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return true;
    }();
    (void)attr;
    const int64_t blocks = (gauss_total + kProjBlock - 1) / kProjBlock;
    k_bwd_batch<DEG><<<(unsigned)blocks, kProjBlock, smem, s>>>(renders, scenes, S, gauss_total, items, sc, grads);
    return 1;
}

int launch_bwd_batch(const RenderDesc* renders, const SceneDesc* scenes, int S, int deg, int64_t gauss_total,
                     int64_t items, const Scratch& sc, const pgs_gaussians* grads, cudaStream_t s) {
    if (gauss_total == 0) return 0;
    switch (deg) {
        case 0: return launch_bwd_batch_deg<0>(renders, scenes, S, gauss_total, items, sc, grads, s);
        case 1: return launch_bwd_batch_deg<1>(renders, scenes, S, gauss_total, items, sc, grads, s);
        case 2: return launch_bwd_batch_deg<2>(renders, scenes, S, gauss_total, items, sc, grads, s);
        default: return launch_bwd_batch_deg<3>(renders, scenes, S, gauss_total, items, sc, grads, s);
    }
}

}  // namespace pgs
