// Single-reference cost-volume MVS of the geometry prior (Sec. III-A): depth range from the
// projected sparse points ([0.5 q.05, 1.5 q.95]), reference keyframe by Eq. 4, census matching
// cost over a fronto-parallel plane sweep, SGM aggregation, confidence filter (0.4), fusion.
//
// Readings (the paper names the ingredients; the rest is fixed here):
//   luma Y = 0.299 R + 0.587 G + 0.114 B; census over a 7 x 7 window, 48 bits in raster order of
//   the neighbours (centre skipped), set when the neighbour is darker, outside neighbours clear;
//   D planes uniform in inverse depth, plane 0 the farthest; plane map H_k = K_r (R + t e3^T / d_k)
//   K_t^-1 built in FP64 in a fixed order, rounded to FP32, applied to pixel centres in FP32
//   (products and sums rounded separately, IEEE division: the reference pixel is an integer
//   decided in floating point, so the order is part of the definition); cost = Hamming distance,
//   24 when the point is behind the reference or outside it; SGM over 4 paths with P1 = 8,
//   P2 = 32 in integers; winner-take-all with S2 the best cost two or more planes away, kept when
//   the minimum is interior and 5 (S2 - S1) >= 2 S2 (confidence 1 - S1 / S2 >= 0.4); parabola
//   refinement in inverse depth; kept pixels back-projected in FP64.
//
// Layout: census codes [H][W] u64; cost C [H][W][D] u8, the four paths' L [4][H][W][D] u8 and the
// aggregated cost S [H][W][D] u16, the plane index innermost so a pixel's costs are one contiguous
// run for every path direction.
#include <cmath>

#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int kR = 3;                    // census radius
constexpr int kInvalid = 24;
constexpr int kP1 = 8, kP2 = 32;
constexpr int kCtx = 32, kCty = 8;       // census tile
constexpr int kRun = 32;                 // pixels per cost-volume CTA

__device__ __forceinline__ float luma(float r, float g, float b) {
    return __fadd_rn(__fadd_rn(__fmul_rn(0.299f, r), __fmul_rn(0.587f, g)), __fmul_rn(0.114f, b));
}

__global__ void __launch_bounds__(kCtx * kCty)
k_census(const float* __restrict__ rgb, int W, int H, uint64_t* __restrict__ code) {
    __shared__ float s[kCty + 2 * kR][kCtx + 2 * kR];
    const int x0 = blockIdx.x * kCtx, y0 = blockIdx.y * kCty;
    const size_t plane = (size_t)W * H;
    for (int k = threadIdx.y * kCtx + threadIdx.x; k < (kCty + 2 * kR) * (kCtx + 2 * kR); k += kCtx * kCty) {
        const int r = k / (kCtx + 2 * kR), c = k % (kCtx + 2 * kR);
        const int y = y0 - kR + r, x = x0 - kR + c;
        float v = __int_as_float(0x7f800000);  // outside: +inf, never darker
        if (x >= 0 && x < W && y >= 0 && y < H) {
            const size_t p = (size_t)y * W + x;
            v = luma(rgb[p], rgb[plane + p], rgb[2 * plane + p]);
        }
        s[r][c] = v;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= W || y >= H) return;
    const float ctr = s[threadIdx.y + kR][threadIdx.x + kR];
    uint64_t out = 0;
    int bit = 0;
#pragma unroll
    for (int dy = -kR; dy <= kR; ++dy)
#pragma unroll
        for (int dx = -kR; dx <= kR; ++dx) {
            if (dy == 0 && dx == 0) continue;
            out |= (uint64_t)(s[threadIdx.y + kR + dy][threadIdx.x + kR + dx] < ctr) << bit;
            ++bit;
        }
    code[(size_t)y * W + x] = out;
}

struct CamF {
    float fx, fy, cx, cy;
    float v[12];
};

CamF camf(const pgs_camera& c) {
    CamF o;
    o.fx = c.fx;
    o.fy = c.fy;
    o.cx = c.cx;
    o.cy = c.cy;
    for (int i = 0; i < 12; ++i) o.v[i] = c.viewmat[i];
    return o;
}

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dadd_rn(a, -b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// plane maps H_k (FP64 in the order of the definition, rounded to FP32), thread per plane
__global__ void k_plane_maps(CamF t, CamF r, double inv_far, double step, int D, float* __restrict__ maps) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    double Rt[3][3], tt[3], Rr[3][3], tr[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            Rt[i][j] = t.v[4 * i + j];
            Rr[i][j] = r.v[4 * i + j];
        }
        tt[i] = t.v[4 * i + 3];
        tr[i] = r.v[4 * i + 3];
    }
    double R[3][3], tv[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            R[i][j] = dadd(dadd(dmul(Rr[i][0], Rt[j][0]), dmul(Rr[i][1], Rt[j][1])), dmul(Rr[i][2], Rt[j][2]));
    for (int i = 0; i < 3; ++i)
        tv[i] = dsub(tr[i], dadd(dadd(dmul(R[i][0], tt[0]), dmul(R[i][1], tt[1])), dmul(R[i][2], tt[2])));
    const double fxt = t.fx, fyt = t.fy, cxt = t.cx, cyt = t.cy;
    const double fxr = r.fx, fyr = r.fy, cxr = r.cx, cyr = r.cy;
    const double ax = ddiv(cxt, fxt), ay = ddiv(cyt, fyt);
    const double inv = dadd(inv_far, dmul((double)k, step));
    double g[3][3];
    for (int i = 0; i < 3; ++i) {
        const double m0 = R[i][0], m1 = R[i][1], m2 = dadd(R[i][2], dmul(tv[i], inv));
        g[i][0] = ddiv(m0, fxt);
        g[i][1] = ddiv(m1, fyt);
        g[i][2] = dsub(dsub(m2, dmul(m0, ax)), dmul(m1, ay));
    }
    float* h = maps + 9 * k;
    for (int j = 0; j < 3; ++j) {
        h[j] = __double2float_rn(dadd(dmul(fxr, g[0][j]), dmul(cxr, g[2][j])));
        h[3 + j] = __double2float_rn(dadd(dmul(fyr, g[1][j]), dmul(cyr, g[2][j])));
        h[6 + j] = __double2float_rn(g[2][j]);
    }
}

// cost volume: CTA = D threads (thread k = plane k, its map in registers) over a run of pixels
__global__ void k_cost(const uint64_t* __restrict__ cen_t, const uint64_t* __restrict__ cen_r, int W, int H,
                       int D, const float* __restrict__ maps, uint8_t* __restrict__ C) {
    const int k = threadIdx.x;
    const int y = blockIdx.y, xs = blockIdx.x * kRun;
    float h[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) h[q] = maps[9 * k + q];
    const float fW = (float)W, fH = (float)H;
    const float yc = (float)y + 0.5f;
    for (int x = xs; x < xs + kRun && x < W; ++x) {
        const float xc = (float)x + 0.5f;
        const float a = __fadd_rn(__fadd_rn(__fmul_rn(h[0], xc), __fmul_rn(h[1], yc)), h[2]);
        const float b = __fadd_rn(__fadd_rn(__fmul_rn(h[3], xc), __fmul_rn(h[4], yc)), h[5]);
        const float c = __fadd_rn(__fadd_rn(__fmul_rn(h[6], xc), __fmul_rn(h[7], yc)), h[8]);
        int cost = kInvalid;
        if (c > 0.f) {
            const float u = __fdiv_rn(a, c), v = __fdiv_rn(b, c);
            if (u >= 0.f && u < fW && v >= 0.f && v < fH) {
                const int iu = (int)floorf(u), iv = (int)floorf(v);
                cost = __popcll(cen_t[(size_t)y * W + x] ^ cen_r[(size_t)iv * W + iu]);
            }
        }
        C[((size_t)y * W + x) * D + k] = (uint8_t)cost;
    }
}

// the four SGM paths in one launch (blockIdx.y = direction: 0 left to right, 1 right to left,
// 2 top down, 3 bottom up), warp per scanline, lane holding planes lane * KPL .. + KPL - 1; each
// path writes its own L (<= 48 + P2 = 80, a byte) so the directions run concurrently, and the
// costs of the next steps are loaded ahead (the walk along a line is the only serial part)
template <int KPL>
__global__ void __launch_bounds__(128)
k_sgm(const uint8_t* __restrict__ C, uint8_t* __restrict__ Lall, int W, int H, int D) {
    const int dir = blockIdx.y;
    const int line = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const bool horiz = dir < 2;
    const int lines = horiz ? H : W, len = horiz ? W : H;
    if (line >= lines) return;
    uint8_t* __restrict__ Lout = Lall + (size_t)dir * W * H * D;
    constexpr int kBig = 1 << 20, kAhead = 4;
    auto base_of = [&](int s) {
        const int pos = (dir == 0 || dir == 2) ? s : len - 1 - s;
        const int x = horiz ? pos : line, y = horiz ? line : pos;
        return ((size_t)y * W + x) * D;
    };
    auto load = [&](int s, int (&c)[KPL]) {
        if (s < len) {
            const size_t b = base_of(s);
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane * KPL + j;
                c[j] = k < D ? (int)__ldg(C + b + k) : 0;
            }
        }
    };
    int ring[kAhead][KPL];
#pragma unroll
    for (int a = 0; a < kAhead; ++a) load(a, ring[a]);
    int L[KPL];
    for (int s0 = 0; s0 < len; s0 += kAhead) {
#pragma unroll
        for (int a = 0; a < kAhead; ++a) {
            const int s = s0 + a;
            if (s >= len) break;
            int c[KPL];
#pragma unroll
            for (int j = 0; j < KPL; ++j) c[j] = ring[a][j];
            load(s + kAhead, ring[a]);
            if (s == 0) {
#pragma unroll
                for (int j = 0; j < KPL; ++j) L[j] = lane * KPL + j < D ? c[j] : kBig;
            } else {
                int mloc = kBig;
#pragma unroll
                for (int j = 0; j < KPL; ++j) mloc = min(mloc, L[j]);
                const int m = __reduce_min_sync(0xffffffffu, mloc);
                const int below = __shfl_up_sync(0xffffffffu, L[KPL - 1], 1);   // plane lane*KPL - 1
                const int above = __shfl_down_sync(0xffffffffu, L[0], 1);       // plane lane*KPL + KPL
                int nl[KPL];
#pragma unroll
                for (int j = 0; j < KPL; ++j) {
                    const int k = lane * KPL + j;
                    const int lm = j > 0 ? L[j - 1] : (lane > 0 ? below : kBig);
                    const int lp = j < KPL - 1 ? L[j + 1] : (lane < 31 ? above : kBig);
                    const int best = min(min(L[j], min(lm, lp) + kP1), m + kP2);
                    nl[j] = k < D ? c[j] + best - m : kBig;
                }
#pragma unroll
                for (int j = 0; j < KPL; ++j) L[j] = nl[j];
            }
            const size_t b = base_of(s);
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane * KPL + j;
                if (k < D) Lout[b + k] = (uint8_t)L[j];
            }
        }
    }
}

// S = the sum of the four paths (written out), winner-take-all, confidence, parabola refinement;
// depth (NaN where not kept) and kept flags.  A warp takes 32 consecutive pixels: for each, lanes
// over the planes (as in the SGM walk: coalesced loads and stores) find the minimiser, S2 and the
// neighbours by warp reductions and leave them with lane i for pixel i; then every lane refines its
// own pixel, so the FP64 refinement runs on full warps (GB300's FP64 pipe costs a warp instruction
// the same with one lane or thirty-two).
constexpr int kSelectThreads = 256;

template <int KPL>
__global__ void __launch_bounds__(kSelectThreads)
k_select(const uint8_t* __restrict__ Lall, uint16_t* __restrict__ S, int W, int H, int D, double inv_far,
         double step, float* __restrict__ depth, uint8_t* __restrict__ kept, unsigned long long* __restrict__ count) {
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)W * H;
    const size_t plane = (size_t)n * D;
    const int64_t chunks = (n + 31) / 32, warps = (int64_t)gridDim.x * (kSelectThreads / 32);
    constexpr int kBig = 1 << 30;
    for (int64_t ch = (int64_t)blockIdx.x * (kSelectThreads / 32) + (threadIdx.x >> 5); ch < chunks; ch += warps) {
        int my_k1 = 0, my_s1 = 0, my_s2 = 0, my_sm = 0, my_sp = 0;
        for (int i = 0; i < 32; ++i) {
            const int64_t p = ch * 32 + i;
            if (p >= n) break;  // warp-uniform
            int v[KPL];
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane * KPL + j;
                v[j] = kBig;
                if (k < D) {
                    int t = 0;
#pragma unroll
                    for (int d = 0; d < 4; ++d) t += __ldg(Lall + d * plane + (size_t)p * D + k);
                    v[j] = t;
                    S[(size_t)p * D + k] = (uint16_t)t;
                }
            }
            int loc = kBig;
#pragma unroll
            for (int j = 0; j < KPL; ++j) loc = min(loc, v[j]);
            const int s1 = __reduce_min_sync(0xffffffffu, loc);
            int kloc = kBig;
#pragma unroll
            for (int j = KPL - 1; j >= 0; --j)
                if (v[j] == s1) kloc = lane * KPL + j;
            const int k1 = __reduce_min_sync(0xffffffffu, kloc);  // first minimiser
            int far = kBig, mm = 0, mp = 0;
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int k = lane * KPL + j;
                if (k < D && abs(k - k1) >= 2) far = min(far, v[j]);
                if (k == k1 - 1) mm = v[j];
                if (k == k1 + 1) mp = v[j];
            }
            const int s2 = __reduce_min_sync(0xffffffffu, far);
            const int sm = __reduce_add_sync(0xffffffffu, mm), sp = __reduce_add_sync(0xffffffffu, mp);
            if (lane == i) {
                my_k1 = k1;
                my_s1 = s1;
                my_s2 = s2 == kBig ? s1 : s2;
                my_sm = sm;
                my_sp = sp;
            }
        }
        const int64_t p = ch * 32 + lane;
        const bool live = p < n;
        const bool keep =
            live && my_k1 > 0 && my_k1 < D - 1 && my_s2 > 0 && 5 * (my_s2 - my_s1) >= 2 * my_s2;
        float out = __int_as_float(0x7fc00000);
        if (keep) {
            const int den = my_sm - 2 * my_s1 + my_sp;
            const float delta = den > 0 ? __fdiv_rn((float)(my_sm - my_sp), __fmul_rn(2.f, (float)den)) : 0.f;
            const double inv = dadd(inv_far, dmul(dadd((double)my_k1, (double)delta), step));
            out = __double2float_rn(ddiv(1.0, inv));
        }
        if (live) {
            depth[p] = out;
            kept[p] = keep ? 1 : 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0 && bal) atomicAdd(&s_count, __popc(bal));
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_count) atomicAdd(count, (unsigned long long)s_count);
}

// kept-pixel counts per CTA (pixel order), then an exclusive scan in one CTA, then the points
constexpr int kFuseThreads = 256;

__global__ void __launch_bounds__(kFuseThreads)
k_fuse_count(const float* __restrict__ depth, int64_t n, uint32_t* __restrict__ cta_count) {
    const int64_t p = (int64_t)blockIdx.x * kFuseThreads + threadIdx.x;
    const bool keep = p < n && depth[p] == depth[p];
    const int c = __syncthreads_count(keep);
    if (threadIdx.x == 0) cta_count[blockIdx.x] = (uint32_t)c;
}

__global__ void __launch_bounds__(1024)
k_fuse_scan(uint32_t* __restrict__ cta_count, int ctas, int64_t* __restrict__ total) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < ctas; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < ctas ? cta_count[i] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if ((threadIdx.x & 31) >= o) incl += u;
        }
        if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += s_warp[w];
        const uint64_t carry = s_carry;
        if (i < ctas) cta_count[i] = (uint32_t)(carry + before + incl - v);
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = (int64_t)s_carry;
}

__global__ void __launch_bounds__(kFuseThreads)
k_fuse_points(const float* __restrict__ depth, int W, int64_t n, CamF cam, const uint32_t* __restrict__ cta_off,
              int64_t capacity, float* __restrict__ points, int32_t* __restrict__ pix) {
    __shared__ uint32_t s_warp[kFuseThreads / 32];
    const int64_t p = (int64_t)blockIdx.x * kFuseThreads + threadIdx.x;
    const float d = p < n ? depth[p] : __int_as_float(0x7fc00000);
    const bool keep = d == d;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    if (!keep) return;
    const int64_t o = (int64_t)cta_off[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    if (o >= capacity) return;
    const int y = (int)(p / W), x = (int)(p % W);
    const double dd = d;
    const double X0 = dsub(dmul(dd, ddiv(dsub((double)x + 0.5, (double)cam.cx), (double)cam.fx)), (double)cam.v[3]);
    const double X1 = dsub(dmul(dd, ddiv(dsub((double)y + 0.5, (double)cam.cy), (double)cam.fy)), (double)cam.v[7]);
    const double X2 = dsub(dd, (double)cam.v[11]);
    for (int j = 0; j < 3; ++j) {
        const double w =
            dadd(dadd(dmul((double)cam.v[j], X0), dmul((double)cam.v[4 + j], X1)), dmul((double)cam.v[8 + j], X2));
        points[3 * o + j] = __double2float_rn(w);
    }
    pix[o] = (int32_t)p;
}

// camera-z (FP64) of the sparse points in front of the target and inside its image, compacted
__global__ void k_sparse_depths(const float* __restrict__ P, int64_t n, CamF cam, int W, int H, double* __restrict__ z,
                                unsigned long long* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double X = P[3 * i], Y = P[3 * i + 1], Z = P[3 * i + 2];
    double Xc[3];
    for (int r = 0; r < 3; ++r)
        Xc[r] = dadd(dadd(dadd(dmul((double)cam.v[4 * r], X), dmul((double)cam.v[4 * r + 1], Y)),
                          dmul((double)cam.v[4 * r + 2], Z)),
                     (double)cam.v[4 * r + 3]);
    const double zz = Xc[2];
    if (!(zz > 0.2)) return;
    const double u = dadd(dmul((double)cam.fx, ddiv(Xc[0], zz)), (double)cam.cx);
    const double v = dadd(dmul((double)cam.fy, ddiv(Xc[1], zz)), (double)cam.cy);
    if (!(u >= 0.0 && u < (double)W && v >= 0.0 && v < (double)H)) return;
    z[atomicAdd(count, 1ull)] = zz;
}

// one CTA: the order statistics of the quantiles 0.05, 0.5, 0.95 of z[0..m) by radix selection on
// the FP64 bit patterns (positive values order like their bits), eight 8-bit passes for all six
// ranks at once; out = (0.5 q.05, 1.5 q.95, q.5)
__global__ void __launch_bounds__(1024)
k_quantiles(const double* __restrict__ z, const unsigned long long* __restrict__ count, double* __restrict__ out,
            int* __restrict__ status) {
    constexpr int kQ = 6;
    __shared__ unsigned s_hist[kQ][256];
    __shared__ unsigned long long s_prefix[kQ];
    __shared__ long long s_rank[kQ];
    const long long m = (long long)*count;
    if (m == 0) {
        if (threadIdx.x == 0) atomicOr(status, 1);
        return;
    }
    const double ps[3] = {0.05, 0.5, 0.95};
    if (threadIdx.x < kQ) {
        const double h = dmul((double)(m - 1), ps[threadIdx.x >> 1]);
        const long long lo = (long long)floor(h);
        s_rank[threadIdx.x] = (threadIdx.x & 1) ? (lo + 1 < m ? lo + 1 : m - 1) : lo;
        s_prefix[threadIdx.x] = 0ull;
    }
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int e = threadIdx.x; e < kQ * 256; e += blockDim.x) (&s_hist[0][0])[e] = 0u;
        __syncthreads();
        const unsigned long long hmask = shift == 56 ? 0ull : (~0ull << (shift + 8));
        // the values cluster, so most lanes of a warp hit the same bin: one atomic per distinct bin
        // of a warp (lanes grouped by __match_any_sync) instead of one per lane
        const long long mend = (m + 31) & ~31ll;
        for (long long i = threadIdx.x; i < mend; i += blockDim.x) {
            const bool live = i < m;
            const unsigned long long b = live ? (unsigned long long)__double_as_longlong(z[i]) : 0ull;
            const unsigned d = (unsigned)((b >> shift) & 255ull);
            const unsigned lane = threadIdx.x & 31;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const unsigned key = (live && (b & hmask) == s_prefix[q]) ? d : 256u;
                const unsigned grp = __match_any_sync(0xffffffffu, key);
                if (key < 256u && lane == (unsigned)(__ffs(grp) - 1)) atomicAdd(&s_hist[q][key], (unsigned)__popc(grp));
            }
        }
        __syncthreads();
        if (threadIdx.x < kQ) {
            const int q = threadIdx.x;
            long long r = s_rank[q];
            int d = 0;
            for (; d < 255; ++d) {
                if (r < (long long)s_hist[q][d]) break;
                r -= s_hist[q][d];
            }
            s_rank[q] = r;
            s_prefix[q] |= (unsigned long long)d << shift;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double q[3];
        for (int j = 0; j < 3; ++j) {
            const double h = dmul((double)(m - 1), ps[j]);
            const double lo = floor(h);
            const double a = __longlong_as_double((long long)s_prefix[2 * j]);
            const double b = __longlong_as_double((long long)s_prefix[2 * j + 1]);
            q[j] = dadd(a, dmul(dsub(h, lo), dsub(b, a)));
        }
        out[0] = dmul(0.5, q[0]);
        out[1] = dmul(1.5, q[2]);
        out[2] = q[1];
    }
}

// Eq. 4 score of every keyframe as the reference of `target`, and the best (ties: lowest index)
__global__ void __launch_bounds__(1024)
k_reference(const CamF* __restrict__ cams, int count, int target, double median, double* __restrict__ scores,
            int* __restrict__ best) {
    __shared__ double s_val[1024];
    __shared__ int s_idx[1024];
    const int j = threadIdx.x;
    auto centre = [&](const CamF& c, double o[3]) {
        for (int q = 0; q < 3; ++q)
            o[q] = -dadd(dadd(dmul((double)c.v[q], (double)c.v[3]), dmul((double)c.v[4 + q], (double)c.v[7])),
                         dmul((double)c.v[8 + q], (double)c.v[11]));
    };
    double sc = -INFINITY;
    if (j < count && j != target) {
        double ct[3], cj[3];
        centre(cams[target], ct);
        centre(cams[j], cj);
        const double dx = dsub(cj[0], ct[0]), dy = dsub(cj[1], ct[1]), dz = dsub(cj[2], ct[2]);
        const double b = sqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
        const CamF& A = cams[target];
        const CamF& B = cams[j];
        const double cosang = dadd(dadd(dmul((double)B.v[8], (double)A.v[8]), dmul((double)B.v[9], (double)A.v[9])),
                                   dmul((double)B.v[10], (double)A.v[10]));
        const double alpha = acos(fmax(-1.0, fmin(1.0, cosang)));
        const double bt = dmul(0.1, median), sb = dmul(0.5, bt);
        const double alpha_min = dmul(5.0, 0.017453292519943295);
        const double e = dsub(b, bt);
        sc = dmul(exp(ddiv(-dmul(e, e), dmul(dmul(2.0, sb), sb))), fmax(ddiv(alpha, alpha_min), 1.0));
    }
    if (j < count) scores[j] = sc;
    s_val[j] = sc;
    s_idx[j] = j;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (j < w) {
            const double a = s_val[j], b2 = s_val[j + w];
            if (b2 > a || (b2 == a && s_idx[j + w] < s_idx[j])) {
                s_val[j] = b2;
                s_idx[j] = s_idx[j + w];
            }
        }
        __syncthreads();
    }
    if (j == 0) *best = s_idx[0];
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int launch_mvs_census(const float* rgb, int W, int H, uint64_t* code, cudaStream_t s) {
    k_census<<<dim3(blocks(W, kCtx), blocks(H, kCty)), dim3(kCtx, kCty), 0, s>>>(rgb, W, H, code);
    return 1;
}

int launch_mvs_cost(const pgs_camera& t, const pgs_camera& r, const uint64_t* cen_t, const uint64_t* cen_r, int W,
                    int H, int D, double inv_far, double step, float* maps, uint8_t* C, cudaStream_t s) {
    k_plane_maps<<<blocks(D, 64), 64, 0, s>>>(camf(t), camf(r), inv_far, step, D, maps);
    k_cost<<<dim3(blocks(W, kRun), H), D, 0, s>>>(cen_t, cen_r, W, H, D, maps, C);
    return 2;
}

int launch_mvs_sgm(const uint8_t* C, uint8_t* L, int W, int H, int D, cudaStream_t s) {
    const int lines = W > H ? W : H;
    const dim3 g(blocks((int64_t)lines * 32, 128), 4);
    if (D <= 32) k_sgm<1><<<g, 128, 0, s>>>(C, L, W, H, D);
    else if (D <= 64) k_sgm<2><<<g, 128, 0, s>>>(C, L, W, H, D);
    else if (D <= 96) k_sgm<3><<<g, 128, 0, s>>>(C, L, W, H, D);
    else k_sgm<4><<<g, 128, 0, s>>>(C, L, W, H, D);
    return 1;
}

int launch_mvs_select(const uint8_t* L, uint16_t* S, int W, int H, int D, double inv_far, double step, float* depth,
                      uint8_t* kept, unsigned long long* count, cudaStream_t s) {
    cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    const int64_t n = (int64_t)W * H;
    int64_t g = ((n + 31) / 32 + kSelectThreads / 32 - 1) / (kSelectThreads / 32);
    if (g > 152 * 8) g = 152 * 8;  // grid-stride: 8 resident CTAs an SM
    if (D <= 32) k_select<1><<<(unsigned)g, kSelectThreads, 0, s>>>(L, S, W, H, D, inv_far, step, depth, kept, count);
    else if (D <= 64) k_select<2><<<(unsigned)g, kSelectThreads, 0, s>>>(L, S, W, H, D, inv_far, step, depth, kept, count);
    else if (D <= 96) k_select<3><<<(unsigned)g, kSelectThreads, 0, s>>>(L, S, W, H, D, inv_far, step, depth, kept, count);
    else k_select<4><<<(unsigned)g, kSelectThreads, 0, s>>>(L, S, W, H, D, inv_far, step, depth, kept, count);
    return 1;
}

int launch_mvs_fuse(const float* depth, int W, int H, const pgs_camera& cam, uint32_t* cta_scratch, int64_t* total,
                    int64_t capacity, float* points, int32_t* pix, cudaStream_t s) {
    const int64_t n = (int64_t)W * H;
    const unsigned g = blocks(n, kFuseThreads);
    k_fuse_count<<<g, kFuseThreads, 0, s>>>(depth, n, cta_scratch);
    k_fuse_scan<<<1, 1024, 0, s>>>(cta_scratch, (int)g, total);
    k_fuse_points<<<g, kFuseThreads, 0, s>>>(depth, W, n, camf(cam), cta_scratch, capacity, points, pix);
    return 3;
}

int mvs_fuse_ctas(int W, int H) { return (int)blocks((int64_t)W * H, kFuseThreads); }

int launch_mvs_range(const float* P, int64_t n, const pgs_camera& cam, double* zbuf, unsigned long long* count,
                     double* out, int* status, cudaStream_t s) {
    cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (n > 0)
        k_sparse_depths<<<blocks(n, 256), 256, 0, s>>>(P, n, camf(cam), cam.width, cam.height, zbuf, count);
    k_quantiles<<<1, 1024, 0, s>>>(zbuf, count, out, status);
    return n > 0 ? 2 : 1;
}

int launch_mvs_reference(const void* cams_f, int count, int target, double median, double* scores, int* best,
                         cudaStream_t s) {
    k_reference<<<1, 1024, 0, s>>>(static_cast<const CamF*>(cams_f), count, target, median, scores, best);
    return 1;
}

size_t mvs_camf_bytes() { return sizeof(CamF); }

void mvs_pack_cameras(const pgs_camera* cams, int count, void* host_out) {
    CamF* o = static_cast<CamF*>(host_out);
    for (int i = 0; i < count; ++i) o[i] = camf(cams[i]);
}

}  // namespace pgs
