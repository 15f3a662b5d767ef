// K6 composite_fwd and K8 composite_bwd: one CTA per 16x16 screen tile; each thread owns a
// vertical strip of kPix pixels (128 threads per tile at kPix = 2), so every entry staged in
// shared memory and every warp reduction serves kPix times more pixels than one pixel per thread.
// Tiles are scheduled heaviest first (tile_order).
//
// Forward (Eq. 7, evaluated front to back with transmittance T): the tile's depth-ordered list
// [range.x, range.y) is staged in shared memory in batches (projected record gathered through
// the canonical index, i.e. through pi of Eq. 10); each pixel composites
//     alpha = min(0.99, o exp(power)),  skip if alpha < 1/255,
//     stop (without compositing) when T (1 - alpha) < 1e-4,  C += alpha T c,  T *= 1 - alpha,
// and keeps only T_final, last = 1 + list position of the last composited entry, and the number
// of composited entries.
//
// Backward: instead of the paper's per-pixel replay cache S = {id, C_in, alpha} (Eq. 9) the
// kernel re-traverses the list back to front from `last`, rebuilding the transmittance in front
// of each entry from T_final (T_i = T_{i+1} / (1 - alpha_i); alpha <= 0.99 bounds the growth) and
// the colour behind it with Eq. 7 itself (C_in of the last entry is the background), then applies
// Eq. 8:  dL/dc = alpha dL/dC_out,  dL/dalpha = <dL/dC_out, c - C_in>,  dL/dC_out = T_i dL/dC.
// Each thread first sums its strip's nine screen-space gradients; the warp's 32 partial sums are
// then added by a transpose-reduction (9 shuffles for 8 values; with two pixels per thread two
// consecutive entries share one 18-value reduction) and scattered with one atomic per value per
// warp to the canonical index (Eq. 10: grad_{pi(i)} += g_i).  Each warp stops at its own deepest
// `last`, not the tile's.
//
// The exponent is evaluated base 2: the conic is pre-scaled by -log2(e)/2 (and -log2(e) for the
// cross term) when an entry is staged, and alpha uses ex2.approx.  Forward and backward stage and
// evaluate with the same instruction sequence, so they take identical skip decisions.
#include <cstdlib>
#include <type_traits>

#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// conic (a, b, c) -> base-2 exponent coefficients: power * log2(e) = A dx^2 + B dx dy + C dy^2
__device__ __forceinline__ float4 scaled_conic(float4 con) {
    return make_float4(__fmul_rn(-0.5f * kLog2e, con.x), __fmul_rn(-kLog2e, con.y),
                       __fmul_rn(-0.5f * kLog2e, con.z), 0.0f);
}

// alpha of one (pixel, entry) with the shared part adx2 = A dx^2 precomputed; explicit roundings
// so the forward and the backward evaluate it identically.  og = o * G before the clamp.
__device__ __forceinline__ float entry_alpha(float dx, float dy, float adx2, float4 s2, float o,
                                             float& G, float& og) {
    const float p = __fmaf_rn(s2.z, __fmul_rn(dy, dy), __fmaf_rn(s2.y, __fmul_rn(dx, dy), adx2));
    G = ex2_approx(p);
    og = __fmul_rn(o, G);
    return fminf(kAlphaMax, og);
}

__device__ __forceinline__ uint32_t checked_id(uint32_t id, int64_t n, int32_t* status) {
    if (id >= n) {
        atomicOr(status, kStatusInternal);
        return 0;
    }
    return id;
}

// Where one tile reads and writes.
struct TileJob {
    int W, H, TX;  // image of the render
    int tile;      // tile index inside the render
    float3 bg;
    uint2 range;   // [first, last) in the sorted pairs
    float* image;  // [3][H][W] (forward)
    const float* dL;  // [3][H][W] (backward)
    float* T_final;
    uint32_t* last;
    uint32_t* ncomp;
    // forward with the L1 loss fused (target != nullptr): dL_out = sign(image - target) * inv_n
    const float* target = nullptr;
    float* dL_out = nullptr;
    float inv_n = 0.f;
};

// L1 terms of one pixel's three values (the loss kernel's arithmetic): gradient written, |d| and
// d^2 added to the thread's sums
__device__ __forceinline__ void l1_pixel(const TileJob& J, size_t p, size_t plane, float r, float g, float b,
                                         float& l1, float& l2) {
    const float v[3] = {r, g, b};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float d = v[c] - J.target[c * plane + p];
        l1 += fabsf(d);
        l2 = fmaf(d, d, l2);
        J.dL_out[c * plane + p] = d > 0.f ? J.inv_n : (d < 0.f ? -J.inv_n : 0.f);
    }
}

// Replay cache of the paper's training operator (the per-pixel record S = {id, C_in, alpha} of
// Eq. 9 with a per-pixel count reset every render), in front-to-back form: for each pixel the
// first K composited entries as one 16-byte record {list position | clamp flag << 31, alpha,
// T in front of the entry, unused}, [pixel][K] (one vector store per recorded entry), and the
// count (K + 1 when the pixel composited more than K entries: its backward falls back to
// recomputing).  The colour behind an entry (Eq. 7's C_in) is rebuilt back to front in the
// backward, as in the recompute path.
struct ReplayCache {
    float4* rec = nullptr;
    uint32_t* count = nullptr;
    int K = 0;
};

// Thread t's pixel column and first row inside the tile: each warp takes a block 8 pixels wide and
// 4 kPix rows high (lane: column lane % 8, strip of kPix rows from kPix (lane / 8)), the blocks
// tiling the tile row by row.  Compact blocks end their pixels' lists at more similar depths than
// kT-wide strips, so a warp walks fewer entries only some of its pixels need (16-pixel tiles, two
// pixels a thread: 8 x 8 blocks instead of 16 x 4 strips, backward 0.574 -> 0.536 ms).
template <int kT, int kPix>
__device__ __forceinline__ void strip_origin(int t, int& dx, int& dy0) {
    constexpr int kAcross = kT / 8;  // blocks per block row
    const int w = t >> 5, lane = t & 31;
    dx = (w % kAcross) * 8 + (lane & 7);
    dy0 = (w / kAcross) * (4 * kPix) + (lane >> 3) * kPix;
}

template <int kDepth>
struct FwdSmem {
    float4 xyo[kDepth], s2[kDepth], rgb[kDepth];
};

// One tile of the forward.  kPix: pixels per thread (vertical strip); kDepth: entries staged per
// batch.  Every thread of the CTA calls it with the same job.
// Returns the thread's L1 sums (|d|, d^2) when J.target is set, else zeros.
template <int kT, int kPix, int kDepth, bool kRecord = false>
__device__ __forceinline__ float2 fwd_tile_scalar(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                         const Scratch& sc, FwdSmem<kDepth>& S, ReplayCache rc = {}) {
    static_assert(!kRecord || kPix == 1, "the replay cache records one pixel per thread");
    constexpr int kThreads = kT * kT / kPix;
    constexpr int kBatch = kDepth;
    float4* s_xyo = S.xyo;
    float4* s_s2 = S.s2;
    float4* s_rgb = S.rgb;
    const int W = J.W, H = J.H;
    int sdx, sdy0;
    strip_origin<kT, kPix>((int)threadIdx.x, sdx, sdy0);
    const int px = (J.tile % J.TX) * kT + sdx;
    const int py0 = (J.tile / J.TX) * kT + sdy0;
    const float fx = (float)px + 0.5f, fy0 = (float)py0 + 0.5f;
    const uint2 range = J.range;
    const float3 bg = J.bg;
    float T[kPix], C0[kPix], C1[kPix], C2[kPix];
    uint32_t last[kPix], ncomp[kPix];
    bool done[kPix];
    bool all_done = true;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = ncomp[k] = 0;
        done[k] = !(px < W && py0 + k < H);
        all_done = all_done && done[k];
    }
    for (uint32_t base = range.x; base < range.y; base += kBatch) {
        if (__syncthreads_count(all_done) == kThreads) break;
#pragma unroll
        for (int e = threadIdx.x; e < kBatch; e += kThreads) {
            const uint32_t idx = base + e;
            if (idx < range.y) {
                const uint32_t id = checked_id(vals[idx], n, sc.status);
                s_xyo[e] = sc.xyo[id];
                s_s2[e] = scaled_conic(sc.conic[id]);
                s_rgb[e] = sc.rgb[id];
            }
        }
        __syncthreads();
        const int cnt = min((uint32_t)kBatch, range.y - base);
        for (int j = 0; !all_done && j < cnt; ++j) {
            const float4 p = s_xyo[j];
            const float4 s2 = s_s2[j];
            const float4 c = s_rgb[j];
            const float dx = fx - p.x;
            const float adx2 = __fmul_rn(s2.x, __fmul_rn(dx, dx));
            const float dy0 = fy0 - p.y;
            all_done = true;
#pragma unroll
            for (int k = 0; k < kPix; ++k) {
                if (!done[k]) {
                    float G, og;
                    const float alpha = entry_alpha(dx, dy0 + (float)k, adx2, s2, p.z, G, og);
                    if (alpha >= kAlphaMin) {
                        const float Tn = T[k] * (1.0f - alpha);
                        if (Tn < kTMin) {
                            done[k] = true;
                        } else {
                            if constexpr (kRecord) {
                                if (ncomp[k] < (uint32_t)rc.K) {
                                    const uint32_t word = (base + j - range.x) | (og > kAlphaMax ? 0x80000000u : 0u);
                                    rc.rec[((size_t)(py0 + k) * W + px) * rc.K + ncomp[k]] =
                                        make_float4(__uint_as_float(word), alpha, T[k], 0.0f);
                                }
                            }
                            const float w = alpha * T[k];
                            C0[k] = fmaf(c.x, w, C0[k]);
                            C1[k] = fmaf(c.y, w, C1[k]);
                            C2[k] = fmaf(c.z, w, C2[k]);
                            T[k] = Tn;
                            last[k] = base + j - range.x + 1;
                            ++ncomp[k];
                        }
                    }
                }
                all_done = all_done && done[k];
            }
        }
    }
    float l1 = 0.f, l2 = 0.f;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        const int py = py0 + k;
        if (px < W && py < H) {
            const size_t p = (size_t)py * W + px, plane = (size_t)W * H;
            const float r = fmaf(T[k], bg.x, C0[k]), g = fmaf(T[k], bg.y, C1[k]), b = fmaf(T[k], bg.z, C2[k]);
            J.image[p] = r;
            J.image[plane + p] = g;
            J.image[2 * plane + p] = b;
            J.T_final[p] = T[k];
            J.last[p] = last[k];
            J.ncomp[p] = ncomp[k];
            if constexpr (kRecord) rc.count[p] = ncomp[k] > (uint32_t)rc.K ? (uint32_t)rc.K + 1 : ncomp[k];
            if (J.target) l1_pixel(J, p, plane, r, g, b, l1, l2);
        }
    }
    return make_float2(l1, l2);
}

// Sum v[0..8] over the warp.  Afterwards lane l with l % 4 == 0 holds the sum of v[l >> 2]
// (values 0..7) and every lane holds the sum of v[8].
__device__ __forceinline__ void warp_sum9(const float v[9], int lane, float& s8, float& s9) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b4 ? v[k] : v[k + 4];
        const float keep = b4 ? v[k + 4] : v[k];
        u[k] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    float w[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b3 ? u[k] : u[k + 2];
        const float keep = b3 ? u[k + 2] : u[k];
        w[k] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    float s = (b2 ? w[1] : w[0]) + __shfl_xor_sync(kFull, b2 ? w[0] : w[1], 4);
    s += __shfl_xor_sync(kFull, s, 2);
    s += __shfl_xor_sync(kFull, s, 1);
    float t = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    s8 = s;
    s9 = t;
}

// Sum a[0..8] and b[0..8] (values 0..8 and 9..17) over the warp by one transpose-reduction: at
// each level (xor 16, 8, 4, 2, 1) a lane keeps the half of its values selected by that lane bit
// (odd counts padded with a zero) and adds the partner's copy of it, 9 + 5 + 3 + 2 + 1 = 20
// shuffles.  Afterwards lane l holds the warp sum of value idx, or idx = -1 (a padding slot).
__device__ __forceinline__ void warp_sum18(const float a[9], const float b[9], int lane, float& s, int& idx) {
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2, b1 = lane & 1;
    float x9[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) x9[k] = (b16 ? b[k] : a[k]) + __shfl_xor_sync(kFull, b16 ? a[k] : b[k], 16);
    float x5[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float lo = x9[k], hi = k + 5 < 9 ? x9[k + 5] : 0.0f;
        x5[k] = (b8 ? hi : lo) + __shfl_xor_sync(kFull, b8 ? lo : hi, 8);
    }
    float x3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = x5[k], hi = k + 3 < 5 ? x5[k + 3] : 0.0f;
        x3[k] = (b4 ? hi : lo) + __shfl_xor_sync(kFull, b4 ? lo : hi, 4);
    }
    float x2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float lo = x3[k], hi = k + 2 < 3 ? x3[k + 2] : 0.0f;
        x2[k] = (b2 ? hi : lo) + __shfl_xor_sync(kFull, b2 ? lo : hi, 2);
    }
    s = (b1 ? x2[1] : x2[0]) + __shfl_xor_sync(kFull, b1 ? x2[0] : x2[1], 1);
    const int r2 = (b2 ? 2 : 0) + (b1 ? 1 : 0);  // index in the 3-value level (4 with the pad)
    const int r4 = (b4 ? 3 : 0) + r2;            // in the 5-value level
    const int r8 = (b8 ? 5 : 0) + r4;            // in the 9-value level
    idx = (r2 < 3 && r4 < 5 && r8 < 9) ? (b16 ? 9 : 0) + r8 : -1;
}

// factor from the summed (dpow dx^2, dpow dx dy, dpow dy^2) to d power / d(a, b, c) =
// (-dx^2 / 2, -dx dy, -dy^2 / 2); 1 for the other screen-space gradients
__device__ __forceinline__ float grad_factor(int q) { return q == 2 || q == 4 ? -0.5f : (q == 3 ? -1.0f : 1.0f); }

// One entry's nine warp-summed screen-space gradients added to its canonical index
__device__ __forceinline__ void scatter9(const float v[9], int lane, uint32_t id, int64_t n, float* grad2d) {
    float s8, s9;
    warp_sum9(v, lane, s8, s9);
    if ((lane & 3) == 0) atomicAdd(&grad2d[(size_t)(lane >> 2) * n + id], grad_factor(lane >> 2) * s8);
    if (lane == 1) atomicAdd(&grad2d[(size_t)8 * n + id], s9);
}

template <int kDepth>
struct BwdSmem {
    float4 xyo[kDepth], s2[kDepth], con[kDepth], rgb[kDepth];
    uint32_t id[kDepth];
    uint32_t wmax[32];  // per warp (at most 32 warps per CTA)
};

// Eq. 8 for one composited (pixel, entry): the colour behind B is updated by Eq. 7, T becomes
// the transmittance in front Tb, and the strip's partial sums v gain the nine screen-space
// gradient terms (mean and conic only when alpha was not clamped at 0.99).
__device__ __forceinline__ void eq8_accumulate(float alpha, float Tb, float G, bool unclamped, float dx,
                                               float dy, float4 c, float4 con, float g0, float g1,
                                               float g2, float& B0, float& B1, float& B2, float& T,
                                               float v[9]) {
    const float r0 = c.x - B0, r1 = c.y - B1, r2 = c.z - B2;
    const float dLda = Tb * (r0 * g0 + r1 * g1 + r2 * g2);
    const float wgt = alpha * Tb;
    v[6] = fmaf(wgt, g0, v[6]);
    v[7] = fmaf(wgt, g1, v[7]);
    v[8] = fmaf(wgt, g2, v[8]);
    B0 = fmaf(alpha, r0, B0);
    B1 = fmaf(alpha, r1, B1);
    B2 = fmaf(alpha, r2, B2);
    T = Tb;
    if (unclamped) {  // zero gradient through the 0.99 clamp
        v[5] = fmaf(dLda, G, v[5]);
        const float dpow = dLda * alpha;
        v[0] = fmaf(dpow, con.x * dx + con.y * dy, v[0]);
        v[1] = fmaf(dpow, con.z * dy + con.y * dx, v[1]);
        v[2] = fmaf(dpow, dx * dx, v[2]);
        v[3] = fmaf(dpow, dx * dy, v[3]);
        v[4] = fmaf(dpow, dy * dy, v[4]);
    }
}

template <int kT, int kPix, int kDepth, bool kReplay = false>
__device__ __forceinline__ void bwd_tile_scalar(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                         const Scratch& sc, BwdSmem<kDepth>& S, ReplayCache rc = {}) {
    static_assert(!kReplay || kPix == 1, "the replay cache holds one pixel per thread");
    constexpr int kThreads = kT * kT / kPix;
    constexpr int kBatch = kDepth;
    float4* s_xyo = S.xyo;
    float4* s_s2 = S.s2;
    float4* s_con = S.con;
    float4* s_rgb = S.rgb;
    uint32_t* s_id = S.id;
    uint32_t* s_max = S.wmax;
    const int W = J.W, H = J.H;
    const float3 bg = J.bg;
    const float* __restrict__ dL_dimage = J.dL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int sdx, sdy0;
    strip_origin<kT, kPix>((int)threadIdx.x, sdx, sdy0);
    const int px = (J.tile % J.TX) * kT + sdx;
    const int py0 = (J.tile / J.TX) * kT + sdy0;
    const float fx = (float)px + 0.5f, fy0 = (float)py0 + 0.5f;
    const uint2 range = J.range;
    const size_t plane = (size_t)W * H;
    float T[kPix], g0[kPix], g1[kPix], g2[kPix], B0[kPix], B1[kPix], B2[kPix];
    uint32_t my_last[kPix];
    uint32_t tmax = 0;
    // replay state (kReplay): the pixel's next cached record from the back
    bool replay[kPix];
    int ci[kPix];
    float4 cr[kPix];
    size_t cbase[kPix];
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        const int py = py0 + k;
        T[k] = 1.0f;
        g0[k] = g1[k] = g2[k] = 0.f;
        my_last[k] = 0;
        replay[k] = false;
        ci[k] = -1;
        cr[k] = make_float4(__uint_as_float(0xffffffffu), 0.f, 0.f, 0.f);
        cbase[k] = 0;
        if (px < W && py < H) {
            const size_t p = (size_t)py * W + px;
            T[k] = J.T_final[p];
            my_last[k] = J.last[p];
            g0[k] = dL_dimage[p];
            g1[k] = dL_dimage[plane + p];
            g2[k] = dL_dimage[2 * plane + p];
            if constexpr (kReplay) {
                const uint32_t count = rc.count[p];
                replay[k] = count <= (uint32_t)rc.K;
                cbase[k] = p * rc.K;
                if (replay[k]) {
                    ci[k] = (int)count - 1;
                    if (ci[k] >= 0) cr[k] = rc.rec[cbase[k] + ci[k]];
                }
            }
        }
        B0[k] = bg.x;  // colour behind the current entry (Eq. 7 C_in)
        B1[k] = bg.y;
        B2[k] = bg.z;
        tmax = max(tmax, my_last[k]);
    }
    const uint32_t wmax = __reduce_max_sync(kFull, tmax);
    if (lane == 0) s_max[warp] = wmax;
    __syncthreads();
    uint32_t end = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) end = max(end, s_max[w]);

    while (end > 0) {
        const uint32_t start = end > (uint32_t)kBatch ? end - kBatch : 0u;
        const int cnt = (int)(end - start);
        __syncthreads();
#pragma unroll
        for (int e = threadIdx.x; e < kBatch; e += kThreads) {
            if (e < cnt) {
                const uint32_t id = checked_id(vals[range.x + start + e], n, sc.status);
                s_id[e] = id;
                s_xyo[e] = sc.xyo[id];
                const float4 con = sc.conic[id];
                s_con[e] = con;
                s_s2[e] = scaled_conic(con);
                s_rgb[e] = sc.rgb[id];
            }
        }
        __syncthreads();
        // this warp's entries: positions below its deepest `last`
        const int jtop = (int)min((uint32_t)cnt, wmax > start ? wmax - start : 0u);
        for (int j = jtop - 1; j >= 0; --j) {
            const uint32_t pos = start + j;
            const float4 pm = s_xyo[j];
            const float4 s2 = s_s2[j];
            const float4 con = s_con[j];
            const float4 c = s_rgb[j];
            const float dx = fx - pm.x;
            const float adx2 = __fmul_rn(s2.x, __fmul_rn(dx, dx));
            const float dy0 = fy0 - pm.y;
            float v[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) v[q] = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < kPix; ++k) {
                const float dy = dy0 + (float)k;
                if (kReplay && replay[k]) {
                    // cached entry at this position: alpha and T in front from the forward
                    const uint32_t word = __float_as_uint(cr[k].x);
                    if (ci[k] >= 0 && (word & 0x7fffffffu) == pos) {
                        const float alpha = cr[k].y;
                        contrib = true;
                        eq8_accumulate(alpha, cr[k].z, __fdividef(alpha, pm.z), (word >> 31) == 0u, dx, dy, c,
                                       con, g0[k], g1[k], g2[k], B0[k], B1[k], B2[k], T[k], v);
                        --ci[k];
                        if (ci[k] >= 0) cr[k] = rc.rec[cbase[k] + ci[k]];
                    }
                } else if (pos < my_last[k]) {
                    float G, og;
                    const float alpha = entry_alpha(dx, dy, adx2, s2, pm.z, G, og);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        const float Tb = __fdividef(T[k], 1.0f - alpha);  // transmittance in front
                        eq8_accumulate(alpha, Tb, G, og <= kAlphaMax, dx, dy, c, con, g0[k], g1[k], g2[k],
                                       B0[k], B1[k], B2[k], T[k], v);
                    }
                }
            }
            if (__any_sync(kFull, contrib)) {
                float s8, s9;
                warp_sum9(v, lane, s8, s9);
                const uint32_t id = s_id[j];
                if ((lane & 3) == 0) {
                    // d power / d(a, b, c) = (-dx^2 / 2, -dx dy, -dy^2 / 2)
                    const int q = lane >> 2;
                    const float f = q == 2 || q == 4 ? -0.5f : (q == 3 ? -1.0f : 1.0f);
                    atomicAdd(&sc.grad2d[(size_t)q * n + id], f * s8);
                }
                if (lane == 1) atomicAdd(&sc.grad2d[(size_t)8 * n + id], s9);
            }
        }
        end = start;
    }
}


// ---------------------------------------------------------------------------------------------
// Paired-pixel tiles (kPix = 2, 4): a thread's strip is processed two pixels at a time with the
// packed fp32 instructions of sm_100+ (add/sub/mul/fma .rn .f32x2).  Every packed lane rounds
// exactly as the scalar instruction does and takes the same operands (dx = column - x,
// dy = row - y per pixel), so the alpha, skip and stop decisions and the forward image are
// bit-identical to the one-pixel tiles; per pixel the work is branch-free (a pixel that
// does not composite an entry contributes alpha = 0, which leaves T, C and the colour behind
// unchanged), and the pair shares one branch.
struct F2 {
    unsigned long long r;
};
__device__ __forceinline__ F2 f2(float a, float b) {
    F2 o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(a), "f"(b));
    return o;
}
__device__ __forceinline__ F2 f2(float a) { return f2(a, a); }
__device__ __forceinline__ float2 un(F2 a) {
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(a.r));
    return o;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}

// alpha of the pixel pair (dy, dy + 1) below one entry: the packed form of entry_alpha
__device__ __forceinline__ void pair_alpha(F2 dy, F2 DX, F2 ADX2, F2 S2Y, F2 S2Z, F2 O, float2& G,
                                           float2& og, float2& alpha) {
    const float2 p = un(fma2(S2Z, mul2(dy, dy), fma2(S2Y, mul2(DX, dy), ADX2)));
    G = make_float2(ex2_approx(p.x), ex2_approx(p.y));
    og = un(mul2(O, f2(G.x, G.y)));
    alpha = make_float2(fminf(kAlphaMax, og.x), fminf(kAlphaMax, og.y));
}

template <int kT, int kPix, int kDepth>
__device__ __forceinline__ float2 fwd_tile_pairs(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                                 const Scratch& sc, FwdSmem<kDepth>& S) {
    constexpr int kThreads = kT * kT / kPix;
    constexpr int kBatch = kDepth;
    constexpr int NP = kPix / 2;
    float4* s_xyo = S.xyo;
    float4* s_s2 = S.s2;
    float4* s_rgb = S.rgb;
    const int W = J.W, H = J.H;
    int sdx, sdy0;
    strip_origin<kT, kPix>((int)threadIdx.x, sdx, sdy0);
    const int px = (J.tile % J.TX) * kT + sdx;
    const int py0 = (J.tile / J.TX) * kT + sdy0;
    const float fx = (float)px + 0.5f;
    F2 FY[NP];  // pixel-centre rows of the pairs: dy = row - y exactly as the one-pixel strips
#pragma unroll
    for (int q = 0; q < NP; ++q) FY[q] = f2((float)(py0 + 2 * q) + 0.5f, (float)(py0 + 2 * q + 1) + 0.5f);
    const uint2 range = J.range;
    const float3 bg = J.bg;
    F2 T[NP], C0[NP], C1[NP], C2[NP];
    uint32_t last[kPix], ncomp[kPix];
    bool done[kPix];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        T[q] = f2(1.0f);
        C0[q] = C1[q] = C2[q] = f2(0.0f);
    }
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        last[k] = ncomp[k] = 0;
        done[k] = !(px < W && py0 + k < H);
        all_done = all_done && done[k];
    }
    for (uint32_t base = range.x; base < range.y; base += kBatch) {
        if (__syncthreads_count(all_done) == kThreads) break;
#pragma unroll
        for (int e = threadIdx.x; e < kBatch; e += kThreads) {
            const uint32_t idx = base + e;
            if (idx < range.y) {
                const uint32_t id = checked_id(vals[idx], n, sc.status);
                s_xyo[e] = sc.xyo[id];
                s_s2[e] = scaled_conic(sc.conic[id]);
                s_rgb[e] = sc.rgb[id];
            }
        }
        __syncthreads();
        const int cnt = min((uint32_t)kBatch, range.y - base);
        for (int j = 0; !all_done && j < cnt; ++j) {
            const float4 p = s_xyo[j];
            const float4 s2 = s_s2[j];
            const float dx = fx - p.x;
            const F2 DX = f2(dx), ADX2 = f2(__fmul_rn(s2.x, __fmul_rn(dx, dx)));
            const F2 S2Y = f2(s2.y), S2Z = f2(s2.z), O = f2(p.z), Y = f2(p.y);
            const uint32_t pos = base + j - range.x + 1;
            all_done = true;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int k0 = 2 * q, k1 = 2 * q + 1;
                const F2 dy = sub2(FY[q], Y);
                float2 G, og, a;
                pair_alpha(dy, DX, ADX2, S2Y, S2Z, O, G, og, a);
                const bool p0 = !done[k0] && a.x >= kAlphaMin, p1 = !done[k1] && a.y >= kAlphaMin;
                if (p0 || p1) {
                    const float2 tv = un(T[q]);
                    const float2 tn = un(mul2(T[q], sub2(f2(1.0f), f2(a.x, a.y))));
                    const bool s0 = p0 && tn.x < kTMin, s1 = p1 && tn.y < kTMin;  // stop, not composited
                    const bool c0 = p0 && !s0, c1 = p1 && !s1;
                    done[k0] = done[k0] || s0;
                    done[k1] = done[k1] || s1;
                    const F2 w = mul2(f2(c0 ? a.x : 0.0f, c1 ? a.y : 0.0f), T[q]);
                    const float4 c = s_rgb[j];
                    C0[q] = fma2(f2(c.x), w, C0[q]);
                    C1[q] = fma2(f2(c.y), w, C1[q]);
                    C2[q] = fma2(f2(c.z), w, C2[q]);
                    T[q] = f2(c0 ? tn.x : tv.x, c1 ? tn.y : tv.y);
                    last[k0] = c0 ? pos : last[k0];
                    last[k1] = c1 ? pos : last[k1];
                    ncomp[k0] += c0;
                    ncomp[k1] += c1;
                }
                all_done = all_done && done[k0] && done[k1];
            }
        }
    }
    float l1 = 0.f, l2 = 0.f;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float2 t = un(T[q]), c0 = un(C0[q]), c1 = un(C1[q]), c2 = un(C2[q]);
        const float tk[2] = {t.x, t.y}, r[2] = {c0.x, c0.y}, g[2] = {c1.x, c1.y}, b[2] = {c2.x, c2.y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * q + h;
            const int py = py0 + k;
            if (px < W && py < H) {
                const size_t pp = (size_t)py * W + px, plane = (size_t)W * H;
                const float ir = fmaf(tk[h], bg.x, r[h]), ig = fmaf(tk[h], bg.y, g[h]), ib = fmaf(tk[h], bg.z, b[h]);
                J.image[pp] = ir;
                J.image[plane + pp] = ig;
                J.image[2 * plane + pp] = ib;
                J.T_final[pp] = tk[h];
                J.last[pp] = last[k];
                J.ncomp[pp] = ncomp[k];
                if (J.target) l1_pixel(J, pp, plane, ir, ig, ib, l1, l2);
            }
        }
    }
    return make_float2(l1, l2);
}

// Backward tiles of 32 x 32 pixels with two or four pixels per thread (the two-phase routine
// below would need 128 KB of shared memory for a round of entries at this edge).  The pixels of a
// tile are first ordered by
// `last` (a counting sort into 256 buckets of last * 255 / the tile's deepest last), and each warp
// takes 32 kPix consecutive pixels of that order: a warp walks the list from its own deepest `last`,
// so pixels of similar depth share a walk and few evaluations fall past a pixel's `last` (on the
// 500k/1080p view 90 % of a warp's walk is inside its pixels' lists with 64 pixels per warp, 82 %
// with 128, against 83 % for compact 8 x 8 blocks).  A thread's pixels are processed two at a time
// with the packed f32x2 instructions; every operand that is the same for the pair is staged
// duplicated in shared memory, so it loads as a ready pair.
//
// Eq. 8 is carried per pixel with two scalars: the transmittance T in front of the current entry
// and S = <C_behind, dL/dC>, the colour behind the entry (Eq. 7's C_in) projected on the pixel's
// upstream gradient: dL/dalpha = T_i (<c_i, dL/dC> - S) and S <- S + alpha_i (<c_i, dL/dC> - S),
// the same recurrence as C_in <- C_in (1 - alpha) + alpha c.  A pixel that does not composite an
// entry takes alpha = 0 (its T, S and sums unchanged).  Per entry the thread sums over its pixels
// dpow = dL/dalpha alpha (zero through the 0.99 clamp) times (1, dx, dy, dx^2, dx dy, dy^2) and
// alpha T dL/dC; d opacity = sum(dpow) / o and the mean gradient (a dx + b dy, c dy + b dx)
// follow from those moments.
template <int kT, int kDepth>
struct BwdSmemPacked {
    float4 xy[kDepth];  // (u, u, v, v)
    float4 ab[kDepth];  // (A, A, B, B): base-2 exponent coefficients (scaled conic)
    float4 co[kDepth];  // (C, C, o, o)
    float4 rg[kDepth];  // (r, r, g, g) colour
    float4 bz[kDepth];  // (b, b, conic a, conic c) colour blue, conic
    float2 bi[kDepth];  // (conic b, canonical index bits)
    uint32_t order[kT * kT];  // tile pixels (row-major index) in the order of their `last`
    uint32_t count[256];
    uint32_t wmax[32];
};

template <int kT, int kPix, int kDepth>
__device__ __forceinline__ void bwd_tile_sorted(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                                const Scratch& sc, BwdSmemPacked<kT, kDepth>& S) {
    static_assert(kPix == 2 || kPix == 4, "pairs of pixels");
    constexpr int kThreads = kT * kT / kPix;
    constexpr int kWarps = kThreads / 32;
    constexpr int NP = kPix / 2;
    const int W = J.W, H = J.H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = (J.tile % J.TX) * kT, y0 = (J.tile / J.TX) * kT;
    const uint2 range = J.range;
    // ---- order the tile's pixels by `last`
    uint32_t lst[kPix];
    uint32_t tmax = 0;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        const int i = tid * kPix + k, px = x0 + i % kT, py = y0 + i / kT;
        lst[k] = (px < W && py < H) ? J.last[(size_t)py * W + px] : 0u;
        tmax = max(tmax, lst[k]);
    }
    for (int b = tid; b < 256; b += kThreads) S.count[b] = 0;
    tmax = __reduce_max_sync(kFull, tmax);
    if (lane == 0) S.wmax[warp] = tmax;
    __syncthreads();
    uint32_t end = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) end = max(end, S.wmax[w]);
    uint32_t bucket[kPix];
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        bucket[k] = end ? (uint32_t)(((uint64_t)lst[k] * 255u) / end) : 0u;
        atomicAdd(&S.count[bucket[k]], 1u);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 256 bucket counts, 8 per lane
        uint32_t c[8], run = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = run;
            run += S.count[lane * 8 + k];
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t base = incl - run;
#pragma unroll
        for (int k = 0; k < 8; ++k) S.count[lane * 8 + k] = base + c[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPix; ++k) S.order[atomicAdd(&S.count[bucket[k]], 1u)] = (uint32_t)(tid * kPix + k);
    __syncthreads();
    // ---- this thread's pixels: kPix consecutive positions of the order
    const size_t plane = (size_t)W * H;
    const float3 bg = J.bg;
    F2 FX[NP], FY[NP], T[NP], Sb[NP], g0[NP], g1[NP], g2[NP];
    uint32_t my_last[kPix];
    uint32_t wlast = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float fx[2], fy[2], t[2] = {1.0f, 1.0f}, a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f}, c[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * q + h;
            const uint32_t i = S.order[tid * kPix + k];
            const int px = x0 + (int)(i % kT), py = y0 + (int)(i / kT);
            fx[h] = (float)px + 0.5f;
            fy[h] = (float)py + 0.5f;
            my_last[k] = 0;
            if (px < W && py < H) {
                const size_t pp = (size_t)py * W + px;
                t[h] = J.T_final[pp];
                my_last[k] = J.last[pp];
                a[h] = J.dL[pp];
                b[h] = J.dL[plane + pp];
                c[h] = J.dL[2 * plane + pp];
            }
            wlast = max(wlast, my_last[k]);
        }
        FX[q] = f2(fx[0], fx[1]);
        FY[q] = f2(fy[0], fy[1]);
        T[q] = f2(t[0], t[1]);
        g0[q] = f2(a[0], a[1]);
        g1[q] = f2(b[0], b[1]);
        g2[q] = f2(c[0], c[1]);
        // S = <C_behind, dL/dC>, the background behind the last entry
        Sb[q] = fma2(f2(bg.z), g2[q], fma2(f2(bg.y), g1[q], mul2(f2(bg.x), g0[q])));
    }
    const uint32_t wmax = __reduce_max_sync(kFull, wlast);
    const F2 ONE = f2(1.0f);

    while (end > 0) {
        const uint32_t start = end > (uint32_t)kDepth ? end - kDepth : 0u;
        const int cnt = (int)(end - start);
        __syncthreads();
#pragma unroll
        for (int e = tid; e < kDepth; e += kThreads) {
            if (e < cnt) {
                const uint32_t id = checked_id(vals[range.x + start + e], n, sc.status);
                const float4 xyo = sc.xyo[id];
                const float4 con = sc.conic[id];
                const float4 s2 = scaled_conic(con);
                const float4 c = sc.rgb[id];
                S.xy[e] = make_float4(xyo.x, xyo.x, xyo.y, xyo.y);
                S.ab[e] = make_float4(s2.x, s2.x, s2.y, s2.y);
                S.co[e] = make_float4(s2.z, s2.z, xyo.z, xyo.z);
                S.rg[e] = make_float4(c.x, c.x, c.y, c.y);
                S.bz[e] = make_float4(c.z, c.z, con.x, con.z);
                S.bi[e] = make_float2(con.y, __uint_as_float(id));
            }
        }
        __syncthreads();
        const int jtop = (int)min((uint32_t)cnt, wmax > start ? wmax - start : 0u);
        // one entry, back to front: the thread's per-pixel state moves in front of it and its
        // sums over the thread's pixels come back in v (mean terms already through the conic);
        // returns whether a pixel of the warp composited it (the same for every lane)
        auto entry = [&](int j, float (&v)[9]) -> bool {
            const uint32_t pos = start + j;
            const float4 xy = S.xy[j], ab = S.ab[j], co = S.co[j];
            const F2 X2 = f2(xy.x, xy.y), Y2 = f2(xy.z, xy.w);
            const F2 A2 = f2(ab.x, ab.y), B2 = f2(ab.z, ab.w), C2 = f2(co.x, co.y), O2 = f2(co.z, co.w);
            F2 DX[NP], DY[NP];
            float2 og[NP], al[NP];
            bool p0[NP], p1[NP];
            bool any = false;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                DX[q] = sub2(FX[q], X2);
                DY[q] = sub2(FY[q], Y2);
                // the forward's exponent, term for term: A dx^2 + B dx dy + C dy^2
                const float2 p = un(fma2(C2, mul2(DY[q], DY[q]), fma2(B2, mul2(DX[q], DY[q]), mul2(A2, mul2(DX[q], DX[q])))));
                og[q] = un(mul2(O2, f2(ex2_approx(p.x), ex2_approx(p.y))));
                al[q] = make_float2(fminf(kAlphaMax, og[q].x), fminf(kAlphaMax, og[q].y));
                p0[q] = pos < my_last[2 * q] && al[q].x >= kAlphaMin;
                p1[q] = pos < my_last[2 * q + 1] && al[q].y >= kAlphaMin;
                any = any || p0[q] || p1[q];
            }
            // warp-uniform: an entry no pixel of the warp composites costs no more
            if (!__any_sync(kFull, any)) return false;
            const float4 rg = S.rg[j], bz = S.bz[j];
            const F2 Cr = f2(rg.x, rg.y), Cg = f2(rg.z, rg.w), Cb = f2(bz.x, bz.y);
            F2 acc[9];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                // a pixel that does not composite the entry takes alpha = 0: T, S and its sums unchanged
                const F2 A = f2(p0[q] ? al[q].x : 0.0f, p1[q] ? al[q].y : 0.0f);
                // alpha through which the gradient flows: zero at the 0.99 clamp
                const F2 AQ = f2(p0[q] && og[q].x <= kAlphaMax ? al[q].x : 0.0f,
                                 p1[q] && og[q].y <= kAlphaMax ? al[q].y : 0.0f);
                const float2 om = un(sub2(ONE, A));
                float rx, ry;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(om.x));
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(om.y));
                const F2 Tb = mul2(T[q], f2(p0[q] ? rx : 1.0f, p1[q] ? ry : 1.0f));  // transmittance in front
                const F2 cg = fma2(Cb, g2[q], fma2(Cg, g1[q], mul2(Cr, g0[q])));
                const F2 r = sub2(cg, Sb[q]);
                const F2 dLda = mul2(Tb, r);
                const F2 wgt = mul2(A, Tb);
                Sb[q] = fma2(A, r, Sb[q]);
                T[q] = Tb;
                const F2 dpow = mul2(dLda, AQ);
                const F2 dpx = mul2(dpow, DX[q]), dpy = mul2(dpow, DY[q]);
                if (q == 0) {
                    acc[6] = mul2(wgt, g0[q]);
                    acc[7] = mul2(wgt, g1[q]);
                    acc[8] = mul2(wgt, g2[q]);
                    acc[5] = dpow;
                    acc[0] = dpx;
                    acc[1] = dpy;
                    acc[2] = mul2(dpx, DX[q]);
                    acc[3] = mul2(dpx, DY[q]);
                    acc[4] = mul2(dpy, DY[q]);
                } else {
                    acc[6] = fma2(wgt, g0[q], acc[6]);
                    acc[7] = fma2(wgt, g1[q], acc[7]);
                    acc[8] = fma2(wgt, g2[q], acc[8]);
                    acc[5] = add2(acc[5], dpow);
                    acc[0] = add2(acc[0], dpx);
                    acc[1] = add2(acc[1], dpy);
                    acc[2] = fma2(dpx, DX[q], acc[2]);
                    acc[3] = fma2(dpx, DY[q], acc[3]);
                    acc[4] = fma2(dpy, DY[q], acc[4]);
                }
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float2 h = un(acc[k]);
                v[k] = h.x + h.y;
            }
            // d power / d mean2D = (a dx + b dy, c dy + b dx) with the entry's conic (a, b, c)
            const float cb = S.bi[j].x;
            const float m0 = fmaf(bz.z, v[0], cb * v[1]);
            const float m1 = fmaf(bz.w, v[1], cb * v[0]);
            v[0] = m0;
            v[1] = m1;
            return true;
        };
        // factor from a summed value to its screen-space gradient: d power / d(a, b, c) =
        // (-dx^2 / 2, -dx dy, -dy^2 / 2); d opacity = sum(dpow) / o
        auto factor = [&](int q, int j) -> float {
            if (q == 5) return __fdividef(1.0f, S.co[j].z);
            return q == 2 || q == 4 ? -0.5f : (q == 3 ? -1.0f : 1.0f);
        };
        if constexpr (NP == 1) {
            // entries in pairs: two entries' gradients share one transpose-reduction and one
            // atomic instruction (an entry no lane composited is not added)
            for (int j = jtop - 1; j >= 0; j -= 2) {
                float va[9], vb[9];
                const bool ca = entry(j, va);
                const bool cb = j >= 1 && entry(j - 1, vb);
                if (ca && cb) {
                    float s;
                    int idx;
                    warp_sum18(va, vb, lane, s, idx);
                    if (idx >= 0) {
                        const int q = idx >= 9 ? idx - 9 : idx;
                        const int jj = idx >= 9 ? j - 1 : j;
                        atomicAdd(&sc.grad2d[(size_t)q * n + __float_as_uint(S.bi[jj].y)], factor(q, jj) * s);
                    }
                } else if (ca || cb) {
                    const int jj = ca ? j : j - 1;
                    float s8, s9;
                    warp_sum9(ca ? va : vb, lane, s8, s9);
                    const uint32_t id = __float_as_uint(S.bi[jj].y);
                    if ((lane & 3) == 0) atomicAdd(&sc.grad2d[(size_t)(lane >> 2) * n + id], factor(lane >> 2, jj) * s8);
                    if (lane == 1) atomicAdd(&sc.grad2d[(size_t)8 * n + id], s9);
                }
            }
        } else {
            for (int j = jtop - 1; j >= 0; --j) {
                float v[9];
                if (entry(j, v)) {
                    float s8, s9;
                    warp_sum9(v, lane, s8, s9);
                    const uint32_t id = __float_as_uint(S.bi[j].y);
                    if ((lane & 3) == 0) atomicAdd(&sc.grad2d[(size_t)(lane >> 2) * n + id], factor(lane >> 2, j) * s8);
                    if (lane == 1) atomicAdd(&sc.grad2d[(size_t)8 * n + id], s9);
                }
            }
        }
        end = start;
    }
}

// Backward tiles with two or four pixels per thread, in two phases per round of kBwdRound list
// entries, each warp on its own pixels.
//
// Phase 1 (per pixel, back to front, as Eq. 8 orders it): each thread carries its pixels' state
// and, for every entry some pixel of the warp composites, writes two scalars per pixel to a row of
// the warp's round in shared memory:
// dpow = dL/dalpha alpha (zero through the 0.99 clamp) and wgt = alpha T (the weight of the entry's
// colour).  The state is the transmittance T in front of the current entry and S = <C_behind,
// dL/dC>, the colour behind the entry (Eq. 7's C_in) projected on the pixel's upstream gradient:
// dL/dalpha = T_i (<c_i, dL/dC> - S) and S <- S + alpha_i (<c_i, dL/dC> - S), the recurrence
// C_in <- C_in (1 - alpha) + alpha c.  A pixel that does not composite an entry takes alpha = 0.
//
// Phase 2 (per entry): the lanes of an entry sum over the warp's pixels the moments
// sum dpow (1, x, y, x^2, x y, y^2) (pixel centres relative to the tile centre) and
// sum wgt dL/dC, add them over those lanes and turn them into the nine screen-space gradients:
// with dx = x - u, dy = y - v,
//   sum dpow dx = Mx - u M0,  sum dpow dx^2 = Mxx - 2 u Mx + u^2 M0,  ...,
//   d mean = (a sum dpow dx + b sum dpow dy, c sum dpow dy + b sum dpow dx),
//   d conic = -(sum dpow dx^2 / 2, sum dpow dx dy, sum dpow dy^2 / 2),  d opacity = M0 / o,
// added to the canonical index with one atomic per value (Eq. 10's scatter).  No per-entry
// reduction across the warp's 32 lanes and no per-pixel moment arithmetic in the walk.
//
// The pixels of a tile are ordered by `last` first (a counting sort into 256 buckets of
// last * 255 / the tile's deepest last) and each warp takes 32 kPix consecutive pixels of that
// order, so a warp stops at its own deepest `last` (on the 500k/1080p view 90 % of a warp's walk
// lies inside its pixels' lists with 64 pixels per warp, against 83 % for compact 8 x 8 blocks).
// Pixel pairs run on the packed f32x2 instructions; every operand that is the same for the pair
// is staged duplicated, so it loads as a ready pair.
constexpr int kBwdRound = 8;  // entries per phase-1 / phase-2 round

template <int kT, int kPix, int kDepth>
struct Bwd2Smem {
    static constexpr int kWarps = kT * kT / kPix / 32;
    static constexpr int kPW = 16 * kPix;      // pixel pairs per warp
    static constexpr int kRow = kPW + 4;       // a round row, padded so that phase 2's reads of two
                                               // rows fall in different banks
    float4 xy[kDepth];  // (u, u, v, v)
    float4 ab[kDepth];  // (A, A, B, B): base-2 exponent coefficients (scaled conic)
    float4 co[kDepth];  // (C, C, o, o)
    float4 rg[kDepth];  // (r, r, g, g) colour
    float4 bz[kDepth];  // (b, b, conic a, conic c) colour blue, conic
    float2 bi[kDepth];  // (conic b, canonical index bits)
    float4 m0[kWarps * kPW];  // pixel pair (x, x, y, y) relative to the tile centre
    float4 gg0[kWarps * kPW]; // dL/dC (r, r, g, g)
    float2 gg1[kWarps * kPW]; // (b, b)
    uint32_t wmax[32];
    int rowj[kWarps][kBwdRound];  // staged entry of each row of a warp's round
    union {
        float4 D[kWarps][kBwdRound][kRow];  // per warp, row of the round and pixel pair: (dpow x2, wgt x2)
        struct {
            uint32_t order[kT * kT];  // tile pixels (row-major index) in the order of their `last`
            uint32_t count[256];
        } sort;  // only while the tile's pixels are ordered
    };
};

template <int kT, int kPix, int kDepth>
__device__ __forceinline__ void bwd_tile_2p(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                            const Scratch& sc, Bwd2Smem<kT, kPix, kDepth>& S) {
    static_assert(kPix == 2 || kPix == 4, "pairs of pixels");
    using Sm = Bwd2Smem<kT, kPix, kDepth>;
    constexpr int kThreads = kT * kT / kPix;
    constexpr int kWarps = kThreads / 32;
    constexpr int NP = kPix / 2;
    constexpr int kPW = Sm::kPW;
    constexpr int kE = kBwdRound;
    constexpr int L = 32 / kE;       // phase 2: lanes per entry
    constexpr int kPL = kPW / L;     // pairs per lane
    static_assert(L >= 1 && (L & (L - 1)) == 0 && kPW % L == 0, "phase-2 lanes");
    const int W = J.W, H = J.H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = (J.tile % J.TX) * kT, y0 = (J.tile / J.TX) * kT;
    const float cxt = (float)x0 + 0.5f * kT, cyt = (float)y0 + 0.5f * kT;  // tile centre
    const uint2 range = J.range;
    // ---- order the tile's pixels by `last`
    uint32_t end = 0;
    {
        uint32_t lst[kPix];
        uint32_t tmax = 0;
#pragma unroll
        for (int k = 0; k < kPix; ++k) {
            const int i = tid * kPix + k, px = x0 + i % kT, py = y0 + i / kT;
            lst[k] = (px < W && py < H) ? J.last[(size_t)py * W + px] : 0u;
            tmax = max(tmax, lst[k]);
        }
        for (int b = tid; b < 256; b += kThreads) S.sort.count[b] = 0;
        tmax = __reduce_max_sync(kFull, tmax);
        if (lane == 0) S.wmax[warp] = tmax;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kWarps; ++w) end = max(end, S.wmax[w]);
        uint32_t bucket[kPix];
#pragma unroll
        for (int k = 0; k < kPix; ++k) {
            bucket[k] = end ? (uint32_t)(((uint64_t)lst[k] * 255u) / end) : 0u;
            atomicAdd(&S.sort.count[bucket[k]], 1u);
        }
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the 256 bucket counts, 8 per lane
            uint32_t c[8], run = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                c[k] = run;
                run += S.sort.count[lane * 8 + k];
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t base = incl - run;
#pragma unroll
            for (int k = 0; k < 8; ++k) S.sort.count[lane * 8 + k] = base + c[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPix; ++k) S.sort.order[atomicAdd(&S.sort.count[bucket[k]], 1u)] = (uint32_t)(tid * kPix + k);
        __syncthreads();
    }
    // ---- this thread's pixels: kPix consecutive positions of the order = the warp's pairs lane NP + q
    const size_t plane = (size_t)W * H;
    const float3 bg = J.bg;
    F2 FX[NP], FY[NP], T[NP], Sb[NP], g0[NP], g1[NP], g2[NP];
    uint32_t my_last[kPix];
    uint32_t wlast = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float fx[2], fy[2], t[2] = {1.0f, 1.0f}, a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f}, c[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * q + h;
            const uint32_t i = S.sort.order[tid * kPix + k];
            const int px = x0 + (int)(i % kT), py = y0 + (int)(i / kT);
            fx[h] = (float)px + 0.5f;
            fy[h] = (float)py + 0.5f;
            my_last[k] = 0;
            if (px < W && py < H) {
                const size_t pp = (size_t)py * W + px;
                t[h] = J.T_final[pp];
                my_last[k] = J.last[pp];
                a[h] = J.dL[pp];
                b[h] = J.dL[plane + pp];
                c[h] = J.dL[2 * plane + pp];
            }
            wlast = max(wlast, my_last[k]);
        }
        FX[q] = f2(fx[0], fx[1]);
        FY[q] = f2(fy[0], fy[1]);
        T[q] = f2(t[0], t[1]);
        g0[q] = f2(a[0], a[1]);
        g1[q] = f2(b[0], b[1]);
        g2[q] = f2(c[0], c[1]);
        // S = <C_behind, dL/dC>, the background behind the last entry
        Sb[q] = fma2(f2(bg.z), g2[q], fma2(f2(bg.y), g1[q], mul2(f2(bg.x), g0[q])));
        // the pair's phase-2 operands; pair q of lane l is the warp's pair q 32 + l
        const int gp = warp * kPW + q * 32 + lane;
        const float rx0 = fx[0] - cxt, rx1 = fx[1] - cxt, ry0 = fy[0] - cyt, ry1 = fy[1] - cyt;
        S.m0[gp] = make_float4(rx0, rx1, ry0, ry1);
        S.gg0[gp] = make_float4(a[0], a[1], b[0], b[1]);
        S.gg1[gp] = make_float2(c[0], c[1]);
    }
    const uint32_t wmax = __reduce_max_sync(kFull, wlast);
    const F2 ONE = f2(1.0f);
    const int pe = lane / L, pl = lane % L;  // phase 2: entry of the round, lane inside the entry
    float4(* __restrict__ Dw)[Sm::kRow] = S.D[warp];

    while (end > 0) {
        const uint32_t start = end > (uint32_t)kDepth ? end - kDepth : 0u;
        const int cnt = (int)(end - start);
        __syncthreads();
#pragma unroll
        for (int e = tid; e < kDepth; e += kThreads) {
            if (e < cnt) {
                const uint32_t id = checked_id(vals[range.x + start + e], n, sc.status);
                const float4 xyo = sc.xyo[id];
                const float4 con = sc.conic[id];
                const float4 s2 = scaled_conic(con);
                const float4 c = sc.rgb[id];
                S.xy[e] = make_float4(xyo.x, xyo.x, xyo.y, xyo.y);
                S.ab[e] = make_float4(s2.x, s2.x, s2.y, s2.y);
                S.co[e] = make_float4(s2.z, s2.z, xyo.z, xyo.z);
                S.rg[e] = make_float4(c.x, c.x, c.y, c.y);
                S.bz[e] = make_float4(c.z, c.z, con.x, con.z);
                S.bi[e] = make_float2(con.y, __uint_as_float(id));
            }
        }
        __syncthreads();
        // this warp's entries: positions below its deepest `last`, back to front; the entries some
        // pixel of the warp composites fill rounds of kE rows, each summed by phase 2 when full
        const int jtop = (int)min((uint32_t)cnt, wmax > start ? wmax - start : 0u);
        int nrow = 0;
        for (int j = jtop - 1; j >= 0; --j) {
            // ---- phase 1: entry j for this thread's pixels
            const uint32_t pos = start + j;
            const float4 xy = S.xy[j], ab = S.ab[j], co = S.co[j], rg = S.rg[j], bz = S.bz[j];
            const F2 X2 = f2(xy.x, xy.y), Y2 = f2(xy.z, xy.w);
            const F2 A2 = f2(ab.x, ab.y), B2 = f2(ab.z, ab.w), C2 = f2(co.x, co.y), O2 = f2(co.z, co.w);
            const F2 Cr = f2(rg.x, rg.y), Cg = f2(rg.z, rg.w), Cb = f2(bz.x, bz.y);
            float4 out1[NP];
            bool mine = false;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const F2 DX = sub2(FX[q], X2), DY = sub2(FY[q], Y2);
                // the forward's exponent, term for term: A dx^2 + B dx dy + C dy^2
                const float2 p = un(fma2(C2, mul2(DY, DY), fma2(B2, mul2(DX, DY), mul2(A2, mul2(DX, DX)))));
                const float2 og = un(mul2(O2, f2(ex2_approx(p.x), ex2_approx(p.y))));
                const float ax = fminf(kAlphaMax, og.x), ay = fminf(kAlphaMax, og.y);
                const bool p0 = pos < my_last[2 * q] && ax >= kAlphaMin;
                const bool p1 = pos < my_last[2 * q + 1] && ay >= kAlphaMin;
                mine = mine || p0 || p1;
                // a pixel that does not composite the entry takes alpha = 0
                const F2 A = f2(p0 ? ax : 0.0f, p1 ? ay : 0.0f);
                // alpha through which the gradient flows: zero at the 0.99 clamp
                const F2 AQ = f2(p0 && og.x <= kAlphaMax ? ax : 0.0f, p1 && og.y <= kAlphaMax ? ay : 0.0f);
                const float2 om = un(sub2(ONE, A));
                float rx, ry;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(om.x));
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(om.y));
                const F2 Tb = mul2(T[q], f2(p0 ? rx : 1.0f, p1 ? ry : 1.0f));  // transmittance in front
                const F2 cg = fma2(Cb, g2[q], fma2(Cg, g1[q], mul2(Cr, g0[q])));
                const F2 r = sub2(cg, Sb[q]);
                const float2 dpow = un(mul2(mul2(Tb, r), AQ));
                const float2 wgt = un(mul2(A, Tb));
                Sb[q] = fma2(A, r, Sb[q]);
                T[q] = Tb;
                out1[q] = make_float4(dpow.x, dpow.y, wgt.x, wgt.y);
            }
            if (__any_sync(kFull, mine)) {  // warp-uniform: the entry gets a row of the round
#pragma unroll
                for (int q = 0; q < NP; ++q) Dw[nrow][q * 32 + lane] = out1[q];
                if (lane == 0) S.rowj[warp][nrow] = j;
                ++nrow;
            }
            if (nrow < kE && j > 0) continue;
            if (nrow == 0) break;
            __syncwarp();
            // ---- phase 2: row pe (entry rowj[pe]), summed over the warp's pairs pl, pl + L, ...
            // (consecutive lanes read consecutive pairs: no bank conflict)
            if (pe < nrow) {
                const float4* __restrict__ Drow = Dw[pe];
                F2 acc[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = f2(0.0f);
#pragma unroll 4
                for (int k = 0; k < kPL; ++k) {
                    const int lp = pl + L * k, gp = warp * kPW + lp;
                    const float4 d = Drow[lp], m0 = S.m0[gp], q0 = S.gg0[gp];
                    const float2 q1 = S.gg1[gp];
                    const F2 DP = f2(d.x, d.y), WG = f2(d.z, d.w), X = f2(m0.x, m0.y), Y = f2(m0.z, m0.w);
                    const F2 DX = mul2(DP, X), DY = mul2(DP, Y);
                    acc[0] = add2(acc[0], DP);
                    acc[1] = add2(acc[1], DX);
                    acc[2] = add2(acc[2], DY);
                    acc[3] = fma2(DX, X, acc[3]);
                    acc[4] = fma2(DX, Y, acc[4]);
                    acc[5] = fma2(DY, Y, acc[5]);
                    acc[6] = fma2(WG, f2(q0.x, q0.y), acc[6]);
                    acc[7] = fma2(WG, f2(q0.z, q0.w), acc[7]);
                    acc[8] = fma2(WG, f2(q1.x, q1.y), acc[8]);
                }
                float v[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float2 h = un(acc[k]);
                    v[k] = h.x + h.y;
                }
                // add over the L lanes of the entry (all of them end with the totals)
                const unsigned gmask = L == 32 ? kFull : (((1u << L) - 1u) << (lane & ~(L - 1)));
#pragma unroll
                for (int o = 1; o < L; o <<= 1)
#pragma unroll
                    for (int k = 0; k < 9; ++k) v[k] += __shfl_xor_sync(gmask, v[k], o);
                const int je = S.rowj[warp][pe];
                const float M0 = v[0], Mx = v[1], My = v[2], Mxx = v[3], Mxy = v[4], Myy = v[5];
                const float u = S.xy[je].x - cxt, vv = S.xy[je].z - cyt;  // mean relative to the tile centre
                const float sdx = fmaf(-u, M0, Mx), sdy = fmaf(-vv, M0, My);  // sum dpow dx, sum dpow dy
                float out[9];
                const float ca = S.bz[je].z, cc = S.bz[je].w, cb = S.bi[je].x;
                out[0] = fmaf(ca, sdx, cb * sdy);
                out[1] = fmaf(cc, sdy, cb * sdx);
                out[2] = -0.5f * fmaf(-u, sdx, fmaf(-u, Mx, Mxx));    // sum dpow dx^2
                out[3] = -fmaf(-vv, sdx, fmaf(-u, My, Mxy));          // sum dpow dx dy
                out[4] = -0.5f * fmaf(-vv, sdy, fmaf(-vv, My, Myy));  // sum dpow dy^2
                out[5] = __fdividef(M0, S.co[je].z);
                out[6] = v[6];
                out[7] = v[7];
                out[8] = v[8];
                const uint32_t id = __float_as_uint(S.bi[je].y);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    if (k % L == pl) atomicAdd(&sc.grad2d[(size_t)k * n + id], out[k]);
            }
            __syncwarp();
            nrow = 0;
        }
        end = start;
    }
}

template <int kT, int kPix, int kDepth>
__device__ __forceinline__ float2 fwd_tile(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                           const Scratch& sc, FwdSmem<kDepth>& S) {
    if constexpr (kPix == 1) return fwd_tile_scalar<kT, kPix, kDepth>(J, n, vals, sc, S);
    else return fwd_tile_pairs<kT, kPix, kDepth>(J, n, vals, sc, S);
}

// shared memory of a backward tile: one pixel per thread stages plain records, pairs the packed ones
template <int kT, int kPix, int kDepth>
using BwdSmemOf = typename std::conditional<
    kPix == 1, BwdSmem<kDepth>,
    typename std::conditional<kT == 32, BwdSmemPacked<kT, kDepth>, Bwd2Smem<kT, kPix, kDepth>>::type>::type;

template <int kT, int kPix, int kDepth, bool kBackward>
using BatchSmem = typename std::conditional<kBackward, BwdSmemOf<kT, kPix, kDepth>, FwdSmem<kDepth>>::type;

// Shared memory of a compositing kernel comes dynamically (the two-phase backward needs more than
// the 48 KB a static allocation may take); the limit is raised once per kernel.
template <class Kernel>
static size_t dynamic_smem(Kernel k, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return bytes;
}

template <int kT, int kPix, int kDepth>
__device__ __forceinline__ void bwd_tile(const TileJob& J, int64_t n, const uint32_t* __restrict__ vals,
                                         const Scratch& sc, BwdSmemOf<kT, kPix, kDepth>& S) {
    if constexpr (kPix == 1) bwd_tile_scalar<kT, kPix, kDepth>(J, n, vals, sc, S);
    else if constexpr (kT == 32) bwd_tile_sorted<kT, kPix, kDepth>(J, n, vals, sc, S);
    else bwd_tile_2p<kT, kPix, kDepth>(J, n, vals, sc, S);
}


__device__ __forceinline__ int render_of_tile(const RenderDesc* __restrict__ renders, int R, int64_t gt) {
    int lo = 0, hi = R - 1;  // last render whose tile_base <= gt
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (renders[mid].tile_base <= gt) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ TileJob batch_job(const RenderDesc& rd, int64_t gt, const Scratch& sc) {
    TileJob J;
    J.W = rd.cam.width;
    J.H = rd.cam.height;
    J.TX = rd.TX;
    J.tile = (int)(gt - rd.tile_base);
    J.bg = make_float3(rd.cam.bg[0], rd.cam.bg[1], rd.cam.bg[2]);
    J.range = sc.ranges[gt];
    J.image = rd.image;
    J.dL = rd.dL;
    J.T_final = sc.T_final + rd.pixel_base;
    J.last = sc.last + rd.pixel_base;
    J.ncomp = sc.ncomp + rd.pixel_base;
    return J;
}

template <int kT, int kPix, int kDepth>
__global__ void __launch_bounds__(kT * kT / kPix)
k_composite_fwd(int W, int H, int TX, float3 bg, int64_t n, const uint32_t* __restrict__ vals,
                Scratch sc, float* __restrict__ image, int64_t zero_grad, L1Fused l1f) {
    __shared__ FwdSmem<kDepth> S;
    TileJob J;
    J.W = W;
    J.H = H;
    J.TX = TX;
    J.tile = (int)sc.tile_order[blockIdx.x];
    J.bg = bg;
    J.range = sc.ranges[J.tile];
    J.image = image;
    J.dL = nullptr;
    J.T_final = sc.T_final;
    J.last = sc.last;
    J.ncomp = sc.ncomp;
    J.target = l1f.target;
    J.dL_out = l1f.dL;
    J.inv_n = l1f.inv_n;
    const float2 l = fwd_tile<kT, kPix, kDepth>(J, n, vals, sc, S);
    if (l1f.target) {  // the tile's L1 sums into the render's double accumulators; the last CTA reports
        constexpr int kWarps = kT * kT / kPix / 32;
        __shared__ float s_l1[kWarps], s_l2[kWarps];
        __shared__ bool s_last;
        float a = l.x, b = l.y;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(kFull, a, o);
            b += __shfl_xor_sync(kFull, b, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_l1[threadIdx.x >> 5] = a;
            s_l2[threadIdx.x >> 5] = b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ta = 0.0, tb = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                ta += (double)s_l1[w];
                tb += (double)s_l2[w];
            }
            atomicAdd(&l1f.acc[0], ta);
            atomicAdd(&l1f.acc[1], tb);
            __threadfence();
            s_last = atomicAdd(l1f.ticket, 1u) == gridDim.x - 1;
            if (s_last) {
                __threadfence();
                l1f.out[0] = (float)(atomicAdd(&l1f.acc[0], 0.0) / (double)l1f.n);
                l1f.out[1] = (float)atomicAdd(&l1f.acc[1], 0.0);
            }
        }
    }
    if (zero_grad > 0) {  // grad2d is 256-byte aligned: 16-byte stores, the tail by block 0
        float4* g4 = reinterpret_cast<float4*>(sc.grad2d);
        const int64_t n4 = zero_grad >> 2;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n4; w += stride)
            g4[w] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (blockIdx.x == 0 && threadIdx.x < (zero_grad & 3)) sc.grad2d[(n4 << 2) + threadIdx.x] = 0.f;
    }
}

template <int kT, int kPix, int kDepth>
__global__ void __launch_bounds__(kT * kT / kPix)
k_composite_bwd(int W, int H, int TX, float3 bg, int64_t n, const uint32_t* __restrict__ vals,
                Scratch sc, const float* __restrict__ dL_dimage) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    auto& S = *reinterpret_cast<BwdSmemOf<kT, kPix, kDepth>*>(dyn_smem);
    TileJob J;
    J.W = W;
    J.H = H;
    J.TX = TX;
    J.tile = (int)sc.tile_order[blockIdx.x];
    J.bg = bg;
    J.range = sc.ranges[J.tile];
    J.image = nullptr;
    J.dL = dL_dimage;
    J.T_final = sc.T_final;
    J.last = sc.last;
    J.ncomp = sc.ncomp;
    bwd_tile<kT, kPix, kDepth>(J, n, vals, sc, S);
}

// Replay-cache forward and backward (one pixel per thread, 256 entries staged per batch).
template <int kT>
__global__ void __launch_bounds__(kT * kT)
k_composite_fwd_record(int W, int H, int TX, float3 bg, int64_t n, const uint32_t* __restrict__ vals,
                       Scratch sc, float* __restrict__ image, ReplayCache rc) {
    __shared__ FwdSmem<256> S;
    TileJob J;
    J.W = W;
    J.H = H;
    J.TX = TX;
    J.tile = (int)sc.tile_order[blockIdx.x];
    J.bg = bg;
    J.range = sc.ranges[J.tile];
    J.image = image;
    J.dL = nullptr;
    J.T_final = sc.T_final;
    J.last = sc.last;
    J.ncomp = sc.ncomp;
    fwd_tile_scalar<kT, 1, 256, true>(J, n, vals, sc, S, rc);
}

template <int kT>
__global__ void __launch_bounds__(kT * kT)
k_composite_bwd_replay(int W, int H, int TX, float3 bg, int64_t n, const uint32_t* __restrict__ vals,
                       Scratch sc, const float* __restrict__ dL_dimage, ReplayCache rc) {
    __shared__ BwdSmem<256> S;
    TileJob J;
    J.W = W;
    J.H = H;
    J.TX = TX;
    J.tile = (int)sc.tile_order[blockIdx.x];
    J.bg = bg;
    J.range = sc.ranges[J.tile];
    J.image = nullptr;
    J.dL = dL_dimage;
    J.T_final = sc.T_final;
    J.last = sc.last;
    J.ncomp = sc.ncomp;
    bwd_tile_scalar<kT, 1, 256, true>(J, n, vals, sc, S, rc);
}

// Batched compositing: persistent CTAs take global tiles, heaviest first, until every tile of
// every render is done.  A CTA's first job is its own index, so the first (heaviest) round is
// spread over the SMs in launch order as a one-tile-per-CTA grid would be; later jobs come from a
// device work counter (an atomic ticket offset by the grid size; no CTA ever waits for another).
// Taking the first round from the ticket too let the heaviest tiles gather on a few SMs (the
// CTAs of one SM reach the ticket together) and left the other SMs idle at the end.
template <int kT, int kPix, int kDepth, bool kBackward>
__global__ void __launch_bounds__(kT * kT / kPix)
k_composite_batch(const RenderDesc* __restrict__ renders, int R, int64_t total_tiles, int64_t n,
                  const uint32_t* __restrict__ vals, Scratch sc, uint32_t* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    auto& S = *reinterpret_cast<BatchSmem<kT, kPix, kDepth, kBackward>*>(dyn_smem);
    __shared__ int64_t s_job;
    int64_t job = blockIdx.x;
    while (job < total_tiles) {
        const int64_t gt = sc.tile_order[job];
        const TileJob J = batch_job(renders[render_of_tile(renders, R, gt)], gt, sc);
        if constexpr (kBackward) bwd_tile<kT, kPix, kDepth>(J, n, vals, sc, S);
        else fwd_tile<kT, kPix, kDepth>(J, n, vals, sc, S);
        __syncthreads();
        if (threadIdx.x == 0) s_job = (int64_t)atomicAdd(work, 1u) + gridDim.x;
        __syncthreads();
        job = s_job;
    }
}

// Decision trace of listed pixels (one thread per pixel): walk the pixel's tile list front to back
// with the forward kernels' own evaluation (entry_alpha, the same staging of the conic, dx, dy,
// T (1 - alpha)), and record per evaluated entry o G before the clamp and the decision taken:
// 0 skipped (alpha < 1/255), 1 composited, 2 composited clamped at 0.99, 3 stop (T (1 - alpha)
// < 1e-4; the walk ends there).  count = entries evaluated (recorded up to max_entries);
// T_out / last_out / ncomp_out = the fp32 transmittance, 1 + position of the last composited entry
// and the composited count, which equal the forward's T_final, last and ncomp.  A pixel outside
// the image gets count -1.
__global__ void k_trace_pixels(int W, int H, int TX, int T, int64_t n, const uint32_t* __restrict__ vals,
                               Scratch sc, const int32_t* __restrict__ pix, int64_t npix, int max_entries,
                               float* __restrict__ og_out, uint8_t* __restrict__ code_out,
                               int32_t* __restrict__ count_out, float* __restrict__ T_out,
                               uint32_t* __restrict__ last_out, uint32_t* __restrict__ ncomp_out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npix) return;
    const int px = pix[2 * k], py = pix[2 * k + 1];
    if (px < 0 || py < 0 || px >= W || py >= H) {
        count_out[k] = -1;
        return;
    }
    const uint2 range = sc.ranges[(py / T) * TX + px / T];
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    float Tr = 1.0f;
    uint32_t last = 0, ncomp = 0;
    int32_t count = 0;
    for (uint32_t idx = range.x; idx < range.y; ++idx) {
        const uint32_t id = checked_id(vals[idx], n, sc.status);
        const float4 p = sc.xyo[id];
        const float4 s2 = scaled_conic(sc.conic[id]);
        const float dx = fx - p.x;
        const float adx2 = __fmul_rn(s2.x, __fmul_rn(dx, dx));
        float G, og;
        const float alpha = entry_alpha(dx, fy - p.y, adx2, s2, p.z, G, og);
        uint8_t code = 0;
        bool stop = false;
        if (alpha >= kAlphaMin) {
            const float Tn = Tr * (1.0f - alpha);
            if (Tn < kTMin) {
                code = 3;
                stop = true;
            } else {
                code = og > kAlphaMax ? 2 : 1;
                Tr = Tn;
                last = idx - range.x + 1;
                ++ncomp;
            }
        }
        if (count < max_entries) {
            og_out[k * max_entries + count] = og;
            code_out[k * max_entries + count] = code;
        }
        ++count;
        if (stop) break;
    }
    count_out[k] = count;
    T_out[k] = Tr;
    last_out[k] = last;
    ncomp_out[k] = ncomp;
}

}  // namespace

// pixels per thread and staging depth (64, 128, 256 entries) of the compositing kernels; default
// (2, 256), the autotuner's choice on the 500k-Gaussian 1080p workload, valid for every tile edge.
// PGS_COMPOSITE_PIXELS / PGS_COMPOSITE_DEPTH override the default (read once per process).
CompositeVariant default_variant() {
    static CompositeVariant v = [] {
        CompositeVariant c{2, 256};
        if (const char* e = getenv("PGS_COMPOSITE_PIXELS")) c.pix = atoi(e);
        if (const char* e = getenv("PGS_COMPOSITE_DEPTH")) c.depth = atoi(e);
        if (!valid_variant(c, kTileDefault) || !valid_variant(c, 8) || !valid_variant(c, 32))
            c = CompositeVariant{2, 256};
        return c;
    }();
    return v;
}

// Strips per tile edge: T = 8 takes 1 or 2 pixels per thread (64 or 32 threads per tile), T = 16
// takes 1, 2 or 4 (256, 128, 64 threads), T = 32 takes 2 or 4 (512, 256 threads), so every CTA
// is whole warps.
bool valid_variant(CompositeVariant v, int T) {
    const bool depth = v.depth == 64 || v.depth == 128 || v.depth == 256;
    if (T == 8) return depth && (v.pix == 1 || v.pix == 2);
    if (T == 16) return depth && (v.pix == 1 || v.pix == 2 || v.pix == 4);
    if (T == 32) return depth && (v.pix == 2 || v.pix == 4);
    return false;
}

#define PGS_VARIANTS(X)                                                                           \
    X(8, 1, 64) X(8, 1, 128) X(8, 1, 256) X(8, 2, 64) X(8, 2, 128) X(8, 2, 256)                   \
    X(16, 1, 64) X(16, 1, 128) X(16, 1, 256) X(16, 2, 64) X(16, 2, 128) X(16, 2, 256)             \
    X(16, 4, 64) X(16, 4, 128) X(16, 4, 256)                                                      \
    X(32, 2, 64) X(32, 2, 128) X(32, 2, 256) X(32, 4, 64) X(32, 4, 128) X(32, 4, 256)

int launch_composite_fwd(const pgs_camera& cam, int TX, int TY, int T, int buf, int64_t n,
                         const Scratch& sc, float* image, cudaStream_t s, CompositeVariant v, int64_t zero_grad,
                         const L1Fused& l1f) {
    const float3 bg = make_float3(cam.bg[0], cam.bg[1], cam.bg[2]);
#define X(TT, P, D)                                                                               \
    if (T == TT && v.pix == P && v.depth == D) {                                                  \
        k_composite_fwd<TT, P, D><<<TX * TY, TT * TT / P, 0, s>>>(cam.width, cam.height, TX, bg, n, \
                                                                  sc.vals[buf], sc, image, zero_grad, l1f); \
        return 1;                                                                                 \
    }
    PGS_VARIANTS(X)
#undef X
    return 0;
}

int launch_composite_bwd(const pgs_camera& cam, int TX, int TY, int T, int buf, int64_t n,
                         const Scratch& sc, const float* dL_dimage, cudaStream_t s, CompositeVariant v) {
    const float3 bg = make_float3(cam.bg[0], cam.bg[1], cam.bg[2]);
#define X(TT, P, D)                                                                               \
    if (T == TT && v.pix == P && v.depth == D) {                                                  \
        static const size_t smem = dynamic_smem(k_composite_bwd<TT, P, D>, sizeof(BwdSmemOf<TT, P, D>)); \
        k_composite_bwd<TT, P, D><<<TX * TY, TT * TT / P, smem, s>>>(cam.width, cam.height, TX, bg, n, \
                                                                     sc.vals[buf], sc, dL_dimage); \
        return 1;                                                                                 \
    }
    PGS_VARIANTS(X)
#undef X
    return 0;
}

int launch_composite_replay(const pgs_camera& cam, int TX, int TY, int T, int buf, int64_t n,
                            const Scratch& sc, float* image, const float* dL_dimage, float4* rec,
                            uint32_t* count, int K, bool backward, cudaStream_t s) {
    const float3 bg = make_float3(cam.bg[0], cam.bg[1], cam.bg[2]);
    ReplayCache rc;
    rc.rec = rec;
    rc.count = count;
    rc.K = K;
    const unsigned grid = (unsigned)(TX * TY);
#define X(TT)                                                                                     \
    if (T == TT) {                                                                                \
        if (backward)                                                                             \
            k_composite_bwd_replay<TT><<<grid, TT * TT, 0, s>>>(cam.width, cam.height, TX, bg, n, \
                                                               sc.vals[buf], sc, dL_dimage, rc);  \
        else                                                                                      \
            k_composite_fwd_record<TT><<<grid, TT * TT, 0, s>>>(cam.width, cam.height, TX, bg, n, \
                                                               sc.vals[buf], sc, image, rc);      \
        return 1;                                                                                 \
    }
    X(8) X(16) X(32)
#undef X
    return 0;
}

template <int TT, int P, int D, bool B>
static int launch_batch_variant(const RenderDesc* renders, int R, int64_t total_tiles, int buf,
                                int64_t n, const Scratch& sc, uint32_t* work, cudaStream_t s) {
    static const size_t smem = dynamic_smem(k_composite_batch<TT, P, D, B>, sizeof(BatchSmem<TT, P, D, B>));
    static int grid = [] {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite_batch<TT, P, D, B>, TT * TT / P, smem);
        return sms * (per_sm > 0 ? per_sm : 1);
    }();
    const int64_t g = grid < total_tiles ? grid : total_tiles;  // every CTA has a first job
    if (g < 1) return 0;
    k_composite_batch<TT, P, D, B><<<(unsigned)g, TT * TT / P, smem, s>>>(renders, R, total_tiles, n,
                                                                          sc.vals[buf], sc, work);
    return 1;
}

int launch_composite_batch(const RenderDesc* renders, int R, int64_t total_tiles, int T, int buf,
                           int64_t n, const Scratch& sc, uint32_t* work, bool backward,
                           cudaStream_t s, CompositeVariant v) {
#define X(TT, P, D)                                                                               \
    if (T == TT && v.pix == P && v.depth == D)                                                    \
        return backward ? launch_batch_variant<TT, P, D, true>(renders, R, total_tiles, buf, n, sc, work, s) \
                        : launch_batch_variant<TT, P, D, false>(renders, R, total_tiles, buf, n, sc, work, s);
    PGS_VARIANTS(X)
#undef X
    return 0;
}


int launch_trace_pixels(const pgs_camera& cam, int TX, int T, int buf, int64_t n, const Scratch& sc,
                        const int32_t* pix, int64_t npix, int max_entries, float* og, uint8_t* code,
                        int32_t* count, float* T_out, uint32_t* last, uint32_t* ncomp, cudaStream_t s) {
    if (npix <= 0) return 0;
    const int threads = 128;
    k_trace_pixels<<<(unsigned)((npix + threads - 1) / threads), threads, 0, s>>>(
        cam.width, cam.height, TX, T, n, sc.vals[buf], sc, pix, npix, max_entries, og, code, count, T_out, last,
        ncomp);
    return 1;
}

}  // namespace pgs
