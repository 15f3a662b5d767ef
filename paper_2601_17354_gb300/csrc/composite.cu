// K6 composite_fwd and K8 composite_bwd: one CTA per 16x16 screen tile, one pixel per thread.
//
// Forward (Eq. 7, evaluated front to back with transmittance T): the tile's depth-ordered list
// [range.x, range.y) is staged in shared memory in batches of 256 entries (projected record
// gathered through the canonical index, i.e. through pi of Eq. 10); each pixel composites
//     alpha = min(0.99, o exp(power)),  skip if alpha < 1/255,
//     stop (without compositing) when T (1 - alpha) < 1e-4,  C += alpha T c,  T *= 1 - alpha,
// and keeps only T_final and last = 1 + list position of the last composited entry.
//
// Backward: instead of the paper's per-pixel replay cache S = {id, C_in, alpha} (Eq. 9) the
// kernel re-traverses the list back to front from `last`, rebuilding the transmittance in front
// of each entry from T_final (T_i = T_{i+1} / (1 - alpha_i); alpha <= 0.99 bounds the growth) and
// the colour behind it with Eq. 7 itself (C_in of the last entry is the background), then applies
// Eq. 8:  dL/dc = alpha dL/dC_out,  dL/dalpha = <dL/dC_out, c - C_in>,  dL/dC_out = T_i dL/dC.
// Per entry, the nine screen-space gradients of the warp's 32 pixels are summed by a
// transpose-reduction (9 shuffles for 8 values) and scattered with one atomic per value per
// warp to the canonical index (Eq. 10: grad_{pi(i)} += g_i).
#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBatch = kTilePixels;  // entries staged per batch (one per thread)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// alpha of one (pixel, entry), written with explicit roundings so the forward and the backward
// take identical decisions.  og = o * exp(power) before the clamp.
__device__ __forceinline__ float entry_alpha(float dx, float dy, float4 con, float o, float& G,
                                             float& og) {
    const float quad = __fmaf_rn(con.x, __fmul_rn(dx, dx), __fmul_rn(con.z, __fmul_rn(dy, dy)));
    const float power = __fmaf_rn(-0.5f, quad, -__fmul_rn(con.y, __fmul_rn(dx, dy)));
    G = __expf(power);
    og = __fmul_rn(o, G);
    return fminf(kAlphaMax, og);
}

__global__ void __launch_bounds__(kTilePixels)
k_composite_fwd(int W, int H, int TX, float3 bg, int64_t n, const uint32_t* __restrict__ vals,
                Scratch sc, float* __restrict__ image) {
    __shared__ float4 s_xyo[kBatch];
    __shared__ float4 s_con[kBatch];
    __shared__ float4 s_rgb[kBatch];
    const int tile = blockIdx.x;
    const int px = (tile % TX) * kTile + (threadIdx.x % kTile);
    const int py = (tile / TX) * kTile + (threadIdx.x / kTile);
    const bool inside = px < W && py < H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 range = sc.ranges[tile];
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0, ncomp = 0;
    bool done = !inside;
    for (uint32_t base = range.x; base < range.y; base += kBatch) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const uint32_t k = base + threadIdx.x;
        if (k < range.y) {
            uint32_t id = vals[k];
            if (id >= n) {
                atomicOr(sc.status, kStatusInternal);
                id = 0;
            }
            s_xyo[threadIdx.x] = sc.xyo[id];
            s_con[threadIdx.x] = sc.conic[id];
            s_rgb[threadIdx.x] = sc.rgb[id];
        }
        __syncthreads();
        const int cnt = min((uint32_t)kBatch, range.y - base);
        for (int j = 0; !done && j < cnt; ++j) {
            const float4 p = s_xyo[j];
            float G, og;
            const float alpha = entry_alpha(fx - p.x, fy - p.y, s_con[j], p.z, G, og);
            if (alpha < kAlphaMin) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < kTMin) {
                done = true;
                break;
            }
            const float4 c = s_rgb[j];
            const float w = alpha * T;
            C0 = fmaf(c.x, w, C0);
            C1 = fmaf(c.y, w, C1);
            C2 = fmaf(c.z, w, C2);
            T = Tn;
            last = base + j - range.x + 1;
            ++ncomp;
        }
    }
    if (inside) {
        const size_t p = (size_t)py * W + px, plane = (size_t)W * H;
        image[p] = fmaf(T, bg.x, C0);
        image[plane + p] = fmaf(T, bg.y, C1);
        image[2 * plane + p] = fmaf(T, bg.z, C2);
        sc.T_final[p] = T;
        sc.last[p] = last;
        sc.ncomp[p] = ncomp;
    }
}

// Sum v[0..8] over the warp.  Afterwards lane l with l % 4 == 0 holds the sum of v[l >> 2]
// (values 0..7) and every lane holds the sum of v[8].
__device__ __forceinline__ void warp_sum9(float v[9], int lane, float& s8, float& s9) {
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

__global__ void __launch_bounds__(kTilePixels)
k_composite_bwd(int W, int H, int TX, float3 bg, int64_t n, const uint32_t* __restrict__ vals,
                Scratch sc, const float* __restrict__ dL_dimage) {
    __shared__ float4 s_xyo[kBatch];
    __shared__ float4 s_con[kBatch];
    __shared__ float4 s_rgb[kBatch];
    __shared__ uint32_t s_id[kBatch];
    __shared__ uint32_t s_max[kTilePixels / 32];
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int px = (tile % TX) * kTile + (threadIdx.x % kTile);
    const int py = (tile / TX) * kTile + (threadIdx.x / kTile);
    const bool inside = px < W && py < H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 range = sc.ranges[tile];
    const size_t p = (size_t)py * W + px, plane = (size_t)W * H;
    float T = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t my_last = 0;
    if (inside) {
        T = sc.T_final[p];
        my_last = sc.last[p];
        g0 = dL_dimage[p];
        g1 = dL_dimage[plane + p];
        g2 = dL_dimage[2 * plane + p];
    }
    float B0 = bg.x, B1 = bg.y, B2 = bg.z;  // colour behind the current entry (Eq. 7 C_in)
    const uint32_t wmax = __reduce_max_sync(kFull, my_last);
    if (lane == 0) s_max[threadIdx.x >> 5] = wmax;
    __syncthreads();
    uint32_t end = 0;
#pragma unroll
    for (int w = 0; w < kTilePixels / 32; ++w) end = max(end, s_max[w]);

    for (; end > 0;) {
        const uint32_t start = end > (uint32_t)kBatch ? end - kBatch : 0u;
        const int cnt = (int)(end - start);
        __syncthreads();
        if (threadIdx.x < cnt) {
            uint32_t id = vals[range.x + start + threadIdx.x];
            if (id >= n) {
                atomicOr(sc.status, kStatusInternal);
                id = 0;
            }
            s_id[threadIdx.x] = id;
            s_xyo[threadIdx.x] = sc.xyo[id];
            s_con[threadIdx.x] = sc.conic[id];
            s_rgb[threadIdx.x] = sc.rgb[id];
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            float v[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = 0.f;
            bool contrib = false;
            if (start + j < my_last) {
                const float4 pm = s_xyo[j];
                const float4 con = s_con[j];
                const float dx = fx - pm.x, dy = fy - pm.y;
                float G, og;
                const float alpha = entry_alpha(dx, dy, con, pm.z, G, og);
                if (alpha >= kAlphaMin) {
                    contrib = true;
                    const float4 c = s_rgb[j];
                    const float Tb = __fdividef(T, 1.0f - alpha);  // transmittance in front
                    const float dLda = Tb * ((c.x - B0) * g0 + (c.y - B1) * g1 + (c.z - B2) * g2);
                    const float wgt = alpha * Tb;
                    v[6] = wgt * g0;
                    v[7] = wgt * g1;
                    v[8] = wgt * g2;
                    B0 = fmaf(alpha, c.x - B0, B0);
                    B1 = fmaf(alpha, c.y - B1, B1);
                    B2 = fmaf(alpha, c.z - B2, B2);
                    T = Tb;
                    if (og <= kAlphaMax) {  // zero gradient through the 0.99 clamp
                        v[5] = dLda * G;
                        const float dpow = dLda * alpha;
                        v[0] = dpow * (con.x * dx + con.y * dy);
                        v[1] = dpow * (con.z * dy + con.y * dx);
                        v[2] = -0.5f * dpow * dx * dx;
                        v[3] = -dpow * dx * dy;
                        v[4] = -0.5f * dpow * dy * dy;
                    }
                }
            }
            if (__any_sync(kFull, contrib)) {
                float s8, s9;
                warp_sum9(v, lane, s8, s9);
                const uint32_t id = s_id[j];
                if ((lane & 3) == 0) atomicAdd(&sc.grad2d[(size_t)(lane >> 2) * n + id], s8);
                if (lane == 1) atomicAdd(&sc.grad2d[(size_t)8 * n + id], s9);
            }
        }
        end = start;
    }
}

}  // namespace

int launch_composite_fwd(const pgs_camera& cam, int TX, int TY, int buf, int64_t n,
                         const Scratch& sc, float* image, cudaStream_t s) {
    k_composite_fwd<<<TX * TY, kTilePixels, 0, s>>>(cam.width, cam.height, TX,
                                                     make_float3(cam.bg[0], cam.bg[1], cam.bg[2]), n,
                                                     sc.vals[buf], sc, image);
    return 1;
}

int launch_composite_bwd(const pgs_camera& cam, int TX, int TY, int buf, int64_t n,
                          const Scratch& sc, const float* dL_dimage, cudaStream_t s) {
    k_composite_bwd<<<TX * TY, kTilePixels, 0, s>>>(cam.width, cam.height, TX,
                                                     make_float3(cam.bg[0], cam.bg[1], cam.bg[2]), n,
                                                     sc.vals[buf], sc, dL_dimage);
    return 1;
}

}  // namespace pgs
