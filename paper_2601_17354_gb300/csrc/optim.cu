// K7 L1 loss and K10 fused Adam.
//
// Adam (Kingma & Ba 2015) runs over every parameter group of the canonical buffer in one launch,
// in canonical order, so the moments stay aligned with their parameters (Sec. III-C, "keeping
// Adam states aligned with their parameters without CPU intervention"); it also zeroes the
// gradients it consumed.
#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int kThreads = 256;

// mean |x - y| and sum (x - y)^2 over n values, gradient sign(x - y) / n.  Partial sums per
// CTA; the last CTA to finish (ticket counter) adds them in a fixed order, so the result does
// not depend on scheduling.  No CTA waits for another.
__global__ void __launch_bounds__(kThreads)
k_loss_l1(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
          float* __restrict__ grad, float* __restrict__ out, float* partials, uint32_t* ticket) {
    const float inv_n = 1.0f / (float)n;
    float l1 = 0.f, l2 = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        const float d = x[k] - y[k];
        l1 += fabsf(d);
        l2 = fmaf(d, d, l2);
        grad[k] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    }
    __shared__ float s1[kThreads / 32], s2[kThreads / 32];
    __shared__ bool s_last;
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s1[threadIdx.x >> 5] = l1;
        s2[threadIdx.x >> 5] = l2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) {
            a += s1[w];
            b += s2[w];
        }
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA: fixed-order sum of the partials (strided per thread, then a fixed tree)
    __shared__ double d1[kThreads], d2[kThreads];
    double a = 0.0, b = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += kThreads) {
        a += (double)__ldcg(partials + k);
        b += (double)__ldcg(partials + gridDim.x + k);
    }
    d1[threadIdx.x] = a;
    d2[threadIdx.x] = b;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            d1[threadIdx.x] += d1[threadIdx.x + w];
            d2[threadIdx.x] += d2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = (float)(d1[0] / (double)n);
        out[1] = (float)d2[0];
        *ticket = 0;
    }
}

struct AdamArgs {
    float* p[5];
    float* g[5];
    float* m[5];
    float* v[5];
    float lr[6];
    int64_t n;
    int K;
    float b1, b2, omb1, omb2, eps, isb;  // omb = 1 - b, isb = 1 / sqrt(1 - b2^t), in double on the host
};

// row r of the (11 + 3K) x n parameter matrix -> group, row inside the group, learning rate
__device__ __forceinline__ void row_of(const AdamArgs& a, int r, int& grp, int& sub, float& lr) {
    if (r < 3) { grp = 0; sub = r; lr = a.lr[0]; }
    else if (r < 6) { grp = 1; sub = r - 3; lr = a.lr[1]; }
    else if (r < 10) { grp = 2; sub = r - 6; lr = a.lr[2]; }
    else if (r == 10) { grp = 3; sub = 0; lr = a.lr[3]; }
    else { grp = 4; sub = r - 11; lr = (sub % a.K) == 0 ? a.lr[4] : a.lr[5]; }
}

// lr: the row's learning rate already divided by 1 - b1^t
__device__ __forceinline__ void adam1(float& p, float& g, float& m, float& v, float lr,
                                      const AdamArgs& a) {
    adam_update(p, m, v, g, a.b1, a.b2, a.omb1, a.omb2, lr, a.isb, a.eps);
    g = 0.0f;
}

// grid.y = row, grid.x x 4 threads' worth of float4 per row
__global__ void __launch_bounds__(kThreads) k_adam_vec4(AdamArgs a) {
    int grp, sub;
    float lr;
    row_of(a, blockIdx.y, grp, sub, lr);
    const int64_t off = (int64_t)sub * a.n;
    float4* __restrict__ P = reinterpret_cast<float4*>(a.p[grp] + off);
    float4* __restrict__ Gd = reinterpret_cast<float4*>(a.g[grp] + off);
    float4* __restrict__ M = reinterpret_cast<float4*>(a.m[grp] + off);
    float4* __restrict__ V = reinterpret_cast<float4*>(a.v[grp] + off);
    const int64_t n4 = a.n >> 2;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    // two float4 of each array in flight per thread per iteration
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < n4; k += 2 * stride) {
        const bool two = k + stride < n4;
        float4 p0 = P[k], g0 = Gd[k], m0 = M[k], v0 = V[k];
        float4 p1, g1, m1, v1;
        if (two) {
            p1 = P[k + stride];
            g1 = Gd[k + stride];
            m1 = M[k + stride];
            v1 = V[k + stride];
        }
        adam1(p0.x, g0.x, m0.x, v0.x, lr, a);
        adam1(p0.y, g0.y, m0.y, v0.y, lr, a);
        adam1(p0.z, g0.z, m0.z, v0.z, lr, a);
        adam1(p0.w, g0.w, m0.w, v0.w, lr, a);
        P[k] = p0;
        M[k] = m0;
        V[k] = v0;
        Gd[k] = g0;
        if (two) {
            adam1(p1.x, g1.x, m1.x, v1.x, lr, a);
            adam1(p1.y, g1.y, m1.y, v1.y, lr, a);
            adam1(p1.z, g1.z, m1.z, v1.z, lr, a);
            adam1(p1.w, g1.w, m1.w, v1.w, lr, a);
            P[k + stride] = p1;
            M[k + stride] = m1;
            V[k + stride] = v1;
            Gd[k + stride] = g1;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_adam_scalar(AdamArgs a) {
    int grp, sub;
    float lr;
    row_of(a, blockIdx.y, grp, sub, lr);
    const int64_t off = (int64_t)sub * a.n;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < a.n; k += (int64_t)gridDim.x * kThreads) {
        float p = a.p[grp][off + k], g = a.g[grp][off + k], m = a.m[grp][off + k], v = a.v[grp][off + k];
        adam1(p, g, m, v, lr, a);
        a.p[grp][off + k] = p;
        a.m[grp][off + k] = m;
        a.v[grp][off + k] = v;
        a.g[grp][off + k] = g;
    }
}

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

// Batched L1: one pass over every render's image values (renders' values are numbered
// consecutively); gradient sign / (3 H W) of the value's render; per-render sums of |d| and d^2
// (losses[2 r], losses[2 r + 1], zeroed by the caller).  Each CTA covers a contiguous chunk and
// walks the render segments inside it (usually one, two at a render boundary): per segment the
// threads' float partials are reduced across the CTA and added with one double atomic per sum,
// so a render receives about 3 H W / 4096 atomics.
constexpr int kLossChunk = kThreads * 16;

__device__ __forceinline__ double block_sum(double x, double* s_red) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();  // s_red is free again
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
    return t;
}

__global__ void __launch_bounds__(kThreads)
k_loss_batch(const RenderDesc* __restrict__ renders, int R, int64_t values, double* __restrict__ losses) {
    __shared__ double s_red[kThreads / 32];
    const int64_t begin = (int64_t)blockIdx.x * kLossChunk;
    const int64_t end = begin + kLossChunk < values ? begin + kLossChunk : values;
    int lo = 0, hi = R - 1;  // last render whose values start at or before `begin`
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (renders[mid].value_base <= begin) lo = mid;
        else hi = mid - 1;
    }
    for (int r = lo; r < R; ++r) {
        const RenderDesc& rd = renders[r];
        const int64_t vbase = rd.value_base;
        if (vbase >= end) break;
        const int64_t nv = 3ll * rd.cam.width * rd.cam.height;
        const int64_t a = begin > vbase ? begin - vbase : 0;
        const int64_t b = end - vbase < nv ? end - vbase : nv;
        if (a >= b) continue;
        const float* __restrict__ img = rd.image;
        const float* __restrict__ tgt = rd.target;
        float* __restrict__ grad = rd.dL;
        const float inv_n = 1.0f / (float)nv;
        float l1 = 0.f, l2 = 0.f;
        auto one = [&](float xv, float yv) {
            const float d = xv - yv;
            l1 += fabsf(d);
            l2 = fmaf(d, d, l2);
            return d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
        };
        // the 4-aligned middle of [a, b) with 16-byte accesses when the three planes are 16-byte
        // aligned, the ends one value at a time
        const bool aligned = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(tgt) |
                               reinterpret_cast<uintptr_t>(grad)) % 16) == 0;
        const int64_t q0 = aligned ? min((a + 3) & ~int64_t(3), b) : b;
        const int64_t q1 = aligned ? max(q0, b & ~int64_t(3)) : b;
        for (int64_t q = a + threadIdx.x; q < q0; q += kThreads) grad[q] = one(img[q], tgt[q]);
        for (int64_t q = q0 / 4 + threadIdx.x; q < q1 / 4; q += kThreads) {
            const float4 u = reinterpret_cast<const float4*>(img)[q], w = reinterpret_cast<const float4*>(tgt)[q];
            float4 g;
            g.x = one(u.x, w.x);
            g.y = one(u.y, w.y);
            g.z = one(u.z, w.z);
            g.w = one(u.w, w.w);
            reinterpret_cast<float4*>(grad)[q] = g;
        }
        for (int64_t q = q1 + threadIdx.x; q < b; q += kThreads) grad[q] = one(img[q], tgt[q]);
        const double t1 = block_sum((double)l1, s_red);
        const double t2 = block_sum((double)l2, s_red);
        if (threadIdx.x == 0) {
            atomicAdd(&losses[2 * r], t1);
            atomicAdd(&losses[2 * r + 1], t2);
        }
    }
}

}  // namespace

int launch_loss_l1(const float* image, const float* target, int64_t n, float* grad,
                    float* loss_out, const Scratch& sc, cudaStream_t s) {
    int blocks = (int)((n + kThreads * 8 - 1) / (kThreads * 8));
    blocks = blocks < 1 ? 1 : (blocks > kLossBlocks ? kLossBlocks : blocks);
    k_loss_l1<<<blocks, kThreads, 0, s>>>(image, target, n, grad, loss_out, sc.loss_partials,
                                          sc.loss_ticket);
    return 1;
}

int launch_adam(pgs_gaussians& p, pgs_gaussians& g, pgs_gaussians& m, pgs_gaussians& v,
                 const float lr[6], float b1, float b2, float eps, int64_t t, cudaStream_t s) {
    AdamArgs a;
    pgs_gaussians* src[4] = {&p, &g, &m, &v};
    float** dst[4] = {a.p, a.g, a.m, a.v};
    bool vec = (p.n % 4) == 0;
    for (int q = 0; q < 4; ++q) {
        float* ptrs[5] = {src[q]->means, src[q]->log_scales, src[q]->quats, src[q]->opacity_logits, src[q]->sh};
        for (int k = 0; k < 5; ++k) {
            dst[q][k] = ptrs[k];
            vec = vec && aligned16(ptrs[k]);
        }
    }
    const double bc1 = 1.0 - pow((double)b1, (double)t), bc2 = 1.0 - pow((double)b2, (double)t);
    for (int k = 0; k < 6; ++k) a.lr[k] = (float)((double)lr[k] / bc1);
    a.n = p.n;
    a.K = sh_coeffs(p.sh_degree);
    a.b1 = b1;
    a.b2 = b2;
    a.omb1 = (float)(1.0 - (double)b1);
    a.omb2 = (float)(1.0 - (double)b2);
    a.eps = eps;
    a.isb = (float)(1.0 / sqrt(bc2));
    const int rows = param_rows(p.sh_degree);
    const int64_t work = vec ? (p.n >> 2) : p.n;
    int64_t bx = (work + kThreads - 1) / kThreads;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    const dim3 grid((unsigned)bx, (unsigned)rows);
    if (vec) k_adam_vec4<<<grid, kThreads, 0, s>>>(a);
    else k_adam_scalar<<<grid, kThreads, 0, s>>>(a);
    return 1;
}

int launch_loss_batch(const RenderDesc* renders, int R, int64_t values, double* losses, cudaStream_t s) {
    const int64_t blocks = (values + kLossChunk - 1) / kLossChunk;
    if (blocks == 0) return 0;
    k_loss_batch<<<(unsigned)blocks, kThreads, 0, s>>>(renders, R, values, losses);
    return 1;
}

}  // namespace pgs
