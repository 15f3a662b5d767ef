// K15: the learned initializer's MLP 16-64-64-8 (GELU), BF16 weights and activations, FP32
// accumulation on the tensor cores (mma.sync m16n8k16, bf16 x bf16 -> f32), operands staged in
// shared memory and loaded with ldmatrix (transposed where a product needs the transpose).
//
// At K = 16 / 64 and N = 8 / 64 each layer is a handful of 16x8x16 products per 16 points; the
// kernels keep every activation of a 64-point slice in shared memory, so a training step reads
// the features and targets once and writes only the loss and the weight gradients.
//
// Training kernel, per CTA slice of 64 points (4 warps x 16):
//   forward  Z1 = X W1^T + b1, H1 = gelu(Z1), Z2 = H1 W2^T + b2, H2 = gelu(Z2), Y = H2 W3^T + b3
//   loss     |Y0..2 - t|^2 + (1 - <Y3..6/|Y3..6|, t_q>^2) + (Y7 - t)^2, mean over points
//   backward dH2 = dY W3, dZ2 = dH2 gelu'(Z2), dH1 = dZ2 W2, dZ1 = dH1 gelu'(Z1)
//   weights  dW3 = dY^T H2, dW2 = dZ2^T H1, dW1 = dZ1^T X (split across the warps, accumulated in
//            registers over the CTA's slices, added to the FP32 gradient once per CTA); bias
//            gradients are FP32 sums of the unrounded dY, dZ2, dZ1.
// BF16 rounding points: X, weights, H1, H2 and the gradients fed to products (dY, dZ2, dZ1).
#include <cuda_bf16.h>

#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int kIn = 16, kHid = 64, kOut = 8;
constexpr int kWarps = 4, kRows = 16 * kWarps;  // points per CTA slice
constexpr int LD16 = kIn + 8, LD64 = kHid + 8;  // padded bf16 row strides (16-byte multiples)
constexpr int kParams = kHid * kIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;  // 5768

// offsets of the flat FP32 parameter vector [W1 | b1 | W2 | b2 | W3 | b3]
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid,
              oW3 = ob2 + kHid, ob3 = oW3 + kOut * kHid;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t r[2], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t r[2], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (16 x 16) of a row-major bf16 matrix at (r0, c0)
__device__ __forceinline__ void frag_a(uint32_t a[4], const __nv_bfloat16* S, int ld, int r0, int c0) {
    const int l = threadIdx.x & 31, i = l >> 3;
    ldsm_x4(a, S + (size_t)(r0 + (i & 1) * 8 + (l & 7)) * ld + c0 + (i >> 1) * 8);
}
// A fragment of the transpose: A[m][k] = S[k][m], block rows (data) k0.., cols m0..
__device__ __forceinline__ void frag_a_t(uint32_t a[4], const __nv_bfloat16* S, int ld, int k0, int m0) {
    const int l = threadIdx.x & 31, i = l >> 3;
    ldsm_x4_t(a, S + (size_t)(k0 + (i >> 1) * 8 + (l & 7)) * ld + m0 + (i & 1) * 8);
}
// B fragment (16 x 8) with B[k][n] = W[n][k], W row-major [n][k]
__device__ __forceinline__ void frag_b(uint32_t b[2], const __nv_bfloat16* W, int ld, int n0, int k0) {
    const int l = threadIdx.x & 31;
    ldsm_x2(b, W + (size_t)(n0 + (l & 7)) * ld + k0 + ((l >> 3) & 1) * 8);
}
// B fragment with B[k][n] = S[k][n], S row-major [k][n]
__device__ __forceinline__ void frag_b_t(uint32_t b[2], const __nv_bfloat16* S, int ld, int k0, int n0) {
    const int l = threadIdx.x & 31;
    ldsm_x2_t(b, S + (size_t)(k0 + ((l >> 3) & 1) * 8 + (l & 7)) * ld + n0);
}

// 1 + erf(x) by the rational approximation 7.1.26 of Abramowitz & Stegun (Handbook of
// Mathematical Functions, 1964): for x >= 0, erf(x) = 1 - (a1 s + a2 s^2 + ... + a5 s^5) e^{-x^2}
// with s = 1 / (1 + p x) and |error| <= 1.5e-7, far below the BF16 rounding of the activations.
// Evaluated as q = polynomial * e^{-x^2}, 1 + erf(x) = 2 - q for x >= 0 and q for x < 0 (the
// odd symmetry), so the left tail keeps its relative accuracy instead of cancelling.
__device__ __forceinline__ float one_plus_erf(float x) {
    const float ax = fabsf(x);
    const float s = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    float poly = fmaf(1.061405429f, s, -1.453152027f);
    poly = fmaf(poly, s, 1.421413741f);
    poly = fmaf(poly, s, -0.284496736f);
    poly = fmaf(poly, s, 0.254829592f);
    const float q = poly * s * __expf(-ax * ax);
    return x >= 0.0f ? 2.0f - q : q;
}
// GELU in the erf form, z Phi(z), and its derivative Phi(z) + z phi(z)
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * one_plus_erf(z * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * one_plus_erf(z * 0.70710678118654752f) + z * __expf(-0.5f * z * z) * 0.3989422804014327f;
}

struct Smem {
    __nv_bfloat16 W1[kHid * LD16], W2[kHid * LD64], W3[16 * LD64];  // W3 rows 8..15 zero
    __nv_bfloat16 X[kRows * LD16], H1[kRows * LD64], H2[kRows * LD64];
    __nv_bfloat16 dY[kRows * LD16], dZ2[kRows * LD64], dZ1[kRows * LD64];
    float Z1[kRows * kHid], Z2[kRows * kHid];
    float Y[kRows * kOut];
    float b1[kHid], b2[kHid], b3[kOut];
};

__device__ void load_weights(Smem& S, const __nv_bfloat16* __restrict__ W1, const __nv_bfloat16* __restrict__ W2,
                             const __nv_bfloat16* __restrict__ W3, const float* __restrict__ b1,
                             const float* __restrict__ b2, const float* __restrict__ b3) {
    for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x) S.W1[(k / kIn) * LD16 + k % kIn] = W1[k];
    for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) S.W2[(k / kHid) * LD64 + k % kHid] = W2[k];
    for (int k = threadIdx.x; k < 16 * kHid; k += blockDim.x)
        S.W3[(k / kHid) * LD64 + k % kHid] = k < kOut * kHid ? W3[k] : __float2bfloat16_rn(0.f);
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        S.b1[k] = b1[k];
        S.b2[k] = b2[k];
    }
    if (threadIdx.x < kOut) S.b3[threadIdx.x] = b3[threadIdx.x];
    for (int k = threadIdx.x; k < kRows * LD16; k += blockDim.x) S.dY[k] = __float2bfloat16_rn(0.f);
}

// Forward of one warp's 16 points (rows r0..r0+15 of the slice): fills X, Z1, H1, Z2, H2, Y.
__device__ void warp_forward(Smem& S, const __nv_bfloat16* __restrict__ x, int64_t n, int64_t p0, int r0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    {   // X rows: 16 rows x 32 bytes, one 16-byte half row per lane
        const int row = lane >> 1, half = lane & 1;
        const int64_t p = p0 + row;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (p < n) v = *reinterpret_cast<const uint4*>(x + p * kIn + half * 8);
        *reinterpret_cast<uint4*>(S.X + (size_t)(r0 + row) * LD16 + half * 8) = v;
    }
    __syncwarp();
    uint32_t a[4];
    frag_a(a, S.X, LD16, r0, 0);
#pragma unroll
    for (int j = 0; j < kHid / 8; ++j) {
        uint32_t b[2];
        frag_b(b, S.W1, LD16, 8 * j, 0);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma(c, a, b);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = r0 + g + (e >> 1) * 8, col = 8 * j + 2 * t + (e & 1);
            const float z = c[e] + S.b1[col];
            S.Z1[row * kHid + col] = z;
            S.H1[row * LD64 + col] = __float2bfloat16_rn(gelu(z));
        }
    }
    __syncwarp();
    uint32_t a4[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) frag_a(a4[kk], S.H1, LD64, r0, 16 * kk);
#pragma unroll
    for (int j = 0; j < kHid / 8; ++j) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t b[2];
            frag_b(b, S.W2, LD64, 8 * j, 16 * kk);
            mma(c, a4[kk], b);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = r0 + g + (e >> 1) * 8, col = 8 * j + 2 * t + (e & 1);
            const float z = c[e] + S.b2[col];
            S.Z2[row * kHid + col] = z;
            S.H2[row * LD64 + col] = __float2bfloat16_rn(gelu(z));
        }
    }
    __syncwarp();
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) frag_a(a4[kk], S.H2, LD64, r0, 16 * kk);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t b[2];
        frag_b(b, S.W3, LD64, 0, 16 * kk);
        mma(c, a4[kk], b);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int row = r0 + g + (e >> 1) * 8, col = 2 * t + (e & 1);
        S.Y[row * kOut + col] = c[e] + S.b3[col];
    }
    __syncwarp();
}

// Inference: activations never leave registers.  The f32 accumulator fragment of a 16 x 8
// product tile (rows g, g + 8; columns 2t, 2t + 1 of lane (g, t)) is, after bias and GELU and
// packing column pairs to bf16x2, exactly the A fragment of the next layer's 16 x 16 k-tile (the
// k-tile of columns 16 kk.. is made of n-tiles 2 kk and 2 kk + 1), so each warp carries its 16
// points through the three layers with no shared-memory round trip; only the weights are staged.
struct WeightSmem {
    __nv_bfloat16 W1[kHid * LD16], W2[kHid * LD64], W3[16 * LD64];  // W3 rows 8..15 zero
    float b1[kHid], b2[kHid], b3[kOut];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// bias + GELU of the eight 16 x 8 accumulator tiles C[j] of a 64-wide layer, packed into the
// four A fragments of the next layer
__device__ __forceinline__ void activate(const float C[8][4], const float* __restrict__ bias, int t,
                                         uint32_t A[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        A[kk][0] = pack_bf16(gelu(C[2 * kk][0] + bias[c0]), gelu(C[2 * kk][1] + bias[c0 + 1]));
        A[kk][1] = pack_bf16(gelu(C[2 * kk][2] + bias[c0]), gelu(C[2 * kk][3] + bias[c0 + 1]));
        A[kk][2] = pack_bf16(gelu(C[2 * kk + 1][0] + bias[c1]), gelu(C[2 * kk + 1][1] + bias[c1 + 1]));
        A[kk][3] = pack_bf16(gelu(C[2 * kk + 1][2] + bias[c1]), gelu(C[2 * kk + 1][3] + bias[c1 + 1]));
    }
}

constexpr int kInferWarps = 4;

__global__ void __launch_bounds__(32 * kInferWarps)
k_mlp_forward(const __nv_bfloat16* __restrict__ x, int64_t n, const __nv_bfloat16* __restrict__ W1,
              const __nv_bfloat16* __restrict__ W2, const __nv_bfloat16* __restrict__ W3,
              const float* __restrict__ b1, const float* __restrict__ b2, const float* __restrict__ b3,
              float* __restrict__ out) {
    __shared__ __align__(16) WeightSmem S;
    for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x) S.W1[(k / kIn) * LD16 + k % kIn] = W1[k];
    for (int k = threadIdx.x; k < kHid * kHid; k += blockDim.x) S.W2[(k / kHid) * LD64 + k % kHid] = W2[k];
    for (int k = threadIdx.x; k < 16 * kHid; k += blockDim.x)
        S.W3[(k / kHid) * LD64 + k % kHid] = k < kOut * kHid ? W3[k] : __float2bfloat16_rn(0.f);
    for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
        S.b1[k] = b1[k];
        S.b2[k] = b2[k];
    }
    if (threadIdx.x < kOut) S.b3[threadIdx.x] = b3[threadIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t* __restrict__ xw = reinterpret_cast<const uint32_t*>(x);  // 8 words per point
    const int64_t slices = (n + 15) / 16;
    for (int64_t sl = (int64_t)blockIdx.x * kInferWarps + warp; sl < slices;
         sl += (int64_t)gridDim.x * kInferWarps) {
        const int64_t p0 = sl * 16, pa = p0 + g, pb = p0 + g + 8;
        uint32_t a[4];
        a[0] = pa < n ? xw[pa * 8 + t] : 0u;
        a[1] = pb < n ? xw[pb * 8 + t] : 0u;
        a[2] = pa < n ? xw[pa * 8 + t + 4] : 0u;
        a[3] = pb < n ? xw[pb * 8 + t + 4] : 0u;
        float C[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t b[2];
            frag_b(b, S.W1, LD16, 8 * j, 0);
            C[j][0] = C[j][1] = C[j][2] = C[j][3] = 0.f;
            mma(C[j], a, b);
        }
        uint32_t A[4][4];
        activate(C, S.b1, t, A);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            C[j][0] = C[j][1] = C[j][2] = C[j][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                uint32_t b[2];
                frag_b(b, S.W2, LD64, 8 * j, 16 * kk);
                mma(C[j], A[kk], b);
            }
        }
        activate(C, S.b2, t, A);
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t b[2];
            frag_b(b, S.W3, LD64, 0, 16 * kk);
            mma(y, A[kk], b);
        }
        const int c = 2 * t;
        if (pa < n) *reinterpret_cast<float2*>(out + pa * kOut + c) = make_float2(y[0] + S.b3[c], y[1] + S.b3[c + 1]);
        if (pb < n) *reinterpret_cast<float2*>(out + pb * kOut + c) = make_float2(y[2] + S.b3[c], y[3] + S.b3[c + 1]);
    }
}

__global__ void __launch_bounds__(32 * kWarps)
k_mlp_train(const __nv_bfloat16* __restrict__ x, const float* __restrict__ target, int64_t n,
            const __nv_bfloat16* __restrict__ W1, const __nv_bfloat16* __restrict__ W2,
            const __nv_bfloat16* __restrict__ W3, const float* __restrict__ b1, const float* __restrict__ b2,
            const float* __restrict__ b3, float* __restrict__ grad, double* __restrict__ loss_sum) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    Smem& S = *reinterpret_cast<Smem*>(s_raw);
    load_weights(S, W1, W2, W3, b1, b2, b3);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = 16 * warp;
    const float inv_n = 1.0f / (float)n;
    float accW2[8][4], accW1[2][4], accW3[2][4];
    float db1[16], db2[16], db3[kOut];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) accW2[j][e] = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) accW1[j][e] = accW3[j][e] = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) db1[k] = db2[k] = 0.f;
#pragma unroll
    for (int k = 0; k < kOut; ++k) db3[k] = 0.f;
    double lsum = 0.0;

    for (int64_t p0 = (int64_t)blockIdx.x * kRows; p0 < n; p0 += (int64_t)gridDim.x * kRows) {
        warp_forward(S, x, n, p0 + r0, r0);
        // loss head: lane = point of the warp
        if (lane < 16) {
            const int row = r0 + lane;
            const int64_t p = p0 + row;
            float dy[kOut] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (p < n) {
                const float* y = S.Y + row * kOut;
                const float* tg = target + p * kOut;
                float L = 0.f;
                for (int k = 0; k < 3; ++k) {
                    const float d = y[k] - tg[k];
                    L += d * d;
                    dy[k] = 2.f * d * inv_n;
                }
                const float qn = sqrtf(y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
                const float iq = qn > 0.f ? 1.0f / qn : 0.f;
                float f = 0.f;
                for (int k = 0; k < 4; ++k) f += y[3 + k] * iq * tg[3 + k];
                L += 1.f - f * f;
                float dq[4], dot = 0.f;
                for (int k = 0; k < 4; ++k) {
                    dq[k] = -2.f * f * tg[3 + k];
                    dot += dq[k] * y[3 + k] * iq;
                }
                for (int k = 0; k < 4; ++k) dy[3 + k] = (dq[k] - y[3 + k] * iq * dot) * iq * inv_n;
                const float d = y[7] - tg[7];
                L += d * d;
                dy[7] = 2.f * d * inv_n;
                lsum += (double)L;
            }
            for (int k = 0; k < kOut; ++k) {
                db3[k] += dy[k];
                S.dY[row * LD16 + k] = __float2bfloat16_rn(dy[k]);
            }
        }
        __syncwarp();
        // dZ2 = (dY W3) gelu'(Z2)
        uint32_t a[4];
        frag_a(a, S.dY, LD16, r0, 0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t b[2];
            frag_b_t(b, S.W3, LD64, 0, 8 * j);
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma(c, a, b);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = r0 + g + (e >> 1) * 8, col = 8 * j + 2 * t + (e & 1);
                const float dz = c[e] * gelu_d(S.Z2[row * kHid + col]);
                db2[2 * j + (e & 1)] += dz;
                S.dZ2[row * LD64 + col] = __float2bfloat16_rn(dz);
            }
        }
        __syncwarp();
        // dZ1 = (dZ2 W2) gelu'(Z1)
        uint32_t a4[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) frag_a(a4[kk], S.dZ2, LD64, r0, 16 * kk);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                uint32_t b[2];
                frag_b_t(b, S.W2, LD64, 16 * kk, 8 * j);
                mma(c, a4[kk], b);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = r0 + g + (e >> 1) * 8, col = 8 * j + 2 * t + (e & 1);
                const float dz = c[e] * gelu_d(S.Z1[row * kHid + col]);
                db1[2 * j + (e & 1)] += dz;
                S.dZ1[row * LD64 + col] = __float2bfloat16_rn(dz);
            }
        }
        __syncthreads();
        // weight gradients over the slice's 64 points (K = data rows)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t at[4];
            frag_a_t(at, S.dZ2, LD64, 16 * kk, 16 * warp);  // rows of dW2 owned by this warp
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                uint32_t b[2];
                frag_b_t(b, S.H1, LD64, 16 * kk, 8 * j);
                mma(accW2[j], at, b);
            }
            frag_a_t(at, S.dZ1, LD64, 16 * kk, 16 * warp);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t b[2];
                frag_b_t(b, S.X, LD16, 16 * kk, 8 * j);
                mma(accW1[j], at, b);
            }
            frag_a_t(at, S.dY, LD16, 16 * kk, 0);  // dY^T padded to 16 rows
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t b[2];
                frag_b_t(b, S.H2, LD64, 16 * kk, 8 * (2 * warp + j));
                mma(accW3[j], at, b);
            }
        }
        __syncthreads();
    }
    // flush: weight gradients (C fragment rows g / g + 8, cols 2t, 2t + 1)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = 16 * warp + g + (e >> 1) * 8, col = 8 * j + 2 * t + (e & 1);
            atomicAdd(&grad[oW2 + m * kHid + col], accW2[j][e]);
        }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = 16 * warp + g + (e >> 1) * 8, col = 8 * j + 2 * t + (e & 1);
            atomicAdd(&grad[oW1 + m * kIn + col], accW1[j][e]);
            if (e < 2) {  // dW3 has 8 rows: the fragment's upper half
                const int col3 = 8 * (2 * warp + j) + 2 * t + (e & 1);
                atomicAdd(&grad[oW3 + g * kHid + col3], accW3[j][e]);
            }
        }
    // bias gradients: reduce over the lanes sharing t (rows), then over lanes (db3)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        for (int o = 4; o < 32; o <<= 1) {
            db1[k] += __shfl_xor_sync(0xffffffffu, db1[k], o);
            db2[k] += __shfl_xor_sync(0xffffffffu, db2[k], o);
        }
    }
    if (g == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                atomicAdd(&grad[ob1 + 8 * j + 2 * t + q], db1[2 * j + q]);
                atomicAdd(&grad[ob2 + 8 * j + 2 * t + q], db2[2 * j + q]);
            }
    }
#pragma unroll
    for (int k = 0; k < kOut; ++k)
        for (int o = 1; o < 32; o <<= 1) db3[k] += __shfl_xor_sync(0xffffffffu, db3[k], o);
    if (lane == 0)
        for (int k = 0; k < kOut; ++k) atomicAdd(&grad[ob3 + k], db3[k]);
    for (int o = 1; o < 32; o <<= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(loss_sum, lsum);
}

// Adam on the FP32 master parameters; refreshes the BF16 weight copies and zeroes the gradient.
__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1,
                           float bc2, __nv_bfloat16* __restrict__ W1, __nv_bfloat16* __restrict__ W2,
                           __nv_bfloat16* __restrict__ W3) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kParams; k += gridDim.x * blockDim.x) {
        const float gk = grad[k];
        const float mm = b1 * m[k] + (1.f - b1) * gk;
        const float vv = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mm;
        v[k] = vv;
        const float p = master[k] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
        master[k] = p;
        grad[k] = 0.f;
        if (k < ob1) W1[k - oW1] = __float2bfloat16_rn(p);
        else if (k >= oW2 && k < ob2) W2[k - oW2] = __float2bfloat16_rn(p);
        else if (k >= oW3 && k < ob3) W3[k - oW3] = __float2bfloat16_rn(p);
    }
}

__global__ void k_mlp_pack(const float* __restrict__ master, __nv_bfloat16* __restrict__ W1,
                           __nv_bfloat16* __restrict__ W2, __nv_bfloat16* __restrict__ W3) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kParams; k += gridDim.x * blockDim.x) {
        const float p = master[k];
        if (k < ob1) W1[k - oW1] = __float2bfloat16_rn(p);
        else if (k >= oW2 && k < ob2) W2[k - oW2] = __float2bfloat16_rn(p);
        else if (k >= oW3 && k < ob3) W3[k - oW3] = __float2bfloat16_rn(p);
    }
}

int grid_for(int64_t n) {
    static int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v;
    }();
    const int64_t slices = (n + kRows - 1) / kRows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(slices, (int64_t)sms * 2));
}

void enable_smem() {
    static bool done = [] {
        cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
        return true;
    }();
    (void)done;
}

}  // namespace

int mlp_param_count() { return kParams; }

int launch_mlp_forward(const void* x, int64_t n, const float* master, const void* W1, const void* W2,
                       const void* W3, float* out, cudaStream_t s) {
    if (n <= 0) return 0;
    enable_smem();
    static int grid = [] {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_forward, 32 * kInferWarps, 0);
        return sms * (per_sm > 0 ? per_sm : 1);
    }();
    const int64_t slices = (n + 15) / 16;
    const int64_t blocks = std::min<int64_t>(grid, (slices + kInferWarps - 1) / kInferWarps);
    k_mlp_forward<<<(unsigned)blocks, 32 * kInferWarps, 0, s>>>(
        static_cast<const __nv_bfloat16*>(x), n, static_cast<const __nv_bfloat16*>(W1),
        static_cast<const __nv_bfloat16*>(W2), static_cast<const __nv_bfloat16*>(W3), master + ob1,
        master + ob2, master + ob3, out);
    return 1;
}

int launch_mlp_train(const void* x, const float* target, int64_t n, const float* master, const void* W1,
                     const void* W2, const void* W3, float* grad, double* loss_sum, cudaStream_t s) {
    if (n <= 0) return 0;
    enable_smem();
    k_mlp_train<<<grid_for(n), 32 * kWarps, sizeof(Smem), s>>>(
        static_cast<const __nv_bfloat16*>(x), target, n, static_cast<const __nv_bfloat16*>(W1),
        static_cast<const __nv_bfloat16*>(W2), static_cast<const __nv_bfloat16*>(W3), master + ob1,
        master + ob2, master + ob3, grad, loss_sum);
    return 1;
}

int launch_mlp_adam(float* master, float* grad, float* m, float* v, float lr, float b1, float b2,
                    float eps, int64_t t, void* W1, void* W2, void* W3, cudaStream_t s) {
    const float bc1 = (float)(1.0 - pow((double)b1, (double)t));
    const float bc2 = (float)(1.0 - pow((double)b2, (double)t));
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, s>>>(master, grad, m, v, lr, b1, b2, eps, bc1, bc2,
                                                      static_cast<__nv_bfloat16*>(W1),
                                                      static_cast<__nv_bfloat16*>(W2),
                                                      static_cast<__nv_bfloat16*>(W3));
    return 1;
}

int launch_mlp_pack(const float* master, void* W1, void* W2, void* W3, cudaStream_t s) {
    k_mlp_pack<<<(kParams + 255) / 256, 256, 0, s>>>(master, static_cast<__nv_bfloat16*>(W1),
                                                      static_cast<__nv_bfloat16*>(W2),
                                                      static_cast<__nv_bfloat16*>(W3));
    return 1;
}

}  // namespace pgs
