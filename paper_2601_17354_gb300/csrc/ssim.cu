// L1 + D-SSIM loss of a rendered image against its target and the loss gradient (the paper
// reports SSIM, Sec. IV, and names no training loss; this is the 3DGS-style alternative to the
// plain L1 of K7).  Per colour plane, with G the 11 x 11 Gaussian window (sigma 1.5, taps
// normalised to sum 1) and zero padding:
//   mu_x = G*x, sigma_x^2 = G*x^2 - mu_x^2, sigma_xy = G*(xy) - mu_x mu_y,
//   SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),
//   loss = (1 - lam) mean|x - y| + lam (1 - mean SSIM).
// Two tiled kernels, 32 x 32 output pixels of one plane per CTA with the 5-pixel halo staged in
// shared memory and the window applied separably (rows, then columns):
//   forward  the five filtered moments, SSIM, and per pixel the SSIM's derivatives with respect
//            to the three filtered moments of x (m1 = G*x, m2 = G*x^2, m12 = G*xy), written as
//            three planes; L1 and SSIM sums per CTA added in double;
//   backward filters the three derivative planes with the same window and combines them,
//            d(sum SSIM)/dx = G*ds/dm1 + 2 x G*ds/dm2 + y G*ds/dm12, with the L1 sign term.
#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr int kR = 5;                 // window radius
constexpr int kTw = 32;               // output tile edge
constexpr int kIn = kTw + 2 * kR;     // staged edge with the halo
constexpr int kThreadsX = 32, kThreadsY = 8;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Taps {
    float w[2 * kR + 1];
};

// stage plane[y0 - R .. y0 + 32 + R) x [x0 - R .. x0 + 32 + R) with zeros outside the image
__device__ __forceinline__ void stage(float (*dst)[kIn], const float* __restrict__ plane, int W, int H,
                                      int x0, int y0) {
    for (int k = threadIdx.y * kThreadsX + threadIdx.x; k < kIn * kIn; k += kThreadsX * kThreadsY) {
        const int r = k / kIn, c = k % kIn;
        const int y = y0 - kR + r, x = x0 - kR + c;
        dst[r][c] = (x >= 0 && x < W && y >= 0 && y < H) ? plane[(size_t)y * W + x] : 0.0f;
    }
}

__global__ void __launch_bounds__(kThreadsX * kThreadsY)
k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt, int W, int H, Taps taps,
           float* __restrict__ dm, double* __restrict__ sums) {
    __shared__ float sx[kIn][kIn], sy[kIn][kIn];
    __shared__ float hm[5][kIn][kTw];  // row-filtered x, y, x^2, y^2, xy
    __shared__ double red[2][kThreadsX * kThreadsY / 32];
    const int x0 = blockIdx.x * kTw, y0 = blockIdx.y * kTw, c = blockIdx.z;
    const size_t plane = (size_t)W * H;
    const float* __restrict__ X = img + c * plane;
    const float* __restrict__ Y = tgt + c * plane;
    stage(sx, X, W, H, x0, y0);
    stage(sy, Y, W, H, x0, y0);
    __syncthreads();
    for (int r = threadIdx.y; r < kIn; r += kThreadsY) {
        const int col = threadIdx.x;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float u = sx[r][col + k], v = sy[r][col + k], w = taps.w[k];
            a = fmaf(w, u, a);
            b = fmaf(w, v, b);
            aa = fmaf(w, u * u, aa);
            bb = fmaf(w, v * v, bb);
            ab = fmaf(w, u * v, ab);
        }
        hm[0][r][col] = a;
        hm[1][r][col] = b;
        hm[2][r][col] = aa;
        hm[3][r][col] = bb;
        hm[4][r][col] = ab;
    }
    __syncthreads();
    float l1 = 0.f, ss = 0.f;  // a thread's at most 4 values; per CTA in double
    for (int r = threadIdx.y; r < kTw; r += kThreadsY) {
        const int col = threadIdx.x;
        const int x = x0 + col, y = y0 + r;
        if (x >= W || y >= H) continue;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float w = taps.w[k];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmaf(w, hm[q][r + k][col], m[q]);
        }
        const float mx = m[0], my = m[1];
        const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
        const float rb1 = __fdividef(1.0f, B1), rb2 = __fdividef(1.0f, B2);  // B1, B2 >= C1, C2 > 0
        const float inv = rb1 * rb2;
        const float s = A1 * A2 * inv;
        const float ds_dmu = 2.f * my * A2 * inv - s * 2.f * mx * rb1;  // sigmas held fixed
        const float ds_dsxx = -s * rb2;
        const float ds_dsxy = 2.f * A1 * inv;
        const size_t p = c * plane + (size_t)y * W + x;
        dm[p] = ds_dmu - 2.f * mx * ds_dsxx - my * ds_dsxy;  // d s / d m1
        dm[3 * plane + p] = ds_dsxx;                        // d s / d m2
        dm[6 * plane + p] = ds_dsxy;                        // d s / d m12
        ss += s;
        l1 += fabsf(sx[r + kR][col + kR] - sy[r + kR][col + kR]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    const int lin = threadIdx.y * kThreadsX + threadIdx.x;
    if ((lin & 31) == 0) {
        red[0][lin >> 5] = (double)l1;
        red[1][lin >> 5] = (double)ss;
    }
    __syncthreads();
    if (lin == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kThreadsX * kThreadsY / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        atomicAdd(&sums[0], a);
        atomicAdd(&sums[1], b);
    }
}

__global__ void __launch_bounds__(kThreadsX * kThreadsY)
k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ tgt, int W, int H, Taps taps, float lam,
           const float* __restrict__ dm, const double* __restrict__ sums, float* __restrict__ grad,
           float* __restrict__ loss_out) {
    __shared__ float sd[3][kIn][kIn];
    __shared__ float hd[3][kIn][kTw];
    const int x0 = blockIdx.x * kTw, y0 = blockIdx.y * kTw, c = blockIdx.z;
    const size_t plane = (size_t)W * H;
    const double n = 3.0 * (double)plane;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        // the forward launch has finished: its sums are complete
        const double l1 = sums[0] / n, ssim = sums[1] / n;
        loss_out[0] = (float)((1.0 - lam) * l1 + lam * (1.0 - ssim));
        loss_out[1] = (float)ssim;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) stage(sd[q], dm + (size_t)q * 3 * plane + c * plane, W, H, x0, y0);
    __syncthreads();
    for (int r = threadIdx.y; r < kIn; r += kThreadsY) {
        const int col = threadIdx.x;
        float h[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float w = taps.w[k];
#pragma unroll
            for (int q = 0; q < 3; ++q) h[q] = fmaf(w, sd[q][r][col + k], h[q]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) hd[q][r][col] = h[q];
    }
    __syncthreads();
    const float inv_n = (float)(1.0 / n);
    for (int r = threadIdx.y; r < kTw; r += kThreadsY) {
        const int col = threadIdx.x;
        const int x = x0 + col, y = y0 + r;
        if (x >= W || y >= H) continue;
        float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float w = taps.w[k];
#pragma unroll
            for (int q = 0; q < 3; ++q) g[q] = fmaf(w, hd[q][r + k][col], g[q]);
        }
        const size_t p = c * plane + (size_t)y * W + x;
        const float xv = img[p], yv = tgt[p];
        const float d_ssim = g[0] + 2.f * xv * g[1] + yv * g[2];
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        grad[p] = ((1.f - lam) * sgn - lam * d_ssim) * inv_n;
    }
}

}  // namespace

int launch_loss_dssim(const float* image, const float* target, int W, int H, float lam, float* dm,
                      double* sums, float* grad, float* loss_out, cudaStream_t s) {
    Taps taps;
    double t[2 * kR + 1], tot = 0.0;
    for (int k = -kR; k <= kR; ++k) tot += t[k + kR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
    for (int k = 0; k <= 2 * kR; ++k) taps.w[k] = (float)(t[k] / tot);
    const dim3 grid((unsigned)((W + kTw - 1) / kTw), (unsigned)((H + kTw - 1) / kTw), 3);
    const dim3 block(kThreadsX, kThreadsY);
    cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    k_ssim_fwd<<<grid, block, 0, s>>>(image, target, W, H, taps, dm, sums);
    k_ssim_bwd<<<grid, block, 0, s>>>(image, target, W, H, taps, lam, dm, sums, grad, loss_out);
    return 2;
}

}  // namespace pgs
