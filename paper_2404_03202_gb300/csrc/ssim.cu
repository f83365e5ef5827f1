// Photometric loss with its D-SSIM term (Eq. 17): L = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)).
//
// SSIM per colour plane with an 11 x 11 Gaussian window (sigma 1.5, normalised), "same"-size filtering with zero
// padding, C1 = 0.01^2, C2 = 0.03^2 (the 3DGS conventions the paper defers to). The window is separable, so each
// filtered moment is a horizontal then a vertical 11-tap pass over a shared-memory tile with a 5-pixel halo. Both
// passes are register-blocked: a thread filters 4 adjacent outputs from one run of 14 inputs (read as 16-byte
// vectors in the horizontal pass), so each output costs a few shared-memory loads instead of 11 per moment.
//
// Precision: the moments are formed of the shifted images x' = x - 1/2 and y' = y - 1/2 (padding -1/2, which is what
// zero padding of x means after the shift). Variances and the covariance are shift-invariant, and mid-grey images
// keep x' small, so E[x'^2] - mu'^2 cancels far less than E[x^2] - mu^2 would in FP32.
//
// Forward (dssim_fwd_kernel): per output pixel, the five moments, SSIM, the three sensitivities
//   M1 = dS/dmu_x' = S (2 mu_y / A1 - 2 mu_x / B1 - 2 mu_y' / A2 + 2 mu_x' / B2),
//   M2 = dS/dE[x'^2] = -S / B2,    M3 = dS/dE[x'y'] = 2 S / A2,
// (A1 = 2 mu_x mu_y + C1, A2 = 2 sigma_xy + C2, B1 = mu_x^2 + mu_y^2 + C1, B2 = sigma_x^2 + sigma_y^2 + C2) written to
// the scratch, and per-CTA sums of SSIM and |x - y|.
// Adjoint (dssim_bwd_kernel): each moment is a symmetric zero-padded filter, so its adjoint is the same filter:
//   d mean(S) / dx = (G * M1 + 2 x' (G * M2) + y' (G * M3)) / N.
#include <cmath>

#include "common.cuh"

namespace omnigs {
namespace {

constexpr int kSsimR = 5;                    // window radius (11 taps)
constexpr int kSsimTW = 32, kSsimTH = 32;    // output tile
constexpr int kSsimInW = kSsimTW + 2 * kSsimR, kSsimInH = kSsimTH + 2 * kSsimR;
constexpr int kSsimStride = 44;              // staged row stride (16-byte aligned rows, >= kSsimInW + 2)
constexpr int kSsimRun = 4;                  // adjacent outputs per thread and pass
constexpr int kSsimSpan = kSsimRun + 2 * kSsimR;  // inputs one run reads (14)
constexpr int kSsimThreads = 256;
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;
constexpr float kShift = 0.5f;

// The 11 taps travel as a kernel argument (kernel parameters sit in the constant bank).
struct SsimTaps {
    float g[2 * kSsimR + 1];
};

SsimTaps gaussian_taps() {
    SsimTaps t;
    double s = 0.0, w[2 * kSsimR + 1];
    for (int i = 0; i <= 2 * kSsimR; ++i) {
        const double r = i - kSsimR;
        w[i] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
        s += w[i];
    }
    for (int i = 0; i <= 2 * kSsimR; ++i) t.g[i] = (float)(w[i] / s);
    return t;
}

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kSsimThreads / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Horizontal pass over one staged plane: 16 inputs from row r starting at column c0 (a multiple of 4), as four
// 16-byte loads.
__device__ __forceinline__ void load_run16(const float* row, int c0, float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 f = *reinterpret_cast<const float4*>(row + c0 + 4 * q);
        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
}

// Grid: (ceil(W / 32), ceil(H / 32), V * 3). partials: [2][blocks] (SSIM sum, |x - y| sum).
__global__ void __launch_bounds__(kSsimThreads)
dssim_fwd_kernel(int W, int H, SsimTaps taps, const float* __restrict__ x, const float* __restrict__ y,
                 float* __restrict__ m1, float* __restrict__ m2, float* __restrict__ m3, float* __restrict__ partials) {
    __shared__ __align__(16) float sx[kSsimInH][kSsimStride], sy[kSsimInH][kSsimStride];
    __shared__ float hm[5][kSsimInH][kSsimTW];  // horizontal moments: x', y', x'^2, y'^2, x'y'
    __shared__ float red[kSsimThreads / 32];
    const size_t plane = (size_t)blockIdx.z * H * W;
    const int ox = blockIdx.x * kSsimTW, oy = blockIdx.y * kSsimTH;
    for (int i = threadIdx.x; i < kSsimInH * kSsimStride; i += kSsimThreads) {
        const int r = i / kSsimStride, c = i - r * kSsimStride;
        const int gy = oy + r - kSsimR, gx = ox + c - kSsimR;
        const bool in = c < kSsimInW && gx >= 0 && gx < W && gy >= 0 && gy < H;
        sx[r][c] = (in ? __ldg(x + plane + (size_t)gy * W + gx) : 0.f) - kShift;
        sy[r][c] = (in ? __ldg(y + plane + (size_t)gy * W + gx) : 0.f) - kShift;
    }
    __syncthreads();
    // horizontal: run (r, 4 s .. 4 s + 3) of the 32 output columns, for every staged row
    for (int i = threadIdx.x; i < kSsimInH * (kSsimTW / kSsimRun); i += kSsimThreads) {
        const int r = i / (kSsimTW / kSsimRun), c0 = (i - r * (kSsimTW / kSsimRun)) * kSsimRun;
        float a[16], b[16];
        load_run16(sx[r], c0, a);
        load_run16(sy[r], c0, b);
#pragma unroll
        for (int o = 0; o < kSsimRun; ++o) {
            float ax = 0.f, ay = 0.f, axx = 0.f, ayy = 0.f, axy = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * kSsimR; ++t) {
                const float g = taps.g[t], u = a[o + t], w = b[o + t];
                const float gu = g * u, gw = g * w;
                ax += gu;
                ay += gw;
                axx = fmaf(gu, u, axx);
                ayy = fmaf(gw, w, ayy);
                axy = fmaf(gu, w, axy);
            }
            hm[0][r][c0 + o] = ax; hm[1][r][c0 + o] = ay; hm[2][r][c0 + o] = axx; hm[3][r][c0 + o] = ayy;
            hm[4][r][c0 + o] = axy;
        }
    }
    __syncthreads();
    // vertical: rows 4 q .. 4 q + 3 of output column c
    float s_sum = 0.f, l1_sum = 0.f;
    for (int i = threadIdx.x; i < kSsimTW * (kSsimTH / kSsimRun); i += kSsimThreads) {
        const int c = i % kSsimTW, r0 = (i / kSsimTW) * kSsimRun;
        float mom[5][kSsimRun];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float v[kSsimSpan];
#pragma unroll
            for (int t = 0; t < kSsimSpan; ++t) v[t] = hm[k][r0 + t][c];
#pragma unroll
            for (int o = 0; o < kSsimRun; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t <= 2 * kSsimR; ++t) acc = fmaf(taps.g[t], v[o + t], acc);
                mom[k][o] = acc;
            }
        }
        const int gx = ox + c;
#pragma unroll
        for (int o = 0; o < kSsimRun; ++o) {
            const int gy = oy + r0 + o;
            if (gx >= W || gy >= H) continue;
            const float mx = mom[0][o], my = mom[1][o];
            const float vx = fmaf(-mx, mx, mom[2][o]), vy = fmaf(-my, my, mom[3][o]), cxy = fmaf(-mx, my, mom[4][o]);
            const float Mx = mx + kShift, My = my + kShift;  // the means of the unshifted images
            const float a1 = fmaf(2.f * Mx, My, kSsimC1), a2 = fmaf(2.f, cxy, kSsimC2);
            const float b1 = fmaf(Mx, Mx, fmaf(My, My, kSsimC1)), b2 = vx + vy + kSsimC2;
            const float S = (a1 * a2) / (b1 * b2);
            const size_t pix = plane + (size_t)gy * W + gx;
            m1[pix] = S * (2.f * My / a1 - 2.f * Mx / b1 - 2.f * my / a2 + 2.f * mx / b2);
            m2[pix] = -S / b2;
            m3[pix] = 2.f * S / a2;
            s_sum += S;
            l1_sum += fabsf(sx[r0 + o + kSsimR][c + kSsimR] - sy[r0 + o + kSsimR][c + kSsimR]);
        }
    }
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const size_t nblk = (size_t)gridDim.x * gridDim.y * gridDim.z;
    const float ts = block_sum(s_sum, red);
    const float tl = block_sum(l1_sum, red);
    if (threadIdx.x == 0) {
        partials[blk] = ts;
        partials[nblk + blk] = tl;
    }
}

// dL/dx = (1 - lambda) sign(x - y) / N - lambda (G * M1 + 2 x' (G * M2) + y' (G * M3)) / N.
__global__ void __launch_bounds__(kSsimThreads)
dssim_bwd_kernel(int W, int H, SsimTaps taps, float lambda, float inv_n, const float* __restrict__ x,
                 const float* __restrict__ y, const float* __restrict__ m1, const float* __restrict__ m2,
                 const float* __restrict__ m3, float* __restrict__ dL) {
    __shared__ __align__(16) float sm[3][kSsimInH][kSsimStride];
    __shared__ float hm[3][kSsimInH][kSsimTW];
    const size_t plane = (size_t)blockIdx.z * H * W;
    const int ox = blockIdx.x * kSsimTW, oy = blockIdx.y * kSsimTH;
    for (int i = threadIdx.x; i < kSsimInH * kSsimStride; i += kSsimThreads) {
        const int r = i / kSsimStride, c = i - r * kSsimStride;
        const int gy = oy + r - kSsimR, gx = ox + c - kSsimR;
        const bool in = c < kSsimInW && gx >= 0 && gx < W && gy >= 0 && gy < H;
        const size_t p = plane + (size_t)gy * W + gx;
        sm[0][r][c] = in ? __ldg(m1 + p) : 0.f;
        sm[1][r][c] = in ? __ldg(m2 + p) : 0.f;
        sm[2][r][c] = in ? __ldg(m3 + p) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSsimInH * (kSsimTW / kSsimRun); i += kSsimThreads) {
        const int r = i / (kSsimTW / kSsimRun), c0 = (i - r * (kSsimTW / kSsimRun)) * kSsimRun;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float a[16];
            load_run16(sm[k][r], c0, a);
#pragma unroll
            for (int o = 0; o < kSsimRun; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t <= 2 * kSsimR; ++t) acc = fmaf(taps.g[t], a[o + t], acc);
                hm[k][r][c0 + o] = acc;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSsimTW * (kSsimTH / kSsimRun); i += kSsimThreads) {
        const int c = i % kSsimTW, r0 = (i / kSsimTW) * kSsimRun;
        float f[3][kSsimRun];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float v[kSsimSpan];
#pragma unroll
            for (int t = 0; t < kSsimSpan; ++t) v[t] = hm[k][r0 + t][c];
#pragma unroll
            for (int o = 0; o < kSsimRun; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t <= 2 * kSsimR; ++t) acc = fmaf(taps.g[t], v[o + t], acc);
                f[k][o] = acc;
            }
        }
        const int gx = ox + c;
#pragma unroll
        for (int o = 0; o < kSsimRun; ++o) {
            const int gy = oy + r0 + o;
            if (gx >= W || gy >= H) continue;
            const size_t pix = plane + (size_t)gy * W + gx;
            const float xv = __ldg(x + pix), yv = __ldg(y + pix);
            const float diff = xv - yv;
            const float sg = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
            const float dssim = f[0][o] + 2.f * (xv - kShift) * f[1][o] + (yv - kShift) * f[2][o];
            dL[pix] = inv_n * ((1.f - lambda) * sg - lambda * dssim);
        }
    }
}

__global__ void __launch_bounds__(1024)
dssim_finish_kernel(const float* __restrict__ partials, int nblk, float lambda, double inv_n, float* __restrict__ loss) {
    __shared__ double red_s[32], red_l[32];
    double s = 0.0, l = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        s += partials[i];
        l += partials[nblk + i];
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        l += __shfl_xor_sync(0xffffffffu, l, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_s[threadIdx.x >> 5] = s;
        red_l[threadIdx.x >> 5] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tl = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ts += red_s[w];
            tl += red_l[w];
        }
        *loss = (float)((1.0 - lambda) * tl * inv_n + lambda * (1.0 - ts * inv_n));
    }
}

}  // namespace

size_t dssim_scratch_bytes(const omnigs_config& cfg) {
    const size_t n = (size_t)cfg.num_views * 3 * cfg.height * cfg.width;
    const size_t blocks = (size_t)((cfg.width + kSsimTW - 1) / kSsimTW) * ((cfg.height + kSsimTH - 1) / kSsimTH) *
                          cfg.num_views * 3;
    return 256 + 3 * ((n * sizeof(float) + 255) / 256 * 256) + 2 * blocks * sizeof(float);
}

cudaError_t launch_dssim(const omnigs_config& cfg, float lambda, const float* rgb, const float* target, float* dL,
                         float* loss, char* scratch, cudaStream_t stream) {
    const SsimTaps taps = gaussian_taps();
    const size_t n = (size_t)cfg.num_views * 3 * cfg.height * cfg.width;
    const size_t map = (n * sizeof(float) + 255) / 256 * 256;
    float* m1 = reinterpret_cast<float*>(scratch + 256);
    float* m2 = reinterpret_cast<float*>(scratch + 256 + map);
    float* m3 = reinterpret_cast<float*>(scratch + 256 + 2 * map);
    float* partials = reinterpret_cast<float*>(scratch + 256 + 3 * map);
    const dim3 grid((cfg.width + kSsimTW - 1) / kSsimTW, (cfg.height + kSsimTH - 1) / kSsimTH, cfg.num_views * 3);
    const int nblk = (int)(grid.x * grid.y * grid.z);
    {
        ProfScope prof("dssim_fwd", stream);
        dssim_fwd_kernel<<<grid, kSsimThreads, 0, stream>>>(cfg.width, cfg.height, taps, rgb, target, m1, m2, m3,
                                                            partials);
    }
    {
        ProfScope prof("dssim_bwd", stream, 2);
        dssim_bwd_kernel<<<grid, kSsimThreads, 0, stream>>>(cfg.width, cfg.height, taps, lambda,
                                                            (float)(1.0 / (double)n), rgb, target, m1, m2, m3, dL);
        dssim_finish_kernel<<<1, 1024, 0, stream>>>(partials, nblk, lambda, 1.0 / (double)n, loss);
    }
    return cudaGetLastError();
}

}  // namespace omnigs
