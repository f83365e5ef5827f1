// Perspective crop of equirectangular images (Sec. 5.4: rendered equirectangular views are cropped into perspective
// images before being compared with perspective renders).
//
// One thread per output pixel: the pinhole direction of its centre, d = R^T ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy,
// 1), its longitude and latitude (Eq. 3) and the equirectangular position (Eqs. 4-5), sampled bilinearly between pixel
// centres with the columns wrapping around the seam and the rows clamped at the poles.
#include "common.cuh"

namespace omnigs {
namespace {

__global__ void __launch_bounds__(256)
crop_kernel(int We, int He, const float* __restrict__ eq, const float* __restrict__ rot, int W, int H, float fx,
            float fy, float cx, float cy, float* __restrict__ out) {
    const int v = blockIdx.z;
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    const float* R = rot + 9 * v;
    const float a = (x + 0.5f - cx) / fx, b = (y + 0.5f - cy) / fy;
    const float dx = __ldg(R + 0) * a + __ldg(R + 3) * b + __ldg(R + 6);
    const float dy = __ldg(R + 1) * a + __ldg(R + 4) * b + __ldg(R + 7);
    const float dz = __ldg(R + 2) * a + __ldg(R + 5) * b + __ldg(R + 8);
    const float lon = atan2f(dx, dz);
    const float lat = asinf(fminf(fmaxf(dy / sqrtf(dx * dx + dy * dy + dz * dz), -1.f), 1.f));
    const float u = (lon / kPi + 1.f) * (0.5f * (float)We) - 0.5f;
    const float w = (2.f * lat / kPi + 1.f) * (0.5f * (float)He) - 0.5f;
    const float fu0 = floorf(u), fw0 = floorf(w);
    const float fu = u - fu0, fw = w - fw0;
    int x0 = (int)fu0 % We;
    x0 += x0 < 0 ? We : 0;
    const int x1 = x0 + 1 == We ? 0 : x0 + 1;
    const int y0 = min(max((int)fw0, 0), He - 1), y1 = min(max((int)fw0 + 1, 0), He - 1);
    const size_t plane = (size_t)He * We;
    const float* src = eq + (size_t)v * 3 * plane;
    float* dst = out + (size_t)v * 3 * H * W + (size_t)y * W + x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* p = src + c * plane;
        const float top = fmaf(fu, __ldg(p + (size_t)y0 * We + x1) - __ldg(p + (size_t)y0 * We + x0),
                               __ldg(p + (size_t)y0 * We + x0));
        const float bot = fmaf(fu, __ldg(p + (size_t)y1 * We + x1) - __ldg(p + (size_t)y1 * We + x0),
                               __ldg(p + (size_t)y1 * We + x0));
        dst[(size_t)c * H * W] = fmaf(fw, bot - top, top);
    }
}

}  // namespace

cudaError_t launch_crop(int V, int We, int He, const float* eq, const float* rot, int W, int H, float fx, float fy,
                        float cx, float cy, float* out, cudaStream_t stream) {
    const dim3 grid((W + 31) / 32, (H + 7) / 8, V);
    ProfScope prof("equirect_crop", stream);
    crop_kernel<<<grid, 256, 0, stream>>>(We, He, eq, rot, W, H, fx, fy, cx, cy, out);
    return cudaGetLastError();
}

}  // namespace omnigs
