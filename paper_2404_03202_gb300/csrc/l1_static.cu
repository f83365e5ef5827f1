// A form of the L1 loss gradient that needs no workspace and therefore no device allocation by anyone.
//
// omnigs_l1_loss keeps its per-block partial sums in the caller's workspace. Some callers cannot provide one: code
// that runs where allocation is forbidden or unavailable, such as a host application that hands this library only
// its input and output buffers and manages (or pre-reserves) all other device memory itself, a real-time loop whose
// memory budget is fixed up front, or a plug-in whose host process owns the CUDA allocator. For them,
// omnigs_l1_loss_static keeps the partial sums in a fixed array that is part of this library's device image.
//
// The array is sized for kStaticBlocks partial sums of kPerBlock elements each, i.e. images of up to
// kStaticBlocks * kPerBlock floats over [V, 3, H, W]; larger requests are rejected with OMNIGS_E_INVALID before any
// work is enqueued. Every call writes every partial sum it reads, so nothing has to be cleared between calls. All
// calls on a device share the one array: calls that may overlap on the GPU (different streams, or several host
// threads) race with each other and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace omnigs {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticBlocks = 4096;          // partial sums held by the fixed array (16 KiB)
constexpr int64_t kPerBlock = 65536;         // floats reduced by one block
constexpr int64_t kStaticMaxElements = (int64_t)kStaticBlocks * kPerBlock;  // 268,435,456 floats

static __device__ __align__(256) float g_l1_partials[kStaticBlocks];

__device__ __forceinline__ float block_sum(float x, float* red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kStaticThreads / 32; ++w) s += red[w];
    return s;
}

// Block b reduces elements [b * kPerBlock, (b + 1) * kPerBlock) and writes its partial sum; the gradient is written
// elementwise, exactly as omnigs_l1_loss writes it.
__global__ void __launch_bounds__(kStaticThreads)
l1_static_kernel(int64_t n4, const float4* __restrict__ rgb, const float4* __restrict__ target,
                 float4* __restrict__ dL, float inv_total, float* __restrict__ partials) {
    __shared__ float red[kStaticThreads / 32];
    const int64_t b0 = (int64_t)blockIdx.x * (kPerBlock / 4);
    const int64_t b1 = min(b0 + kPerBlock / 4, n4);
    float acc = 0.f;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kStaticThreads) {
        const float4 a = __ldg(rgb + i), b = __ldg(target + i);
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        auto sg = [inv_total](float d) { return d > 0.f ? inv_total : (d < 0.f ? -inv_total : 0.f); };
        dL[i] = make_float4(sg(d0), sg(d1), sg(d2), sg(d3));
    }
    const float s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void l1_static_finish_kernel(const float* __restrict__ partials, int nb, float inv_total,
                                        float* __restrict__ loss) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += partials[i];
        *loss = (float)(s * inv_total);
    }
}

// Device address of g_l1_partials, looked up once per device with that device current. (In host code the symbol
// names a host-side stand-in, not device memory, so kernels must be given this address.)
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
float* g_addr[kMaxDevices] = {};

cudaError_t partials_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_l1_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<float*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool valid_static_cfg(const omnigs_config* c) {
    if (!c) return false;
    if (c->tile != 8 && c->tile != 16 && c->tile != 32) return false;
    if (c->width <= 0 || c->height <= 0 || c->width % c->tile || c->height % c->tile) return false;
    return c->num_views >= 1;
}

}  // namespace
}  // namespace omnigs

using namespace omnigs;

extern "C" omnigs_status omnigs_l1_loss_static(const omnigs_config* cfg, const float* rgb, const float* target,
                                               float* dL_drgb, float* loss, omnigs_stream_t stream) {
    if (!valid_static_cfg(cfg) || !rgb || !target || !dL_drgb || !loss) return OMNIGS_E_INVALID;
    if (((uintptr_t)rgb | (uintptr_t)target | (uintptr_t)dL_drgb) % 16) return OMNIGS_E_INVALID;
    const int64_t total = (int64_t)cfg->num_views * 3 * cfg->height * cfg->width;
    if (total > kStaticMaxElements) return OMNIGS_E_INVALID;  // beyond the fixed scratch array
    float* partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) return OMNIGS_E_CUDA;
    const int nb = (int)((total + kPerBlock - 1) / kPerBlock);
    const float inv = (float)(1.0 / (double)total);
    cudaStream_t s = (cudaStream_t)stream;
    {
        ProfScope prof("l1_loss_static", s);
        l1_static_kernel<<<nb, kStaticThreads, 0, s>>>(total / 4, reinterpret_cast<const float4*>(rgb),
                                                        reinterpret_cast<const float4*>(target),
                                                        reinterpret_cast<float4*>(dL_drgb), inv, partials);
    }
    {
        ProfScope prof("l1_finish_static", s);
        l1_static_finish_kernel<<<1, 32, 0, s>>>(partials, nb, inv, loss);
    }
    return cudaGetLastError() == cudaSuccess ? OMNIGS_OK : OMNIGS_E_CUDA;
}
