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
// work is enqueued, and so is every configuration omnigs_l1_loss rejects. Every call writes every partial sum it
// reads, so nothing has to be cleared between calls. All calls on a device share the one array: calls that may
// overlap on the GPU (different streams, or several host threads) race with each other and must be serialised by
// the caller.
//
// The array's device address is looked up (cudaGetSymbolAddress) on the first call in each CUDA context and kept
// with that context's id, so a context created anew (after cudaDeviceReset, say) gets a fresh lookup. The first
// call in a context also loads this library's module onto the device if nothing has loaded it yet, which needs
// device memory for the module image; it should therefore come before the caller reserves all device memory and
// before any stream capture.
#include <cuda.h>  // driver types only: the two driver functions used are fetched through the runtime

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

// One block of 1024 threads adds the nb <= kStaticBlocks partial sums in double precision.
__global__ void __launch_bounds__(1024)
l1_static_finish_kernel(const float* __restrict__ partials, int nb, float inv_total, float* __restrict__ loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 1024) s += (double)partials[i];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = red[threadIdx.x];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *loss = (float)(s * (double)inv_total);
    }
}

// Device address of g_l1_partials in the current context. (In host code the symbol names a host-side stand-in, not
// device memory, so kernels must be given this address.) It is cached per device together with the id of the
// context it was looked up in, and looked up again when the current context's id differs. Without the driver's
// context functions (an old driver) it is looked up on every call.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
struct AddrSlot {
    unsigned long long ctx_id;
    float* addr;
};
AddrSlot g_addr[kMaxDevices] = {};
bool g_ctx_fns_tried = false;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the current context, 0 when it cannot be told (no driver function, or no context current yet).
unsigned long long current_context_id() {
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

cudaError_t partials_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    const unsigned long long id = current_context_id();
    if (id == 0 || g_addr[dev].ctx_id != id || !g_addr[dev].addr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_l1_partials);  // makes the device's primary context current if none is
        if (e != cudaSuccess) return e;
        g_addr[dev].addr = static_cast<float*>(p);
        g_addr[dev].ctx_id = id != 0 ? id : current_context_id();
    }
    *out = g_addr[dev].addr;
    return cudaSuccess;
}

}  // namespace
}  // namespace omnigs

using namespace omnigs;

extern "C" omnigs_status omnigs_l1_loss_static(const omnigs_config* cfg, const float* rgb, const float* target,
                                               float* dL_drgb, float* loss, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !rgb || !target || !dL_drgb || !loss) return OMNIGS_E_INVALID;
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
        l1_static_finish_kernel<<<1, 1024, 0, s>>>(partials, nb, inv, loss);
    }
    return cudaGetLastError() == cudaSuccess ? OMNIGS_OK : OMNIGS_E_CUDA;
}
