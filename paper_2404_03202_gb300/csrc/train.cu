// Per-iteration bookkeeping of the reconstruction loop (Sec. 4, Algorithm 1): the Adam step, densification
// statistics from dL/ds, clone / split / prune, and the periodic opacity reset.
//
// The optimiser keeps every Gaussian as one row of P = 11 + 3K raw floats: mean (3), log-scale (3), quaternion (4,
// normalised only when used), logit-opacity (1), SH (3K, coefficient-major as [K][3]). Its Adam moments m and v have
// the same layout. The renderer reads the activated arrays (scales = exp(log-scale), opacity = sigmoid(logit)) in its
// own [n, 3] / [n, 4] / [n] / [n, K, 3] layout, which omnigs_adam_step (and omnigs_publish_params) write.
//
// Thresholds follow the 3DGS conventions the paper says its densification resembles (its supplement, which holds
// the values, is not available); they are inputs (omnigs_densify_config).
#include <cmath>

#include "common.cuh"

namespace omnigs {
namespace {

constexpr int kTrainThreads = 256;

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + __expf(-x)); }

// Column c of a parameter row: 0-2 mean, 3-5 log-scale, 6-9 quaternion, 10 logit-opacity, 11.. SH.
__device__ __forceinline__ void publish_one(int64_t g, int c, int K, float raw, float* __restrict__ means,
                                            float* __restrict__ scales, float* __restrict__ quats,
                                            float* __restrict__ opacity, float* __restrict__ sh) {
    if (c < 3) means[g * 3 + c] = raw;
    else if (c < 6) scales[g * 3 + (c - 3)] = expf(raw);
    else if (c < 10) quats[g * 4 + (c - 6)] = raw;
    else if (c == 10) opacity[g] = sigmoidf_(raw);
    else sh[g * 3 * K + (c - 11)] = raw;
}

__global__ void __launch_bounds__(kTrainThreads)
adam_kernel(int64_t n, int K, omnigs_adam_config cfg, float bias1, float bias2, float* __restrict__ params,
            float* __restrict__ m, float* __restrict__ v, const float* __restrict__ d_means,
            const float* __restrict__ d_scales, const float* __restrict__ d_quats, const float* __restrict__ d_opacity,
            const float* __restrict__ d_sh, float* __restrict__ means, float* __restrict__ scales,
            float* __restrict__ quats, float* __restrict__ opacity, float* __restrict__ sh) {
    const int P = 11 + 3 * K;
    const int64_t total = n * P;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / P;
        const int c = (int)(e - g * P);
        const float raw = params[e];
        float grad, lr;  // gradient with respect to the raw value (chain rule through the activation)
        if (c < 3) {
            grad = d_means[g * 3 + c];
            lr = cfg.lr_means;
        } else if (c < 6) {
            grad = d_scales[g * 3 + (c - 3)] * expf(raw);
            lr = cfg.lr_scales;
        } else if (c < 10) {
            grad = d_quats[g * 4 + (c - 6)];
            lr = cfg.lr_quats;
        } else if (c == 10) {
            const float o = sigmoidf_(raw);
            grad = d_opacity[g] * o * (1.f - o);
            lr = cfg.lr_opacity;
        } else {
            grad = d_sh[g * 3 * K + (c - 11)];
            lr = c < 14 ? cfg.lr_sh_dc : cfg.lr_sh_rest;  // coefficient 0 = columns 11..13
        }
        const float mk = fmaf(cfg.beta1, m[e], (1.f - cfg.beta1) * grad);
        const float vk = fmaf(cfg.beta2, v[e], (1.f - cfg.beta2) * grad * grad);
        const float mhat = mk / bias1, vhat = vk / bias2;
        const float nr = raw - lr * mhat / (sqrtf(vhat) + cfg.eps);
        m[e] = mk;
        v[e] = vk;
        params[e] = nr;
        publish_one(g, c, K, nr, means, scales, quats, opacity, sh);
    }
}

__global__ void __launch_bounds__(kTrainThreads)
publish_kernel(int64_t n, int K, const float* __restrict__ params, float* __restrict__ means,
               float* __restrict__ scales, float* __restrict__ quats, float* __restrict__ opacity,
               float* __restrict__ sh) {
    const int P = 11 + 3 * K;
    const int64_t total = n * P;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / P;
        publish_one(g, (int)(e - g * P), K, params[e], means, scales, quats, opacity, sh);
    }
}

// One render's statistics: for every view in which Gaussian g has instances, |dL/ds| (dL/ds = dL/dp diag(W/2, H/2))
// is added to accum[g], count[g] is incremented and max_radius[g] keeps the largest instance half-extent.
__global__ void __launch_bounds__(kTrainThreads)
densify_stats_kernel(int64_t n, int V, float half_w, float half_h, const float4* __restrict__ splats,
                     const float4* __restrict__ grads, float* __restrict__ accum, int* __restrict__ count,
                     float* __restrict__ max_radius) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float a = accum[g], r = max_radius[g];
    int k = count[g];
    for (int v = 0; v < V; ++v) {
        const size_t i = (size_t)v * n + g;
        const float4 c = __ldg(splats + 3 * i + 1);  // c2, depth, radii, q
        const unsigned radii = __float_as_uint(c.z);
        const int rx = (int)(radii & 0xffffu), ry = (int)(radii >> 16);
        if (rx <= 0) continue;
        const float4 gr = __ldg(grads + 3 * i);
        a += hypotf(gr.x * half_w, gr.y * half_h);
        ++k;
        r = fmaxf(r, (float)max(rx, ry));
    }
    accum[g] = a;
    count[g] = k;
    max_radius[g] = r;
}

struct Decision {
    bool clone, split, keep, clone_kept, child_kept;
};

__device__ __forceinline__ bool pruned(float logit, float max_scale, const omnigs_densify_config& cfg) {
    return sigmoidf_(logit) < cfg.min_opacity || max_scale > cfg.max_scale_frac * cfg.extent;
}

__device__ __forceinline__ Decision decide(const float* __restrict__ row, float accum, int count, float max_radius,
                                           const omnigs_densify_config& cfg) {
    Decision d;
    const float s_max = fmaxf(expf(row[3]), fmaxf(expf(row[4]), expf(row[5])));
    const bool hot = count > 0 && accum / (float)count >= cfg.grad_threshold;
    const bool big = s_max > cfg.percent_dense * cfg.extent;
    d.clone = hot && !big;
    d.split = hot && big;
    const bool gone = pruned(row[10], s_max, cfg);
    d.keep = !d.split && !gone && !(max_radius > cfg.max_screen_radius);
    d.clone_kept = d.clone && !gone;
    d.child_kept = d.split && !pruned(row[10], s_max / 1.6f, cfg);
    return d;
}

__device__ __forceinline__ unsigned out_rows(const Decision& d) {
    return (d.keep ? 1u : 0u) + (d.clone_kept ? 1u : 0u) + (d.child_kept ? 2u : 0u);
}

template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* scratch, T* total) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= (unsigned)o) s += y;
    }
    if (lane == 31) scratch[warp] = s;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kTrainThreads / 32 ? scratch[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (unsigned)o) w += y;
        }
        if (lane < kTrainThreads / 32) scratch[lane] = w;
    }
    __syncthreads();
    const T base = warp ? scratch[warp - 1] : T(0);
    *total = scratch[kTrainThreads / 32 - 1];
    __syncthreads();
    return base + s - x;
}

__global__ void __launch_bounds__(kTrainThreads)
densify_count_kernel(int64_t n, int K, omnigs_densify_config cfg, const float* __restrict__ params,
                     const float* __restrict__ accum, const int* __restrict__ count,
                     const float* __restrict__ max_radius, unsigned* __restrict__ block_sums) {
    __shared__ unsigned scratch[kTrainThreads / 32];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int P = 11 + 3 * K;
    unsigned c = 0;
    if (g < n) c = out_rows(decide(params + g * P, accum[g], count[g], max_radius[g], cfg));
    unsigned tot;
    block_excl_scan<unsigned>(c, scratch, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Exclusive scan of the per-block sums by one CTA (grid-stride over the blocks); the total goes to *n_out.
__global__ void __launch_bounds__(kTrainThreads)
densify_scan_kernel(int nblocks, const unsigned* __restrict__ block_sums, long long* __restrict__ block_offsets,
                    long long* __restrict__ n_out) {
    __shared__ long long scratch[kTrainThreads / 32];
    long long carry = 0;
    for (int base = 0; base < nblocks; base += kTrainThreads) {
        const int i = base + threadIdx.x;
        const long long x = i < nblocks ? (long long)block_sums[i] : 0ll;
        long long tot;
        const long long ex = block_excl_scan<long long>(x, scratch, &tot);
        if (i < nblocks) block_offsets[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *n_out = carry;
}

__device__ __forceinline__ void copy_row(float* __restrict__ dst, const float* __restrict__ src, int P) {
    for (int c = 0; c < P; ++c) dst[c] = src[c];
}

__device__ __forceinline__ void zero_row(float* __restrict__ dst, int P) {
    for (int c = 0; c < P; ++c) dst[c] = 0.f;
}

// Rows out, per original in index order: itself (if kept), its clone, its two split children.
__global__ void __launch_bounds__(kTrainThreads)
densify_emit_kernel(int64_t n, int K, omnigs_densify_config cfg, const float* __restrict__ params,
                    const float* __restrict__ m, const float* __restrict__ v, const float* __restrict__ accum,
                    const int* __restrict__ count, const float* __restrict__ max_radius,
                    const float* __restrict__ normals, const long long* __restrict__ block_offsets,
                    float* __restrict__ params_out, float* __restrict__ m_out, float* __restrict__ v_out) {
    __shared__ unsigned scratch[kTrainThreads / 32];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int P = 11 + 3 * K;
    Decision d{};
    unsigned c = 0;
    if (g < n) {
        d = decide(params + g * P, accum[g], count[g], max_radius[g], cfg);
        c = out_rows(d);
    }
    unsigned tot;
    const unsigned ex = block_excl_scan<unsigned>(c, scratch, &tot);
    if (g >= n || c == 0) return;
    long long o = block_offsets[blockIdx.x] + ex;
    const float* row = params + g * P;
    if (d.keep) {
        copy_row(params_out + o * P, row, P);
        copy_row(m_out + o * P, m + g * P, P);
        copy_row(v_out + o * P, v + g * P, P);
        ++o;
    }
    if (d.clone_kept) {
        copy_row(params_out + o * P, row, P);
        zero_row(m_out + o * P, P);
        zero_row(v_out + o * P, P);
        ++o;
    }
    if (d.child_kept) {
        // R(q) of the normalised quaternion (w, x, y, z)
        const float qw = row[6], qx = row[7], qy = row[8], qz = row[9];
        const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
        const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                            2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                            2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        const float s[3] = {expf(row[3]), expf(row[4]), expf(row[5])};
        const float ln16 = 0.47000362924573558f;  // ln(1.6)
        for (int k = 0; k < 2; ++k) {
            const float* z3 = normals + (g * 2 + k) * 3;
            float* dst = params_out + o * P;
            copy_row(dst, row, P);
#pragma unroll
            for (int i = 0; i < 3; ++i)
                dst[i] = row[i] + R[3 * i] * (s[0] * z3[0]) + R[3 * i + 1] * (s[1] * z3[1]) + R[3 * i + 2] * (s[2] * z3[2]);
#pragma unroll
            for (int i = 0; i < 3; ++i) dst[3 + i] = row[3 + i] - ln16;
            zero_row(m_out + o * P, P);
            zero_row(v_out + o * P, P);
            ++o;
        }
    }
}

__global__ void __launch_bounds__(kTrainThreads)
reset_opacity_kernel(int64_t n, int K, float cap, float* __restrict__ params, float* __restrict__ m,
                     float* __restrict__ v, float* __restrict__ opacity) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int P = 11 + 3 * K;
    const float l = fminf(params[g * P + 10], cap);
    params[g * P + 10] = l;
    m[g * P + 10] = 0.f;
    v[g * P + 10] = 0.f;
    if (opacity) opacity[g] = sigmoidf_(l);
}

int grid_for(int64_t work) {
    const int64_t b = (work + kTrainThreads - 1) / kTrainThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 16));
}

}  // namespace

size_t densify_workspace_bytes(int64_t n) {
    const size_t nb = (size_t)((n + kTrainThreads - 1) / kTrainThreads);
    return 256 + (nb * sizeof(unsigned) + 255) / 256 * 256 + nb * sizeof(long long);
}

cudaError_t launch_adam(int64_t n, int K, const omnigs_adam_config& cfg, int64_t step, float* params, float* m,
                        float* v, const float* d_means, const float* d_scales, const float* d_quats,
                        const float* d_opacity, const float* d_sh, float* means, float* scales, float* quats,
                        float* opacity, float* sh, cudaStream_t stream) {
    const float bias1 = (float)(1.0 - std::pow((double)cfg.beta1, (double)step));
    const float bias2 = (float)(1.0 - std::pow((double)cfg.beta2, (double)step));
    ProfScope prof("adam_step", stream);
    adam_kernel<<<grid_for(n * (11 + 3 * K)), kTrainThreads, 0, stream>>>(
        n, K, cfg, bias1, bias2, params, m, v, d_means, d_scales, d_quats, d_opacity, d_sh, means, scales, quats,
        opacity, sh);
    return cudaGetLastError();
}

cudaError_t launch_publish(int64_t n, int K, const float* params, float* means, float* scales, float* quats,
                           float* opacity, float* sh, cudaStream_t stream) {
    ProfScope prof("publish_params", stream);
    publish_kernel<<<grid_for(n * (11 + 3 * K)), kTrainThreads, 0, stream>>>(n, K, params, means, scales, quats,
                                                                             opacity, sh);
    return cudaGetLastError();
}

cudaError_t launch_densify_stats(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats,
                                 const omnigs_splat_grad* grads, float* accum, int* count, float* max_radius,
                                 cudaStream_t stream) {
    ProfScope prof("densify_stats", stream);
    densify_stats_kernel<<<(unsigned)((n + kTrainThreads - 1) / kTrainThreads), kTrainThreads, 0, stream>>>(
        n, cfg.num_views, 0.5f * (float)cfg.width, 0.5f * (float)cfg.height,
        reinterpret_cast<const float4*>(splats), reinterpret_cast<const float4*>(grads), accum, count, max_radius);
    return cudaGetLastError();
}

cudaError_t launch_densify(int64_t n, int K, const omnigs_densify_config& cfg, const float* params, const float* m,
                           const float* v, const float* accum, const int* count, const float* max_radius,
                           const float* normals, float* params_out, float* m_out, float* v_out, long long* n_out,
                           char* ws, cudaStream_t stream) {
    const int nb = (int)((n + kTrainThreads - 1) / kTrainThreads);
    unsigned* sums = reinterpret_cast<unsigned*>(ws + 256);
    long long* offs = reinterpret_cast<long long*>(ws + 256 + ((size_t)nb * sizeof(unsigned) + 255) / 256 * 256);
    ProfScope prof("densify", stream, 3);
    densify_count_kernel<<<nb, kTrainThreads, 0, stream>>>(n, K, cfg, params, accum, count, max_radius, sums);
    densify_scan_kernel<<<1, kTrainThreads, 0, stream>>>(nb, sums, offs, n_out);
    densify_emit_kernel<<<nb, kTrainThreads, 0, stream>>>(n, K, cfg, params, m, v, accum, count, max_radius, normals,
                                                          offs, params_out, m_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_reset_opacity(int64_t n, int K, float value, float* params, float* m, float* v, float* opacity,
                                 cudaStream_t stream) {
    const float cap = (float)std::log((double)value / (1.0 - (double)value));
    ProfScope prof("reset_opacity", stream);
    reset_opacity_kernel<<<(unsigned)((n + kTrainThreads - 1) / kTrainThreads), kTrainThreads, 0, stream>>>(
        n, K, cap, params, m, v, opacity);
    return cudaGetLastError();
}

}  // namespace omnigs
