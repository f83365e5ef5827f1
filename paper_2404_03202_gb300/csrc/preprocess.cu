// Per-Gaussian projection onto the equirectangular image (Sec. 3.2-3.3, Eqs. 1, 3-5, 9-16; colour from SH, Sec. 3.1)
// and its adjoint (Sec. 3.4, Eqs. 18-20).
//
// One thread per Gaussian loops over the V views, so the 59 parameter floats are read from HBM once per launch.
// The forward stages the SH block of a CTA through shared memory with coalesced loads (rows padded to an odd stride
// so the per-thread reads are bank-conflict free). The adjoint walks only the views that passed the Gaussian a
// gradient and copies its SH row into the same layout at the first of them. The 2x2 covariance is formed as (M R S)(M R S)^T with M = J W, and its
// determinant as |T0 x T1|^2 + 0.3 (|T0|^2 + |T1|^2) + 0.09, a sum of non-negative terms, so that FP32 keeps full
// relative accuracy for elongated splats (a c - b^2 would cancel). With the pinhole camera a Gaussian whose instance
// box misses the image is culled (the frustum cull of 3DGS), and the adjoint, specialised per camera model, skips it.
#include "common.cuh"

namespace omnigs {
namespace {

constexpr int kPreThreads = 128;
// The adjoint's CTA: one warp. Few Gaussians take gradients in most views, and a CTA's final barrier (the d_sh rows
// written out through shared memory) waits for its slowest thread: one-warp CTAs wait on fewer (measured on the
// 8-view egocentric step: 0.182 ms against 0.188 with 64 threads and 0.200 with 128).
constexpr int kPreBwdThreads = 32;

// Real orthonormal SH, degree <= 3, no Condon-Shortley phase; normalisations
// sqrt((2l+1)/(4pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for m != 0.
constexpr float kY00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15/pi)/2
constexpr float kY2b = 0.31539156525252005f;   // sqrt(5/pi)/4
constexpr float kY2c = 0.54627421529603959f;   // sqrt(15/pi)/4
constexpr float kY3a = 0.59004358992664352f;   // sqrt(35/(2 pi))/4
constexpr float kY3b = 2.8906114426405538f;    // sqrt(105/pi)/2
constexpr float kY3c = 0.45704579946446572f;   // sqrt(21/(2 pi))/4
constexpr float kY3d = 0.37317633259011546f;   // sqrt(7/pi)/4
constexpr float kY3e = 1.4453057213202769f;    // sqrt(105/pi)/4

template <int K>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
    Y[0] = kY00;
    if (K > 1) {
        Y[1] = kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = kY1 * x;
    }
    if (K > 4) {
        Y[4] = kY2a * x * y;
        Y[5] = kY2a * y * z;
        Y[6] = kY2b * (3.f * z * z - 1.f);
        Y[7] = kY2a * x * z;
        Y[8] = kY2c * (x * x - y * y);
    }
    if (K > 9) {
        Y[9] = kY3a * y * (3.f * x * x - y * y);
        Y[10] = kY3b * x * y * z;
        Y[11] = kY3c * y * (5.f * z * z - 1.f);
        Y[12] = kY3d * z * (5.f * z * z - 3.f);
        Y[13] = kY3c * x * (5.f * z * z - 1.f);
        Y[14] = kY3e * z * (x * x - y * y);
        Y[15] = kY3a * x * (x * x - 3.f * y * y);
    }
}

// sum_k w_k grad Y_k(x, y, z) (gradient of the polynomial forms above)
template <int K>
__device__ __forceinline__ float3 sh_grad_dot(float x, float y, float z, const float* w) {
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (K > 1) {
        g.x += kY1 * w[3];
        g.y += kY1 * w[1];
        g.z += kY1 * w[2];
    }
    if (K > 4) {
        g.x += kY2a * (y * w[4] + z * w[7]) + 2.f * kY2c * x * w[8];
        g.y += kY2a * (x * w[4] + z * w[5]) - 2.f * kY2c * y * w[8];
        g.z += kY2a * (y * w[5] + x * w[7]) + 6.f * kY2b * z * w[6];
    }
    if (K > 9) {
        float zz5 = 5.f * z * z;
        g.x += 6.f * kY3a * x * y * w[9] + kY3b * y * z * w[10] + kY3c * (zz5 - 1.f) * w[13] +
               2.f * kY3e * x * z * w[14] + 3.f * kY3a * (x * x - y * y) * w[15];
        g.y += 3.f * kY3a * (x * x - y * y) * w[9] + kY3b * x * z * w[10] + kY3c * (zz5 - 1.f) * w[11] -
               2.f * kY3e * y * z * w[14] - 6.f * kY3a * x * y * w[15];
        g.z += kY3b * x * y * w[10] + 10.f * kY3c * y * z * w[11] + kY3d * (3.f * zz5 - 3.f) * w[12] +
               10.f * kY3c * x * z * w[13] + kY3e * (x * x - y * y) * w[14];
    }
    return g;
}

struct View {
    float Wr[9], t[3];
};

__device__ __forceinline__ View load_view(const float* s_view, int v) {
    View w;
    const float* m = s_view + 16 * v;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) w.Wr[3 * i + j] = m[4 * i + j];
        w.t[i] = m[4 * i + 3];
    }
    return w;
}

// Camera model of the config: the equirectangular camera (Eqs. 3-5) or the pinhole of Eq. 2 with the 3DGS bound on
// the ratios t_x / t_z and t_y / t_z inside J (limx, limy = 1.3 half-fields of view).
struct Cam {
    int pinhole;
    float fx, fy, cx, cy, limx, limy;
};

constexpr float kMaxCoord = 8388608.f;  // 2^23: pinhole Gaussians projected beyond this are culled

Cam make_cam(const omnigs_config& cfg) {
    Cam c{};
    c.pinhole = cfg.camera == OMNIGS_CAMERA_PINHOLE;
    if (c.pinhole) {
        c.fx = cfg.fx; c.fy = cfg.fy; c.cx = cfg.cx; c.cy = cfg.cy;
        c.limx = 1.3f * (float)cfg.width / (2.f * cfg.fx);
        c.limy = 1.3f * (float)cfg.height / (2.f * cfg.fy);
    }
    return c;
}

// Quantities of one (view, Gaussian) pair shared by the forward pass and its adjoint.
struct Proj {
    float t[3], tr, rho, rg;  // tr: the depth that orders Gaussians (t_r, or t_z for the pinhole camera)
    float J[6];       // the covariance Jacobian, 2 x 3 (J[1] = 0); dp/dt itself for the equirectangular camera
    float M[6];       // J W
    float Tm[6];      // M R diag(s)
    float A, B, C;    // Sigma~ entries 00, 01, 11 (with dilation)
    float det;
};

// Eq. 2 (pinhole) position and Jacobian; returns false when culled.
__device__ __forceinline__ bool project_pinhole(const Cam& cam, float near_r, Proj& P, float& px, float& py) {
    const float tx = P.t[0], ty = P.t[1], tz = P.t[2];
    P.tr = tz;
    P.rho = P.rg = 0.f;
    if (!(tz > near_r)) return false;
    const float iz = 1.f / tz;
    px = fmaf(cam.fx, tx * iz, cam.cx);
    py = fmaf(cam.fy, ty * iz, cam.cy);
    if (!(fabsf(px) < kMaxCoord && fabsf(py) < kMaxCoord)) return false;
    const float u = fminf(fmaxf(tx * iz, -cam.limx), cam.limx), v = fminf(fmaxf(ty * iz, -cam.limy), cam.limy);
    P.J[0] = cam.fx * iz; P.J[1] = 0.f; P.J[2] = -cam.fx * u * iz;
    P.J[3] = 0.f; P.J[4] = cam.fy * iz; P.J[5] = -cam.fy * v * iz;
    return true;
}

// Eqs. 3-5 and 10-16; returns false when culled.
__device__ __forceinline__ bool project_equirect(int W, int H, float near_r, Proj& P, float& px, float& py) {
    const float tx = P.t[0], ty = P.t[1], tz = P.t[2];
    P.tr = sqrtf(tx * tx + ty * ty + tz * tz);
    if (!(P.tr > near_r)) return false;
    float lon = atan2f(tx, tz);
    if (lon >= kPi) lon = -kPi;
    float sl = fminf(fmaxf(ty / P.tr, -1.f), 1.f);
    float lat = asinf(sl);
    px = (lon / kPi + 1.f) * (0.5f * (float)W);
    py = (2.f * lat / kPi + 1.f) * (0.5f * (float)H);
    if (!(isfinite(px) && isfinite(py))) return false;
    const float a = (float)W / (2.f * kPi), b = (float)H / kPi;
    P.rho = sqrtf(tx * tx + tz * tz);
    P.rg = fmaxf(P.rho, kPoleGuard * P.tr);
    const float rg = P.rg, rg2 = rg * rg, tr2 = P.tr * P.tr;
    P.J[0] = a * tz / rg2;
    P.J[1] = 0.f;
    P.J[2] = -a * tx / rg2;
    P.J[3] = -b * tx * ty / (tr2 * rg);
    P.J[4] = b * rg / tr2;
    P.J[5] = -b * tz * ty / (tr2 * rg);
    return true;
}

// Eq. 9: Sigma~ = (J W M3)(J W M3)^T + 0.3 I with its determinant as a sum of non-negative terms.
__device__ __forceinline__ bool covariance(const View& w, const float M3[9], Proj& P) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        P.M[j] = P.J[0] * w.Wr[j] + P.J[2] * w.Wr[6 + j];
        P.M[3 + j] = P.J[3] * w.Wr[j] + P.J[4] * w.Wr[3 + j] + P.J[5] * w.Wr[6 + j];
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P.Tm[3 * r + j] = P.M[3 * r] * M3[j] + P.M[3 * r + 1] * M3[3 + j] + P.M[3 * r + 2] * M3[6 + j];
    const float* T0 = P.Tm;
    const float* T1 = P.Tm + 3;
    const float n0 = T0[0] * T0[0] + T0[1] * T0[1] + T0[2] * T0[2];
    const float n1 = T1[0] * T1[0] + T1[1] * T1[1] + T1[2] * T1[2];
    const float cx = T0[1] * T1[2] - T0[2] * T1[1];
    const float cy = T0[2] * T1[0] - T0[0] * T1[2];
    const float cz = T0[0] * T1[1] - T0[1] * T1[0];
    P.A = n0 + kDilation;
    P.B = T0[0] * T1[0] + T0[1] * T1[1] + T0[2] * T1[2];
    P.C = n1 + kDilation;
    P.det = (cx * cx + cy * cy + cz * cz) + kDilation * (n0 + n1) + kDilation * kDilation;
    return P.det > 0.f;
}

// Eqs. 1, 3-5 (position) and 9-16 (covariance), or Eq. 2 for the pinhole camera. Returns false when culled (near
// plane or det <= 0).
__device__ __forceinline__ bool project(const View& w, const Cam& cam, const float m[3], const float M3[9], int W,
                                        int H, float near_r, Proj& P, float& px, float& py) {
#pragma unroll
    for (int i = 0; i < 3; ++i) P.t[i] = fmaf(w.Wr[3 * i], m[0], fmaf(w.Wr[3 * i + 1], m[1], fmaf(w.Wr[3 * i + 2], m[2], w.t[i])));
    if (cam.pinhole) {
        if (!project_pinhole(cam, near_r, P, px, py)) return false;
    } else if (!project_equirect(W, H, near_r, P, px, py)) {
        return false;
    }
    return covariance(w, M3, P);
}

// R(q) for the unit quaternion (w, x, y, z); M3 = R diag(s).
__device__ __forceinline__ void rot_scale(const float qn[4], const float s[3], float R[9], float M3[9]) {
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M3[3 * i + j] = R[3 * i + j] * s[j];
}

__device__ __forceinline__ void load_params(int g, const float* __restrict__ means, const float* __restrict__ scales,
                                            const float* __restrict__ quats, float m[3], float s[3], float qn[4],
                                            float& qnorm) {
    m[0] = __ldg(means + 3 * g); m[1] = __ldg(means + 3 * g + 1); m[2] = __ldg(means + 3 * g + 2);
    s[0] = __ldg(scales + 3 * g); s[1] = __ldg(scales + 3 * g + 1); s[2] = __ldg(scales + 3 * g + 2);
    const float4 q = __ldg(reinterpret_cast<const float4*>(quats) + g);
    qnorm = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float inv = 1.f / qnorm;
    qn[0] = q.x * inv; qn[1] = q.y * inv; qn[2] = q.z * inv; qn[3] = q.w * inv;
}

// Camera centre c = -W^T t_cw and unit direction from it to m.
__device__ __forceinline__ float view_dir(const View& w, const float m[3], float d[3]) {
    float v[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float c = -(w.Wr[j] * w.t[0] + w.Wr[3 + j] * w.t[1] + w.Wr[6 + j] * w.t[2]);
        v[j] = m[j] - c;
    }
    const float dist = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float inv = 1.f / dist;
    d[0] = v[0] * inv; d[1] = v[1] * inv; d[2] = v[2] * inv;
    return dist;
}

template <int K>
__device__ __forceinline__ void stage_sh(float* s_sh, const float* __restrict__ sh, int g0, int cnt) {
    constexpr int KK = 3 * K, STRIDE = KK + 1;
    const float* src = sh + (size_t)g0 * KK;
    for (int e = threadIdx.x; e < cnt * KK; e += blockDim.x) {
        const int t = e / KK;
        s_sh[t * STRIDE + (e - t * KK)] = __ldg(src + e);
    }
}

// The instance box (rx, ry): the 3-sigma square of half-side ceil(3 sqrt(lambda_max)) narrowed to the box of the
// alpha >= 1/255 ellipse dp^T conic dp <= q, q = 2 ln(255 o), whose half-extents are sqrt(q Sigma~_00) and
// sqrt(q Sigma~_11) (slightly widened), held at kMaxRadius. Returns q.
__device__ __forceinline__ float instance_box(const Proj& P, float o, int& rx, int& ry) {
    const float mid = 0.5f * (P.A + P.C);
    const float hd = 0.5f * (P.A - P.C);
    const float disc = fmaxf(0.1f, hd * hd + P.B * P.B);   // = mid^2 - det
    const float lam = mid + sqrtf(disc);
    const float rr = ceilf(3.f * sqrtf(lam));
    const float q = fmaxf(2.f * logf(255.f * o), 0.f);
    const float hx = ceilf(fmaf(sqrtf(q * P.A), 1.0001f, 1e-3f));
    const float hy = ceilf(fmaf(sqrtf(q * P.C), 1.0001f, 1e-3f));
    const float lim = fminf(rr, (float)kMaxRadius);
    rx = (int)fminf(hx, lim);
    ry = (int)fminf(hy, lim);
    return q;
}

// The pinhole's frustum cull: a box [floor(p) -+ r] that misses the image has no tile (|p| < 2^23 here).
__device__ __forceinline__ bool box_off_image(float px, float py, int rx, int ry, int W, int H) {
    const int ix = (int)floorf(px), iy = (int)floorf(py);
    return ix + rx < 0 || ix - rx >= W || iy + ry < 0 || iy - ry >= H;
}

// kKeys: also write the depth sort's packed key of every splat, ((view << 32 | t_r bits) << gbits) | splat index, and
// the splat count (omnigs_preprocess_bin), so that the binning does not read every splat record back for its depth.
template <int K, bool kKeys>
__global__ void __launch_bounds__(kPreThreads)
preprocess_kernel(int n, int V, int W, int H, float near_r, Cam cam, const float* __restrict__ means,
                  const float* __restrict__ scales, const float* __restrict__ quats, const float* __restrict__ opacity,
                  const float* __restrict__ sh, const float* __restrict__ viewmats, float4* __restrict__ splats,
                  unsigned long long* __restrict__ depth_keys, int gbits,
                  unsigned long long* __restrict__ splat_count) {
    constexpr int STRIDE = 3 * K + 1;
    extern __shared__ float smem[];
    float* s_sh = smem;
    float* s_view = smem + kPreThreads * STRIDE;
    const int g0 = blockIdx.x * kPreThreads;
    const int cnt = min(kPreThreads, n - g0);
    stage_sh<K>(s_sh, sh, g0, cnt);
    for (int e = threadIdx.x; e < 16 * V; e += blockDim.x) s_view[e] = __ldg(viewmats + e);
    __syncthreads();
    const int g = g0 + threadIdx.x;
    if (threadIdx.x >= cnt) return;
    if (kKeys && g == 0) *splat_count = (unsigned long long)n * V;

    float m[3], s[3], qn[4], qnorm, R[9], M3[9];
    load_params(g, means, scales, quats, m, s, qn, qnorm);
    rot_scale(qn, s, R, M3);
    const float o = __ldg(opacity + g);
    const float* shc = s_sh + threadIdx.x * STRIDE;

    for (int v = 0; v < V; ++v) {
        const View w = load_view(s_view, v);
        Proj P;
        float px, py;
        float4* out = splats + 3 * ((size_t)v * n + g);
        const bool visible = project(w, cam, m, M3, W, H, near_r, P, px, py);  // sets t_r either way
        if constexpr (kKeys) {
            const unsigned long long i = (unsigned long long)v * n + g;
            depth_keys[i] = ((((unsigned long long)v << 32) | __float_as_uint(P.tr)) << gbits) | i;
        }
        if (!visible) {
            out[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            out[1] = make_float4(0.f, P.tr, __uint_as_float(0u), 0.f);
            out[2] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float inv = 1.f / P.det;
        const float c0 = P.C * inv, c1 = -P.B * inv, c2 = P.A * inv;
        int rx, ry;
        const float q = instance_box(P, o, rx, ry);
        const bool off = cam.pinhole && box_off_image(px, py, rx, ry, W, H);
        if (!(255.f * o >= 1.f) || off) {  // alpha < 1/255 everywhere, or no tile: no instance
            out[0] = make_float4(px, py, c0, c1);
            out[1] = make_float4(c2, P.tr, __uint_as_float(0u), 0.f);
            out[2] = make_float4(o, 0.f, 0.f, 0.f);
            continue;
        }

        float d[3], Y[16];
        view_dir(w, m, d);
        sh_eval<K>(d[0], d[1], d[2], Y);
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fmaf(Y[k], shc[3 * k + ch], acc);
            rgb[ch] = fmaxf(acc + 0.5f, 0.f);
        }
        out[0] = make_float4(px, py, c0, c1);
        out[1] = make_float4(c2, P.tr, __uint_as_float((unsigned)rx | ((unsigned)ry << 16)), q);
        out[2] = make_float4(o, rgb[0], rgb[1], rgb[2]);
    }
}

// ---------------------------------------------------------------------------------------------------- adjoint

template <int K, bool kPin>
// 20 one-warp CTAs per SM: 96 registers a thread (12 bytes spilled), against 128 at 16 CTAs: the kernel waits on
// memory, and the extra warps cover it (0.168 ms against 0.180 on the 8-view egocentric step; 80 registers spill
// 136 bytes and measured 0.188)
__global__ void __launch_bounds__(kPreBwdThreads, 20)
preprocess_bwd_kernel(int n, int V, int W, int H, float near_r, Cam cam, const float* __restrict__ means,
                      const float* __restrict__ scales, const float* __restrict__ quats,
                      const float* __restrict__ opacity, const float* __restrict__ sh,
                      const float* __restrict__ viewmats,
                      const float4* __restrict__ grads, float* __restrict__ d_means, float* __restrict__ d_scales,
                      float* __restrict__ d_quats, float* __restrict__ d_opacity, float* __restrict__ d_sh,
                      float* __restrict__ d_screen) {
    constexpr int KK = 3 * K, STRIDE = KK + 1;
    cam.pinhole = kPin;  // the camera model as a compile-time constant
    extern __shared__ float smem[];
    float* s_sh = smem;
    float* s_dsh = smem + kPreBwdThreads * STRIDE;
    float* s_view = s_dsh + kPreBwdThreads * STRIDE;
    const int g0 = blockIdx.x * kPreBwdThreads;
    const int cnt = min(kPreBwdThreads, n - g0);
    for (int e = threadIdx.x; e < 16 * V; e += blockDim.x) s_view[e] = __ldg(viewmats + e);
    float* dshc = s_dsh + threadIdx.x * STRIDE;
    for (int k = 0; k < KK; ++k) dshc[k] = 0.f;
    __syncthreads();
    const int g = g0 + threadIdx.x;
    if (threadIdx.x < cnt) {
        float m[3], s[3], qn[4], qnorm, R[9], M3[9];
        load_params(g, means, scales, quats, m, s, qn, qnorm);
        rot_scale(qn, s, R, M3);
        // the thread's SH row, copied to its shared-memory slot at its first view with a gradient (most Gaussians
        // have none)
        float* shc = s_sh + threadIdx.x * STRIDE;
        bool sh_here = false;
        float dm[3] = {0.f, 0.f, 0.f}, dM3[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float dop = 0.f, dsx = 0.f, dsy = 0.f;
        const float a = (float)W / (2.f * kPi), b = (float)H / kPi;
        // culled in every view when alpha < 1/255 everywhere (255 o < 1): no gradient reaches it
        const int views = 255.f * __ldg(opacity + g) >= 1.f ? V : 0;

        // Every term of a view's contribution is a product with one of its nine splat-gradient fields, so a view
        // that passed this splat no gradient (culled, occluded, or reaching no pixel) adds exactly nothing. The
        // views with some gradient are collected 32 at a time (their loads all in flight), and only those are
        // walked: most splats are hidden in most views.
        for (int v0 = 0; v0 < views; v0 += 32) {
            const int vn = min(32, views - v0);
            unsigned live = 0;
#pragma unroll 8
            for (int i = 0; i < vn; ++i) {
                const float4* gp = grads + 3 * ((size_t)(v0 + i) * n + g);
                const float4 a0 = __ldg(gp), a1 = __ldg(gp + 1);
                const float a2 = __ldg(reinterpret_cast<const float*>(gp + 2));
                const bool some = a0.x != 0.f || a0.y != 0.f || a0.z != 0.f || a0.w != 0.f || a1.x != 0.f ||
                                  a1.y != 0.f || a1.z != 0.f || a1.w != 0.f || a2 != 0.f;
                live |= some ? 1u << i : 0u;
            }
            if (live && !sh_here) {
                const float* src = sh + (size_t)g * KK;
                for (int k = 0; k < KK; ++k) shc[k] = __ldg(src + k);
                sh_here = true;
            }
            while (live) {
                const int v = v0 + __ffs(live) - 1;
                live &= live - 1;
                const float4 g0v = __ldg(grads + 3 * ((size_t)v * n + g));
                const float4 g1v = __ldg(grads + 3 * ((size_t)v * n + g) + 1);
                const float4 g2v = __ldg(grads + 3 * ((size_t)v * n + g) + 2);
                const View w = load_view(s_view, v);
                Proj P;
                float px, py;
                if (!project(w, cam, m, M3, W, H, near_r, P, px, py)) continue;
                if (kPin) {  // culled in the forward when its box misses the image: no gradient
                    int rx, ry;
                    instance_box(P, __ldg(opacity + g), rx, ry);
                    if (box_off_image(px, py, rx, ry, W, H)) continue;
                }
                const float gpx = g0v.x, gpy = g0v.y, gc0 = g0v.z, gc1 = g0v.w, gc2 = g1v.x;
                dop += g1v.y;
                const float grgb[3] = {g1v.z, g1v.w, g2v.x};
                dsx += gpx * 0.5f * (float)W;
                dsy += gpy * 0.5f * (float)H;

                // conic -> Sigma~: dSigma~ = -conic dconic conic (symmetric parametrisation of the off-diagonal)
                const float inv = 1.f / P.det;
                const float c0 = P.C * inv, c1 = -P.B * inv, c2 = P.A * inv;
                const float dA = -(gc0 * c0 * c0 + gc1 * c0 * c1 + gc2 * c1 * c1);
                const float dB = -(2.f * gc0 * c0 * c1 + gc1 * (c0 * c2 + c1 * c1) + 2.f * gc2 * c1 * c2);
                const float dC = -(gc0 * c1 * c1 + gc1 * c1 * c2 + gc2 * c2 * c2);
                // Sigma~ = Tm Tm^T + 0.3 I: dTm0 = 2 dA Tm0 + dB Tm1, dTm1 = dB Tm0 + 2 dC Tm1
                float dTm[6];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    dTm[j] = 2.f * dA * P.Tm[j] + dB * P.Tm[3 + j];
                    dTm[3 + j] = dB * P.Tm[j] + 2.f * dC * P.Tm[3 + j];
                }
                // Tm = M M3: dM = dTm M3^T, dM3 += M^T dTm
                float dM[6];
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        dM[3 * r + k] =
                            dTm[3 * r] * M3[3 * k] + dTm[3 * r + 1] * M3[3 * k + 1] + dTm[3 * r + 2] * M3[3 * k + 2];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int j = 0; j < 3; ++j) dM3[3 * k + j] += P.M[k] * dTm[j] + P.M[3 + k] * dTm[3 + j];
                // M = J W: dJ = dM W^T
                float dJ[6];
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        dJ[3 * r + k] =
                            dM[3 * r] * w.Wr[3 * k] + dM[3 * r + 1] * w.Wr[3 * k + 1] + dM[3 * r + 2] * w.Wr[3 * k + 2];
                float dt[3];
                if (kPin) {
                    // dp/dt of Eq. 2 (unclamped), then dJ/dt: a ratio held at its bound is a constant
                    const float tx = P.t[0], ty = P.t[1], tz = P.t[2], iz = 1.f / tz, iz2 = iz * iz;
                    dt[0] = gpx * cam.fx * iz;
                    dt[1] = gpy * cam.fy * iz;
                    dt[2] = -(gpx * cam.fx * tx + gpy * cam.fy * ty) * iz2;
                    const float u = tx * iz, v = ty * iz;
                    dt[2] -= (dJ[0] * cam.fx + dJ[4] * cam.fy) * iz2;
                    if (u < -cam.limx || u > cam.limx) {
                        dt[2] += dJ[2] * cam.fx * fminf(fmaxf(u, -cam.limx), cam.limx) * iz2;
                    } else {
                        dt[0] -= dJ[2] * cam.fx * iz2;
                        dt[2] += dJ[2] * 2.f * cam.fx * tx * iz2 * iz;
                    }
                    if (v < -cam.limy || v > cam.limy) {
                        dt[2] += dJ[5] * cam.fy * fminf(fmaxf(v, -cam.limy), cam.limy) * iz2;
                    } else {
                        dt[1] -= dJ[5] * cam.fy * iz2;
                        dt[2] += dJ[5] * 2.f * cam.fy * ty * iz2 * iz;
                    }
                } else {
                    // dJ/dt (quotient rule on Eqs. 11-16; rho replaced by the guarded rg)
                    const float tx = P.t[0], ty = P.t[1], tz = P.t[2], tr = P.tr, rg = P.rg;
                    float drg[3];
                    if (P.rho >= kPoleGuard * tr) {
                        drg[0] = tx / rg; drg[1] = 0.f; drg[2] = tz / rg;
                    } else {
                        drg[0] = kPoleGuard * tx / tr; drg[1] = kPoleGuard * ty / tr; drg[2] = kPoleGuard * tz / tr;
                    }
                    const float tr2 = tr * tr, tr4 = tr2 * tr2, rg2 = rg * rg, rg3 = rg2 * rg;
                    // p(t): dp/dt = J (Eqs. 11-16 are exactly dp/ds * ds/dt)
#pragma unroll
                    for (int k = 0; k < 3; ++k) dt[k] = gpx * P.J[k] + gpy * P.J[3 + k];
                    const float e00 = dJ[0], e02 = dJ[2], e10 = dJ[3], e11 = dJ[4], e12 = dJ[5];
                    // J00 = a tz / rg^2
                    const float k00 = -2.f * a * tz / rg3;
                    // J02 = -a tx / rg^2
                    const float k02 = 2.f * a * tx / rg3;
                    // J10 = -b tx ty / (tr^2 rg), J12 = -b tz ty / (tr^2 rg)
                    const float q1 = b / (tr2 * rg);
                    const float q1t = 2.f * b / (tr4 * rg);     // derivative of 1/tr^2 part: + 2 b tx ty t / (tr^4 rg)
                    const float q1r = b / (tr2 * rg2);          // derivative of 1/rg part:  + b tx ty drg / (tr^2 rg^2)
                    // J11 = b rg / tr^2
                    const float k11r = b / tr2, k11t = -2.f * b * rg / tr4;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float ex = (k == 0) ? 1.f : 0.f, ey = (k == 1) ? 1.f : 0.f, ez = (k == 2) ? 1.f : 0.f;
                        float acc = e00 * (a * ez / rg2 + k00 * drg[k]);
                        acc += e02 * (-a * ex / rg2 + k02 * drg[k]);
                        acc += e10 * (-q1 * (ty * ex + tx * ey) + q1t * tx * ty * P.t[k] + q1r * tx * ty * drg[k]);
                        acc += e11 * (k11r * drg[k] + k11t * P.t[k]);
                        acc += e12 * (-q1 * (ty * ez + tz * ey) + q1t * tz * ty * P.t[k] + q1r * tz * ty * drg[k]);
                        dt[k] += acc;
                    }
                }
                // t = W m + t_cw
#pragma unroll
                for (int j = 0; j < 3; ++j) dm[j] += w.Wr[j] * dt[0] + w.Wr[3 + j] * dt[1] + w.Wr[6 + j] * dt[2];

                // colour: c = max(sum_k Y_k(d) sh_k + 0.5, 0), d = (m - c_cam) / |m - c_cam|
                float d[3], Y[16];
                const float dist = view_dir(w, m, d);
                sh_eval<K>(d[0], d[1], d[2], Y);
                float wk[16];
                float gm[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < K; ++k) acc = fmaf(Y[k], shc[3 * k + ch], acc);
                    gm[ch] = (acc + 0.5f > 0.f) ? grgb[ch] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    wk[k] = shc[3 * k] * gm[0] + shc[3 * k + 1] * gm[1] + shc[3 * k + 2] * gm[2];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) dshc[3 * k + ch] += Y[k] * gm[ch];
                }
                const float3 gd = sh_grad_dot<K>(d[0], d[1], d[2], wk);
                const float dd = gd.x * d[0] + gd.y * d[1] + gd.z * d[2];
                const float idist = 1.f / dist;
                dm[0] += (gd.x - d[0] * dd) * idist;
                dm[1] += (gd.y - d[1] * dd) * idist;
                dm[2] += (gd.z - d[2] * dd) * idist;
            }
        }

        // M3 = R diag(s): ds_j = sum_i dM3_ij R_ij, dR_ij = dM3_ij s_j
        float dR[9], ds[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            ds[j] = dM3[j] * R[j] + dM3[3 + j] * R[3 + j] + dM3[6 + j] * R[6 + j];
#pragma unroll
            for (int i = 0; i < 3; ++i) dR[3 * i + j] = dM3[3 * i + j] * s[j];
        }
        // R(q^) -> q^
        const float qw = qn[0], qx = qn[1], qy = qn[2], qz = qn[3];
        float dq[4];
        dq[0] = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
        dq[1] = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] + qw * dR[7] - 2.f * qx * dR[8]);
        dq[2] = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] + qz * dR[7] - 2.f * qy * dR[8]);
        dq[3] = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] + qy * dR[5] + qx * dR[6] + qy * dR[7]);
        // through q^ = q / |q|
        const float dot = dq[0] * qw + dq[1] * qx + dq[2] * qy + dq[3] * qz;
        const float iq = 1.f / qnorm;
        reinterpret_cast<float4*>(d_quats)[g] =
            make_float4((dq[0] - qw * dot) * iq, (dq[1] - qx * dot) * iq, (dq[2] - qy * dot) * iq, (dq[3] - qz * dot) * iq);
        d_means[3 * g] = dm[0];
        d_means[3 * g + 1] = dm[1];
        d_means[3 * g + 2] = dm[2];
        d_scales[3 * g] = ds[0];
        d_scales[3 * g + 1] = ds[1];
        d_scales[3 * g + 2] = ds[2];
        d_opacity[g] = dop;
        reinterpret_cast<float2*>(d_screen)[g] = make_float2(dsx, dsy);
    }
    __syncthreads();
    float* dst = d_sh + (size_t)g0 * KK;
    for (int e = threadIdx.x; e < cnt * KK; e += blockDim.x) {
        const int t = e / KK;
        dst[e] = s_dsh[t * STRIDE + (e - t * KK)];
    }
}

template <int K>
cudaError_t preprocess_k(const omnigs_config& cfg, int64_t n, const float* means, const float* scales,
                         const float* quats, const float* opacity, const float* sh, const float* viewmats,
                         omnigs_splat* splats, uint64_t* depth_keys, int gbits, uint64_t* splat_count,
                         cudaStream_t stream) {
    const size_t smem = sizeof(float) * (kPreThreads * (3 * K + 1) + 16 * cfg.num_views);
    auto kern = depth_keys ? preprocess_kernel<K, true> : preprocess_kernel<K, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((n + kPreThreads - 1) / kPreThreads);
    ProfScope prof("preprocess_fwd", stream);
    kern<<<blocks, kPreThreads, smem, stream>>>((int)n, cfg.num_views, cfg.width, cfg.height, cfg.near_r, make_cam(cfg),
                                                means, scales, quats, opacity, sh, viewmats,
                                                reinterpret_cast<float4*>(splats),
                                                reinterpret_cast<unsigned long long*>(depth_keys), gbits,
                                                reinterpret_cast<unsigned long long*>(splat_count));
    return cudaGetLastError();
}

template <int K>
cudaError_t preprocess_bwd_k(const omnigs_config& cfg, int64_t n, const float* means, const float* scales,
                             const float* quats, const float* opacity, const float* sh, const float* viewmats,
                             const omnigs_splat_grad* grads,
                             float* d_means, float* d_scales, float* d_quats, float* d_opacity, float* d_sh,
                             float* d_screen, cudaStream_t stream) {
    const size_t smem = sizeof(float) * (2 * kPreBwdThreads * (3 * K + 1) + 16 * cfg.num_views);
    auto kern = cfg.camera == OMNIGS_CAMERA_PINHOLE ? preprocess_bwd_kernel<K, true> : preprocess_bwd_kernel<K, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((n + kPreBwdThreads - 1) / kPreBwdThreads);
    ProfScope prof("preprocess_bwd", stream);
    kern<<<blocks, kPreBwdThreads, smem, stream>>>((int)n, cfg.num_views, cfg.width, cfg.height, cfg.near_r, make_cam(cfg),
                                                means, scales, quats, opacity, sh, viewmats,
                                                reinterpret_cast<const float4*>(grads), d_means, d_scales, d_quats,
                                                d_opacity, d_sh, d_screen);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_preprocess(const omnigs_config& cfg, int64_t n, const float* means, const float* scales,
                              const float* quats, const float* opacity, const float* sh, const float* viewmats,
                              omnigs_splat* splats, cudaStream_t stream, uint64_t* depth_keys, int gbits,
                              uint64_t* splat_count) {
    if (n == 0) return cudaSuccess;
#define OMNIGS_PRE(K) preprocess_k<K>(cfg, n, means, scales, quats, opacity, sh, viewmats, splats, depth_keys, gbits, \
                                      splat_count, stream)
    switch (cfg.sh_degree) {
        case 0: return OMNIGS_PRE(1);
        case 1: return OMNIGS_PRE(4);
        case 2: return OMNIGS_PRE(9);
        default: return OMNIGS_PRE(16);
    }
#undef OMNIGS_PRE
}

cudaError_t launch_preprocess_bwd(const omnigs_config& cfg, int64_t n, const float* means, const float* scales,
                                  const float* quats, const float* opacity, const float* sh, const float* viewmats,
                                  const omnigs_splat_grad* grads, float* d_means, float* d_scales, float* d_quats,
                                  float* d_opacity, float* d_sh, float* d_screen, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    switch (cfg.sh_degree) {
        case 0: return preprocess_bwd_k<1>(cfg, n, means, scales, quats, opacity, sh, viewmats, grads, d_means, d_scales, d_quats, d_opacity, d_sh, d_screen, stream);
        case 1: return preprocess_bwd_k<4>(cfg, n, means, scales, quats, opacity, sh, viewmats, grads, d_means, d_scales, d_quats, d_opacity, d_sh, d_screen, stream);
        case 2: return preprocess_bwd_k<9>(cfg, n, means, scales, quats, opacity, sh, viewmats, grads, d_means, d_scales, d_quats, d_opacity, d_sh, d_screen, stream);
        default: return preprocess_bwd_k<16>(cfg, n, means, scales, quats, opacity, sh, viewmats, grads, d_means, d_scales, d_quats, d_opacity, d_sh, d_screen, stream);
    }
}

}  // namespace omnigs
