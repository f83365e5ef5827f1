// C-ABI entry points of the rasterizer: argument validation, workspace layout, the optional kernel profiler and the
// dispatch to the stage launchers. See include/omnigs.h for the contract of every call.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

static_assert(sizeof(omnigs_splat) == 48, "omnigs_splat is three float4");

namespace omnigs {

int num_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 148;
    return sms;
}

WsLayout ws_layout(const omnigs_config& cfg, int64_t n, int64_t capacity) {
    WsLayout L;
    const size_t total = (size_t)n * cfg.num_views;
    const size_t nb = std::max<size_t>(1, (total + kBinThreads - 1) / kBinThreads);
    L.loss_blocks = kLossBlocks;
    size_t off = 0;
    L.header = off;         off += align256(sizeof(WsHeader));
    L.loss_partials = off;  off += align256(sizeof(float) * L.loss_blocks);
    // per-tile sums of the forward with the L1 loss fused in (omnigs_render_fwd_l1)
    L.loss_tiles = off;     off += align256(sizeof(float) * (size_t)cfg.num_views * (cfg.width / cfg.tile) *
                                            (cfg.height / cfg.tile));
    L.hist = off;           off += align256(sizeof(unsigned) * kRadixMax * ((size_t)num_sms() * kSortCtasPerSm + 1));
    const bool bk = bucketed_binning(cfg, n);  // bucket entries are 32 bits, radix-sort keys 64
    // (+16 bytes: the column pass's bulk copies read whole 16-byte words, up to 12 bytes past the last entry)
    const size_t alt_bytes = (bk ? sizeof(unsigned) : sizeof(unsigned long long)) * (size_t)capacity + 16;
    L.alt_keys = off;       off += align256(alt_bytes);
    L.depth_keys = off;     off += align256(sizeof(unsigned long long) * total);
    L.depth_keys_alt = off; off += align256(sizeof(unsigned long long) * total);
    L.depth_vals_alt = off; off += align256(sizeof(uint32_t) * total);
    L.block_sums = off;     off += align256(sizeof(unsigned) * nb);
    L.block_offsets = off;  off += align256(sizeof(unsigned long long) * nb);
    L.piece_start = off;    off += align256(sizeof(unsigned) * nb);
    L.row_base = off;       off += align256(sizeof(unsigned) * nb);
    L.row_count = off;      off += align256(sizeof(unsigned) * nb);
    L.piece_block = off;    off += align256(sizeof(unsigned) * ((size_t)capacity / kEmitPiece + 1));
    // visibility blocks per view, their counts and one ballot word per 32 slots
    const size_t nbv = std::max<size_t>(1, ((size_t)n + kVisSlots - 1) / kVisSlots);
    L.vis_sums = off;       off += align256(sizeof(unsigned) * nbv * cfg.num_views);
    L.vis_start = off;      off += align256(sizeof(unsigned) * ((size_t)cfg.num_views + 1));
    L.vis_mask = off;       off += align256(sizeof(unsigned) * (kVisSlots / 32) * nbv * cfg.num_views);
    // bucketed instance order: row words in their own region (the emission fills alt_keys)
    const size_t nbkt = bk ? (size_t)cfg.num_views * (cfg.height / cfg.tile) : 0;
    const size_t chunks = bk ? (size_t)capacity / kColChunk + nbkt + 1 : 0;
    L.row_cap = bk ? (size_t)capacity / 2 + 1 : 0;
    L.rows = off;           off += align256(sizeof(unsigned long long) * L.row_cap);
    L.rows_off = off;       off += align256(sizeof(unsigned) * L.row_cap);
    L.bkt_counts = off;     off += align256(sizeof(unsigned) * nbkt * (bk ? blocks_per_view_max(n) : 0));
    L.bkt_total = off;      off += align256(sizeof(unsigned long long) * nbkt);
    L.bkt_base = off;       off += align256(sizeof(unsigned long long) * nbkt);
    L.bkt_eff = off;        off += align256(sizeof(unsigned long long) * nbkt);
    L.col_start = off;      off += align256(sizeof(unsigned) * (nbkt + 1));
    L.col_hist = off;       off += align256(sizeof(unsigned) * chunks * (bk ? cfg.width / cfg.tile : 0));
    L.unstored_list = off;  off += align256(sizeof(unsigned) * (bk ? nb : 0));
    L.total = off;
    return L;
}

// ------------------------------------------------------------------------------------------------ profiler

namespace {
struct ProfRecord {
    std::string name;
    int kernels;
    cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_prof_records;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_pool;
size_t g_prof_used = 0;

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return true;
    return st != cudaStreamCaptureStatusNone;
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t s, int kernels) : slot(-1), stream(s) {
    if (!g_prof_on || capturing(s)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_used == g_prof_pool.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
        g_prof_pool.push_back({a, b});
    }
    auto ev = g_prof_pool[g_prof_used++];
    g_prof_records.push_back({name, kernels, ev.first, ev.second});
    slot = (int)g_prof_records.size() - 1;
    cudaEventRecord(ev.first, s);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof_records[slot].stop, stream);
}

// The configuration checks shared by every entry point that takes an omnigs_config.
bool valid_cfg(const omnigs_config* c) {
    if (!c) return false;
    if (c->tile != 8 && c->tile != 16 && c->tile != 32) return false;
    if (c->width <= 0 || c->height <= 0 || c->width % c->tile || c->height % c->tile) return false;
    if (c->width > 65536 || c->height > 65536) return false;  // instance-box half-extents are 16-bit
    if (c->num_views < 1 || c->num_views > 4096) return false;
    if (c->sh_degree < 0 || c->sh_degree > 3) return false;
    if (!std::isfinite(c->near_r) || c->near_r < 0.f) return false;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(c->bg[i])) return false;
    for (const int ppt : {c->pixels_per_thread, c->adjoint_pixels_per_thread}) {
        if (ppt != 0 && ppt != 2 && ppt != 4 && ppt != 8) return false;
        if (ppt > 2 && c->tile == 8) return false;
    }
    if (c->camera != OMNIGS_CAMERA_EQUIRECT && c->camera != OMNIGS_CAMERA_PINHOLE) return false;
    if (c->camera == OMNIGS_CAMERA_PINHOLE &&
        !(std::isfinite(c->fx) && std::isfinite(c->fy) && c->fx > 0.f && c->fy > 0.f && std::isfinite(c->cx) &&
          std::isfinite(c->cy)))
        return false;
    const uint64_t tiles = (uint64_t)(c->width / c->tile) * (uint64_t)(c->height / c->tile) * (uint64_t)c->num_views;
    return tiles < (1ull << 31);
}

}  // namespace omnigs

using namespace omnigs;

namespace {

bool valid_n(const omnigs_config* c, int64_t n) {
    return n >= 0 && (uint64_t)n * (uint64_t)c->num_views < (1ull << 32) && n < (1ll << 31);
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

omnigs_status from_cuda(cudaError_t e) { return e == cudaSuccess ? OMNIGS_OK : OMNIGS_E_CUDA; }

}  // namespace

extern "C" {

int omnigs_version(void) { return 100; }

const char* omnigs_status_string(omnigs_status s) {
    switch (s) {
        case OMNIGS_OK: return "ok";
        case OMNIGS_E_INVALID: return "invalid argument";
        case OMNIGS_E_CAPACITY: return "instance capacity exceeded";
        case OMNIGS_E_CUDA: return "CUDA error";
        case OMNIGS_E_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

size_t omnigs_workspace_size(const omnigs_config* cfg, int64_t n, int64_t capacity) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n) || capacity < 0 || capacity >= (1ll << 32)) return 0;
    return ws_layout(*cfg, n, capacity).total;
}

omnigs_status omnigs_preprocess(const omnigs_config* cfg, int64_t n, const float* means, const float* scales,
                                const float* quats, const float* opacity, const float* sh, const float* viewmats,
                                omnigs_splat* splats, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n)) return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    if (!means || !scales || !quats || !opacity || !sh || !viewmats || !splats) return OMNIGS_E_INVALID;
    if (!aligned(quats, 16) || !aligned(splats, 16)) return OMNIGS_E_INVALID;
    return from_cuda(launch_preprocess(*cfg, n, means, scales, quats, opacity, sh, viewmats, splats,
                                       (cudaStream_t)stream));
}

omnigs_status omnigs_bin(const omnigs_config* cfg, int64_t n, const omnigs_splat* splats, uint32_t* order,
                         uint64_t* keys, int64_t capacity, void* workspace, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n) || capacity < 0 || capacity >= (1ll << 32)) return OMNIGS_E_INVALID;
    if (!workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    if (n > 0 && (!splats || !order || !aligned(splats, 16))) return OMNIGS_E_INVALID;
    if (capacity > 0 && (!keys || !aligned(keys, 8))) return OMNIGS_E_INVALID;
    const WsLayout L = ws_layout(*cfg, n, capacity);
    return from_cuda(launch_bin(*cfg, n, splats, order, keys, capacity, L, (char*)workspace, (cudaStream_t)stream));
}

omnigs_status omnigs_preprocess_bin(const omnigs_config* cfg, int64_t n, const float* means, const float* scales,
                                    const float* quats, const float* opacity, const float* sh, const float* viewmats,
                                    omnigs_splat* splats, uint32_t* order, uint64_t* keys, int64_t capacity,
                                    void* workspace, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n) || capacity < 0 || capacity >= (1ll << 32)) return OMNIGS_E_INVALID;
    if (!workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    if (n > 0 && (!means || !scales || !quats || !opacity || !sh || !viewmats || !splats || !order))
        return OMNIGS_E_INVALID;
    if (n > 0 && (!aligned(quats, 16) || !aligned(splats, 16))) return OMNIGS_E_INVALID;
    if (capacity > 0 && (!keys || !aligned(keys, 8))) return OMNIGS_E_INVALID;
    const WsLayout L = ws_layout(*cfg, n, capacity);
    char* ws = (char*)workspace;
    const cudaStream_t st = (cudaStream_t)stream;
    int gbits = 0;
    if (n == 0 || !packed_depth_keys(*cfg, n, &gbits)) {  // the two calls one after the other
        cudaError_t e = launch_preprocess(*cfg, n, means, scales, quats, opacity, sh, viewmats, splats, st);
        if (e != cudaSuccess) return from_cuda(e);
        return from_cuda(launch_bin(*cfg, n, splats, order, keys, capacity, L, ws, st));
    }
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
    if (e == cudaSuccess)
        e = launch_preprocess(*cfg, n, means, scales, quats, opacity, sh, viewmats, splats, st,
                              reinterpret_cast<uint64_t*>(ws + L.depth_keys), gbits,
                              reinterpret_cast<uint64_t*>(&hdr->splat_count));
    if (e == cudaSuccess) e = launch_bin(*cfg, n, splats, order, keys, capacity, L, ws, st, true);
    return from_cuda(e);
}

omnigs_status omnigs_sort(const omnigs_config* cfg, int64_t n, int64_t capacity, uint64_t* keys, uint32_t* ranges,
                          void* workspace, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n) || capacity < 0 || capacity >= (1ll << 32)) return OMNIGS_E_INVALID;
    if (!ranges || !workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    if (capacity > 0 && (!keys || !aligned(keys, 8))) return OMNIGS_E_INVALID;
    const WsLayout L = ws_layout(*cfg, n, capacity);
    return from_cuda(launch_sort(*cfg, n, capacity, keys, ranges, L, (char*)workspace, (cudaStream_t)stream));
}

omnigs_status omnigs_render_fwd(const omnigs_config* cfg, int64_t n, const omnigs_splat* splats,
                                const uint32_t* ranges, const uint64_t* keys, const uint32_t* order, float* out_rgb,
                                float* out_T, uint32_t* out_ncontrib, uint32_t* out_count, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n)) return OMNIGS_E_INVALID;
    if (!ranges || !out_rgb || !out_T || !out_ncontrib) return OMNIGS_E_INVALID;
    if (n > 0 && (!splats || !keys || !order || !aligned(splats, 16))) return OMNIGS_E_INVALID;
    return from_cuda(launch_render_fwd(*cfg, n, splats, ranges, keys, order, out_rgb, out_T, out_ncontrib, out_count,
                                       nullptr, (cudaStream_t)stream));
}

omnigs_status omnigs_render_fwd_l1(const omnigs_config* cfg, int64_t n, const omnigs_splat* splats,
                                   const uint32_t* ranges, const uint64_t* keys, const uint32_t* order,
                                   const float* target, float* out_rgb, float* out_T, uint32_t* out_ncontrib,
                                   float* dL_drgb, float* loss, void* workspace, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n)) return OMNIGS_E_INVALID;
    if (!ranges || !out_rgb || !out_T || !out_ncontrib) return OMNIGS_E_INVALID;
    if (n > 0 && (!splats || !keys || !order || !aligned(splats, 16))) return OMNIGS_E_INVALID;
    if (!target || !dL_drgb || !loss || !workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    const WsLayout L = ws_layout(*cfg, 0, 0);  // the per-tile sums sit at a fixed offset
    const FwdL1 l1 = {target, dL_drgb, loss, reinterpret_cast<float*>((char*)workspace + L.loss_tiles)};
    return from_cuda(launch_render_fwd(*cfg, n, splats, ranges, keys, order, out_rgb, out_T, out_ncontrib, nullptr,
                                       &l1, (cudaStream_t)stream));
}

omnigs_status omnigs_l1_loss(const omnigs_config* cfg, const float* rgb, const float* target, float* dL_drgb,
                             float* loss, void* workspace, omnigs_stream_t stream) {
    if (!valid_cfg(cfg)) return OMNIGS_E_INVALID;
    if (!rgb || !target || !dL_drgb || !loss || !workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    if (!aligned(rgb, 16) || !aligned(target, 16) || !aligned(dL_drgb, 16)) return OMNIGS_E_INVALID;
    const WsLayout L = ws_layout(*cfg, 0, 0);  // the header and the loss partials sit at fixed offsets
    return from_cuda(launch_l1(*cfg, 0, cfg->height, rgb, target, dL_drgb, loss, L, (char*)workspace,
                               (cudaStream_t)stream));
}

omnigs_status omnigs_l1_loss_rows(const omnigs_config* cfg, int32_t row_begin, int32_t row_end, const float* rgb,
                                  const float* target, float* dL_drgb, float* loss, void* workspace,
                                  omnigs_stream_t stream) {
    if (!valid_cfg(cfg)) return OMNIGS_E_INVALID;
    if (row_begin < 0 || row_end > cfg->height || row_begin >= row_end) return OMNIGS_E_INVALID;
    if (!rgb || !target || !dL_drgb || !loss || !workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    if (!aligned(rgb, 16) || !aligned(target, 16) || !aligned(dL_drgb, 16)) return OMNIGS_E_INVALID;
    const WsLayout L = ws_layout(*cfg, 0, 0);
    return from_cuda(launch_l1(*cfg, row_begin, row_end, rgb, target, dL_drgb, loss, L, (char*)workspace,
                               (cudaStream_t)stream));
}

size_t omnigs_dssim_scratch_size(const omnigs_config* cfg) {
    if (!valid_cfg(cfg)) return 0;
    return dssim_scratch_bytes(*cfg);
}

omnigs_status omnigs_dssim_loss(const omnigs_config* cfg, float lambda, const float* rgb, const float* target,
                                float* dL_drgb, float* loss, void* scratch, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !(lambda >= 0.f && lambda <= 1.f)) return OMNIGS_E_INVALID;
    if (!rgb || !target || !dL_drgb || !loss || !scratch || !aligned(scratch, 256)) return OMNIGS_E_INVALID;
    return from_cuda(launch_dssim(*cfg, lambda, rgb, target, dL_drgb, loss, (char*)scratch, (cudaStream_t)stream));
}

namespace {
bool valid_rows(int64_t n, int32_t K) {
    return n >= 0 && n < (1ll << 31) && (K == 1 || K == 4 || K == 9 || K == 16);
}
}  // namespace

omnigs_status omnigs_adam_step(int64_t n, int32_t K, const omnigs_adam_config* cfg, int64_t step, float* params,
                               float* m, float* v, const float* d_means, const float* d_scales, const float* d_quats,
                               const float* d_opacity, const float* d_sh, float* means, float* scales, float* quats,
                               float* opacity, float* sh, omnigs_stream_t stream) {
    if (!cfg || !valid_rows(n, K) || step < 1) return OMNIGS_E_INVALID;
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f))
        return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    if (!params || !m || !v || !d_means || !d_scales || !d_quats || !d_opacity || !d_sh || !means || !scales ||
        !quats || !opacity || !sh)
        return OMNIGS_E_INVALID;
    return from_cuda(launch_adam(n, K, *cfg, step, params, m, v, d_means, d_scales, d_quats, d_opacity, d_sh, means,
                                 scales, quats, opacity, sh, (cudaStream_t)stream));
}

omnigs_status omnigs_publish_params(int64_t n, int32_t K, const float* params, float* means, float* scales,
                                    float* quats, float* opacity, float* sh, omnigs_stream_t stream) {
    if (!valid_rows(n, K)) return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    if (!params || !means || !scales || !quats || !opacity || !sh) return OMNIGS_E_INVALID;
    return from_cuda(launch_publish(n, K, params, means, scales, quats, opacity, sh, (cudaStream_t)stream));
}

omnigs_status omnigs_densify_stats(const omnigs_config* cfg, int64_t n, const omnigs_splat* splats,
                                   const omnigs_splat_grad* grads, float* accum, int32_t* count, float* max_radius,
                                   omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n)) return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    if (!splats || !grads || !accum || !count || !max_radius || !aligned(splats, 16) || !aligned(grads, 16))
        return OMNIGS_E_INVALID;
    return from_cuda(launch_densify_stats(*cfg, n, splats, grads, accum, count, max_radius, (cudaStream_t)stream));
}

size_t omnigs_densify_workspace_size(int64_t n) {
    if (n < 0 || n >= (1ll << 31)) return 0;
    return densify_workspace_bytes(n);
}

omnigs_status omnigs_densify(int64_t n, int32_t K, const omnigs_densify_config* cfg, const float* params,
                             const float* m, const float* v, const float* accum, const int32_t* count,
                             const float* max_radius, const float* normals, float* params_out, float* m_out,
                             float* v_out, int64_t* n_out, void* workspace, omnigs_stream_t stream) {
    if (!cfg || !valid_rows(n, K) || !n_out) return OMNIGS_E_INVALID;
    if (!(cfg->extent > 0.f)) return OMNIGS_E_INVALID;
    if (n == 0) return from_cuda(cudaMemsetAsync(n_out, 0, sizeof(int64_t), (cudaStream_t)stream));
    if (!params || !m || !v || !accum || !count || !max_radius || !normals || !params_out || !m_out || !v_out ||
        !workspace || !aligned(workspace, 256))
        return OMNIGS_E_INVALID;
    return from_cuda(launch_densify(n, K, *cfg, params, m, v, accum, count, max_radius, normals, params_out, m_out,
                                    v_out, reinterpret_cast<long long*>(n_out), (char*)workspace,
                                    (cudaStream_t)stream));
}

omnigs_status omnigs_reset_opacity(int64_t n, int32_t K, float value, float* params, float* m, float* v,
                                   float* opacity, omnigs_stream_t stream) {
    if (!valid_rows(n, K) || !(value > 0.f && value < 1.f)) return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    if (!params || !m || !v) return OMNIGS_E_INVALID;
    return from_cuda(launch_reset_opacity(n, K, value, params, m, v, opacity, (cudaStream_t)stream));
}

omnigs_status omnigs_equirect_crop(int32_t V, int32_t eq_width, int32_t eq_height, const float* equirect,
                                   const float* rotations, int32_t width, int32_t height, float fx, float fy, float cx,
                                   float cy, float* out, omnigs_stream_t stream) {
    if (V < 0 || eq_width <= 0 || eq_height <= 0 || width <= 0 || height <= 0) return OMNIGS_E_INVALID;
    if (eq_width > (1 << 20) || eq_height > (1 << 20) || width > (1 << 20) || height > (1 << 20) || V > 65535)
        return OMNIGS_E_INVALID;
    if (!(std::isfinite(fx) && std::isfinite(fy) && fx > 0.f && fy > 0.f && std::isfinite(cx) && std::isfinite(cy)))
        return OMNIGS_E_INVALID;
    if (V == 0) return OMNIGS_OK;
    if (!equirect || !rotations || !out) return OMNIGS_E_INVALID;
    return from_cuda(launch_crop(V, eq_width, eq_height, equirect, rotations, width, height, fx, fy, cx, cy, out,
                                 (cudaStream_t)stream));
}

omnigs_status omnigs_render_bwd(const omnigs_config* cfg, int64_t n, const omnigs_splat* splats,
                                const uint32_t* ranges, const uint64_t* keys, const uint32_t* order,
                                const float* out_T, const uint32_t* ncontrib, const float* dL_drgb,
                                omnigs_splat_grad* grads, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n)) return OMNIGS_E_INVALID;
    if (!ranges || !out_T || !ncontrib || !dL_drgb) return OMNIGS_E_INVALID;
    if (n > 0 && (!splats || !keys || !order || !grads || !aligned(splats, 16) || !aligned(grads, 16)))
        return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    return from_cuda(launch_render_bwd(*cfg, n, splats, ranges, keys, order, out_T, ncontrib, dL_drgb, grads,
                                       (cudaStream_t)stream));
}

omnigs_status omnigs_preprocess_bwd(const omnigs_config* cfg, int64_t n, const float* means, const float* scales,
                                    const float* quats, const float* opacity, const float* sh,
                                    const float* viewmats, const omnigs_splat_grad* grads, float* d_means,
                                    float* d_scales, float* d_quats, float* d_opacity, float* d_sh,
                                    float* d_screen, omnigs_stream_t stream) {
    if (!valid_cfg(cfg) || !valid_n(cfg, n)) return OMNIGS_E_INVALID;
    if (n == 0) return OMNIGS_OK;
    if (!means || !scales || !quats || !opacity || !sh || !viewmats || !grads) return OMNIGS_E_INVALID;
    if (!d_means || !d_scales || !d_quats || !d_opacity || !d_sh || !d_screen) return OMNIGS_E_INVALID;
    if (!aligned(quats, 16) || !aligned(grads, 16) || !aligned(d_quats, 16) || !aligned(d_screen, 8))
        return OMNIGS_E_INVALID;
    return from_cuda(launch_preprocess_bwd(*cfg, n, means, scales, quats, opacity, sh, viewmats, grads, d_means,
                                           d_scales, d_quats, d_opacity, d_sh, d_screen, (cudaStream_t)stream));
}

omnigs_status omnigs_instance_count(const void* workspace, int64_t* count, omnigs_stream_t stream) {
    if (!workspace || !count || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    WsHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return OMNIGS_E_CUDA;
    *count = (int64_t)h.count;
    return OMNIGS_OK;
}

omnigs_status omnigs_last_error(void* workspace, omnigs_stream_t stream) {
    if (!workspace || !aligned(workspace, 256)) return OMNIGS_E_INVALID;
    WsHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return OMNIGS_E_CUDA;
    if (h.error == 0) return OMNIGS_OK;
    const unsigned zero = 0;
    e = cudaMemcpyAsync((char*)workspace + offsetof(WsHeader, error), &zero, sizeof(zero), cudaMemcpyHostToDevice,
                        (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (h.error & kErrCapacity) return OMNIGS_E_CAPACITY;
    if (h.error & kErrConsistency) return OMNIGS_E_CUDA;
    return OMNIGS_E_TIMEOUT;
}

omnigs_status omnigs_profiler_enable(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = enable != 0;
    return OMNIGS_OK;
}

int omnigs_profiler_collect(omnigs_kernel_time* out, int max) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<omnigs_kernel_time> agg;
    for (auto& r : g_prof_records) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess)
            ms = 0.f;
        size_t k = 0;
        while (k < agg.size() && std::strncmp(agg[k].name, r.name.c_str(), sizeof(agg[k].name)) != 0) ++k;
        if (k == agg.size()) {
            omnigs_kernel_time t;
            std::memset(&t, 0, sizeof(t));
            std::strncpy(t.name, r.name.c_str(), sizeof(t.name) - 1);
            agg.push_back(t);
        }
        agg[k].launches += r.kernels;
        agg[k].total_ms += ms;
    }
    g_prof_records.clear();
    g_prof_used = 0;
    const int m = (int)std::min<size_t>(agg.size(), (size_t)std::max(max, 0));
    for (int i = 0; i < m; ++i) out[i] = agg[i];
    return (int)agg.size();
}

}  // extern "C"
