// Shared device definitions of the sm_103a rasterizer: constants of the method, the tile rectangle of a splat,
// the workspace layout and the kernel-launch helpers. Arithmetic of the individual stages lives in its own .cu file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "omnigs.h"

namespace omnigs {

// Method constants (3DGS conventions the paper inherits, Sec. 3.3).
constexpr float kPi = 3.14159265358979323846f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kDilation = 0.3f;        // low-pass dilation added to the 2x2 covariance
constexpr float kAlphaMax = 0.99f;       // alpha clamp (alphas below 1/255 are skipped: the factor 255 in the
                                         // pass threshold -log2(255 o) and in the box's q = 2 ln(255 o))
constexpr float kTStop = 1e-4f;          // stop once accumulated alpha would reach 0.9999
constexpr float kPoleGuard = 1e-6f;      // rho is kept >= 1e-6 t_r inside J
constexpr int kMaxRadius = 65535;        // instance-box half-extents are stored in 16 bits

constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrConsistency = 2u;  // a device-side consistency check failed (the access was skipped)
constexpr uint32_t kErrTimeout = 4u;      // a bounded device-side wait ran out (the data it guarded was skipped)

// Workspace header (first 256 bytes of every workspace).
struct WsHeader {
    unsigned long long count;        // total instances of the last bin (may exceed capacity)
    unsigned long long splat_count;  // V * n of the last bin
    unsigned int error;              // sticky device-side error bits
    unsigned int extra_pieces;       // bin_emit CTAs beyond one per block (blocks with many instances)
    float loss;
    unsigned int unstored;           // blocks whose row items did not fit the rows region (bucketed order)
    unsigned long long rows_used;    // row items bin_count has stored for bin_emit
};

struct Rect {
    int x0, nx, y0, ny;
};

// Tiles covered by the box of half-extents (rx, ry) around pixel floor(p): columns x0 .. x0 + nx - 1 modulo the
// column count (all columns, from 0, once the box is at least as wide as the image) when `wrap` (the equirectangular
// longitude seam), clipped to the image like the rows otherwise (pinhole camera).
// tile_shift = log2(tile) (tiles are powers of two): an arithmetic right shift is the floor quotient.
__device__ inline Rect splat_rect(float px, float py, int rx, int ry, int tiles_x, int tiles_y, int tile_shift,
                                  bool wrap) {
    Rect R;
    int ix = (int)floorf(px), iy = (int)floorf(py);
    int x0 = (ix - rx) >> tile_shift, x1 = (ix + rx) >> tile_shift;
    if (!wrap) {
        x0 = x0 < 0 ? 0 : x0;
        x1 = x1 > tiles_x - 1 ? tiles_x - 1 : x1;
    }
    int nx = x1 >= x0 ? x1 - x0 + 1 : 0;
    if (nx >= tiles_x) {
        x0 = 0;
        nx = tiles_x;
    }
    int y0 = (iy - ry) >> tile_shift, y1 = (iy + ry) >> tile_shift;
    y0 = y0 < 0 ? 0 : y0;
    y1 = y1 > tiles_y - 1 ? tiles_y - 1 : y1;
    R.x0 = x0;
    R.nx = nx;
    R.y0 = y0;
    R.ny = y1 >= y0 ? y1 - y0 + 1 : 0;
    return R;
}

// Workspace layout (all offsets 256-byte aligned). Every region depends on the configuration and the capacity only.
// Order: fixed-size regions, then those sized by the capacity, then those sized by n, so that calls which do not take
// n or the capacity find their regions at the same offsets as omnigs_bin.
struct WsLayout {
    size_t header, loss_partials, loss_tiles, hist, alt_keys, depth_keys, depth_keys_alt, depth_vals_alt, block_sums,
        block_offsets, piece_start, piece_block, row_base, row_count, vis_sums, vis_start, vis_mask,
        // bucketed instance order (see bucketed_binning): stored row words and their bucket offsets, per-block
        // bucket counts, bucket totals and bases, chunk starts and the column pass's per-chunk histograms
        rows, rows_off, bkt_counts, bkt_total, bkt_base, bkt_eff, col_start, col_hist, unstored_list, total;
    size_t row_cap;  // row words the rows region holds
    int loss_blocks;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kBinThreads = 256;
constexpr int kSplatsPerThread = 1;  // splats per thread in the instance passes
constexpr int kBinSplats = kBinThreads * kSplatsPerThread;
constexpr int kEmitPiece = 16384;  // instances one bin_emit CTA writes at most (a block with more is split)
constexpr int kVisPerThread = 4;                      // slots per thread of the visibility pass (pinhole views)
constexpr int kVisSlots = kBinThreads * kVisPerThread;
constexpr int kRadixMax = 512;       // radix-sort digits of up to 9 bits
constexpr int kSortCtasPerSm = 12;   // radix-sort grid: up to this many CTAs per SM
constexpr int kMaxBucketRows = 128;  // tile rows per view of the bucketed instance order
constexpr int kMaxBucketCols = 256;  // tile columns per view of its column pass (digits of at most 8 bits)
constexpr int kColChunk = 4096;        // keys per CTA of the column pass
constexpr int kBucketRankBitsMax = 24;  // bucket entries: 8 tile-column bits + up to 24 rank bits
constexpr int kLossThreads = 256;
constexpr int kLossBlocks = 1024;

int num_sms();
WsLayout ws_layout(const omnigs_config &cfg, int64_t n, int64_t capacity);

// Whether omnigs_bin emits the instances bucketed by (view, tile row), so that omnigs_sort orders them with one
// counting pass over the tile column within each bucket (instead of a radix sort over all tile-key bits): when every
// CTA of 256 consecutive splats of the (view, depth) order spans at most two views (n >= 256), a view has at most
// kMaxBucketRows tile rows and kMaxBucketCols tile columns, and a bucket entry (tile column << rank bits | depth rank)
// fits 32 bits (n <= 2^24).
int rank_bits_for(int64_t n);
inline bool bucketed_binning(const omnigs_config &cfg, int64_t n) {
    return n >= kBinSplats && n <= (int64_t(1) << kBucketRankBitsMax) && cfg.height / cfg.tile <= kMaxBucketRows &&
           cfg.width / cfg.tile <= kMaxBucketCols;
}
// Blocks of 256 positions a view's splats can share: its own, plus one straddling the next view.
inline int64_t blocks_per_view_max(int64_t n) { return (n + kBinSplats - 1) / kBinSplats + 1; }

// Whether a configuration is one every entry point accepts (image shape, tile, views, SH degree, camera, schedule).
bool valid_cfg(const omnigs_config *c);

// Kernel launches report their name and stream to the optional profiler.
// Brackets the `kernels` launches of one named stage with CUDA events while the profiler is on.
struct ProfScope {
    int slot;
    cudaStream_t stream;
    ProfScope(const char *name, cudaStream_t s, int kernels = 1);
    ~ProfScope();
};

// Stage launchers (defined in preprocess.cu, binsort.cu, render.cu). Each returns cudaGetLastError().
// depth_keys (optional): also write the depth sort's packed keys (see packed_depth_keys) and the splat count.
cudaError_t launch_preprocess(const omnigs_config &cfg, int64_t n, const float *means, const float *scales,
                              const float *quats, const float *opacity, const float *sh, const float *viewmats,
                              omnigs_splat *splats, cudaStream_t stream, uint64_t *depth_keys = nullptr, int gbits = 0,
                              uint64_t *splat_count = nullptr);
// Whether the depth sort of omnigs_bin orders packed keys ((view << 32 | t_r bits) << gbits | splat index, which the
// equirectangular camera uses when they fit 64 bits); *gbits: the index bits.
bool packed_depth_keys(const omnigs_config &cfg, int64_t n, int *gbits);
cudaError_t launch_preprocess_bwd(const omnigs_config &cfg, int64_t n, const float *means, const float *scales,
                                  const float *quats, const float *opacity, const float *sh, const float *viewmats,
                                  const omnigs_splat_grad *grads, float *d_means, float *d_scales, float *d_quats,
                                  float *d_opacity, float *d_sh, float *d_screen, cudaStream_t stream);
cudaError_t launch_bin(const omnigs_config &cfg, int64_t n, const omnigs_splat *splats, uint32_t *order,
                       uint64_t *keys, int64_t capacity, const WsLayout &L, char *ws, cudaStream_t stream,
                       bool depth_keys_ready = false);
cudaError_t launch_sort(const omnigs_config &cfg, int64_t n, int64_t capacity, uint64_t *keys, uint32_t *ranges,
                        const WsLayout &L, char *ws, cudaStream_t stream);
// The L1 loss fused into the forward blend (omnigs_render_fwd_l1): the target image, the gradient and loss outputs,
// and the per-tile partial sums [V * TILES] in the workspace.
struct FwdL1 {
    const float *target;
    float *dL_drgb;
    float *loss;
    float *tile_sums;
};
cudaError_t launch_render_fwd(const omnigs_config &cfg, int64_t n, const omnigs_splat *splats,
                              const uint32_t *ranges, const uint64_t *keys, const uint32_t *order, float *out_rgb,
                              float *out_T, uint32_t *out_nc, uint32_t *out_count, const FwdL1 *l1,
                              cudaStream_t stream);
cudaError_t launch_render_bwd(const omnigs_config &cfg, int64_t n, const omnigs_splat *splats,
                              const uint32_t *ranges, const uint64_t *keys, const uint32_t *order,
                              const float *out_T, const uint32_t *nc, const float *dL_drgb,
                              omnigs_splat_grad *grads, cudaStream_t stream);
cudaError_t launch_l1(const omnigs_config &cfg, int row_begin, int row_end, const float *rgb, const float *target,
                      float *dL_drgb, float *loss, const WsLayout &L, char *ws, cudaStream_t stream);
size_t densify_workspace_bytes(int64_t n);
cudaError_t launch_adam(int64_t n, int K, const omnigs_adam_config &cfg, int64_t step, float *params, float *m,
                        float *v, const float *d_means, const float *d_scales, const float *d_quats,
                        const float *d_opacity, const float *d_sh, float *means, float *scales, float *quats,
                        float *opacity, float *sh, cudaStream_t stream);
cudaError_t launch_publish(int64_t n, int K, const float *params, float *means, float *scales, float *quats,
                           float *opacity, float *sh, cudaStream_t stream);
cudaError_t launch_densify_stats(const omnigs_config &cfg, int64_t n, const omnigs_splat *splats,
                                 const omnigs_splat_grad *grads, float *accum, int *count, float *max_radius,
                                 cudaStream_t stream);
cudaError_t launch_densify(int64_t n, int K, const omnigs_densify_config &cfg, const float *params, const float *m,
                           const float *v, const float *accum, const int *count, const float *max_radius,
                           const float *normals, float *params_out, float *m_out, float *v_out, long long *n_out,
                           char *ws, cudaStream_t stream);
cudaError_t launch_reset_opacity(int64_t n, int K, float value, float *params, float *m, float *v, float *opacity,
                                 cudaStream_t stream);
cudaError_t launch_crop(int V, int We, int He, const float *eq, const float *rot, int W, int H, float fx, float fy,
                        float cx, float cy, float *out, cudaStream_t stream);
size_t dssim_scratch_bytes(const omnigs_config &cfg);
cudaError_t launch_dssim(const omnigs_config &cfg, float lambda, const float *rgb, const float *target, float *dL,
                         float *loss, char *scratch, cudaStream_t stream);

}  // namespace omnigs
