/*
 * omnigs.h -- C ABI of the GB300 (sm_103a) equirectangular Gaussian-splatting rasterizer.
 *
 * The library renders 3D Gaussians directly onto an equirectangular (spherical-camera) image and back-propagates
 * through that rendering, following OmniGS (arXiv 2404.03202): projection onto longitude / latitude (Sec. 3.2,
 * Eqs. 1, 3-5), the spherical-camera Jacobian and EWA covariance (Sec. 3.3, Eqs. 9-16), tile-based alpha blending
 * sorted by the camera distance t_r (Sec. 3.3, Eqs. 6-8 and the tile procedure that closes Sec. 3.3), and the
 * gradients of Sec. 3.4 (Eqs. 18-20).
 *
 * Conventions for every entry point:
 *   - Pointers named as device buffers must be device memory (or managed memory) of the current device. All
 *     arrays are C-contiguous; float arrays are IEEE float32; "[a, b]" gives the shape.
 *   - The caller owns every buffer, including the workspace. The library never allocates device memory and never
 *     synchronises, except in omnigs_instance_count and omnigs_last_error, which say so.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL means the legacy default stream) and runs asynchronously.
 *   - Invalid arguments are rejected before any work is enqueued, with OMNIGS_E_INVALID. A failed launch returns
 *     OMNIGS_E_CUDA. Conditions found on the device (instance capacity exceeded) set a sticky error word in the
 *     workspace; omnigs_last_error returns and clears it. Outputs are undefined after any error.
 *   - Gradient outputs are overwritten, not accumulated.
 *   - A sequence of calls for one frame must use one workspace and one stream; concurrent frames need separate
 *     workspaces.
 */
#ifndef OMNIGS_H
#define OMNIGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *omnigs_stream_t; /* same type as cudaStream_t */

typedef enum {
    OMNIGS_OK = 0,
    OMNIGS_E_INVALID = 1,  /* bad argument; nothing was enqueued */
    OMNIGS_E_CAPACITY = 2, /* more tile instances than the capacity given to omnigs_bin */
    OMNIGS_E_CUDA = 3,     /* a CUDA launch or call failed */
    OMNIGS_E_TIMEOUT = 4   /* a bounded device-side wait ran out (the tile sort's bulk copies; 2 s each) */
} omnigs_status;

/* Image and camera set-up shared by all calls of one frame. */
typedef struct {
    int32_t width;     /* W, equirectangular width in pixels; a multiple of `tile`, at most 65536 */
    int32_t height;    /* H, height in pixels; a multiple of `tile`, at most 65536 (W = 2H is the usual shape) */
    int32_t tile;      /* square tile side in pixels: 8, 16 or 32 */
    int32_t num_views; /* V >= 1 camera poses rendered in one call */
    int32_t sh_degree; /* 0..3; the SH array holds K = (sh_degree + 1)^2 coefficients per colour channel */
    float near_r;      /* a Gaussian is culled when its camera distance t_r <= near_r */
    float bg[3];       /* background colour added with the final transmittance */
    int32_t pixels_per_thread; /* schedule of the forward blend (omnigs_render_fwd): pixels of one image column each
                                * thread owns (2, 4 or 8; 4 and 8 need tile >= 16); 0 lets the library choose (4, or
                                * 2 on 8-pixel tiles). Results do not depend on it. */
    int32_t camera;            /* OMNIGS_CAMERA_EQUIRECT (0): Eqs. 3-5, the paper's camera. OMNIGS_CAMERA_PINHOLE (1):
                                * Eq. 2, the perspective model of 3DGS: p = (fx tx / tz + cx, fy ty / tz + cy);
                                * Gaussians are ordered by t_z and culled when t_z <= near_r or |p| >= 2^23; J holds
                                * t_x / t_z and t_y / t_z within 1.3 half-fields of view (W / (2 fx), H / (2 fy));
                                * tile columns are clipped like rows and dx is not wrapped. */
    float fx, fy, cx, cy;      /* pinhole intrinsics in pixels (fx, fy > 0); ignored for the equirectangular camera */
    int32_t adjoint_pixels_per_thread; /* schedule of the blend adjoint (omnigs_render_bwd), as pixels_per_thread;
                                        * 0 lets the library choose (8, or 2 on 8-pixel tiles). Gradients depend on
                                        * it only through the order of floating-point additions. */
} omnigs_config;

#define OMNIGS_CAMERA_EQUIRECT 0
#define OMNIGS_CAMERA_PINHOLE 1

/* One projected Gaussian in one view (48 bytes; arrays of it must be 16-byte aligned). The fields binning reads
 * (position, conic, depth, box, q) fill the first 32 bytes, the colour fields the last 16. (px, py): Eq. 5 pixel
 * position, px in [0, W], py in [0, H] (Eq. 2 for the pinhole camera: may lie off the image). (c0, c1, c2): inverse of
 * the 2x2 covariance Sigma~ of Eq. 9 (entries 00, 01, 11). depth = t_r = |t|. (radius_x, radius_y): half-extents in
 * pixels of the box around pixel floor(p) whose tiles receive an instance; 0 when the Gaussian is culled in this view.
 * The box is the square of half-side r = ceil(3 sqrt(lambda_max)) (the radius of influence, Sec. 3.3), narrowed per
 * axis to the box of the ellipse where alpha >= 1/255: with q = 2 ln(255 o), radius_x = min(r, ceil(sqrt(q Sigma~_00)
 * (1 + 1e-4) + 1e-3)) and radius_y likewise with Sigma~_11, both held at 65535. Outside that ellipse alpha < 1/255, so
 * the narrowing removes only instances that contribute to no pixel. A Gaussian with 255 o < 1 is culled, and with the
 * pinhole camera so is one whose box misses the image (it has no tile either way). q = 2 ln(255 o) (0 when culled) is
 * the level of that ellipse, dp^T conic dp <= q, which omnigs_bin uses to cull tiles row by row. */
typedef struct {
    float px, py;
    float c0, c1, c2;
    float depth;
    uint16_t radius_x, radius_y;
    float q;
    float opacity;
    float r, g, b;
} omnigs_splat;

/* Gradient of the loss with respect to one omnigs_splat's differentiable fields (48 bytes, 16-byte aligned). */
typedef struct {
    float px, py;
    float c0, c1, c2;
    float opacity;
    float r, g, b;
    float reserved[3]; /* written as 0 */
} omnigs_splat_grad;

/* Library version, major * 10000 + minor * 100 + patch. */
int omnigs_version(void);

/* Human-readable name of a status code (static storage). */
const char *omnigs_status_string(omnigs_status status);

/* Bytes of device workspace needed for n Gaussians in cfg->num_views views with room for `capacity` tile
 * instances (one instance per (view, Gaussian, covered tile); Sec. 3.3). Returns 0 for invalid arguments. The size
 * depends on the device (it is queried on the current one). The workspace is 256-byte aligned by the caller and
 * need not be initialised; omnigs_bin initialises it. */
size_t omnigs_workspace_size(const omnigs_config *cfg, int64_t n, int64_t capacity);

/* Per-(view, Gaussian) projection, Sec. 3.2-3.3: t = W m + t_cw (Eq. 1); lon, lat (Eq. 3); s (Eq. 4); p (Eq. 5);
 * J (Eqs. 10-16); Sigma~ = J W Sigma W^T J^T + 0.3 I (Eq. 9), Sigma = R(q) diag(s)^2 R(q)^T; conic = Sigma~^-1;
 * the instance box (radius_x, radius_y); colour c = max(sum_k Y_k(d) sh_k + 0.5, 0) with d the unit vector from
 * the camera centre to m (Sec. 3.1).
 *   means   [n, 3]  world positions m                     scales  [n, 3]  linear scales S (> 0)
 *   quats   [n, 4]  rotations q as (w, x, y, z), any norm  opacity [n]     opacities o in [0, 1]
 *   sh      [n, K, 3] SH coefficients                     viewmats [V, 4, 4] row-major world-to-camera T_cw
 *   splats  [V, n]  output (device), index v * n + g
 * All inputs are device buffers. n = 0 is valid and enqueues nothing. */
omnigs_status omnigs_preprocess(const omnigs_config *cfg, int64_t n, const float *means, const float *scales,
                                const float *quats, const float *opacity, const float *sh, const float *viewmats,
                                omnigs_splat *splats, omnigs_stream_t stream);

/* Tile binning, Sec. 3.3 ("one instance per influence"): for every splat with radius_x > 0, one instance per tile
 * covered by the box [floor(px) - radius_x, floor(px) + radius_x] x [floor(py) - radius_y, floor(py) + radius_y]
 * that the splat's alpha >= 1/255 ellipse can reach. Tile columns wrap modulo W / tile (the longitude seam; a box at
 * least as wide as the image covers every column once); rows are clipped to the image. Within a tile row of a box
 * narrower than the image, only the columns whose pixel centres lie within one pixel of the ellipse
 * dp^T conic dp <= q (1.001) + 1e-3, over the row's band of pixel-centre y values, are kept (the widening absorbs
 * the rounding of the single-precision bounds). A dropped tile has alpha < 1/255 at each of its pixels: no image
 * changes. Splats with c0 c2 - c1^2 <= 1e-3 c0 c2 keep whole rows, and so, with the equirectangular camera, do
 * splats with radius_x + tile > W / 2 (whose box offsets can differ from the minimal-image dx of the blend).
 * Splats whose centre lies outside [0, W] x [0, H] (equirectangular camera) or beyond 2^23 px (pinhole camera) are
 * ignored.
 *   splats  [V * n] input (device)
 *   order   [V * n] output (device): the splats of each view by increasing depth t_r, equal depths by splat index:
 *           order[v * n + r] = v * n + g of the r-th nearest splat g of view v ("depth rank" r). With the
 *           equirectangular camera every splat is ranked; with the pinhole camera only those with instances are
 *           (a view sees a fraction of the scene), and the entries past a view's ranked splats are unspecified.
 *   keys    [capacity] device buffer for one key per instance, ((v * TILES + tile) << R) | r, with
 *           TILES = (W / tile) * (H / tile), tile = ty * (W / tile) + tx, r the splat's depth rank and
 *           R = max(1, ceil(log2(n))) rank bits. The keys are generated view by view and splat by splat in depth
 *           order (a splat's tiles row by row, columns in seam order), so within a tile they are already in rank
 *           order. When 256 <= n <= 2^24 and an image has at most 128 tile rows and 256 tile columns,
 *           omnigs_bin writes them into the workspace, grouped by (view, tile row) in that order (as 32-bit entries),
 *           and leaves `keys` for omnigs_sort to fill; otherwise it writes them into `keys` in generation order.
 *           Either way omnigs_sort leaves the sorted keys in `keys`.
 * The total instance count stays on the device (workspace); if it exceeds `capacity`, instances beyond it are dropped
 * and OMNIGS_E_CAPACITY is raised in the workspace. capacity < 2^32, the value given to omnigs_workspace_size. */
omnigs_status omnigs_bin(const omnigs_config *cfg, int64_t n, const omnigs_splat *splats, uint32_t *order,
                         uint64_t *keys, int64_t capacity, void *workspace, omnigs_stream_t stream);

/* omnigs_preprocess followed by omnigs_bin, with the same arguments and the same results (splats, order, keys, the
 * instance count and the errors in the workspace). With the equirectangular camera the projection kernel also writes
 * the depth sort's keys into the workspace, so that the binning does not read every splat record back for its depth
 * (the fused form of Sec. 3.3's depth ordering of the splats of Eqs. 3-5; the paper has no such interface); with the
 * pinhole camera the two calls simply run one after the other. */
omnigs_status omnigs_preprocess_bin(const omnigs_config *cfg, int64_t n, const float *means, const float *scales,
                                    const float *quats, const float *opacity, const float *sh, const float *viewmats,
                                    omnigs_splat *splats, uint32_t *order, uint64_t *keys, int64_t capacity,
                                    void *workspace, omnigs_stream_t stream);

/* Stable sort of the instance keys of omnigs_bin by their (view, tile) bits into `keys` (one counting pass by tile
 * column within each (view, tile row) group when omnigs_bin grouped them, a radix sort of `keys` in place
 * otherwise), which leaves them ordered by (view, tile), then by depth rank, i.e. the blending
 * order of Sec. 3.3 (nearest first by t_r) with equal depths in splat order, the order a stable sort of (tile, t_r)
 * keys gives to instances generated splat by splat. Writes ranges [V * TILES, 2] (device): ranges[2t], ranges[2t+1] =
 * first and one-past-last sorted position of tile t (both 0 for an empty tile). n and capacity as for omnigs_bin. */
omnigs_status omnigs_sort(const omnigs_config *cfg, int64_t n, int64_t capacity, uint64_t *keys, uint32_t *ranges,
                          void *workspace, omnigs_stream_t stream);

/* Forward blending, Eqs. 6-8 with the tile procedure of Sec. 3.3: pixel (x, y) of view v is sampled at
 * (x + 0.5, y + 0.5) and blends its tile's sorted list front to back: dx taken as the minimal image in
 * [-W/2, W/2); alpha = min(0.99, o exp(-1/2 dp^T conic dp)); entries with exponent > 0 or alpha < 1/255 are
 * skipped; blending stops before an entry that would bring T below 1e-4; finally C += T bg.
 *   splats [V * n], ranges [V * TILES, 2] and keys [capacity] (from omnigs_sort), order [V * n] (from omnigs_bin):
 *   inputs (device); the splat of sorted position s of view v is order[v * n + (keys[s] & (2^R - 1))].
 *   out_rgb [V, 3, H, W], out_T [V, H, W] (final transmittance), out_ncontrib [V, H, W] (list position after the
 *   last contributor): outputs (device). out_T and out_ncontrib feed omnigs_render_bwd.
 *   out_count [V, H, W] (device, optional, may be NULL): number of splats blended into each pixel. */
omnigs_status omnigs_render_fwd(const omnigs_config *cfg, int64_t n, const omnigs_splat *splats,
                                const uint32_t *ranges, const uint64_t *keys, const uint32_t *order, float *out_rgb,
                                float *out_T, uint32_t *out_ncontrib, uint32_t *out_count, omnigs_stream_t stream);

/* omnigs_render_fwd followed by omnigs_l1_loss in one pass over the image: the forward blend's epilogue compares
 * each pixel's colour with target [V, 3, H, W] (device) and writes dL_drgb [V, 3, H, W] = sign(rgb - target) /
 * (V * 3 * H * W), bit for bit what omnigs_l1_loss writes for this out_rgb, and per tile the sum of |rgb - target|,
 * which a second kernel adds up in double precision into loss [1] (device) = mean |rgb - target|. The loss differs
 * from omnigs_l1_loss's only in the order of the additions (a few units in the last place of the float result).
 * This saves the loss kernel's read of the image (Eq. 17's L1 term and Eqs. 6-8, fused; the paper has no such
 * interface). Other arguments as for omnigs_render_fwd (no per-pixel count); workspace as for omnigs_l1_loss (the
 * per-tile sums sit at a fixed offset of it). Calls sharing a workspace must not overlap on the GPU. */
omnigs_status omnigs_render_fwd_l1(const omnigs_config *cfg, int64_t n, const omnigs_splat *splats,
                                   const uint32_t *ranges, const uint64_t *keys, const uint32_t *order,
                                   const float *target, float *out_rgb, float *out_T, uint32_t *out_ncontrib,
                                   float *dL_drgb, float *loss, void *workspace, omnigs_stream_t stream);

/* L1 term of the photometric loss (Eq. 17 with lambda = 0): loss = mean |rgb - target| over [V, 3, H, W];
 * dL_drgb = sign(rgb - target) / (V * 3 * H * W) (0 where equal). rgb, target: inputs; dL_drgb [V, 3, H, W] and
 * loss [1]: outputs (device). */
omnigs_status omnigs_l1_loss(const omnigs_config *cfg, const float *rgb, const float *target, float *dL_drgb,
                             float *loss, void *workspace, omnigs_stream_t stream);

/* L1 loss restricted to the image rows [row_begin, row_end), for captures whose band of rows shows the capture rig
 * rather than the scene (Sec. 5.2: in the 360Roam captures the bottom rows, which show the robot carrying the
 * camera, are left out of the loss and its gradient): loss = mean |rgb - target| over [V, 3, row_begin:row_end, W];
 * dL_drgb = sign(rgb - target) / (V * 3 * (row_end - row_begin) * W) inside those rows and 0 outside. Requires
 * 0 <= row_begin < row_end <= H (else OMNIGS_E_INVALID). Buffers as for omnigs_l1_loss. */
omnigs_status omnigs_l1_loss_rows(const omnigs_config *cfg, int32_t row_begin, int32_t row_end, const float *rgb,
                                  const float *target, float *dL_drgb, float *loss, void *workspace,
                                  omnigs_stream_t stream);

/* Photometric loss with its D-SSIM term, Eq. 17: L = (1 - lambda) mean|rgb - target| + lambda (1 - SSIM), SSIM the
 * mean over [V, 3, H, W] of the per-pixel structural similarity of each colour plane with an 11 x 11 Gaussian window
 * (sigma 1.5, normalised; zero padding at the image border), C1 = 0.01^2, C2 = 0.03^2 (the conventions of the 3DGS
 * renderer the paper builds on; lambda = 0.2 there). Writes loss [1] and dL_drgb [V, 3, H, W] (device). lambda must
 * lie in [0, 1]. scratch: device buffer of omnigs_dssim_scratch_size(cfg) bytes, 256-byte aligned, owned by the
 * caller, no initialisation needed; calls sharing one scratch must not overlap on the GPU. */
size_t omnigs_dssim_scratch_size(const omnigs_config *cfg);
omnigs_status omnigs_dssim_loss(const omnigs_config *cfg, float lambda, const float *rgb, const float *target,
                                float *dL_drgb, float *loss, void *scratch, omnigs_stream_t stream);

/* The same loss and gradient as omnigs_l1_loss without a workspace, for callers that cannot allocate device memory
 * or hand the library any beyond their inputs and outputs (a host application that owns the CUDA allocator or has
 * reserved all device memory, a loop with a fixed memory budget). The paper has no counterpart; this is an interface
 * convenience. Its scratch (4096 partial sums) is a fixed array inside the library, so it allocates nothing and calls
 * no allocating routine. Limit: V * 3 * H * W <= 268,435,456 floats; larger requests, and every configuration
 * omnigs_l1_loss rejects, return OMNIGS_E_INVALID before anything is enqueued. The first call in a CUDA context
 * looks up the array's device address (cudaGetSymbolAddress; again after the context is re-created) and, if nothing
 * has loaded this library onto the device yet, loads its module, which takes device memory for the module image:
 * make that first call before reserving all device memory and before any stream capture on that device. All calls
 * on a device share the array: calls that may overlap on the GPU race and must be serialised by the caller. rgb,
 * target, dL_drgb: 16-byte aligned device buffers [V, 3, H, W]; loss [1] device. */
omnigs_status omnigs_l1_loss_static(const omnigs_config *cfg, const float *rgb, const float *target, float *dL_drgb,
                                    float *loss, omnigs_stream_t stream);

/* Adjoint of omnigs_render_fwd (Sec. 3.4, the blending part of Eqs. 18-20): per pixel, back to front from its
 * last contributor, recovering T by division by (1 - alpha). Writes grads [V * n] (device): dL/d(px, py, c0, c1,
 * c2, opacity, r, g, b) of every splat, summed over the pixels it reaches. The derivative of alpha is 0 where it is
 * clamped at 0.99. Inputs are those of omnigs_render_fwd plus its out_T, out_ncontrib and dL_drgb [V, 3, H, W]. */
omnigs_status omnigs_render_bwd(const omnigs_config *cfg, int64_t n, const omnigs_splat *splats,
                                const uint32_t *ranges, const uint64_t *keys, const uint32_t *order,
                                const float *out_T, const uint32_t *ncontrib, const float *dL_drgb,
                                omnigs_splat_grad *grads, omnigs_stream_t stream);

/* Adjoint of omnigs_preprocess (Sec. 3.4, Eqs. 18-20): chain rule from the splat gradients through conic,
 * Sigma~ (dSigma~/dSigma), the spherical Jacobian (dJ/dt), p (dp/ds, ds/dt), t = W m + t_cw, R(q), S and the SH
 * colour (dc/dm), summed over views. Same parameter inputs as omnigs_preprocess, plus grads [V * n].
 *   d_means [n, 3], d_scales [n, 3], d_quats [n, 4], d_opacity [n], d_sh [n, K, 3]: outputs (device)
 *   d_screen [n, 2]: dL/ds, the gradient with respect to the uniform screen-space position s of Eq. 4 (which
 *   drives densification, Sec. 4), summed over views; output (device). */
omnigs_status omnigs_preprocess_bwd(const omnigs_config *cfg, int64_t n, const float *means, const float *scales,
                                    const float *quats, const float *opacity, const float *sh,
                                    const float *viewmats, const omnigs_splat_grad *grads, float *d_means,
                                    float *d_scales, float *d_quats, float *d_opacity, float *d_sh,
                                    float *d_screen, omnigs_stream_t stream);

/* Total instance count of the last omnigs_bin on this workspace (may exceed the capacity). Synchronises `stream`. */
omnigs_status omnigs_instance_count(const void *workspace, int64_t *count, omnigs_stream_t stream);

/* Returns and clears the sticky device-side error of the workspace (OMNIGS_OK if none), after synchronising
 * `stream`; also reports a pending CUDA error as OMNIGS_E_CUDA. */
omnigs_status omnigs_last_error(void *workspace, omnigs_stream_t stream);

/* Perspective crops of equirectangular images (Sec. 5.4 compares rendered equirectangular views with perspective
 * renders after cropping them into perspective images). Output pixel (x, y) of view v looks along the camera-frame
 * direction d = R_v^T ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1) (a pinhole of Eq. 2 rotated by R_v); its longitude
 * and latitude (Eq. 3) place it on the equirectangular image (Eqs. 4-5), which is sampled bilinearly between pixel
 * centres, columns wrapping across the seam and rows clamped at the poles.
 *   equirect [V, 3, eq_height, eq_width], rotations [V, 3, 3] (row-major), out [V, 3, height, width]: device. */
omnigs_status omnigs_equirect_crop(int32_t V, int32_t eq_width, int32_t eq_height, const float *equirect,
                                   const float *rotations, int32_t width, int32_t height, float fx, float fy, float cx,
                                   float cy, float *out, omnigs_stream_t stream);

/* ---------------------------------------------------------------- reconstruction loop (Sec. 4, Algorithm 1)
 *
 * The optimiser keeps each Gaussian as one row of P = 11 + 3K raw floats: mean (3), log-scale (3), quaternion (4,
 * normalised only when used), logit-opacity (1), SH coefficients (3K, laid out [K][3]). Adam moments m and v share
 * that layout. The renderer reads the activated arrays means [n, 3], scales = exp(log-scale) [n, 3], quats [n, 4],
 * opacity = sigmoid(logit) [n], sh [n, K, 3]. The densification thresholds live in the paper's missing supplement;
 * the defaults a caller would pass are those of the 3DGS renderer the paper says its strategy resembles. */
typedef struct {
    float lr_means, lr_scales, lr_quats, lr_opacity, lr_sh_dc, lr_sh_rest; /* per parameter group */
    float beta1, beta2, eps;                                               /* Adam */
} omnigs_adam_config;

typedef struct {
    float grad_threshold;    /* densify when mean |dL/ds| over the views that saw the Gaussian reaches this */
    float percent_dense;     /* clone when the largest scale is at most percent_dense * extent, else split */
    float extent;            /* scene extent (world units) */
    float min_opacity;       /* prune below this opacity */
    float max_scale_frac;    /* prune when the largest scale exceeds max_scale_frac * extent */
    float max_screen_radius; /* prune an original whose instance half-extent exceeded this (pixels) */
} omnigs_densify_config;

/* "Advance optimizer by one step" (Algorithm 1): Adam with bias correction (step counts from 1) on the raw rows,
 * from gradients with respect to the activated parameters (the outputs of omnigs_preprocess_bwd; the chain rule
 * through exp and sigmoid is applied here). Updates params, m, v in place and writes the activated arrays for the
 * next render. All pointers are device buffers; n = 0 enqueues nothing. */
omnigs_status omnigs_adam_step(int64_t n, int32_t K, const omnigs_adam_config *cfg, int64_t step, float *params,
                               float *m, float *v, const float *d_means, const float *d_scales, const float *d_quats,
                               const float *d_opacity, const float *d_sh, float *means, float *scales, float *quats,
                               float *opacity, float *sh, omnigs_stream_t stream);

/* Writes the activated arrays of `params` (after a densification, before the next render). */
omnigs_status omnigs_publish_params(int64_t n, int32_t K, const float *params, float *means, float *scales,
                                    float *quats, float *opacity, float *sh, omnigs_stream_t stream);

/* Densification statistics of one render (Sec. 4: densify by dL/ds): for every view in which Gaussian g has tile
 * instances, accum[g] += |dL/ds| with dL/ds = dL/dp diag(W/2, H/2) (Eq. 4) from the 2D gradients of
 * omnigs_render_bwd, count[g] += 1, and max_radius[g] = max(max_radius[g], radius_x, radius_y). accum, count,
 * max_radius [n] are device buffers the caller zeroes after each densification. */
omnigs_status omnigs_densify_stats(const omnigs_config *cfg, int64_t n, const omnigs_splat *splats,
                                   const omnigs_splat_grad *grads, float *accum, int32_t *count, float *max_radius,
                                   omnigs_stream_t stream);

/* Bytes of device workspace omnigs_densify needs for n Gaussians. */
size_t omnigs_densify_workspace_size(int64_t n);

/* Densify and prune (Algorithm 1). A Gaussian whose mean |dL/ds| reaches grad_threshold is cloned if its largest
 * scale is at most percent_dense * extent and split into two otherwise. A split child has mean m + R(q) (S z), with
 * z = normals[g][k] (standard normal draws given by the caller), scales S / 1.6 and the parent's rotation, opacity
 * and SH; the parent is removed. Pruned: any row whose opacity is below min_opacity or whose largest scale exceeds
 * max_scale_frac * extent, and an original whose max_radius exceeded max_screen_radius. Rows out, for each original
 * in index order: itself if kept, its clone, its two children. Moments follow kept originals and are zero for new
 * rows. params_out, m_out, v_out need room for 2n rows; *n_out (device, int64) receives the row count. */
omnigs_status omnigs_densify(int64_t n, int32_t K, const omnigs_densify_config *cfg, const float *params,
                             const float *m, const float *v, const float *accum, const int32_t *count,
                             const float *max_radius, const float *normals, float *params_out, float *m_out,
                             float *v_out, int64_t *n_out, void *workspace, omnigs_stream_t stream);

/* "Reset large o" (Algorithm 1): logit-opacity <- min(logit-opacity, logit(value)) with its Adam moments zeroed;
 * opacity (optional, may be NULL) receives the activated opacities. 0 < value < 1. */
omnigs_status omnigs_reset_opacity(int64_t n, int32_t K, float value, float *params, float *m, float *v,
                                   float *opacity, omnigs_stream_t stream);

/* Kernel timing. While enabled, every stage the library runs (one kernel, or a few back-to-back kernels under one
 * name) is bracketed by CUDA events on its launching stream. omnigs_profiler_collect synchronises those events,
 * writes up to `max` per-stage totals (kernel launches and summed milliseconds, in first-launch order) and clears
 * the record; it returns the number of stages. Host-side
 * state is global to the process and not thread-safe; use it from one thread, outside CUDA graph capture. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} omnigs_kernel_time;
omnigs_status omnigs_profiler_enable(int enable);
int omnigs_profiler_collect(omnigs_kernel_time *out, int max);

#ifdef __cplusplus
}
#endif

#endif /* OMNIGS_H */
