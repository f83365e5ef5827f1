// Tile-based alpha blending onto the equirectangular image (Sec. 3.3, Eqs. 6-8) and its adjoint (Sec. 3.4).
//
// One CTA per (view, tile). The tile's sorted instance list is walked in batches of one entry per thread: each thread
// gathers one splat (two 16-byte loads and one 4-byte load) into shared memory with
//   * the conic pre-scaled by -log2(e)/2, so that G = 2^e with e = dx (c0' dx + c1' dy) + c2' dy^2 costs one ex2;
//   * the longitude-seam shift decided once per (entry, tile): 0 or +-W for the whole tile, or a flag for the rare
//     splat whose minimal-image boundary falls inside the tile;
//   * the exponent threshold thr = -log2(255 o): alpha = min(0.99, o 2^e) < 1/255 exactly when e < thr, so with the
//     exponent > 0 guard a pair passes only if thr <= e <= 0, tested as |e - thr/2| <= -thr/2 with one subtraction
//     and one compare before the ex2.
// Each thread owns PPT vertically adjacent pixels of one column: they share dx, the per-entry products and every
// shared-memory load. The forward's per-pixel update is branch-free (a pair that fails the test or stops the pixel
// adds with weight 0), which costs an ex2 per examined pair but removes the divergent branch. The CTA leaves the
// list once every pixel has stopped (__syncthreads_count).
//
// The adjoint walks the same list back to front from each pixel's last contributor, recovers T by division by
// (1 - alpha), keeps per pixel one scalar for everything behind the current entry (the upstream gradient dotted with
// the colour behind it), and accumulates per entry over the thread's pixels dL/do, dL/d(r, g, b) and the exponent
// moments (the pixels share dx, so the moments in dx follow per thread). The warp then reduces them (a transposed reduce-scatter of 8 fields plus a butterfly for the ninth:
// 14 shuffles, after which 9 lanes hold one field's total each and write it with one shared-memory atomic), the CTA
// sums warps in shared memory, the conic turns the moments into dL/d(px, py, c0, c1, c2) once per entry, and the
// CTA's sum goes to the splat's gradient with 16-byte vector atomics (red.global.add.v4.f32).
// A thread owns PPT = 2, 4 or 8 pixels of one column (the blend schedule of the config): more pixels per thread share
// more of the per-entry work and the warp reduction, fewer give more threads per tile. At 8 pixels one warp covers a
// 16 x 16 tile. The adjoint interleaves the rows of a column's threads within the warp (InterleavedRows), so that
// the pixel pairs it may skip together are bands of adjacent rows. Forward and adjoint evaluate alpha with identical
// arithmetic, so their skip / stop decisions agree.
#include "common.cuh"

namespace omnigs {
namespace {

constexpr float kPerPixelWrap = 1.0f;  // seam-shift value meaning "wrap per pixel" (real shifts are 0 or +-W)

__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The forward's update works on pairs of a thread's vertically adjacent pixels with packed FP32 (f32x2) adds,
// multiplies and FMAs, one instruction per pair. Opacity and colour are staged negated so that every packed step
// rounds exactly like the scalar form it replaces: T' = fma(T, -alpha, T), -alpha = max(-0.99, (-o) G) and
// C' = fma(-w, -c, C) equal fma(-T, alpha, T), -min(0.99, o G) and fma(w, c, C) bit for bit, so the adjoint's
// recomputed alphas and stop decisions still match. The pair operands come from shared memory already duplicated
// in both halves (one 16-byte load gives two pairs).
struct FwdStaged {
    float4 s;   // px, seam shift, c0', c1'     (per-thread dx and the exponent's dx terms)
    float4 p0;  // py, py, c2', c2'
    float4 p1;  // -m, -m, -o, -o              (pass interval centre, opacity)
    float4 p2;  // -r, -r, -g, -g
    float4 p3;  // -b, -b, h, per-pixel wrap flag   (h: pass interval half-width)
};

__device__ __forceinline__ float2 lo2(const float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 v) { return make_float2(v.z, v.w); }

struct Staged {
    float4 a;  // px, py, c0', c1'   (c' = conic scaled to the base-2 exponent)
    float4 b;  // c2', m, h, seam shift; the pass interval thr <= e <= 0 is written |e - m| <= h (m = thr/2, h = -m)
    float4 c;  // opacity, r, g, b
    float4 d;  // raw conic c0, c1, c2, unused (for the adjoint)
};

// Splat of sorted list position s: the key's low rank bits are the splat's depth rank within its view.
__device__ __forceinline__ unsigned entry_splat(const unsigned long long* __restrict__ keys,
                                                const uint32_t* __restrict__ view_order, uint32_t s,
                                                unsigned long long rank_mask) {
    return __ldg(view_order + (__ldg(keys + s) & rank_mask));
}

__device__ __forceinline__ Staged stage_entry(const float4* __restrict__ splats, unsigned vg, float x_first,
                                              float x_last, float halfW, float fW) {
    const float4 a = __ldg(splats + 3 * (size_t)vg);                                   // px, py, c0, c1
    const float c2 = __ldg(reinterpret_cast<const float*>(splats + 3 * (size_t)vg + 1));
    const float4 col = __ldg(splats + 3 * (size_t)vg + 2);                             // opacity, r, g, b
    const float hi = a.x - x_first, lo = a.x - x_last;  // extreme dx over the tile's pixel columns
    float shift;
    if (lo >= -halfW && hi < halfW) shift = 0.f;
    else if (lo >= halfW) shift = -fW;
    else if (hi < -halfW) shift = fW;
    else shift = kPerPixelWrap;
    const float c0 = a.z, c1 = a.w, o = col.x;
    const float thr = -__log2f(255.f * o);  // may be +inf (o = 0): then nothing passes
    Staged s;
    s.a = make_float4(a.x, a.y, -0.5f * kLog2e * c0, -kLog2e * c1);
    s.b = make_float4(-0.5f * kLog2e * c2, 0.5f * thr, -0.5f * thr, shift);
    s.c = col;
    s.d = make_float4(c0, c1, c2, 0.f);
    return s;
}

// The tile's seam shift of the entry (0 when the shift is decided per pixel), and the flag (1) of a per-pixel wrap.
// dx = (px - xs) + shift rounds like the per-pixel wrap (px - xs) -+ W, so a pixel's dx, and its alpha, do not depend
// on which of the two its tile took (nor, then, on the tile size); px - xs is exact for the nearby pixels.
__device__ __forceinline__ float seam_shift(const Staged& st) { return st.b.w != kPerPixelWrap ? st.b.w : 0.f; }
__device__ __forceinline__ float wrap_flag(const Staged& st) { return st.b.w != kPerPixelWrap ? 0.f : 1.f; }

// Minimal-image wrap of a per-pixel dx.
__device__ __forceinline__ float wrap_dx(float dx, float halfW, float fW) {
    if (dx >= halfW) dx -= fW;
    else if (dx < -halfW) dx += fW;
    return dx;
}

// Pixels of a thread: column lx = t % TS, rows (t / TS) * PPT + k for k < PPT, so a warp covers a compact
// TS x (32 / TS * PPT) block.
template <int TS, int PPT>
struct PixelMap {
    static constexpr int NT = TS * TS / PPT;  // threads per CTA
    static_assert(NT % 32 == 0, "a CTA must hold whole warps");
    int x, y0;
    __device__ PixelMap(int txi, int tyi) {
        x = txi * TS + (int)threadIdx.x % TS;
        y0 = tyi * TS + ((int)threadIdx.x / TS) * PPT;
    }
};

// The adjoint's pixels: within each warp, the threads of a column interleave their rows. A warp covers
// RW = 32 / TS threads per column; its thread l / TS of column l % TS takes rows l / TS + RW k of the warp's band
// of RW PPT rows, so the warp's k-th pixels (and its pixel pairs) form one band of RW (2 RW) adjacent rows. The
// adjoint skips a pixel pair when no pixel of the warp's pair passes the entry, and a splat's footprint in the tile
// is a compact blob: it meets fewer of the warp's pair bands than with each thread's pixels stacked.
template <int TS, int PPT>
struct InterleavedRows {
    static constexpr int NT = TS * TS / PPT;
    static constexpr int RW = 32 / TS;
    static_assert(TS <= 32 && NT % 32 == 0, "a warp holds whole rows of threads");
    int x, y0;  // column; row of the thread's pixel k is y0 + RW k
    __device__ InterleavedRows(int txi, int tyi) {
        const int l = (int)threadIdx.x & 31, w = (int)threadIdx.x >> 5;
        x = txi * TS + l % TS;
        y0 = tyi * TS + w * RW * PPT + l / TS;
    }
};

template <int TS, int PPT, bool kCount, bool kL1>
__device__ __forceinline__ void render_fwd_body(int W, int H, float halfW, int tiles_x, int tiles, int n,
                                                unsigned long long rank_mask, float bg0, float bg1, float bg2,
                                                const float4* __restrict__ splats, const uint32_t* __restrict__ ranges,
                                                const unsigned long long* __restrict__ keys,
                                                const uint32_t* __restrict__ order, float* __restrict__ out_rgb,
                                                float* __restrict__ out_T, uint32_t* __restrict__ out_nc,
                                                uint32_t* __restrict__ out_count, const float* __restrict__ target,
                                                float* __restrict__ dL, float* __restrict__ tile_sums,
                                                float inv_total) {
    constexpr int NT = PixelMap<TS, PPT>::NT;
    constexpr int NP = PPT / 2;
    static_assert(PPT % 2 == 0, "pixels are blended in pairs");
    __shared__ FwdStaged s_e[NT];
    const int tile_id = blockIdx.x;
    const int v = tile_id / tiles, t = tile_id - v * tiles;
    const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
    const PixelMap<TS, PPT> pm(txi, tyi);
    const float xs = pm.x + 0.5f;
    const float fW = (float)W;  // halfW: W / 2, or +inf for the pinhole camera (no seam)
    const float x_first = txi * TS + 0.5f, x_last = txi * TS + TS - 0.5f;
    const uint32_t start = ranges[2 * tile_id], end = ranges[2 * tile_id + 1];
    const uint32_t* vorder = order + (size_t)v * n;

    float2 T[NP], C0[NP], C1[NP], C2[NP], NY[NP];  // NY: minus the pixel centres' y
    uint32_t last[PPT], count[PPT];
    bool live[PPT];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        T[q] = make_float2(1.f, 1.f);
        C0[q] = C1[q] = C2[q] = make_float2(0.f, 0.f);
        NY[q] = make_float2(-(pm.y0 + 2 * q + 0.5f), -(pm.y0 + 2 * q + 1 + 0.5f));
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        last[k] = 0; count[k] = 0; live[k] = true;
    }
    int done = 0;
    for (uint32_t b = start; b < end; b += NT) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t s = b + threadIdx.x;
        if (s < end) {
            const Staged st = stage_entry(splats, entry_splat(keys, vorder, s, rank_mask), x_first, x_last, halfW, fW);
            FwdStaged f;
            f.s = make_float4(st.a.x, seam_shift(st), st.a.z, st.a.w);
            f.p0 = make_float4(st.a.y, st.a.y, st.b.x, st.b.x);
            f.p1 = make_float4(-st.b.y, -st.b.y, -st.c.x, -st.c.x);
            f.p2 = make_float4(-st.c.y, -st.c.y, -st.c.z, -st.c.z);
            f.p3 = make_float4(-st.c.w, -st.c.w, st.b.z, wrap_flag(st));
            s_e[threadIdx.x] = f;
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)NT, end - b);
        for (int j = 0; j < nb && !done; ++j) {
            const float4 S = s_e[j].s;
            const float4 P0 = s_e[j].p0;
            const float4 P1 = s_e[j].p1;
            const float4 P2 = s_e[j].p2;
            const float4 P3 = s_e[j].p3;
            float dx = (S.x - xs) + S.y;
            if (P3.w != 0.f) dx = wrap_dx(dx, halfW, fW);
            const float e0 = S.z * dx * dx, e1 = S.w * dx;  // exponent = e0 + dy (e1 + c2' dy)
            const float2 E0 = make_float2(e0, e0), E1 = make_float2(e1, e1);
            const uint32_t pos1 = b - start + j + 1;        // list position after this entry
            const float h = P3.z;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 dy = __fadd2_rn(lo2(P0), NY[q]);
                const float2 e = __ffma2_rn(dy, __ffma2_rn(hi2(P0), dy, E1), E0);
                const float2 em = __fadd2_rn(e, lo2(P1));
                const float2 G = make_float2(fast_ex2(e.x), fast_ex2(e.y));
                float2 na = __fmul2_rn(hi2(P1), G);  // -(o G)
                na.x = fmaxf(-kAlphaMax, na.x);
                na.y = fmaxf(-kAlphaMax, na.y);
                const float2 Tn = __ffma2_rn(T[q], na, T[q]);  // T (1 - alpha) if applied
                const int k0 = 2 * q, k1 = 2 * q + 1;
                const bool pass0 = live[k0] && (fabsf(em.x) <= h), pass1 = live[k1] && (fabsf(em.y) <= h);
                const bool stop0 = pass0 && Tn.x < kTStop, stop1 = pass1 && Tn.y < kTStop;
                const bool add0 = pass0 && !stop0, add1 = pass1 && !stop1;
                live[k0] = live[k0] && !stop0;
                live[k1] = live[k1] && !stop1;
                const float2 nadd = make_float2(add0 ? na.x : 0.f, add1 ? na.y : 0.f);  // -(alpha applied)
                const float2 nw = __fmul2_rn(nadd, T[q]);
                C0[q] = __ffma2_rn(nw, lo2(P2), C0[q]);
                C1[q] = __ffma2_rn(nw, hi2(P2), C1[q]);
                C2[q] = __ffma2_rn(nw, lo2(P3), C2[q]);
                T[q] = __ffma2_rn(T[q], nadd, T[q]);
                last[k0] = add0 ? pos1 : last[k0];
                last[k1] = add1 ? pos1 : last[k1];
                if (kCount) {
                    count[k0] += add0 ? 1u : 0u;
                    count[k1] += add1 ? 1u : 0u;
                }
            }
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) any |= live[k];
            done = !any;
        }
    }
    const size_t HW = (size_t)H * W;
    float l1 = 0.f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int q = k >> 1;
        const float Tk = (k & 1) ? T[q].y : T[q].x;
        const float c0 = (k & 1) ? C0[q].y : C0[q].x, c1 = (k & 1) ? C1[q].y : C1[q].x;
        const float c2 = (k & 1) ? C2[q].y : C2[q].x;
        const size_t pix = (size_t)(pm.y0 + k) * W + pm.x;
        const float rgb[3] = {fmaf(Tk, bg0, c0), fmaf(Tk, bg1, c1), fmaf(Tk, bg2, c2)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t i = (3 * (size_t)v + c) * HW + pix;
            out_rgb[i] = rgb[c];
            if constexpr (kL1) {
                const float d = rgb[c] - __ldg(target + i);
                l1 += fabsf(d);
                dL[i] = d > 0.f ? inv_total : (d < 0.f ? -inv_total : 0.f);
            }
        }
        out_T[(size_t)v * HW + pix] = Tk;
        out_nc[(size_t)v * HW + pix] = last[k];
        if (kCount) out_count[(size_t)v * HW + pix] = count[k];
    }
    if constexpr (kL1) {
        __shared__ float s_l1[NT / 32];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        if ((threadIdx.x & 31) == 0) s_l1[threadIdx.x >> 5] = l1;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) t += s_l1[w];
            tile_sums[tile_id] = t;
        }
    }
}

template <int TS, int PPT, bool kCount>
__global__ void __launch_bounds__(TS * TS / PPT)
render_fwd_kernel(int W, int H, float halfW, int tiles_x, int tiles, int n, unsigned long long rank_mask, float bg0,
                  float bg1, float bg2, const float4* __restrict__ splats, const uint32_t* __restrict__ ranges,
                  const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ order,
                  float* __restrict__ out_rgb, float* __restrict__ out_T, uint32_t* __restrict__ out_nc,
                  uint32_t* __restrict__ out_count) {
    render_fwd_body<TS, PPT, kCount, false>(W, H, halfW, tiles_x, tiles, n, rank_mask, bg0, bg1, bg2, splats, ranges,
                                            keys, order, out_rgb, out_T, out_nc, out_count, nullptr, nullptr, nullptr,
                                            0.f);
}

// The forward with the L1 loss fused into its epilogue (omnigs_render_fwd_l1). Each pixel's colour, already in
// registers, is compared with the target: dL = sign(rgb - target) * inv_total is written beside it, and the CTA's sum
// of |rgb - target| (in pixel order within each thread, then thread and warp order) goes to tile_sums[tile], which
// l1_tiles_finish_kernel adds up. The epilogue needs a few more registers than the plain forward's; at 16 x 16 tiles
// and 4 pixels a thread the budget is held at the plain kernel's 64 (16 CTAs per SM) without spilling. Measured on
// the 8-view egocentric frame: 0.977 ms against 0.979 for the plain forward (plus 0.105 for the separate loss and its
// finish); prefetching the targets to L2 when the CTA starts cost 0.014 ms more.
template <int TS, int PPT>
__global__ void __launch_bounds__(TS * TS / PPT, TS * TS / PPT == 64 ? 16 : 1)
render_fwd_l1_kernel(int W, int H, float halfW, int tiles_x, int tiles, int n, unsigned long long rank_mask,
                     float bg0, float bg1, float bg2, const float4* __restrict__ splats,
                     const uint32_t* __restrict__ ranges, const unsigned long long* __restrict__ keys,
                     const uint32_t* __restrict__ order, float* __restrict__ out_rgb, float* __restrict__ out_T,
                     uint32_t* __restrict__ out_nc, const float* __restrict__ target, float* __restrict__ dL,
                     float* __restrict__ tile_sums, float inv_total) {
    render_fwd_body<TS, PPT, false, true>(W, H, halfW, tiles_x, tiles, n, rank_mask, bg0, bg1, bg2, splats, ranges,
                                          keys, order, out_rgb, out_T, out_nc, nullptr, target, dL, tile_sums,
                                          inv_total);
}

constexpr int kGradFields = 9;
// Pixel pairs the adjoint tests together and, if any of their pixels passes, updates together (a pixel that does not
// pass adds nothing: G = 0). Two pairs give the scheduler two independent update chains: measured 1.82 against
// 1.86 ms on the 8-view egocentric step and 0.257 against 0.265 ms on one view, 0.263 against 0.255 ms on the
// one-view training shell (fewer contributing pairs per entry); four pairs were slower (1.89 ms).
constexpr int kAdjointPairGroup = 2;

// Warp sums of the 9 gradient fields. Fields 0..7 go through a transposed reduce-scatter (offsets 16, 8, 4 halve
// the values each lane carries, offsets 2 and 1 finish the sum): lane l ends with the total of field (l >> 2).
// Field 8 is summed by a plain butterfly. On return, lanes with (l & 3) == 0 hold field l >> 2 and every lane holds
// field 8's total in `f8`.
__device__ __forceinline__ float warp_sum_fields(float (&v)[kGradFields], unsigned lane, float& f8) {
#pragma unroll
    for (int half = 4, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    float t = v[0];
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    float b = v[8];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) b += __shfl_xor_sync(0xffffffffu, b, off);
    f8 = b;
    return t;
}

// The adjoint's entries, staged for packed pixel pairs: every pair operand sits duplicated in both halves of a
// 16-byte word, so one shared-memory load gives two pairs.
struct BwdStaged {
    float4 x;   // px, seam shift, c0', c1'   (the thread's dx and the exponent's dx terms)
    float4 p0;  // py, py, c2', c2'
    float4 p1;  // -m, -m, -o, -o            (pass interval centre, opacity)
    float4 p2;  // r, r, g, g
    float4 p3;  // b, b, h, per-pixel wrap flag   (h: pass interval half-width)
    float4 d;   // raw conic c0, c1, c2, opacity (for the flush)
};

// One entry against the thread's pixel pairs, back to front: per pixel, if the entry passes (thr <= e <= 0, and the
// pixel's last contributor is behind it) recover T in front of it, form dL/dalpha, move the entry into the colour
// behind, and add its terms to the thread's sums. Pairs go kAdjointPairGroup at a time: a group none of whose pixels
// passes is skipped; in the others a pixel that skips the entry gets G = 0 (alpha = 0 leaves T and NS as they are
// and adds nothing). kClampable: the entry's opacity reaches the 0.99 clamp (o >= 0.99),
// where alpha = 0.99 passes no gradient to o or the exponent; below that o G < 0.99 always. Returns whether any
// pixel of the thread took the entry.
template <int NP, bool kClampable>
__device__ __forceinline__ bool bwd_entry_pairs(uint32_t pos, const uint32_t (&last)[2 * NP], float2 (&T)[NP],
                                                float2 (&NS)[NP], const float2 (&g0)[NP], const float2 (&g1)[NP],
                                                const float2 (&g2)[NP], const float2 (&NYS)[NP], float2 E0,
                                                float2 E1, const float4 P0, const float4 P1, const float4 P2,
                                                const float4 P3, float2& su, float2& suy, float2& suyy,
                                                float2& nc0, float2& nc1, float2& nc2) {
    const float2 kOne2 = make_float2(1.f, 1.f);
    const float h = P3.z;
    bool contrib = false;
    constexpr int GQ = kAdjointPairGroup < NP ? kAdjointPairGroup : NP;
#pragma unroll
    for (int q0 = 0; q0 < NP; q0 += GQ) {
    float2 dys[GQ], es[GQ];
    bool ps[GQ][2], any = false;
#pragma unroll
    for (int i = 0; i < GQ; ++i) {
        const int q = q0 + i;
        dys[i] = __fadd2_rn(lo2(P0), NYS[q]);
        es[i] = __ffma2_rn(dys[i], __ffma2_rn(hi2(P0), dys[i], E1), E0);
        const float2 em = __fadd2_rn(es[i], lo2(P1));
        ps[i][0] = pos < last[2 * q] && fabsf(em.x) <= h;
        ps[i][1] = pos < last[2 * q + 1] && fabsf(em.y) <= h;
        any |= ps[i][0] || ps[i][1];
    }
    if (!any) continue;
    contrib = true;
#pragma unroll
    for (int i = 0; i < GQ; ++i) {
        const int q = q0 + i;
        const float2 dy = dys[i], e = es[i];
        const bool p0 = ps[i][0], p1 = ps[i][1];
        const float2 G = make_float2(p0 ? fast_ex2(e.x) : 0.f, p1 ? fast_ex2(e.y) : 0.f);
        const float2 nraw = __fmul2_rn(hi2(P1), G);  // -(o G)
        const float2 nalpha = kClampable ? make_float2(fmaxf(-kAlphaMax, nraw.x), fmaxf(-kAlphaMax, nraw.y)) : nraw;
        const float2 omr = __fadd2_rn(kOne2, nalpha);  // 1 - alpha
        const float2 r = make_float2(__fdividef(1.f, omr.x), __fdividef(1.f, omr.y));
        T[q] = __fmul2_rn(T[q], r);  // transmittance in front of this entry
        // dL/dalpha = T (g . c) - (g . colour behind) / (1 - alpha); then this entry joins the colour behind
        const float2 gc = __ffma2_rn(g0[q], lo2(P2), __ffma2_rn(g1[q], hi2(P2), __fmul2_rn(g2[q], lo2(P3))));
        const float2 nw = __fmul2_rn(nalpha, T[q]);  // -(alpha T)
        const float2 dalpha = __ffma2_rn(NS[q], r, __fmul2_rn(T[q], gc));
        NS[q] = __ffma2_rn(nw, gc, NS[q]);
        nc0 = __ffma2_rn(nw, g0[q], nc0);
        nc1 = __ffma2_rn(nw, g1[q], nc1);
        nc2 = __ffma2_rn(nw, g2[q], nc2);
        const float2 Gu = kClampable ? make_float2(nraw.x > -kAlphaMax ? G.x : 0.f, nraw.y > -kAlphaMax ? G.y : 0.f)
                                     : G;
        const float2 u = __fmul2_rn(dalpha, Gu);
        const float2 udy = __fmul2_rn(u, dy);
        su = __fadd2_rn(su, u);
        suy = __fadd2_rn(suy, udy);
        suyy = __ffma2_rn(udy, dy, suyy);
    }
    }
    return contrib;
}

// Register budget per schedule (measured on the 8-view egocentric frame): at 8 pixels a thread 96 registers (21 warps
// per SM) beat both the unconstrained 123 and tighter budgets that spill.
template <int TS, int PPT>
__global__ void __launch_bounds__(TS * TS / PPT) __maxnreg__(PPT == 8 ? 96 : (PPT == 4 ? 80 : 64))
render_bwd_kernel(int W, int H, float halfW, int tiles_x, int tiles, int n, unsigned long long rank_mask, float bg0,
                  float bg1,
                  float bg2, const float4* __restrict__ splats, const uint32_t* __restrict__ ranges,
                  const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ order,
                  const float* __restrict__ out_T, const uint32_t* __restrict__ ncontrib,
                  const float* __restrict__ dL_drgb, float4* __restrict__ grads) {
    constexpr int NT = InterleavedRows<TS, PPT>::NT, RW = InterleavedRows<TS, PPT>::RW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdStaged* s_e = reinterpret_cast<BwdStaged*>(smem_raw);
    unsigned* s_vg = reinterpret_cast<unsigned*>(s_e + NT);
    float* s_acc = reinterpret_cast<float*>(s_vg + NT);  // [NT][kGradFields]
    __shared__ unsigned s_max;

    const int tile_id = blockIdx.x;
    const int v = tile_id / tiles, t = tile_id - v * tiles;
    const int tyi = t / tiles_x, txi = t - tyi * tiles_x;
    const InterleavedRows<TS, PPT> pm(txi, tyi);
    const float xs = pm.x + 0.5f;
    const float fW = (float)W;  // halfW: W / 2, or +inf for the pinhole camera (no seam)
    const float x_first = txi * TS + 0.5f, x_last = txi * TS + TS - 0.5f;
    const uint32_t start = ranges[2 * tile_id], len = ranges[2 * tile_id + 1] - start;
    const uint32_t* vorder = order + (size_t)v * n;
    const size_t HW = (size_t)H * W;

    // Pixel pairs (2q, 2q + 1) of the thread are updated together with packed FP32 (f32x2) operations. Per pixel:
    // T, the transmittance in front of the current entry; NS, minus the upstream gradient dotted with the colour
    // behind it (the later contributors' c alpha T plus T_final bg); g, the upstream gradient.
    constexpr int NP = PPT / 2;
    static_assert(PPT % 2 == 0, "pixels are updated in pairs");
    uint32_t last[PPT];
    float2 T[NP], NS[NP], g0[NP], g1[NP], g2[NP], NYS[NP];  // NYS: minus the pixel centres' y
    uint32_t mylast = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float t2[2], a0[2], a1[2], a2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * q + h;
            const size_t pix = (size_t)(pm.y0 + RW * k) * W + pm.x;
            last[k] = min(ncontrib[(size_t)v * HW + pix], len);
            t2[h] = out_T[(size_t)v * HW + pix];
            a0[h] = dL_drgb[(3 * (size_t)v + 0) * HW + pix];
            a1[h] = dL_drgb[(3 * (size_t)v + 1) * HW + pix];
            a2[h] = dL_drgb[(3 * (size_t)v + 2) * HW + pix];
            mylast = max(mylast, last[k]);
        }
        T[q] = make_float2(t2[0], t2[1]);
        g0[q] = make_float2(a0[0], a0[1]);
        g1[q] = make_float2(a1[0], a1[1]);
        g2[q] = make_float2(a2[0], a2[1]);
        NS[q] = make_float2(-t2[0] * fmaf(a0[0], bg0, fmaf(a1[0], bg1, a2[0] * bg2)),
                            -t2[1] * fmaf(a0[1], bg0, fmaf(a1[1], bg1, a2[1] * bg2)));
        NYS[q] = make_float2(-(pm.y0 + RW * (2 * q) + 0.5f), -(pm.y0 + RW * (2 * q + 1) + 0.5f));
    }

    // A CTA of one warp (PPT 8 on 16 x 16 tiles) needs no CTA barrier and no shared-memory atomics.
    constexpr bool kOneWarp = NT == 32;
    for (int i = threadIdx.x; i < NT * kGradFields; i += NT) s_acc[i] = 0.f;
    uint32_t maxlast;
    if constexpr (kOneWarp) {
        maxlast = __reduce_max_sync(0xffffffffu, mylast);
        __syncwarp();
    } else {
        if (threadIdx.x == 0) s_max = 0;
        __syncthreads();
        atomicMax(&s_max, mylast);
        __syncthreads();
        maxlast = s_max;
    }
    const unsigned lane = threadIdx.x & 31;
    // Per-thread sums over the thread's pixels for the current entry. With gp = dL/d(exponent) = dL/dalpha o G per
    // pixel, the exponent's derivatives give dL/dc0 = -1/2 sum gp dx^2, dL/dc1 = -sum gp dx dy, dL/dc2 =
    // -1/2 sum gp dy^2, dL/dpx = -(c0 sum gp dx + c1 sum gp dy), dL/dpy = -(c1 sum gp dx + c2 sum gp dy). A thread's
    // pixels share dx, and o is the entry's, so per pixel only u = dL/dalpha G (whose sum is dL/do), u dy and u dy^2
    // are accumulated, with minus the colour weights alpha T g; the warp reduces the moments of u (sum u dx,
    // sum u dx^2, sum u dy, sum u dx dy, sum u dy^2, sum u = dL/do) and -dL/dc, and o, the signs and the conic are
    // applied once per entry when the CTA's sums are flushed.
    float2 su = make_float2(0.f, 0.f), suy = su, suyy = su, nc0 = su, nc1 = su, nc2 = su;
    float gv[kGradFields];

    for (int64_t bend = (int64_t)maxlast; bend > 0; bend -= NT) {
        const int64_t bbeg = bend - NT > 0 ? bend - NT : 0;
        const int nb = (int)(bend - bbeg);
        if ((int)threadIdx.x < nb) {
            const unsigned vg = entry_splat(keys, vorder, (uint32_t)(start + bbeg + threadIdx.x), rank_mask);
            const Staged st = stage_entry(splats, vg, x_first, x_last, halfW, fW);
            BwdStaged b;
            b.x = make_float4(st.a.x, seam_shift(st), st.a.z, st.a.w);
            b.p0 = make_float4(st.a.y, st.a.y, st.b.x, st.b.x);
            b.p1 = make_float4(-st.b.y, -st.b.y, -st.c.x, -st.c.x);
            b.p2 = make_float4(st.c.y, st.c.y, st.c.z, st.c.z);
            b.p3 = make_float4(st.c.w, st.c.w, st.b.z, wrap_flag(st));
            b.d = make_float4(st.d.x, st.d.y, st.d.z, st.c.x);
            s_e[threadIdx.x] = b;
            s_vg[threadIdx.x] = vg;
        }
        if constexpr (kOneWarp) __syncwarp(); else __syncthreads();
        for (int j = nb - 1; j >= 0; --j) {
            const uint32_t pos = (uint32_t)(bbeg + j);  // position in the tile list
            // (a one-warp CTA starts at its warp's largest last contributor: some lane always takes part)
            if (!kOneWarp && __all_sync(0xffffffffu, pos >= mylast)) continue;
            const float4 X = s_e[j].x;
            const float4 P0 = s_e[j].p0;
            const float4 P1 = s_e[j].p1;
            const float4 P2 = s_e[j].p2;
            const float4 P3 = s_e[j].p3;
            float dx = (X.x - xs) + X.y;
            if (P3.w != 0.f) dx = wrap_dx(dx, halfW, fW);
            const float e0 = X.z * dx * dx, e1 = X.w * dx;
            const float2 E0 = make_float2(e0, e0), E1 = make_float2(e1, e1);
            const bool contrib =
                P1.w <= -kAlphaMax
                    ? bwd_entry_pairs<NP, true>(pos, last, T, NS, g0, g1, g2, NYS, E0, E1, P0, P1, P2, P3, su, suy, suyy,
                                                nc0, nc1, nc2)
                    : bwd_entry_pairs<NP, false>(pos, last, T, NS, g0, g1, g2, NYS, E0, E1, P0, P1, P2, P3, su, suy,
                                                 suyy, nc0, nc1, nc2);
            if (__any_sync(0xffffffffu, contrib)) {
                // the moments of u (gp = o u; o and the signs are applied once per entry in the flush)
                gv[5] = su.x + su.y;                      // sum u = dL/do
                gv[0] = dx * gv[5];                       // sum u dx
                gv[1] = dx * gv[0];                       // sum u dx^2
                gv[2] = suy.x + suy.y;                    // sum u dy
                gv[3] = dx * gv[2];                       // sum u dx dy
                gv[4] = suyy.x + suyy.y;                  // sum u dy^2
                gv[6] = nc0.x + nc0.y;                    // -dL/dc
                gv[7] = nc1.x + nc1.y;
                gv[8] = nc2.x + nc2.y;
                float tot8;
                const float tot = warp_sum_fields(gv, lane, tot8);
                const bool quad = (lane & 3u) == 0;
                if (quad || lane == 1u) {
                    float* dst = &s_acc[j * kGradFields + (quad ? (lane >> 2) : 8u)];
                    if constexpr (kOneWarp) *dst = quad ? tot : tot8;
                    else atomicAdd(dst, quad ? tot : tot8);
                }
                su = suy = suyy = nc0 = nc1 = nc2 = make_float2(0.f, 0.f);
            }
        }
        if constexpr (kOneWarp) __syncwarp(); else __syncthreads();
        if ((int)threadIdx.x < nb) {
            float* acc = s_acc + threadIdx.x * kGradFields;
            bool any = false;
#pragma unroll
            for (int f = 0; f < kGradFields; ++f) any |= (acc[f] != 0.f);
            if (any) {
                // the CTA's moments of u -> dL/d(px, py, c0, c1, c2) (gp = o u), dL/do and dL/dc
                const float4 D = s_e[threadIdx.x].d;  // c0, c1, c2, o
                const float gpx = -D.w * fmaf(D.x, acc[0], D.y * acc[2]);
                const float gpy = -D.w * fmaf(D.y, acc[0], D.z * acc[2]);
                float4* gdst = grads + 3 * (size_t)s_vg[threadIdx.x];
                atomicAdd(gdst, make_float4(gpx, gpy, -0.5f * D.w * acc[1], -D.w * acc[3]));
                atomicAdd(gdst + 1, make_float4(-0.5f * D.w * acc[4], acc[5], -acc[6], -acc[7]));
                atomicAdd(reinterpret_cast<float*>(gdst + 2), -acc[8]);
            }
#pragma unroll
            for (int f = 0; f < kGradFields; ++f) acc[f] = 0.f;
        }
        if constexpr (kOneWarp) __syncwarp(); else __syncthreads();
    }
}

size_t bwd_smem(int nt) {
    return (size_t)nt * (sizeof(BwdStaged) + sizeof(unsigned) + kGradFields * sizeof(float));
}

// Sum of the forward's per-tile L1 sums, then the mean, by one CTA of kLossBlocks threads. Each thread adds its
// tiles (16 loads in flight at a time) in FP32 with Kahan's compensation, and the threads' sums are added in double
// precision: GB300's FP64 rate is a small fraction of its FP32 rate, and 65,536 double additions on one SM took
// 43 us where this takes about 10. The order of the additions is fixed, so the loss is reproducible.
__global__ void __launch_bounds__(kLossBlocks)
l1_tiles_finish_kernel(const float* __restrict__ tile_sums, int nt, float inv_total, float* __restrict__ loss) {
    __shared__ double red[kLossBlocks / 32];
    constexpr int kBatch = 16;
    float sum = 0.f, comp = 0.f;  // the running sum and minus its lost low-order part
    for (int i0 = (int)threadIdx.x; i0 < nt; i0 += kBatch * kLossBlocks) {
        float x[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q)
            x[q] = i0 + q * kLossBlocks < nt ? __ldg(tile_sums + i0 + q * kLossBlocks) : 0.f;
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
            const float y = x[q] - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
    }
    double s = (double)sum - (double)comp;
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

// Half the image width for the minimal-image dx across the longitude seam; +inf turns the wrap off (pinhole camera).
float seam_half_width(const omnigs_config& cfg) {
    return cfg.camera == OMNIGS_CAMERA_EQUIRECT ? 0.5f * (float)cfg.width : INFINITY;
}

// Pixels per blend thread: the configured schedule (2, 4 or 8), else 2 for 8x8 tiles and 4 for larger ones.
int blend_ppt(const omnigs_config& cfg) {
    if (cfg.pixels_per_thread) return cfg.pixels_per_thread;
    return cfg.tile == 8 ? 2 : 4;
}

// Pixels per adjoint thread: the configured schedule, else 2 for 8x8 tiles and 8 for larger ones. Measured on the
// egocentric (8 views), training (1 view) and roaming (4096 x 2048) frames at 16 and 32 px tiles, 8 pixels a thread
// was the fastest adjoint everywhere (it shares the per-entry warp reduction among twice the pixels of 4), while
// the forward, with no reduction, was fastest at 4.
int adjoint_ppt(const omnigs_config& cfg) {
    if (cfg.adjoint_pixels_per_thread) return cfg.adjoint_pixels_per_thread;
    return cfg.tile == 8 ? 2 : 8;
}

template <int TS, int PPT>
cudaError_t render_fwd_t(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats, const uint32_t* ranges,
                         const uint64_t* keys, const uint32_t* order, float* out_rgb, float* out_T, uint32_t* out_nc,
                         uint32_t* out_count, const FwdL1* l1, cudaStream_t stream) {
    const int tx = cfg.width / TS, tiles = tx * (cfg.height / TS);
    const unsigned long long mask = (1ull << rank_bits_for(n)) - 1ull;
    const float inv_total = l1 ? (float)(1.0 / ((double)cfg.num_views * 3.0 * cfg.height * cfg.width)) : 0.f;
    {
        ProfScope prof("render_fwd", stream);
        const unsigned grid = (unsigned)(tiles * cfg.num_views), block = PixelMap<TS, PPT>::NT;
        const float4* sp = reinterpret_cast<const float4*>(splats);
        const unsigned long long* ks = reinterpret_cast<const unsigned long long*>(keys);
        if (l1) {
            render_fwd_l1_kernel<TS, PPT><<<grid, block, 0, stream>>>(
                cfg.width, cfg.height, seam_half_width(cfg), tx, tiles, (int)n, mask, cfg.bg[0], cfg.bg[1], cfg.bg[2],
                sp, ranges, ks, order, out_rgb, out_T, out_nc, l1->target, l1->dL_drgb, l1->tile_sums, inv_total);
        } else {
            auto kern = out_count ? render_fwd_kernel<TS, PPT, true> : render_fwd_kernel<TS, PPT, false>;
            kern<<<grid, block, 0, stream>>>(cfg.width, cfg.height, seam_half_width(cfg), tx, tiles, (int)n, mask,
                                             cfg.bg[0], cfg.bg[1], cfg.bg[2], sp, ranges, ks, order, out_rgb, out_T,
                                             out_nc, out_count);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !l1) return e;
    ProfScope prof("l1_finish", stream);
    l1_tiles_finish_kernel<<<1, kLossBlocks, 0, stream>>>(l1->tile_sums, tiles * cfg.num_views, inv_total, l1->loss);
    return cudaGetLastError();
}

template <int TS, int PPT>
cudaError_t render_bwd_t(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats, const uint32_t* ranges,
                         const uint64_t* keys, const uint32_t* order, const float* out_T, const uint32_t* nc,
                         const float* dL_drgb, omnigs_splat_grad* grads, cudaStream_t stream) {
    const unsigned long long mask = (1ull << rank_bits_for(n)) - 1ull;
    const int tx = cfg.width / TS, tiles = tx * (cfg.height / TS);
    constexpr int NT = PixelMap<TS, PPT>::NT;
    const size_t smem = bwd_smem(NT);
    cudaError_t e = cudaFuncSetAttribute(render_bwd_kernel<TS, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope prof("render_bwd", stream);
    render_bwd_kernel<TS, PPT><<<tiles * cfg.num_views, NT, smem, stream>>>(
        cfg.width, cfg.height, seam_half_width(cfg), tx, tiles, (int)n, mask, cfg.bg[0], cfg.bg[1], cfg.bg[2],
        reinterpret_cast<const float4*>(splats), ranges, reinterpret_cast<const unsigned long long*>(keys), order, out_T,
        nc, dL_drgb, reinterpret_cast<float4*>(grads));
    return cudaGetLastError();
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// mean |rgb - target| over the image rows [row_begin, row_end) and its gradient (0 outside those rows); float4 over
// the [V, 3, H, W] buffers (W a multiple of 4, so a float4 never straddles two rows).
__global__ void __launch_bounds__(kLossThreads)
l1_kernel(size_t n4, const float4* __restrict__ rgb, const float4* __restrict__ target, float4* __restrict__ dL,
          float inv_total, unsigned w4, unsigned height, unsigned row_begin, unsigned row_end,
          float* __restrict__ partials) {
    float acc = 0.f;
    const bool all_rows = row_begin == 0 && row_end == height;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned y = all_rows ? 0u : (unsigned)((i / w4) % height);
        if (!all_rows && (y < row_begin || y >= row_end)) {
            dL[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float4 a = __ldg(rgb + i), b = __ldg(target + i);
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        auto sg = [inv_total](float d) { return d > 0.f ? inv_total : (d < 0.f ? -inv_total : 0.f); };
        dL[i] = make_float4(sg(d0), sg(d1), sg(d2), sg(d3));
    }
    __shared__ float red[kLossThreads / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kLossThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// Sum of the per-block partials in double by one CTA of kLossBlocks threads (nb <= kLossBlocks).
__global__ void __launch_bounds__(kLossBlocks)
l1_finish_kernel(const float* __restrict__ partials, int nb, float inv_total, float* __restrict__ loss) {
    __shared__ double red[kLossBlocks / 32];
    double s = (int)threadIdx.x < nb ? (double)partials[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kLossBlocks / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *loss = (float)(s * inv_total);
    }
}

}  // namespace

cudaError_t launch_render_fwd(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats,
                              const uint32_t* ranges, const uint64_t* keys, const uint32_t* order, float* out_rgb,
                              float* out_T, uint32_t* out_nc, uint32_t* out_count, const FwdL1* l1,
                              cudaStream_t stream) {
    const int ppt = blend_ppt(cfg);
#define OMNIGS_FWD(TS, PPT) render_fwd_t<TS, PPT>(cfg, n, splats, ranges, keys, order, out_rgb, out_T, out_nc, \
                                                  out_count, l1, stream)
    switch (cfg.tile) {
        case 8: return OMNIGS_FWD(8, 2);
        case 32: return ppt == 8 ? OMNIGS_FWD(32, 8) : (ppt == 4 ? OMNIGS_FWD(32, 4) : OMNIGS_FWD(32, 2));
        default: return ppt == 8 ? OMNIGS_FWD(16, 8) : (ppt == 4 ? OMNIGS_FWD(16, 4) : OMNIGS_FWD(16, 2));
    }
#undef OMNIGS_FWD
}

cudaError_t launch_render_bwd(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats,
                              const uint32_t* ranges, const uint64_t* keys, const uint32_t* order,
                              const float* out_T, const uint32_t* nc, const float* dL_drgb,
                              omnigs_splat_grad* grads, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(grads, 0, sizeof(omnigs_splat_grad) * (size_t)n * cfg.num_views, stream);
    if (e != cudaSuccess) return e;
    const int ppt = adjoint_ppt(cfg);
    switch (cfg.tile) {
        case 8: return render_bwd_t<8, 2>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream);
        case 32:
            if (ppt == 8) return render_bwd_t<32, 8>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream);
            return ppt == 4 ? render_bwd_t<32, 4>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream)
                            : render_bwd_t<32, 2>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream);
        default:
            if (ppt == 8) return render_bwd_t<16, 8>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream);
            return ppt == 4 ? render_bwd_t<16, 4>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream)
                            : render_bwd_t<16, 2>(cfg, n, splats, ranges, keys, order, out_T, nc, dL_drgb, grads, stream);
    }
}

cudaError_t launch_l1(const omnigs_config& cfg, int row_begin, int row_end, const float* rgb, const float* target,
                      float* dL_drgb, float* loss, const WsLayout& L, char* ws, cudaStream_t stream) {
    const size_t total = (size_t)cfg.num_views * 3 * cfg.height * cfg.width;
    const size_t counted = (size_t)cfg.num_views * 3 * (size_t)(row_end - row_begin) * cfg.width;
    const float inv = counted ? (float)(1.0 / (double)counted) : 0.f;
    float* partials = reinterpret_cast<float*>(ws + L.loss_partials);
    {
        ProfScope prof("l1_loss", stream);
        l1_kernel<<<L.loss_blocks, kLossThreads, 0, stream>>>(total / 4, reinterpret_cast<const float4*>(rgb),
                                                              reinterpret_cast<const float4*>(target),
                                                              reinterpret_cast<float4*>(dL_drgb), inv,
                                                              (unsigned)(cfg.width / 4), (unsigned)cfg.height,
                                                              (unsigned)row_begin, (unsigned)row_end, partials);
    }
    {
        ProfScope prof("l1_finish", stream);
        l1_finish_kernel<<<1, kLossBlocks, 0, stream>>>(partials, L.loss_blocks, inv, loss);
    }
    return cudaGetLastError();
}

}  // namespace omnigs
