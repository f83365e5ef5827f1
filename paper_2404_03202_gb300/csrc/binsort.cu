// Tile binning ("one instance per influence", Sec. 3.3) and the sort of every tile's list by t_r (Sec. 3.3).
//
// The blending order is that of a stable sort of (view * TILES + tile, t_r) keys over instances generated splat by
// splat. Here that order is produced with short keys and coalesced passes only:
//   1. depth_keys + LSD sort: the V * N splats are sorted once by (view, t_r bits), stable, so ties keep splat order.
//      order[v * N + r] is the r-th nearest splat of view v (its depth rank r). Ranks are unique, so comparing ranks
//      equals comparing (t_r, splat index). When view, t_r bits and splat index fit 64 bits the index rides in the
//      key's low bits (keys only; the last pass writes those bits as the order); otherwise it is a value beside the
//      key. Pinhole views rank only the splats they can see (a compaction first).
//   2. bin_count / bin_scan / bin_emit walk the splats in depth order (through `order`), 256 per CTA: bin_count
//      derives the kept columns of every box row (the row culling) and stores the rows, bin_scan takes a 64-bit
//      exclusive scan of the per-CTA counts (overflow checked against the capacity), and bin_emit writes one entry
//      per instance from the stored rows, each chunk's slots in order through a load-balanced search.
//   Bucketed order (the usual case, see bucketed_binning):
//   3. bin_count also ranks every row item within its (view, tile row) bucket among the CTA's items; small scans give
//      each bucket its base and each CTA its offset in the bucket, and bin_emit writes every instance straight to its
//      bucket as a 32-bit entry (tx << rank_bits) | rank. Every bucket is then in rank order.
//   4. omnigs_sort: one stable counting pass by tile column within every bucket (tile_count: per-chunk column counts;
//      tile_ranges: their scans, which are also the tile ranges; tile_scatter: in-CTA stable ranking by column, the
//      lanes sharing a column found by ballots, written out as keys ((v * TILES + tile) << rank_bits) | rank).
//   Otherwise:
//   3. bin_emit writes the keys ((v * TILES + tile) << rank_bits) | rank in generation order, already in rank order
//      within every tile, and a stable LSD radix sort orders them over the tile bits only (ceil(log2(V * TILES))
//      bits above the rank, 2 passes of <= 9 bits: upsweep per-CTA digit counts; two small scans; downsweep with
//      stable in-CTA ranking, staging in shared memory in digit order, runs of equal digits written to HBM).
//   4. tile_ranges: [start, end) of every tile by binary search in the sorted keys.
// The keys carry no payload: the splat is order[v * N + rank].
// No pass waits on another CTA, so there are no spin loops.
#include <algorithm>

#include "common.cuh"

namespace omnigs {
namespace {

typedef unsigned long long u64;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

// Exclusive scan over the CTA; `scratch` holds >= blockDim/32 entries. Returns the CTA total in *total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* scratch, T* total) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nwarps ? scratch[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        if (lane < nwarps) scratch[lane] = s;
    }
    __syncthreads();
    T base = warp > 0 ? scratch[warp - 1] : T(0);
    T tot = scratch[nwarps - 1];
    __syncthreads();
    *total = tot;
    return base + x - v;
}

struct SplatPos {
    float px, py, depth;
    float c0, c1, c2, q;
    int rx, ry;  // instance box half-extents; rx = 0: no instance
};

// Splats whose centre is not a point of [0, W] x [0, H] (which the projection never produces) are treated as culled,
// so malformed input cannot produce a tile index outside the image.
__device__ __forceinline__ SplatPos load_pos(const float4* __restrict__ sp, size_t i, int tiles_x, int tiles_y,
                                             int tile, bool wrap) {
    const float4 a = __ldg(sp + 3 * i);      // px, py, c0, c1
    const float4 c = __ldg(sp + 3 * i + 1);  // c2, depth, radii, q
    SplatPos p;
    p.px = a.x;
    p.py = a.y;
    p.c0 = a.z;
    p.c1 = a.w;
    p.c2 = c.x;
    p.depth = c.y;
    const unsigned radii = __float_as_uint(c.z);
    p.rx = (int)(radii & 0xffffu);
    p.ry = (int)(radii >> 16);
    p.q = c.w;
    // the equirectangular projection lands in [0, W] x [0, H]; a pinhole centre may lie off the image (|p| < 2^23)
    const bool inside = wrap ? (a.x >= 0.f && a.x <= (float)(tiles_x * tile) && a.y >= 0.f &&
                                a.y <= (float)(tiles_y * tile))
                             : (fabsf(a.x) < 8388608.f && fabsf(a.y) < 8388608.f);
    if (!inside) p.rx = 0;
    return p;
}

// Column culling within the tile rows of a box. The alpha >= 1/255 ellipse dp^T conic dp <= q, with q raised to
// q (1.001) + 1e-3, spans, over a band of pixel-centre offsets v = y + 1/2 - py in [v_lo, v_hi], the offsets
// u in [x-(v_L), x+(v_R)], x-+(v) = -s v -+ sqrt(w2 - k v^2) with s = c1 / c0, w2 = q / c0, k = det / c0^2 and
// det = c0 c2 - c1^2, where v_L and v_R (the v of the ellipse's leftmost and rightmost points, +-c1 sqrt(q / (det c2)))
// are clamped to the band intersected with the ellipse's own rows |v| <= sqrt(q c0 / det). A tile column is kept when
// its pixel centres come within one pixel of that span; the widening of q and of the span absorbs the rounding of
// these single-precision steps. The row-invariant part is computed once per splat. Rows keep every column of the box
// when the box spans every column, when the conic is a needle (det <= 1e-3 c0 c2, where the bounds lose precision),
// and, with the longitude seam, when rx + tile > W / 2: only below that do the box's unwrapped column offsets equal
// the minimal-image offsets (|dx| < W / 2) that the blend evaluates, so the span is taken on the copy the blend uses.
// The quotients and square roots are the hardware approximations (relative error a few units in the last place):
// against the widening (one pixel; 0.1 % of q) their error is negligible, and they took bin_count from 0.484 to
// 0.464 ms on the 8-view egocentric frame (the conic entries are far below 2^126, where the fast quotient fails).
__device__ __forceinline__ float approx_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct RowCull {
    float px, py, s, yL;  // centre, shear c1 / c0, leftmost-point offset
    float ey, w2, k;      // ey < 0: no culling (whole rows)
};

__device__ __forceinline__ RowCull row_cull_setup(const SplatPos& p, int nx, int tiles_x, int tile, bool wrap) {
    RowCull rc = {p.px, p.py, 0.f, 0.f, -1.f, 0.f, 0.f};
    if (nx >= tiles_x) return rc;
    if (wrap && 2 * (p.rx + tile) > tiles_x * tile) return rc;
    const float c0c2 = __fmul_rn(p.c0, p.c2), c1c1 = __fmul_rn(p.c1, p.c1);
    const float det = __fsub_rn(c0c2, c1c1);
    const float guard = __fmul_rn(1e-3f, c0c2);
    if (!(det > guard) || !(p.c0 > 0.f) || !(p.c2 > 0.f)) return rc;
    const float qw = __fadd_rn(__fmul_rn(p.q, 1.001f), 1e-3f);
    rc.ey = approx_sqrt(__fdividef(__fmul_rn(qw, p.c0), det));
    rc.yL = __fmul_rn(p.c1, approx_sqrt(__fdividef(qw, __fmul_rn(det, p.c2))));
    rc.s = __fdividef(p.c1, p.c0);
    rc.w2 = __fdividef(qw, p.c0);
    rc.k = __fdividef(__fdividef(det, p.c0), p.c0);
    return rc;
}

// Unwrapped tile columns (first, last) of tile row ty kept by a box with columns x0 .. x0 + nx - 1; first > last: none.
__device__ __forceinline__ int2 row_cols(const RowCull& rc, int x0, int nx, int ty, int tile) {
    if (!(rc.ey >= 0.f)) return make_int2(x0, x0 + nx - 1);
    const float tyT = (float)(ty * tile), fT = (float)tile;
    const float yl = __fsub_rn(__fadd_rn(tyT, 0.5f), rc.py);
    const float yh = __fsub_rn(__fsub_rn(__fadd_rn(tyT, fT), 0.5f), rc.py);
    const float ney = -rc.ey;
    const float lo = yl > ney ? yl : ney;
    const float hi = yh < rc.ey ? yh : rc.ey;
    if (lo > hi) return make_int2(1, 0);
    const float nyL = -rc.yL;
    const float vL = rc.yL < lo ? lo : (rc.yL > hi ? hi : rc.yL);
    const float vR = nyL < lo ? lo : (nyL > hi ? hi : nyL);
    float hL = __fsub_rn(rc.w2, __fmul_rn(rc.k, __fmul_rn(vL, vL)));
    hL = hL > 0.f ? hL : 0.f;
    float hR = __fsub_rn(rc.w2, __fmul_rn(rc.k, __fmul_rn(vR, vR)));
    hR = hR > 0.f ? hR : 0.f;
    const float xl = __fsub_rn(-__fmul_rn(rc.s, vL), approx_sqrt(hL));
    const float xr = __fadd_rn(-__fmul_rn(rc.s, vR), approx_sqrt(hR));
    const float ul = __fsub_rn(__fadd_rn(rc.px, xl), 1.f);
    const float ur = __fadd_rn(__fadd_rn(rc.px, xr), 1.f);
    // tile column c reaches the band when c T + T - 1/2 >= ul and c T + 1/2 <= ur; T is a power of two, so the
    // product with 1 / T (built from its exponent) equals the correctly rounded quotient by T
    const float inv_T = __int_as_float((127 - (__ffs(tile) - 1)) << 23);
    float a = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(ul, 0.5f), fT), inv_T));
    float b = floorf(__fmul_rn(__fsub_rn(ur, 0.5f), inv_T));
    const float fx0 = (float)x0, fx1 = (float)(x0 + nx - 1);
    a = a > fx0 ? a : fx0;
    b = b < fx1 ? b : fx1;
    return make_int2((int)a, (int)b);
}

// The CTAs of the binning passes are dispatched view-interleaved, so that the first blocks of every view, which hold
// its nearest and widest splats and most of its instances, start first instead of forming a tail: dispatch index b
// runs the (b / V)-th block of view b mod V, view v owning the blocks from the one holding its first splat
// (floor(v n / kBinSplats)) up to the next view's. -1: no block (the grid is V times the largest view's block count).
__device__ __forceinline__ int64_t logical_block(int V, int64_t n, unsigned nb, unsigned b) {
    const int64_t v = b % (unsigned)V, j = b / (unsigned)V;
    const int64_t first = v * n / kBinSplats;
    const int64_t next = v + 1 < V ? (v + 1) * n / kBinSplats : (int64_t)nb;
    return first + j < next ? first + j : -1;
}

// ------------------------------------------------------------------------------------------- 1: splat depth order

__global__ void __launch_bounds__(kBinThreads)
depth_keys_kernel(int64_t total, int n, const float4* __restrict__ splats, u64* __restrict__ keys,
                  uint32_t* __restrict__ vals, u64* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    if (i == 0) *count = (u64)total;
    if (i >= total) return;
    const float d = __ldg(reinterpret_cast<const float*>(splats + 3 * i + 1) + 1);
    keys[i] = ((u64)(i / n) << 32) | (u64)__float_as_uint(d);
    vals[i] = (uint32_t)i;
}

// The same order from keys alone, when view, depth and splat index fit one 64-bit word: the index (gbits bits) rides
// below the (view, depth) bits the sort orders by, and index order breaks ties as the stable sort with values does.
// The sort's last pass writes only the index bits, which are the order.
__global__ void __launch_bounds__(kBinThreads)
depth_keys_packed_kernel(int64_t total, int n, int gbits, const float4* __restrict__ splats, u64* __restrict__ keys,
                         u64* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    if (i == 0) *count = (u64)total;
    if (i >= total) return;
    const float d = __ldg(reinterpret_cast<const float*>(splats + 3 * i + 1) + 1);
    keys[i] = ((((u64)(i / n) << 32) | (u64)__float_as_uint(d)) << gbits) | (u64)i;
}

// Pinhole views see a fraction of the scene, so their splats without instances (radius_x = 0: culled, or a box off
// the image) are left out of the depth sort: vis_count / vis_scan / depth_keys_compact write the keys of the others
// densely (view-major; view v's from vis_start[v]), and order_scatter puts the sorted splats back at
// order[v * n + rank]. A block covers kVisSlots slots of one view (4 strided slots per thread), so vis_start[v] is a
// block offset. vis_count reads only the radius word of each splat and leaves one ballot word per warp and slot
// group for the compaction, which keeps the slots in index order (the depth sort breaks ties by it).
constexpr int kVisWords = kVisSlots / 32;

__device__ __forceinline__ bool has_radius(const float4* __restrict__ splats, size_t i) {
    return (__ldg(reinterpret_cast<const unsigned*>(splats + 3 * i + 1) + 2) & 0xffffu) != 0u;
}

__global__ void __launch_bounds__(kBinThreads)
vis_count_kernel(int64_t n, int nbv, const float4* __restrict__ splats, unsigned* __restrict__ sums,
                 unsigned* __restrict__ masks) {
    __shared__ unsigned s_cnt[kBinThreads / 32];
    const int v = blockIdx.x / nbv, j = blockIdx.x - v * nbv;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    bool vis[kVisPerThread];
#pragma unroll
    for (int u = 0; u < kVisPerThread; ++u) {
        const int64_t g = (int64_t)j * kVisSlots + u * kBinThreads + threadIdx.x;
        vis[u] = g < n && has_radius(splats, (size_t)(v * n + g));
    }
    unsigned c = 0;
#pragma unroll
    for (int u = 0; u < kVisPerThread; ++u) {
        const unsigned m = __ballot_sync(0xffffffffu, vis[u]);
        if (lane == 0) masks[(size_t)blockIdx.x * kVisWords + u * (kBinThreads / 32) + warp] = m;
        c += __popc(m);
    }
    if (lane == 0) s_cnt[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kBinThreads / 32; ++w) t += s_cnt[w];
        sums[blockIdx.x] = t;
    }
}

// One CTA: exclusive scan of the per-block counts in place; vis_start[v] (v <= V) and the splat count.
__global__ void __launch_bounds__(1024)
vis_scan_kernel(int nblocks, int nbv, int V, unsigned* __restrict__ sums, unsigned* __restrict__ vis_start,
                u64* __restrict__ count) {
    __shared__ unsigned scratch[32];
    const int per = (nblocks + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nblocks);
    unsigned local = 0;
    for (int b = b0; b < b1; ++b) local += sums[b];
    unsigned tot;
    unsigned run = block_exclusive_scan<unsigned>(local, scratch, &tot);
    for (int b = b0; b < b1; ++b) {
        const unsigned c = sums[b];
        sums[b] = run;
        if (b % nbv == 0) vis_start[b / nbv] = run;
        run += c;
    }
    if (threadIdx.x == 0) {
        vis_start[V] = tot;
        *count = tot;
    }
}

__global__ void __launch_bounds__(kBinThreads)
depth_keys_compact_kernel(int64_t n, int nbv, const float4* __restrict__ splats, const unsigned* __restrict__ offsets,
                          const unsigned* __restrict__ masks, u64* __restrict__ keys, uint32_t* __restrict__ vals) {
    __shared__ unsigned s_word[kVisWords], s_before[kVisWords];
    const int v = blockIdx.x / nbv, j = blockIdx.x - v * nbv;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    static_assert(kVisWords == 32, "one warp scans the block's ballot words");
    if (warp == 0) {
        const unsigned m = __ldg(masks + (size_t)blockIdx.x * kVisWords + lane);
        unsigned x = __popc(m);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        s_word[lane] = m;
        s_before[lane] = x - __popc(m);
    }
    __syncthreads();
    const unsigned base = offsets[blockIdx.x];
#pragma unroll
    for (int u = 0; u < kVisPerThread; ++u) {
        const int w = u * (kBinThreads / 32) + (int)warp;
        const unsigned m = s_word[w];
        if (!((m >> lane) & 1u)) continue;
        const int64_t g = (int64_t)j * kVisSlots + u * kBinThreads + threadIdx.x;
        const size_t i = (size_t)(v * n + g);
        const unsigned c = base + s_before[w] + __popc(m & ((1u << lane) - 1u));
        const float d = __ldg(reinterpret_cast<const float*>(splats + 3 * i + 1) + 1);
        keys[c] = ((u64)v << 32) | (u64)__float_as_uint(d);
        vals[c] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(kBinThreads)
order_scatter_kernel(int64_t n, const u64* __restrict__ keys, const uint32_t* __restrict__ vals,
                     const unsigned* __restrict__ vis_start, const u64* __restrict__ count,
                     uint32_t* __restrict__ order) {
    const u64 i = (u64)blockIdx.x * kBinThreads + threadIdx.x;
    if (i >= *count) return;
    const unsigned v = (unsigned)(keys[i] >> 32);
    order[(u64)v * n + (i - vis_start[v])] = vals[i];
}

// ------------------------------------------------------------------------------------------- 2: instances

// Both instance passes give each CTA kBinSplats consecutive splats of the (view, depth) order (kSplatsPerThread
// consecutive ones per thread, their loads in flight together) and work on their box rows ("row items", in splat
// order), so that the rows of the nearest, widest splats, which depth order puts side by side, are spread over the
// whole CTA: every thread takes kRowsPerThread consecutive row items at a time (owner splat by one binary search over
// the CTA's prefix of row counts, then a forward walk).
constexpr int kRowChunk = 512;
constexpr int kRowsPerThread = kRowChunk / kBinThreads;

struct CtaRows {
    unsigned rexcl[kBinSplats];  // prefix of box-row counts over the CTA's splats
    int4 rect[kBinSplats];       // x0, nx, y0, depth rank
    float4 rc0[kBinSplats];      // RowCull: px, py, s, yL
    float4 rc1[kBinSplats];      //          ey, w2, k; the view's first tile key (bits)
};

// Loads splats i0 + kSplatsPerThread * tid + u (positions in (view, depth) order) and fills S; returns the CTA's
// row-item count.
__device__ __forceinline__ unsigned stage_rows(CtaRows& S, unsigned* scratch, const float4* __restrict__ splats,
                                               const uint32_t* __restrict__ order, int64_t i0, int64_t total, int64_t n,
                                               int tiles_x, int tiles_y, int tile, int wrap,
                                               const unsigned* __restrict__ vis_start) {
    const int s0 = threadIdx.x * kSplatsPerThread;
    unsigned rows[kSplatsPerThread], local = 0;
    uint32_t idx[kSplatsPerThread];
    bool ranked[kSplatsPerThread];  // positions beyond a compacted view's splat count hold no splat
#pragma unroll
    for (int u = 0; u < kSplatsPerThread; ++u) {
        const int64_t i = i0 + s0 + u;
        ranked[u] = i < total && (vis_start == nullptr ||
                                  i - (i / n) * n < (int64_t)(vis_start[i / n + 1] - vis_start[i / n]));
        idx[u] = ranked[u] ? __ldg(order + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kSplatsPerThread; ++u) {
        const int64_t i = i0 + s0 + u;
        rows[u] = 0;
        Rect r = {0, 1, 0, 0};
        int rank = 0;
        unsigned tbase = 0;
        RowCull rc = {0.f, 0.f, 0.f, 0.f, -1.f, 0.f, 0.f};
        if (ranked[u]) {
            const SplatPos p = load_pos(splats, (size_t)idx[u], tiles_x, tiles_y, tile, wrap);
            if (p.rx > 0) {
                r = splat_rect(p.px, p.py, p.rx, p.ry, tiles_x, tiles_y, __ffs(tile) - 1, wrap);
                rows[u] = r.nx > 0 ? (unsigned)r.ny : 0u;
                rc = row_cull_setup(p, r.nx, tiles_x, tile, wrap);
                const int64_t v = i / n;
                rank = (int)(i - v * n);
                tbase = (unsigned)v * (unsigned)(tiles_x * tiles_y);
            }
        }
        S.rect[s0 + u] = make_int4(r.x0, r.nx, r.y0, rank);
        S.rc0[s0 + u] = make_float4(rc.px, rc.py, rc.s, rc.yL);
        S.rc1[s0 + u] = make_float4(rc.ey, rc.w2, rc.k, __uint_as_float(tbase));
        local += rows[u];
    }
    unsigned rows_total;
    unsigned run = block_exclusive_scan<unsigned>(local, scratch, &rows_total);
#pragma unroll
    for (int u = 0; u < kSplatsPerThread; ++u) {
        S.rexcl[s0 + u] = run;
        run += rows[u];
    }
    __syncthreads();
    return rows_total;
}

// The splat owning row item ri: the largest j whose row prefix is <= ri (ri < the CTA's row-item count).
__device__ __forceinline__ int row_owner(const CtaRows& S, unsigned ri) {
    int j = 0;
#pragma unroll
    for (int step = kBinSplats / 2; step >= 1; step >>= 1)
        if (j + step < kBinSplats && S.rexcl[j + step] <= ri) j += step;
    return j;
}

// Kept columns of row item ri, whose owner is j or a later splat (j is advanced to it); tile row in *ty.
__device__ __forceinline__ int2 row_item_cols(const CtaRows& S, unsigned ri, int& j, int tile, int* ty) {
    while (j + 1 < kBinSplats && S.rexcl[j + 1] <= ri) ++j;
    const int4 rr = S.rect[j];
    const float4 a0 = S.rc0[j], a1 = S.rc1[j];
    const RowCull rq = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z};
    *ty = rr.z + (int)(ri - S.rexcl[j]);
    return row_cols(rq, rr.x, rr.y, *ty, tile);
}

// bin_count stores every row item it evaluates (in the tile-sort's spare key buffer, which is free until the sort),
// so that bin_emit reads them instead of re-gathering the splats and re-deriving the rows: first kept column
// (unwrapped, 16 bits), kept-column count, tile row and owner splat (position in the block) in one 64-bit word.
// A block whose rows do not fit (the buffer holds `capacity` items) is recomputed by bin_emit.
__device__ __forceinline__ u64 pack_row(int cl, unsigned cnt, int ty, int j) {
    return (u64)(unsigned short)cl | ((u64)cnt << 16) | ((u64)(unsigned)ty << 32) | ((u64)(unsigned)j << 48);
}

// ------------------------------------------------------------------------------------------- bucketed order
// With bucketed_binning, bin_emit writes every instance straight into its (view, tile row) bucket, in depth order,
// so that omnigs_sort only has to order each bucket by tile column. A block's row items of one bucket take
// consecutive slots after those of the earlier blocks; within the block, the slots follow the items' order
// (splat by splat in depth order). bin_count finds that order by a stable, weighted ranking of the block's row items
// (WarpBuckets); the fallback emission of blocks whose rows were not stored ranks each chunk again (BucketScratch).
constexpr int kBinWarps = kBinThreads / 32;
constexpr int kBucketSlots = 2 * kMaxBucketRows;  // a block's buckets: the tile rows of its (at most two) views

constexpr int kPendRows = 2048;  // row items whose in-warp offsets wait in shared memory for their warp's base

// bin_count's ranking: warp w's row items are the block's items [w * per, (w + 1) * per) in order, ranked 32 at a
// time against the warp's own bucket counters; afterwards every warp's base in a bucket is the count of the earlier
// warps' items there.
struct WarpBuckets {
    unsigned cw[kBinWarps][kBucketSlots];  // per warp: its items' instances in each bucket so far; then its base
    unsigned run[kBucketSlots];            // the block's instances in each bucket
    unsigned lw[kBinWarps][32];            // item weights of the current step, by warp and lane
    unsigned pend[kPendRows];              // row item ri < kPendRows: bucket << 24 | offset within its warp's items
};

struct BucketScratch {
    unsigned run[kBucketSlots];              // the block's instances in each bucket so far
    unsigned wt[kBinWarps][kBucketSlots];    // per-warp bucket totals of the current round (zero between rounds)
    unsigned lw[kBinThreads];                // item weights of the current round, by thread
    unsigned short bl[kRowChunk];            // bucket of each row item of the chunk (view in block * TY + row)
    unsigned w[kRowChunk];                   // its instance count
    unsigned off[kRowChunk];                 // out: its first instance's offset among the block's in the bucket
};

// Bucket offsets of the chunk's n_items row items (B.bl, B.w), in item order; advances B.run. Called by the whole
// CTA; B.wt holds zeros on entry and on return. Round r ranks items r .. r + 255 (one per thread): the lanes of a
// warp sharing a bucket are found by one ballot per bit of the bucket (a padding bucket for missing items
// included), each lane adds the weights of its lower peers, and the warps' totals per bucket are added in warp
// order.
__device__ __forceinline__ void rank_row_buckets(BucketScratch& B, unsigned n_items) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    for (unsigned r = 0; r < n_items; r += kBinThreads) {
        const unsigned i = r + threadIdx.x;
        const bool valid = i < n_items;
        const unsigned bl = valid ? B.bl[i] : (unsigned)kBucketSlots;
        const unsigned w = valid ? B.w[i] : 0u;
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b <= 8; ++b) {  // kBucketSlots = 256: 9 bits with the padding bucket
            const unsigned bit = (bl >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        B.lw[threadIdx.x] = w;
        __syncwarp();
        unsigned pre = 0;
        for (unsigned m = peers & lt; m; m &= m - 1) pre += B.lw[warp * 32 + (__ffs(m) - 1)];
        const bool leader = valid && (peers >> lane) == 1u;  // the highest lane of its group
        if (leader) B.wt[warp][bl] = pre + w;
        __syncthreads();
        if (valid) {
            unsigned xw = 0;
            for (unsigned q = 0; q < warp; ++q) xw += B.wt[q][bl];
            B.off[i] = B.run[bl] + xw + pre;
        }
        __syncthreads();
        if (leader) {
            atomicAdd(&B.run[bl], pre + w);
            B.wt[warp][bl] = 0u;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int64_t view_first_block(int64_t v, int64_t n) { return v * n / kBinSplats; }
__device__ __forceinline__ int64_t view_last_block(int64_t v, int64_t n) { return ((v + 1) * n - 1) / kBinSplats; }

// A block inside one view that starts past the view's ranked splats has nothing to do.
__device__ __forceinline__ bool block_unranked(int64_t blk, int64_t n, const unsigned* __restrict__ vis_start) {
    if (vis_start == nullptr) return false;
    const int64_t i0 = blk * kBinSplats, v = i0 / n;
    return i0 + kBinSplats <= (v + 1) * n && i0 - v * n >= (int64_t)(vis_start[v + 1] - vis_start[v]);
}

// kBuckets: also rank every row item within its (view, tile row) bucket (the offset goes to rows_off beside the row
// word) and write the block's instance count per bucket to bkt_counts[(v * tiles_y + ty) * nbv + block of view v].
template <bool kBuckets>
__global__ void __launch_bounds__(kBinThreads, kBuckets ? 6 : 8)
bin_count_kernel(int64_t total, const float4* __restrict__ splats, const uint32_t* __restrict__ order, int tiles_x,
                 int tiles_y, int tile, int wrap, int V, int64_t n, unsigned nb, const unsigned* __restrict__ vis_start,
                 unsigned* __restrict__ block_sums, u64* __restrict__ rows, u64 row_cap,
                 unsigned* __restrict__ row_base,
                 unsigned* __restrict__ row_count, WsHeader* __restrict__ hdr, unsigned* __restrict__ rows_off,
                 unsigned* __restrict__ bkt_counts, int nbv, unsigned* __restrict__ unstored_list) {
    __shared__ unsigned scratch[32];
    __shared__ CtaRows S;
    __shared__ unsigned s_rbase;
    __shared__ typename std::conditional<kBuckets, WarpBuckets, char>::type B;
    const int64_t blk = logical_block(V, n, nb, blockIdx.x);
    if (blk < 0) return;
    if (block_unranked(blk, n, vis_start)) {
        if (threadIdx.x == 0) {
            block_sums[blk] = 0;
            row_count[blk] = 0;
        }
        return;
    }
    const unsigned rows_total = stage_rows(S, scratch, splats, order, blk * kBinSplats, total, n, tiles_x, tiles_y,
                                           tile, wrap, vis_start);
    if (threadIdx.x == 0) {
        const u64 b = atomicAdd(&hdr->rows_used, (u64)rows_total);
        s_rbase = b + rows_total <= row_cap ? (unsigned)b : 0xffffffffu;
        row_base[blk] = s_rbase;
        row_count[blk] = rows_total;
        if (kBuckets && s_rbase == 0xffffffffu) unstored_list[atomicAdd(&hdr->unstored, 1u)] = (unsigned)blk;
    }
    __syncthreads();
    const unsigned rbase = s_rbase;
    unsigned cnt = 0;
    if constexpr (!kBuckets) {
        for (unsigned ri0 = threadIdx.x * kRowsPerThread; ri0 < rows_total; ri0 += kRowChunk) {
            int j = row_owner(S, ri0);
#pragma unroll
            for (int k = 0; k < kRowsPerThread; ++k) {
                const unsigned ri = ri0 + k;
                if (ri < rows_total) {
                    int ty;
                    const int2 c = row_item_cols(S, ri, j, tile, &ty);
                    const unsigned m = c.y >= c.x ? (unsigned)(c.y - c.x + 1) : 0u;
                    cnt += m;
                    if (rbase != 0xffffffffu) rows[(u64)rbase + ri] = pack_row(c.x, m, ty, j);
                }
            }
        }
    } else {
        // warp w ranks the block's row items [seg0, seg1), 32 at a time, against warp-private bucket counters
        for (int i = threadIdx.x; i < kBinWarps * kBucketSlots; i += kBinThreads) (&B.cw[0][0])[i] = 0u;
        __syncthreads();
        const int64_t p0 = blk * kBinSplats, v_lo = p0 / n, next_view = (v_lo + 1) * n - p0;
        const unsigned lane = lane_id(), warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
        const unsigned per = (rows_total + kBinWarps - 1) / kBinWarps;
        const unsigned seg0 = min(rows_total, warp * per), seg1 = min(rows_total, seg0 + per);
        for (unsigned b0 = seg0; b0 < seg1; b0 += 32) {
            const unsigned ri = b0 + lane;
            const bool valid = ri < seg1;
            unsigned m = 0, bl = kBucketSlots;
            if (valid) {
                int j = row_owner(S, ri), ty;
                const int2 c = row_item_cols(S, ri, j, tile, &ty);
                m = c.y >= c.x ? (unsigned)(c.y - c.x + 1) : 0u;
                bl = (j < next_view ? 0u : (unsigned)tiles_y) + (unsigned)ty;
                if (rbase != 0xffffffffu) rows[(u64)rbase + ri] = pack_row(c.x, m, ty, j);
            }
            cnt += m;
            // the lanes sharing a bucket (measured faster here than one ballot per bucket bit; the column pass,
            // with more keys per warp, is the other way round)
            const unsigned peers = __match_any_sync(0xffffffffu, bl);
            B.lw[warp][lane] = m;
            __syncwarp();
            unsigned pre = 0;
            for (unsigned q = peers & lt; q; q &= q - 1) pre += B.lw[warp][__ffs(q) - 1];
            if (valid) {
                const unsigned intra = B.cw[warp][bl] + pre;
                if (ri < (unsigned)kPendRows) B.pend[ri] = bl << 24 | intra;
                else if (rbase != 0xffffffffu) rows_off[(u64)rbase + ri] = intra;
            }
            __syncwarp();
            if (valid && (peers >> lane) == 1u) B.cw[warp][bl] += pre + m;  // the group's highest lane
            __syncwarp();
        }
        __syncthreads();
        // each warp's base in every bucket (earlier warps' items come first); the block's totals per bucket
        for (int bl = threadIdx.x; bl < kBucketSlots; bl += kBinThreads) {
            unsigned run = 0;
#pragma unroll
            for (int w = 0; w < kBinWarps; ++w) {
                const unsigned x = B.cw[w][bl];
                B.cw[w][bl] = run;
                run += x;
            }
            B.run[bl] = run;
        }
        __syncthreads();
        if (rbase != 0xffffffffu) {
            // the first kPendRows items from shared memory, written once; the rest (blocks of many rows) read back
            for (unsigned ri = seg0 + lane; ri < seg1; ri += 32) {
                if (ri < (unsigned)kPendRows) {
                    const unsigned e = B.pend[ri];
                    rows_off[(u64)rbase + ri] = (e & 0xffffffu) + B.cw[warp][e >> 24];
                } else if (warp > 0) {
                    const u64 w = rows[(u64)rbase + ri];
                    const int ty = (int)((w >> 32) & 0xffffu), j = (int)(w >> 48);
                    const unsigned bl = (j < next_view ? 0u : (unsigned)tiles_y) + (unsigned)ty;
                    rows_off[(u64)rbase + ri] += B.cw[warp][bl];
                }
            }
        }
        for (int i = threadIdx.x; i < 2 * tiles_y; i += kBinThreads) {
            const int lv = i / tiles_y, ty = i - lv * tiles_y;
            const int64_t v = v_lo + lv;
            if (v >= V || blk < view_first_block(v, n) || blk > view_last_block(v, n)) continue;
            bkt_counts[((size_t)v * tiles_y + ty) * nbv + (size_t)(blk - view_first_block(v, n))] = B.run[i];
        }
    }
    unsigned tot;
    block_exclusive_scan<unsigned>(cnt, scratch, &tot);
    if (threadIdx.x == 0) block_sums[blk] = tot;
}

// One CTA: exclusive scan of the per-CTA sums in 64 bits; total to the header, overflow flagged. With piece > 0, a
// block with more than `piece` instances gets ceil(sum / piece) - 1 extra bin_emit CTAs ("pieces"): piece_start[b]
// is the first of block b's extra pieces, piece_block[e] the block of extra piece e (at most max_pieces of them).
__global__ void __launch_bounds__(1024)
bin_scan_kernel(int nblocks, const unsigned* __restrict__ block_sums, u64* __restrict__ block_offsets,
                unsigned piece, unsigned* __restrict__ piece_start, unsigned* __restrict__ piece_block,
                unsigned max_pieces, WsHeader* __restrict__ hdr, u64 capacity) {
    __shared__ u64 scratch[32];
    __shared__ unsigned scratch32[32];
    constexpr int kLoads = 8;  // a thread's sums are read 8 at a time, all in flight (one latency per 8, not per sum)
    const int per = (nblocks + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nblocks);
    u64 local = 0;
    unsigned extra = 0;
    for (int b = b0; b < b1; b += kLoads) {
        unsigned v[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) v[q] = b + q < b1 ? block_sums[b + q] : 0u;
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            local += v[q];
            if (piece) extra += (v[q] + piece - 1) / piece - (v[q] > 0 ? 1u : 0u);
        }
    }
    u64 tot;
    u64 run = block_exclusive_scan<u64>(local, scratch, &tot);
    unsigned extra_tot;
    unsigned erun = block_exclusive_scan<unsigned>(extra, scratch32, &extra_tot);
    for (int b0q = b0; b0q < b1; b0q += kLoads) {
        unsigned v[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) v[q] = b0q + q < b1 ? block_sums[b0q + q] : 0u;
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            const int b = b0q + q;
            if (b >= b1) break;
            block_offsets[b] = run;
            run += v[q];
            if (!piece) continue;
            const unsigned eb = (v[q] + piece - 1) / piece - (v[q] > 0 ? 1u : 0u);
            piece_start[b] = erun;
            for (unsigned k = 0; k < eb; ++k)
                if (erun + k < max_pieces) piece_block[erun + k] = (unsigned)b;
            erun += eb;
        }
    }
    if (threadIdx.x == 0) {
        hdr->count = tot;
        hdr->extra_pieces = min(extra_tot, max_pieces);
        if (tot > capacity) hdr->error |= kErrCapacity;
    }
}

// The splats of a CTA (consecutive in depth order) own one contiguous output range. Their row items are taken
// kRowsPerThread consecutive ones per thread at a time; a CTA scan of the kept-column counts gives every row item its
// output offset. The items of the chunk then go to shared memory, and the CTA writes the chunk's output slots in
// order, thread t taking slots t, t + 256, ...: a binary search over the item offsets finds the slot's row, so every
// store instruction writes 256 consecutive keys whatever the rows' lengths (the nearest splats have rows of hundreds
// of tiles, most others of one to four). Instances of a splat are listed row by row, columns in seam order.

struct EmitBuckets {
    u64 bpos[kBucketSlots];  // output position of the block's first instance in each of its buckets
    u64 pos[kRowChunk];      // output position of each row item's first instance
    BucketScratch R;         // the ranking, for blocks whose rows were not stored
};

// kBuckets: each instance goes to its (view, tile row) bucket: the bucket's base, plus the block's offset in the
// bucket (both from the bucket scans), plus the row item's offset among the block's instances of the bucket (from
// bin_count's ranking, or ranked again here), plus its column index within the item.
template <bool kSplit, bool kBuckets>
__global__ void __launch_bounds__(kBinThreads, kBuckets ? 5 : 8)
bin_emit_kernel(int64_t total, int n, const float4* __restrict__ splats, const uint32_t* __restrict__ order,
                int tiles_x, int tiles_y, int tile, int wrap, int rank_bits, int V, unsigned nb, unsigned piece,
                unsigned max_pieces,
                const unsigned* __restrict__ vis_start, const unsigned* __restrict__ block_sums,
                const u64* __restrict__ block_offsets, const unsigned* __restrict__ piece_start,
                const unsigned* __restrict__ piece_block, const WsHeader* __restrict__ hdr,
                const u64* __restrict__ rows, const unsigned* __restrict__ row_base,
                const unsigned* __restrict__ row_count, void* __restrict__ keys_out, u64 capacity,
                const unsigned* __restrict__ rows_off, const unsigned* __restrict__ bkt_offsets,
                const u64* __restrict__ bkt_base, int nbv, const unsigned* __restrict__ fallback_list) {
    __shared__ unsigned scratch[32];
    __shared__ CtaRows S;
    __shared__ struct {
        unsigned off[kRowChunk];  // output offset of each row item of the chunk, relative to the chunk
        int cl[kRowChunk];        // its first column
        u64 key0[kRowChunk];      // key of its first column, before the column wrap
    } E;
    __shared__ typename std::conditional<kBuckets, EmitBuckets, char>::type EB;
    // The first max_pieces CTAs take the extra pieces of the blocks with more than `piece` instances (the
    // nearest, widest splats, which would otherwise leave one CTA writing hundreds of thousands of keys while the
    // others idle); they start first. The rest take piece 0 of every block, view-interleaved.
    // With kBuckets this kernel writes only the blocks whose row items bin_count could not store (fallback_list):
    // the CTAs take them in turn, whole (no pieces).
    int64_t blk;
    u64 lo = 0;  // output slots [lo, lo + piece) of the block are this CTA's (all of them for a light block)
    unsigned e_fb = blockIdx.x;
    if constexpr (kBuckets) {
        if (e_fb >= hdr->unstored) return;
        blk = fallback_list[e_fb];
    } else if (kSplit && blockIdx.x < max_pieces) {
        const unsigned e = blockIdx.x;
        if (e >= hdr->extra_pieces) return;
        blk = piece_block[e];
        lo = (u64)(1 + e - piece_start[blk]) * piece;
    } else {
        blk = logical_block(V, n, nb, blockIdx.x - max_pieces);
        if (blk < 0 || block_unranked(blk, n, vis_start)) return;
    }
    for (;;) {
    const u64 hi = kSplit && block_sums[blk] > piece ? lo + piece : ~0ull;
    const unsigned rbase = row_base[blk];
    const bool stored = rbase != 0xffffffffu;  // block-uniform: rows from bin_count, or derived again here
    const unsigned rows_total = stored ? row_count[blk]
                                       : stage_rows(S, scratch, splats, order, blk * kBinSplats, total, n, tiles_x,
                                                    tiles_y, tile, wrap, vis_start);
    // depth rank and view of the block's splat j: the block's 256 positions span at most two views
    const int64_t p0 = blk * kBinSplats, v0 = p0 / n, next_view = (v0 + 1) * n - p0;
    const unsigned lane = lane_id();
    const u64 first = block_offsets[blk];
    if constexpr (kBuckets) {
        for (int i = threadIdx.x; i < 2 * tiles_y; i += kBinThreads) {
            const int lv = i / tiles_y, ty = i - lv * tiles_y;
            const int64_t v = v0 + lv;
            u64 p = 0;
            if (v < V && blk >= view_first_block(v, n) && blk <= view_last_block(v, n)) {
                const size_t b = (size_t)v * tiles_y + ty;
                p = bkt_base[b] + bkt_offsets[b * nbv + (size_t)(blk - view_first_block(v, n))];
            }
            EB.bpos[i] = p;
        }
        if (!stored) {
            for (int i = threadIdx.x; i < kBucketSlots; i += kBinThreads) EB.R.run[i] = 0u;
            for (int i = threadIdx.x; i < kBinWarps * kBucketSlots; i += kBinThreads) (&EB.R.wt[0][0])[i] = 0u;
        }
        __syncthreads();
    }
    const u64 plo = first + lo, phi = kSplit && hi != ~0ull ? first + hi : ~0ull;  // this CTA's output positions
    u64 out = first;
    for (unsigned r0 = 0; r0 < rows_total && (!kSplit || out < phi); r0 += kRowChunk) {
        const unsigned ri0 = r0 + threadIdx.x * kRowsPerThread;
        unsigned cnt[kRowsPerThread], local = 0;
        u64 key0[kRowsPerThread];  // key of the item's first column, before the column wrap
        int cl[kRowsPerThread];
        unsigned bl[kRowsPerThread], boff[kRowsPerThread];  // bucketed order: the item's bucket and its offset
        int j = !stored && ri0 < rows_total ? row_owner(S, ri0) : 0;
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const unsigned ri = ri0 + k;
            cnt[k] = 0;
            cl[k] = 0;
            key0[k] = 0;
            bl[k] = 0;
            boff[k] = 0;
            if (ri < rows_total) {
                int ty;
                if (stored) {
                    const u64 w = __ldg(rows + (u64)rbase + ri);
                    cl[k] = (int)(short)(unsigned short)(w & 0xffffu);
                    cnt[k] = (unsigned)(w >> 16) & 0xffffu;
                    ty = (int)((w >> 32) & 0xffffu);
                    j = (int)(w >> 48);
                } else {
                    const int2 c = row_item_cols(S, ri, j, tile, &ty);
                    cnt[k] = c.y >= c.x ? (unsigned)(c.y - c.x + 1) : 0u;
                    cl[k] = c.x;
                }
                const int64_t v = j < next_view ? v0 : v0 + 1;
                const unsigned rank = (unsigned)(p0 + j - v * n);
                const unsigned tb = (unsigned)v * (unsigned)(tiles_x * tiles_y) + (unsigned)(ty * tiles_x);
                key0[k] = kBuckets ? (u64)rank : ((u64)tb << rank_bits) | (u64)rank;  // a bucket entry: no tile bits
                if constexpr (kBuckets) {
                    bl[k] = (j < next_view ? 0u : (unsigned)tiles_y) + (unsigned)ty;
                    boff[k] = stored ? __ldg(rows_off + (u64)rbase + ri) : 0u;
                }
            }
            if constexpr (kBuckets) {
                if (!stored) {
                    const unsigned li = threadIdx.x * kRowsPerThread + k;
                    EB.R.bl[li] = (unsigned short)bl[k];
                    EB.R.w[li] = cnt[k];
                }
            }
            local += cnt[k];
        }
        if constexpr (kBuckets) {
            if (!stored) {  // block-uniform
                __syncthreads();
                rank_row_buckets(EB.R, min((unsigned)kRowChunk, rows_total - r0));
#pragma unroll
                for (int k = 0; k < kRowsPerThread; ++k) boff[k] = EB.R.off[threadIdx.x * kRowsPerThread + k];
            }
        }
        unsigned chunk_total;
        unsigned rel = block_exclusive_scan<unsigned>(local, scratch, &chunk_total);  // offset within the chunk
        if (kSplit && out + chunk_total <= plo) {  // the chunk lies before this CTA's piece
            out += chunk_total;
            continue;
        }
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const int i = threadIdx.x * kRowsPerThread + k;
            E.off[i] = rel;
            E.cl[i] = cl[k];
            E.key0[i] = key0[k];
            if constexpr (kBuckets) EB.pos[i] = EB.bpos[bl[k]] + boff[k];
            rel += cnt[k];
        }
        __syncthreads();
        // output slot s of the chunk belongs to the last row item whose offset is <= s (items without columns share
        // their successor's offset and are passed over)
        unsigned s_lo = 0, s_hi = chunk_total;
        if (kSplit) {
            s_lo = plo > out ? (plo - out < chunk_total ? (unsigned)(plo - out) : chunk_total) : 0u;
            s_hi = phi - out < chunk_total ? (unsigned)(phi - out) : chunk_total;
        }
        for (unsigned sl = s_lo + threadIdx.x; sl < s_hi; sl += kBinThreads) {
            int i = 0;
#pragma unroll
            for (int step = kRowChunk / 2; step >= 1; step >>= 1)
                if (E.off[i + step] <= sl) i += step;
            // a box narrower than the image has columns in (-tiles_x, 2 tiles_x): one wrap at most
            int tx = E.cl[i] + (int)(sl - E.off[i]);
            tx += tx < 0 ? tiles_x : (tx >= tiles_x ? -tiles_x : 0);
            if constexpr (kBuckets) {
                const u64 at = EB.pos[i] + (sl - E.off[i]);
                if (at < capacity)
                    static_cast<unsigned*>(keys_out)[at] = (unsigned)E.key0[i] | ((unsigned)tx << rank_bits);
            } else {
                const u64 at = out + sl;
                if (at < capacity) static_cast<u64*>(keys_out)[at] = E.key0[i] + ((u64)tx << rank_bits);
            }
        }
        __syncthreads();
        out += chunk_total;
    }
    if constexpr (!kBuckets) {
        return;
    } else {
        e_fb += gridDim.x;
        if (e_fb >= hdr->unstored) return;
        blk = fallback_list[e_fb];
        __syncthreads();
    }
    }
}

// Bucketed order, blocks whose row items bin_count stored with their bucket offsets (the others are left to the
// fallback launch of bin_emit_kernel). Same block and piece dispatch as bin_emit_kernel; each row item's first
// instance goes to its bucket's base + the block's offset in the bucket + the item's offset within the block.
template <bool kSplit>
__global__ void __launch_bounds__(kBinThreads, 8)
bin_emit_stored_kernel(int n, int tiles_x, int tiles_y, int rank_bits, int V, unsigned nb, unsigned piece,
                       unsigned max_pieces, const unsigned* __restrict__ block_sums,
                       const u64* __restrict__ block_offsets, const unsigned* __restrict__ piece_start,
                       const unsigned* __restrict__ piece_block, const WsHeader* __restrict__ hdr,
                       const u64* __restrict__ rows, const unsigned* __restrict__ rows_off,
                       const unsigned* __restrict__ row_base, const unsigned* __restrict__ row_count,
                       const unsigned* __restrict__ bkt_offsets, const u64* __restrict__ bkt_base, int nbv,
                       unsigned* __restrict__ entries, u64 capacity) {
    __shared__ unsigned scratch[32];
    __shared__ struct {
        unsigned off[kRowChunk];  // output slot of each row item of the chunk, relative to the chunk
        int cl[kRowChunk];        // its first column
        unsigned rank[kRowChunk];  // its splat's depth rank
        u64 pos[kRowChunk];       // output position of its first instance
    } E;
    __shared__ u64 s_bpos[kBucketSlots];
    int64_t blk;
    u64 lo = 0;
    if (kSplit && blockIdx.x < max_pieces) {
        const unsigned e = blockIdx.x;
        if (e >= hdr->extra_pieces) return;
        blk = piece_block[e];
        lo = (u64)(1 + e - piece_start[blk]) * piece;
    } else {
        blk = logical_block(V, n, nb, blockIdx.x - max_pieces);
        if (blk < 0) return;
    }
    const unsigned rows_total = row_count[blk];
    if (rows_total == 0) return;
    const unsigned rbase = row_base[blk];
    if (rbase == 0xffffffffu) return;  // not stored: the fallback launch writes this block
    const u64 hi = kSplit && block_sums[blk] > piece ? lo + piece : ~0ull;
    const int64_t p0 = blk * kBinSplats, v0 = p0 / n, next_view = (v0 + 1) * n - p0;
    for (int i = threadIdx.x; i < 2 * tiles_y; i += kBinThreads) {
        const int lv = i / tiles_y, ty = i - lv * tiles_y;
        const int64_t v = v0 + lv;
        u64 p = 0;
        if (v < V && blk >= view_first_block(v, n) && blk <= view_last_block(v, n)) {
            const size_t b = (size_t)v * tiles_y + ty;
            p = bkt_base[b] + bkt_offsets[b * nbv + (size_t)(blk - view_first_block(v, n))];
        }
        s_bpos[i] = p;
    }
    __syncthreads();
    u64 out = 0;  // slots of the block before the current chunk
    const u64 slo = lo, shi = hi;
    for (unsigned r0 = 0; r0 < rows_total && (!kSplit || out < shi); r0 += kRowChunk) {
        const unsigned ri0 = r0 + threadIdx.x * kRowsPerThread;
        unsigned cnt[kRowsPerThread], local = 0;
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const unsigned ri = ri0 + k;
            const int i = threadIdx.x * kRowsPerThread + k;
            cnt[k] = 0;
            if (ri < rows_total) {
                const u64 w = __ldg(rows + (u64)rbase + ri);
                const int cl = (int)(short)(unsigned short)(w & 0xffffu);
                const int ty = (int)((w >> 32) & 0xffffu), j = (int)(w >> 48);
                cnt[k] = (unsigned)(w >> 16) & 0xffffu;
                const int64_t v = j < next_view ? v0 : v0 + 1;
                E.cl[i] = cl;
                E.rank[i] = (unsigned)(p0 + j - v * n);
                E.pos[i] = s_bpos[(j < next_view ? 0 : tiles_y) + ty] + __ldg(rows_off + (u64)rbase + ri);
            }
            local += cnt[k];
        }
        unsigned chunk_total;
        unsigned rel = block_exclusive_scan<unsigned>(local, scratch, &chunk_total);
        if (kSplit && out + chunk_total <= slo) {
            out += chunk_total;
            __syncthreads();
            continue;
        }
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            E.off[threadIdx.x * kRowsPerThread + k] = rel;
            rel += cnt[k];
        }
        __syncthreads();
        unsigned s_lo = 0, s_hi = chunk_total;
        if (kSplit) {
            s_lo = slo > out ? (slo - out < chunk_total ? (unsigned)(slo - out) : chunk_total) : 0u;
            s_hi = shi - out < chunk_total ? (unsigned)(shi - out) : chunk_total;
        }
        for (unsigned sl = s_lo + threadIdx.x; sl < s_hi; sl += kBinThreads) {
            int i = 0;
#pragma unroll
            for (int step = kRowChunk / 2; step >= 1; step >>= 1)
                if (E.off[i + step] <= sl) i += step;
            int tx = E.cl[i] + (int)(sl - E.off[i]);
            tx += tx < 0 ? tiles_x : (tx >= tiles_x ? -tiles_x : 0);
            const u64 at = E.pos[i] + (sl - E.off[i]);
            if (at < capacity) entries[at] = E.rank[i] | ((unsigned)tx << rank_bits);
        }
        __syncthreads();
        out += chunk_total;
    }
}

// ------------------------------------------------------------------------------------------- 3: LSD radix sort

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per CTA tile
constexpr int kWarps = kSortThreads / 32;
constexpr int kHistRow = kRadixMax + 1;  // + one bucket for the padding past the end

struct TileSpan {
    u64 begin, end;
};

__device__ __forceinline__ TileSpan cta_tiles(u64 cnt, int G) {
    const u64 tiles_total = (cnt + kSortTile - 1) / kSortTile;
    const u64 tpb = (tiles_total + G - 1) / G;
    TileSpan s;
    s.begin = min((u64)blockIdx.x * tpb, tiles_total);
    s.end = min(s.begin + tpb, tiles_total);
    return s;
}

__global__ void __launch_bounds__(kSortThreads)
lsd_upsweep_kernel(const u64* __restrict__ keys, const u64* __restrict__ count, u64 capacity, int shift, int dbits,
                   unsigned* __restrict__ hist, int G) {
    __shared__ unsigned s_hist[kWarps][kRadixMax];
    const unsigned R = 1u << dbits, mask = R - 1;
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    for (unsigned d = lane; d < R; d += 32) s_hist[warp][d] = 0;
    __syncwarp();
    const u64 cnt = min(*count, capacity);
    const TileSpan span = cta_tiles(cnt, G);
    for (u64 t = span.begin; t < span.end; ++t) {
        const u64 base = t * kSortTile + warp * (kSortItems * 32) + lane;
        unsigned d[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const u64 idx = base + (u64)j * 32;
            d[j] = idx < cnt ? (unsigned)(__ldg(keys + idx) >> shift) & mask : R;
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j)
            if (d[j] < R) atomicAdd(&s_hist[warp][d[j]], 1u);
    }
    __syncthreads();
    for (unsigned d = threadIdx.x; d < R; d += blockDim.x) {
        unsigned s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += s_hist[w][d];
        hist[(size_t)d * G + blockIdx.x] = s;
    }
}

// Exclusive scan of the digit-major histogram [R][G] in two small launches: one CTA per digit scans that digit's G
// per-CTA counts in place and writes the digit total; one CTA scans the R totals into digit starts. The downsweep
// adds both.
__global__ void __launch_bounds__(256) lsd_scan_digit_kernel(unsigned* __restrict__ hist, int G,
                                                            unsigned* __restrict__ totals) {
    __shared__ unsigned scratch[32];
    unsigned* h = hist + (size_t)blockIdx.x * G;
    const int per = (G + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, G);
    unsigned local = 0;
    for (int b = b0; b < b1; ++b) local += h[b];
    unsigned tot;
    unsigned run = block_exclusive_scan<unsigned>(local, scratch, &tot);
    for (int b = b0; b < b1; ++b) {
        const unsigned c = h[b];
        h[b] = run;
        run += c;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRadixMax) lsd_scan_totals_kernel(unsigned* __restrict__ totals, int R) {
    __shared__ unsigned scratch[32];
    const unsigned v = (int)threadIdx.x < R ? totals[threadIdx.x] : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_scan<unsigned>(v, scratch, &tot);
    if ((int)threadIdx.x < R) totals[threadIdx.x] = ex;
}

template <bool kVals>
size_t downsweep_smem() {
    return sizeof(u64) * kSortTile + (kVals ? sizeof(unsigned) * kSortTile : 0) +
           sizeof(unsigned) * (kWarps * kHistRow + 3 * kRadixMax + 32);
}

template <bool kVals>
__global__ void __launch_bounds__(kSortThreads, 3)
lsd_downsweep_kernel(const u64* __restrict__ keys_in, const unsigned* __restrict__ vals_in, u64* __restrict__ keys_out,
                     unsigned* __restrict__ vals_out, const u64* __restrict__ count, u64 capacity, int shift, int dbits,
                     const unsigned* __restrict__ hist, const unsigned* __restrict__ digit_start, int G,
                     uint32_t* __restrict__ low_out, u64 low_mask) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64* s_keys = reinterpret_cast<u64*>(smem_raw);
    unsigned* s_vals = reinterpret_cast<unsigned*>(s_keys + kSortTile);
    unsigned* s_whist = kVals ? s_vals + kSortTile : s_vals;
    unsigned* s_start = s_whist + kWarps * kHistRow;
    unsigned* s_tot = s_start + kRadixMax;
    unsigned* s_gbase = s_tot + kRadixMax;
    unsigned* s_scratch = s_gbase + kRadixMax;

    const unsigned R = 1u << dbits, mask = R - 1;
    const unsigned tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const unsigned lt_mask = (1u << lane) - 1u;
    const u64 cnt = min(*count, capacity);
    const TileSpan span = cta_tiles(cnt, G);
    for (unsigned d = tid; d < R; d += kSortThreads) s_gbase[d] = digit_start[d] + hist[(size_t)d * G + blockIdx.x];
    unsigned* my_hist = s_whist + warp * kHistRow;

    for (u64 t = span.begin; t < span.end; ++t) {
        for (unsigned d = lane; d <= R; d += 32) my_hist[d] = 0;
        __syncwarp();
        const u64 base = t * kSortTile + warp * (kSortItems * 32) + lane;
        u64 k[kSortItems];
        unsigned val[kSortItems], rk[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const u64 idx = base + (u64)j * 32;
            const bool ok = idx < cnt;
            k[j] = ok ? __ldg(keys_in + idx) : ~0ull;
            if (kVals) val[j] = ok ? __ldg(vals_in + idx) : 0u;
        }
        // rank within the warp: the lanes holding the same digit (found by one ballot per digit bit, the padding
        // digit R included) take consecutive slots after the warp's running count of that digit; every lane reads
        // the count, and the lowest lane of each digit advances it (the digits' counters are distinct addresses)
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const u64 idx = base + (u64)j * 32;
            const unsigned d = idx < cnt ? (unsigned)(k[j] >> shift) & mask : R;
            unsigned peers = 0xffffffffu;
            for (int b = 0; b <= dbits; ++b) {
                const unsigned bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            const unsigned before = my_hist[d];
            __syncwarp();
            if ((peers & lt_mask) == 0) my_hist[d] = before + __popc(peers);
            __syncwarp();
            rk[j] = before + __popc(peers & lt_mask);
        }
        __syncthreads();
        for (unsigned d = tid; d < R; d += kSortThreads) {
            unsigned acc = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const unsigned c = s_whist[w * kHistRow + d];
                s_whist[w * kHistRow + d] = acc;
                acc += c;
            }
            s_tot[d] = acc;
        }
        __syncthreads();
        {
            constexpr int PER = kRadixMax / kSortThreads;
            unsigned loc[PER], sum = 0;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const unsigned d = tid * PER + q;
                loc[q] = d < R ? s_tot[d] : 0u;
                sum += loc[q];
            }
            unsigned tile_total;
            unsigned run = block_exclusive_scan<unsigned>(sum, s_scratch, &tile_total);
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const unsigned d = tid * PER + q;
                if (d < R) s_start[d] = run;
                run += loc[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const u64 idx = base + (u64)j * 32;
            if (idx < cnt) {
                const unsigned d = (unsigned)(k[j] >> shift) & mask;
                const unsigned pos = s_start[d] + my_hist[d] + rk[j];
                s_keys[pos] = k[j];
                if (kVals) s_vals[pos] = val[j];
            }
        }
        __syncthreads();
        const unsigned nvalid = (unsigned)min((u64)kSortTile, cnt - t * kSortTile);
        for (unsigned i = tid; i < nvalid; i += kSortThreads) {
            const u64 key = s_keys[i];
            const unsigned d = (unsigned)(key >> shift) & mask;
            const unsigned gpos = s_gbase[d] + (i - s_start[d]);
            if (low_out != nullptr) low_out[gpos] = (uint32_t)(key & low_mask);  // last pass: only the low bits
            else keys_out[gpos] = key;
            if (kVals) vals_out[gpos] = s_vals[i];
        }
        __syncthreads();
        for (unsigned d = tid; d < R; d += kSortThreads) s_gbase[d] += s_tot[d];
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------- 4: tile ranges

// Tile t's range in the sorted keys, by two binary searches over (key >> rank_bits).
__global__ void ranges_kernel(const u64* __restrict__ keys, const WsHeader* __restrict__ hdr, u64 capacity,
                              int rank_bits, u64 ntiles, uint32_t* __restrict__ ranges) {
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const u64 cnt = min(hdr->count, capacity);
    u64 lo = 0, hi = cnt;  // first position with tile >= t
    while (lo < hi) {
        const u64 mid = (lo + hi) >> 1;
        if ((__ldg(keys + mid) >> rank_bits) < t) lo = mid + 1;
        else hi = mid;
    }
    const u64 first = lo;
    hi = cnt;  // first position with tile > t
    while (lo < hi) {
        const u64 mid = (lo + hi) >> 1;
        if ((__ldg(keys + mid) >> rank_bits) <= t) lo = mid + 1;
        else hi = mid;
    }
    ranges[2 * t] = (uint32_t)(first < lo ? first : 0);
    ranges[2 * t + 1] = (uint32_t)(first < lo ? lo : 0);
}

// ------------------------------------------------------------------------------------------- 5: bucketed order

// Per (view, tile row) bucket b = v * tiles_y + ty (one CTA each): exclusive scan, in place, of the instance counts
// of view v's blocks; the bucket's total.
__global__ void __launch_bounds__(256)
bucket_scan_kernel(int tiles_y, int64_t n, int nbv, unsigned* __restrict__ counts, u64* __restrict__ totals) {
    __shared__ u64 scratch[32];
    const int b = blockIdx.x;
    const int64_t v = b / tiles_y;
    const int nblk = (int)(view_last_block(v, n) - view_first_block(v, n) + 1);
    unsigned* c = counts + (size_t)b * nbv;
    constexpr int kLoads = 8;  // read 8 at a time, all in flight
    const int per = (nblk + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nblk);
    u64 local = 0;
    for (int i = b0; i < b1; i += kLoads) {
        unsigned v[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) v[q] = i + q < b1 ? c[i + q] : 0u;
#pragma unroll
        for (int q = 0; q < kLoads; ++q) local += v[q];
    }
    u64 tot;
    u64 run = block_exclusive_scan<u64>(local, scratch, &tot);
    for (int i = b0; i < b1; i += kLoads) {
        unsigned v[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) v[q] = i + q < b1 ? c[i + q] : 0u;
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            if (i + q < b1) c[i + q] = (unsigned)run;
            run += v[q];
        }
    }
    if (threadIdx.x == 0) totals[b] = tot;
}

// One CTA: every bucket's base (exclusive scan of the totals, 64-bit), the part of it below the capacity (`eff`;
// instances past the capacity were not written), and the column pass's chunks of kColChunk keys: bucket b owns
// chunks col_start[b] .. col_start[b + 1] - 1; col_start[nbkt] is their number.
__global__ void __launch_bounds__(1024)
bucket_base_kernel(int nbkt, const u64* __restrict__ totals, u64* __restrict__ base, u64* __restrict__ eff,
                   unsigned* __restrict__ col_start, u64 capacity) {
    __shared__ u64 scratch[32];
    __shared__ unsigned scratch32[32];
    const int per = (nbkt + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nbkt);
    u64 local = 0;
    for (int b = b0; b < b1; ++b) local += totals[b];
    u64 tot;
    u64 run = block_exclusive_scan<u64>(local, scratch, &tot);
    unsigned chunks = 0;
    for (int b = b0; b < b1; ++b) {
        const u64 e = run < capacity ? min(totals[b], capacity - run) : 0ull;
        base[b] = run;
        eff[b] = e;
        chunks += (unsigned)((e + kColChunk - 1) / kColChunk);
        run += totals[b];
    }
    unsigned ctot;
    unsigned crun = block_exclusive_scan<unsigned>(chunks, scratch32, &ctot);
    for (int b = b0; b < b1; ++b) {
        col_start[b] = crun;
        crun += (unsigned)((eff[b] + kColChunk - 1) / kColChunk);
    }
    if (threadIdx.x == 0) col_start[nbkt] = ctot;
}

// One column-pass chunk of bucket entries copied into shared memory by the bulk-copy engine (cp.async.bulk, TMA's
// untiled form): one thread arms an mbarrier with the byte count and issues the copy; every thread waits on the
// barrier's first phase. A bulk copy wants 16-byte aligned addresses and a multiple of 16 bytes, so the window starts
// at the chunk's first entry rounded down to 4 entries and ends at its last rounded up: entry i of the chunk is
// window entry lead + i (lead = first entry mod 4). The window may run up to 3 entries past the chunk; the
// workspace region holding the entries is padded for that. The wait is bounded in time (kBulkWaitNs of the global
// nanosecond timer): on timeout the CTA flags kErrTimeout and reports failure, and the caller skips the chunk.
constexpr int kColWindow = kColChunk + 8;  // entries of the shared-memory window (chunk, lead and rounding)
constexpr unsigned long long kBulkWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool bulk_load_window(unsigned* s_win, unsigned long long* s_bar,
                                                 const unsigned* __restrict__ entries, u64 first, u64 last,
                                                 unsigned* lead, WsHeader* __restrict__ hdr) {
    const u64 a0 = first & ~3ull, a1 = (last + 3) & ~3ull;  // [first, last): the chunk's entries
    const unsigned bytes = (unsigned)(a1 - a0) * 4u;
    *lead = (unsigned)(first - a0);
    const unsigned bar = smem_u32(s_bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(s_win)), "l"(entries + a0), "r"(bytes), "r"(bar)
                     : "memory");
    }
    unsigned done = 0;
    const unsigned long long t0 = global_ns();
    for (;;) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar)
                     : "memory");
        if (done || global_ns() - t0 > kBulkWaitNs) break;
    }
    if (!done) {
        atomicOr(&hdr->error, kErrTimeout);
        return false;
    }
    return true;
}

// Bucket of column-pass chunk c: the last b with col_start[b] <= c (buckets without chunks are passed over).
__device__ __forceinline__ int chunk_bucket(const unsigned* __restrict__ col_start, int nbkt, unsigned c) {
    int lo = 0, hi = nbkt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(col_start + mid) <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Column count of chunk c: hist[c][tx] (one CTA per chunk; CTAs past the last chunk return). A bucket entry is
// (tx << rank_bits) | depth rank; its bucket b = v * tiles_y + ty gives the rest of the tile key, b * tiles_x + tx.
__global__ void __launch_bounds__(kSortThreads)
col_count_kernel(const unsigned* __restrict__ entries, const u64* __restrict__ base, const u64* __restrict__ eff,
                 const unsigned* __restrict__ col_start, int nbkt, int tiles_x, int rank_bits,
                 unsigned* __restrict__ hist, WsHeader* __restrict__ hdr) {
    __shared__ unsigned s_h[kMaxBucketCols];
    __shared__ __align__(128) unsigned s_win[kColWindow];
    __shared__ __align__(8) unsigned long long s_bar;
    const unsigned c = blockIdx.x;
    if (c >= __ldg(col_start + nbkt)) return;
    const int b = chunk_bucket(col_start, nbkt, c);
    const u64 beg = base[b] + (u64)(c - col_start[b]) * kColChunk;
    const u64 end = min(beg + kColChunk, base[b] + eff[b]);
    for (int d = threadIdx.x; d < tiles_x; d += kSortThreads) s_h[d] = 0u;
    unsigned lead;
    const bool ok = bulk_load_window(s_win, &s_bar, entries, beg, end, &lead, hdr);  // syncs the CTA
    const unsigned cnt = ok ? (unsigned)(end - beg) : 0u;
    for (unsigned i = threadIdx.x; i < cnt; i += kSortThreads) {
        const unsigned d = s_win[lead + i] >> rank_bits;
        if (d < (unsigned)tiles_x) atomicAdd(&s_h[d], 1u);
        else atomicOr(&hdr->error, kErrConsistency);  // a key outside its bucket: not counted
    }
    __syncthreads();
    for (int d = threadIdx.x; d < tiles_x; d += kSortThreads) hist[(size_t)c * tiles_x + d] = s_h[d];
}

// Per bucket (one CTA, thread tx per column): exclusive scan over the bucket's chunks of hist[.][tx], then over the
// columns of their totals; hist[c][tx] becomes the output position of chunk c's first key of column tx, and the tile
// ranges of the bucket's tiles are written ([0, 0) for an empty tile). The chunk counts are read kScanBatch at a time,
// all in flight together: a bucket has tens of chunks, and one dependent load after another would take a memory
// latency each.
constexpr int kScanBatch = 16;

__global__ void __launch_bounds__(kMaxBucketCols)
col_scan_kernel(const u64* __restrict__ base, const unsigned* __restrict__ col_start, int tiles_x,
                unsigned* __restrict__ hist, uint32_t* __restrict__ ranges) {
    __shared__ unsigned scratch[32];
    const int b = blockIdx.x;
    const unsigned c0 = col_start[b], c1 = col_start[b + 1];
    const int tx = threadIdx.x;
    const bool col = tx < tiles_x;
    unsigned run = 0;
    if (col)
        for (unsigned c = c0; c < c1; c += kScanBatch) {
            unsigned h[kScanBatch];
#pragma unroll
            for (int q = 0; q < kScanBatch; ++q) h[q] = c + q < c1 ? hist[(size_t)(c + q) * tiles_x + tx] : 0u;
#pragma unroll
            for (int q = 0; q < kScanBatch; ++q) run += h[q];
        }
    unsigned tot;
    const unsigned start = block_exclusive_scan<unsigned>(col ? run : 0u, scratch, &tot);
    if (!col) return;
    const unsigned first = (unsigned)base[b] + start;
    unsigned at = first;
    for (unsigned c = c0; c < c1; c += kScanBatch) {
        unsigned h[kScanBatch];
#pragma unroll
        for (int q = 0; q < kScanBatch; ++q) h[q] = c + q < c1 ? hist[(size_t)(c + q) * tiles_x + tx] : 0u;
#pragma unroll
        for (int q = 0; q < kScanBatch; ++q) {
            if (c + q < c1) hist[(size_t)(c + q) * tiles_x + tx] = at;
            at += h[q];
        }
    }
    const size_t t = (size_t)b * tiles_x + tx;
    ranges[2 * t] = run ? first : 0u;
    ranges[2 * t + 1] = run ? first + run : 0u;
}

// Chunk c of a bucket, ordered by column and written to its final positions as tile keys (one CTA per chunk): the
// entries are ranked stably by column within each warp (the lanes sharing a column found by one ballot per column
// bit, a padding column for missing entries included), the warps' counts are combined in warp order, the entries are
// placed in column order in shared memory, and each is written to hist[c][tx] + its rank within its column.
__global__ void __launch_bounds__(kSortThreads, 4)
col_scatter_kernel(const unsigned* __restrict__ entries, u64* __restrict__ keys_out, const u64* __restrict__ base,
                   const u64* __restrict__ eff, const unsigned* __restrict__ col_start, int nbkt, int tiles_x,
                   int dbits, int rank_bits, const unsigned* __restrict__ hist, u64 capacity,
                   WsHeader* __restrict__ hdr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned* s_ent = reinterpret_cast<unsigned*>(smem_raw);
    unsigned* s_whist = s_ent + kSortTile;  // [kWarps][kHistRow]
    unsigned* s_start = s_whist + kWarps * kHistRow;
    unsigned* s_tot = s_start + kRadixMax;
    unsigned* s_scratch = s_tot + kRadixMax;

    const unsigned c = blockIdx.x;
    if (c >= __ldg(col_start + nbkt)) return;
    const int b = chunk_bucket(col_start, nbkt, c);
    const u64 beg = base[b] + (u64)(c - col_start[b]) * kColChunk;
    const unsigned cnt = (unsigned)(min(beg + kColChunk, base[b] + eff[b]) - beg);
    const u64 tile0 = (u64)b * tiles_x;
    const unsigned R = 1u << dbits, rank_mask = (1u << rank_bits) - 1u;
    const unsigned tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned* my_hist = s_whist + warp * kHistRow;
    for (unsigned d = lane; d <= R; d += 32) my_hist[d] = 0;
    __syncwarp();
    const unsigned base_i = warp * (kSortItems * 32) + lane;
    // (plain loads, all in flight at once: staging the chunk by bulk copy, as col_count does, measured slower here)
    unsigned k[kSortItems], rd[kSortItems];  // rd: rank within the warp's column << 16 | column
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const unsigned idx = base_i + j * 32;
        k[j] = idx < cnt ? __ldg(entries + beg + idx) : 0u;
    }
    unsigned* s_h = s_scratch + 32;  // the chunk's output positions per column, hist[c][.]
    for (int d = tid; d < tiles_x; d += kSortThreads) s_h[d] = __ldg(hist + (size_t)c * tiles_x + d);
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const unsigned idx = base_i + j * 32, dk = k[j] >> rank_bits;
        const unsigned d = idx < cnt && dk < (unsigned)tiles_x ? dk : R;  // an entry outside its columns: left out
        unsigned peers = 0xffffffffu;
        for (int bt = 0; bt <= dbits; ++bt) {
            const unsigned bal = __ballot_sync(0xffffffffu, (d >> bt) & 1u);
            peers &= ((d >> bt) & 1u) ? bal : ~bal;
        }
        const unsigned before = my_hist[d];
        __syncwarp();
        if ((peers & lt_mask) == 0) my_hist[d] = before + __popc(peers);
        __syncwarp();
        rd[j] = (before + __popc(peers & lt_mask)) << 16 | d;
    }
    __syncthreads();
    for (unsigned d = tid; d < R; d += kSortThreads) {
        unsigned acc = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const unsigned x = s_whist[w * kHistRow + d];
            s_whist[w * kHistRow + d] = acc;
            acc += x;
        }
        s_tot[d] = acc;
    }
    __syncthreads();
    {
        constexpr int PER = kRadixMax / kSortThreads;
        unsigned loc[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const unsigned d = tid * PER + q;
            loc[q] = d < R ? s_tot[d] : 0u;
            sum += loc[q];
        }
        unsigned tile_total;
        unsigned run = block_exclusive_scan<unsigned>(sum, s_scratch, &tile_total);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const unsigned d = tid * PER + q;
            if (d < R) s_start[d] = run;
            run += loc[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const unsigned d = rd[j] & 0xffffu;
        if (d < R) s_ent[s_start[d] + my_hist[d] + (rd[j] >> 16)] = k[j];
    }
    __syncthreads();
    const unsigned placed = s_start[R - 1] + s_tot[R - 1];  // entries with a column (all, unless one was left out)
    if (tid == 0 && placed != cnt) atomicOr(&hdr->error, kErrConsistency);
    for (unsigned i = tid; i < placed; i += kSortThreads) {
        const unsigned e = s_ent[i], d = e >> rank_bits;
        const u64 at = (u64)s_h[d] + (i - s_start[d]);
        if (at < capacity) keys_out[at] = ((tile0 + d) << rank_bits) | (u64)(e & rank_mask);
    }
}

// Radix-sort geometry: `bits` key bits in an even number of passes of <= 9 bits.
struct Plan {
    int passes, digit;
};

Plan plan_for(int bits) {
    Plan p;
    p.passes = (bits + 8) / 9;
    if (p.passes < 2) p.passes = 2;
    if (p.passes % 2) ++p.passes;
    p.digit = (bits + p.passes - 1) / p.passes;
    return p;
}

// Stable sort of `count` (device) keys (and values) in (k0, v0) by key bits [lo_bit, lo_bit + bits), through (k1, v1);
// the result lands back in (k0, v0), or, with low_out, only the sorted keys' bits under low_mask land in low_out.
template <bool kVals>
cudaError_t lsd_sort(u64* k0, unsigned* v0, u64* k1, unsigned* v1, const u64* count, u64 capacity, int lo_bit,
                     int bits, int G, unsigned* hist, cudaStream_t stream, const char* tag_up, const char* tag_down,
                     uint32_t* low_out = nullptr, u64 low_mask = 0) {
    const Plan P = plan_for(bits);
    const size_t smem = downsweep_smem<kVals>();
    cudaError_t e = cudaFuncSetAttribute(lsd_downsweep_kernel<kVals>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < P.passes; ++p) {
        const int shift = lo_bit + p * P.digit;
        const int db = std::max(1, std::min(P.digit, lo_bit + bits - shift));
        {
            ProfScope prof(tag_up, stream, 3);
            lsd_upsweep_kernel<<<G, kSortThreads, 0, stream>>>(k0, count, capacity, shift, db, hist, G);
            lsd_scan_digit_kernel<<<1 << db, 256, 0, stream>>>(hist, G, hist + (size_t)kRadixMax * G);
            lsd_scan_totals_kernel<<<1, kRadixMax, 0, stream>>>(hist + (size_t)kRadixMax * G, 1 << db);
        }
        {
            ProfScope prof(tag_down, stream);
            uint32_t* lo = p + 1 == P.passes ? low_out : nullptr;
            lsd_downsweep_kernel<kVals><<<G, kSortThreads, smem, stream>>>(k0, v0, k1, v1, count, capacity, shift, db,
                                                                            hist, hist + (size_t)kRadixMax * G, G, lo,
                                                                            low_mask);
        }
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    return cudaGetLastError();
}

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

int sort_grid(u64 elems) {
    const u64 tiles = (elems + kSortTile - 1) / kSortTile;
    return (int)std::max<u64>(1, std::min<u64>(tiles, (u64)num_sms() * kSortCtasPerSm));
}

}  // namespace

int rank_bits_for(int64_t n) { return std::max(1, ceil_log2((uint64_t)std::max<int64_t>(n, 1))); }

int tile_key_bits(const omnigs_config& cfg) {
    const uint64_t tiles = (uint64_t)(cfg.width / cfg.tile) * (cfg.height / cfg.tile) * cfg.num_views;
    return std::max(1, ceil_log2(tiles));
}

bool packed_depth_keys(const omnigs_config& cfg, int64_t n, int* gbits) {
    const int64_t total = n * cfg.num_views;
    *gbits = std::max(1, ceil_log2((uint64_t)std::max<int64_t>(total, 1)));
    return cfg.camera == OMNIGS_CAMERA_EQUIRECT && ceil_log2(cfg.num_views) + 32 + *gbits <= 64;
}

// depth_keys_ready: the caller zeroed the header and wrote the packed depth keys and the splat count (the fused
// preprocess of omnigs_preprocess_bin; only where packed_depth_keys holds).
cudaError_t launch_bin(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats, uint32_t* order,
                       uint64_t* keys, int64_t capacity, const WsLayout& L, char* ws, cudaStream_t stream,
                       bool depth_keys_ready) {
    const int64_t total = n * cfg.num_views;
    const int tx = cfg.width / cfg.tile, ty = cfg.height / cfg.tile;
    const int wrap = cfg.camera == OMNIGS_CAMERA_EQUIRECT;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    cudaError_t e = depth_keys_ready ? cudaSuccess : cudaMemsetAsync(hdr, 0, sizeof(WsHeader), stream);
    if (e != cudaSuccess || total == 0) return e;
    const float4* sp = reinterpret_cast<const float4*>(splats);
    u64* dk0 = reinterpret_cast<u64*>(ws + L.depth_keys);
    u64* dk1 = reinterpret_cast<u64*>(ws + L.depth_keys_alt);
    unsigned* dv1 = reinterpret_cast<unsigned*>(ws + L.depth_vals_alt);
    unsigned* hist = reinterpret_cast<unsigned*>(ws + L.hist);
    unsigned* bsums = reinterpret_cast<unsigned*>(ws + L.block_sums);
    u64* boffs = reinterpret_cast<u64*>(ws + L.block_offsets);
    const unsigned nb = (unsigned)((total + kBinSplats - 1) / kBinSplats);  // blocks of the instance passes
    const int V = cfg.num_views;
    const unsigned* vis_start = nullptr;  // set when the depth sort ranks only the splats with instances
    int gbits = 0;
    if (packed_depth_keys(cfg, n, &gbits)) {
        if (!depth_keys_ready) {
            const unsigned g = (unsigned)((total + kBinThreads - 1) / kBinThreads);
            ProfScope prof("depth_keys", stream);
            depth_keys_packed_kernel<<<g, kBinThreads, 0, stream>>>(total, (int)n, gbits, sp, dk0, &hdr->splat_count);
        }
        e = lsd_sort<false>(dk0, nullptr, dk1, nullptr, &hdr->splat_count, (u64)total, gbits, 32 + ceil_log2(V),
                            sort_grid((u64)total), hist, stream, "depth_sort", "depth_sort", order,
                            (1ull << gbits) - 1);
        if (e != cudaSuccess) return e;
    } else if (wrap) {
        {
            ProfScope prof("depth_keys", stream);
            const unsigned g = (unsigned)((total + kBinThreads - 1) / kBinThreads);
            depth_keys_kernel<<<g, kBinThreads, 0, stream>>>(total, (int)n, sp, dk0, order, &hdr->splat_count);
        }
        e = lsd_sort<true>(dk0, order, dk1, dv1, &hdr->splat_count, (u64)total, 0, 32 + ceil_log2(V),
                           sort_grid((u64)total), hist, stream, "depth_sort", "depth_sort");
        if (e != cudaSuccess) return e;
    } else {
        const int nbv = (int)((n + kVisSlots - 1) / kVisSlots);
        unsigned* vsums = reinterpret_cast<unsigned*>(ws + L.vis_sums);
        unsigned* vstart = reinterpret_cast<unsigned*>(ws + L.vis_start);
        unsigned* vmask = reinterpret_cast<unsigned*>(ws + L.vis_mask);
        {
            ProfScope prof("depth_keys", stream, 3);
            vis_count_kernel<<<V * nbv, kBinThreads, 0, stream>>>(n, nbv, sp, vsums, vmask);
            vis_scan_kernel<<<1, 1024, 0, stream>>>(V * nbv, nbv, V, vsums, vstart, &hdr->splat_count);
            depth_keys_compact_kernel<<<V * nbv, kBinThreads, 0, stream>>>(n, nbv, sp, vsums, vmask, dk0, dv1);
        }
        // the sorted keys and splats land back in (dk0, dv1); order is the other value buffer meanwhile
        e = lsd_sort<true>(dk0, dv1, dk1, order, &hdr->splat_count, (u64)total, 0, 32 + ceil_log2(V),
                           sort_grid((u64)total), hist, stream, "depth_sort", "depth_sort");
        if (e != cudaSuccess) return e;
        {
            ProfScope prof("depth_keys", stream);
            const unsigned g = (unsigned)((total + kBinThreads - 1) / kBinThreads);
            order_scatter_kernel<<<g, kBinThreads, 0, stream>>>(n, dk0, dv1, vstart, &hdr->splat_count, order);
        }
        vis_start = vstart;
    }
    unsigned per_view = 0;  // the largest number of blocks a view owns
    for (int v = 0; v < V; ++v) {
        const int64_t first = (int64_t)v * n / kBinSplats;
        const int64_t next = v + 1 < V ? (int64_t)(v + 1) * n / kBinSplats : (int64_t)nb;
        per_view = std::max(per_view, (unsigned)(next - first));
    }
    const unsigned grid = per_view * (unsigned)V;
    unsigned* pstart = reinterpret_cast<unsigned*>(ws + L.piece_start);
    unsigned* rbase = reinterpret_cast<unsigned*>(ws + L.row_base);
    unsigned* rcount = reinterpret_cast<unsigned*>(ws + L.row_count);
    unsigned* pblock = reinterpret_cast<unsigned*>(ws + L.piece_block);
    // Splitting heavy blocks pays when few views share the launch; with more, the view-interleaved dispatch already
    // overlaps their heavy first blocks, and the pieces' repeated row work would cost more than it saves.
    const unsigned piece = V <= 2 ? (unsigned)kEmitPiece : 0u;
    const unsigned max_pieces = piece ? (unsigned)((u64)capacity / piece + 1) : 0u;
    const int rb = rank_bits_for(n);
    if (!bucketed_binning(cfg, n)) {
        // instances in emission order into keys; the row words use the tile sort's spare buffer meanwhile
        u64* rows = reinterpret_cast<u64*>(ws + L.alt_keys);
        {
            ProfScope prof("bin_count", stream, 2);
            bin_count_kernel<false><<<grid, kBinThreads, 0, stream>>>(total, sp, order, tx, ty, cfg.tile, wrap, V, n,
                                                                      nb, vis_start, bsums, rows, (u64)capacity,
                                                                      rbase, rcount, hdr, nullptr, nullptr, 0,
                                                                      nullptr);
            bin_scan_kernel<<<1, 1024, 0, stream>>>((int)nb, bsums, boffs, piece, pstart, pblock, max_pieces, hdr,
                                                    (u64)capacity);
        }
        if (capacity > 0) {
            ProfScope prof("bin_emit", stream);
            auto emit = piece ? bin_emit_kernel<true, false> : bin_emit_kernel<false, false>;
            emit<<<grid + max_pieces, kBinThreads, 0, stream>>>(
                total, (int)n, sp, order, tx, ty, cfg.tile, wrap, rb, V, nb, piece, max_pieces, vis_start, bsums,
                boffs, pstart, pblock, hdr, rows, rbase, rcount, reinterpret_cast<u64*>(keys), (u64)capacity, nullptr,
                nullptr, nullptr, 0, nullptr);
        }
        return cudaGetLastError();
    }
    // bucketed: instances go to their (view, tile row) bucket in the spare buffer, as 32-bit entries; omnigs_sort
    // orders each bucket by column into keys
    u64* rows = reinterpret_cast<u64*>(ws + L.rows);
    unsigned* rows_off = reinterpret_cast<unsigned*>(ws + L.rows_off);
    unsigned* bcounts = reinterpret_cast<unsigned*>(ws + L.bkt_counts);
    u64* btotal = reinterpret_cast<u64*>(ws + L.bkt_total);
    u64* bbase = reinterpret_cast<u64*>(ws + L.bkt_base);
    u64* beff = reinterpret_cast<u64*>(ws + L.bkt_eff);
    unsigned* cstart = reinterpret_cast<unsigned*>(ws + L.col_start);
    unsigned* unstored = reinterpret_cast<unsigned*>(ws + L.unstored_list);
    const int nbkt = V * ty;
    const int nbv = (int)blocks_per_view_max(n);
    e = cudaMemsetAsync(bcounts, 0, sizeof(unsigned) * (size_t)nbkt * nbv, stream);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof("bin_count", stream, 4);
        bin_count_kernel<true><<<grid, kBinThreads, 0, stream>>>(total, sp, order, tx, ty, cfg.tile, wrap, V, n, nb,
                                                                 vis_start, bsums, rows, (u64)L.row_cap, rbase, rcount,
                                                                 hdr, rows_off, bcounts, nbv, unstored);
        bin_scan_kernel<<<1, 1024, 0, stream>>>((int)nb, bsums, boffs, piece, pstart, pblock, max_pieces, hdr,
                                                (u64)capacity);
        bucket_scan_kernel<<<nbkt, 256, 0, stream>>>(ty, n, nbv, bcounts, btotal);
        bucket_base_kernel<<<1, 1024, 0, stream>>>(nbkt, btotal, bbase, beff, cstart, (u64)capacity);
    }
    if (capacity > 0) {
        ProfScope prof("bin_emit", stream, 2);
        unsigned* out = reinterpret_cast<unsigned*>(ws + L.alt_keys);  // bucket entries, 32 bits
        auto emit = piece ? bin_emit_stored_kernel<true> : bin_emit_stored_kernel<false>;
        emit<<<grid + max_pieces, kBinThreads, 0, stream>>>((int)n, tx, ty, rb, V, nb, piece, max_pieces, bsums, boffs,
                                                            pstart, pblock, hdr, rows, rows_off, rbase, rcount, bcounts,
                                                            bbase, nbv, out, (u64)capacity);
        // the blocks whose row items did not fit: derived again and ranked here, a few CTAs taking them in turn
        const unsigned fb_grid = std::min<unsigned>(nb, (unsigned)num_sms() * 2);
        bin_emit_kernel<false, true><<<fb_grid, kBinThreads, 0, stream>>>(
            total, (int)n, sp, order, tx, ty, cfg.tile, wrap, rb, V, nb, 0u, 0u, vis_start, bsums, boffs, pstart,
            pblock, hdr, rows, rbase, rcount, out, (u64)capacity, rows_off, bcounts, bbase, nbv, unstored);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort(const omnigs_config& cfg, int64_t n, int64_t capacity, uint64_t* keys, uint32_t* ranges,
                        const WsLayout& L, char* ws, cudaStream_t stream) {
    const u64 ntiles = (u64)(cfg.width / cfg.tile) * (cfg.height / cfg.tile) * cfg.num_views;
    if (capacity == 0 || n == 0) return cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * ntiles, stream);
    cudaError_t e;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    u64* alt = reinterpret_cast<u64*>(ws + L.alt_keys);
    if (bucketed_binning(cfg, n)) {
        // one counting pass by tile column within every (view, tile row) bucket, from the spare buffer into keys
        const int tx = cfg.width / cfg.tile, nbkt = cfg.num_views * (cfg.height / cfg.tile), rb = rank_bits_for(n);
        const u64* bbase = reinterpret_cast<const u64*>(ws + L.bkt_base);
        const u64* beff = reinterpret_cast<const u64*>(ws + L.bkt_eff);
        const unsigned* cstart = reinterpret_cast<const unsigned*>(ws + L.col_start);
        unsigned* chist = reinterpret_cast<unsigned*>(ws + L.col_hist);
        const unsigned chunks = (unsigned)((u64)capacity / kColChunk + nbkt + 1);
        const unsigned* ent = reinterpret_cast<const unsigned*>(ws + L.alt_keys);
        const size_t smem = sizeof(unsigned) * (kSortTile + kWarps * kHistRow + 2 * kRadixMax + 32 + kMaxBucketCols);
        e = cudaFuncSetAttribute(col_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
            ProfScope prof("tile_count", stream);
            col_count_kernel<<<chunks, kSortThreads, 0, stream>>>(ent, bbase, beff, cstart, nbkt, tx, rb, chist, hdr);
        }
        {
            ProfScope prof("tile_ranges", stream);
            col_scan_kernel<<<nbkt, kMaxBucketCols, 0, stream>>>(bbase, cstart, tx, chist, ranges);
        }
        {
            ProfScope prof("tile_scatter", stream);
            col_scatter_kernel<<<chunks, kSortThreads, smem, stream>>>(ent, reinterpret_cast<u64*>(keys), bbase, beff,
                                                                       cstart, nbkt, tx, std::max(1, ceil_log2(tx)),
                                                                       rb, chist, (u64)capacity, hdr);
        }
        return cudaGetLastError();
    }
    unsigned* hist = reinterpret_cast<unsigned*>(ws + L.hist);
    e = lsd_sort<false>(reinterpret_cast<u64*>(keys), nullptr, alt, nullptr, &hdr->count, (u64)capacity,
                        rank_bits_for(n), tile_key_bits(cfg), sort_grid((u64)capacity), hist, stream, "sort_upsweep",
                        "sort_downsweep");
    if (e != cudaSuccess) return e;
    {
        ProfScope prof("tile_ranges", stream);
        ranges_kernel<<<(unsigned)((ntiles + 255) / 256), 256, 0, stream>>>(reinterpret_cast<const u64*>(keys), hdr,
                                                                             (u64)capacity, rank_bits_for(n), ntiles,
                                                                             ranges);
    }
    return cudaGetLastError();
}

}  // namespace omnigs
