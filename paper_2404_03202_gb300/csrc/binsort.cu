// Tile binning ("one instance per influence", Sec. 3.3) and the sort of instances by (view, tile, t_r).
//
// Binning: a count pass reduces per-splat tile counts to per-CTA sums, one CTA scans those (64-bit, so overflow
// is detected), and the emit pass rebuilds the per-splat offsets with a CTA scan and writes the instances warp-
// cooperatively: the 32 splats of a warp own one contiguous output range, and each lane writes every 32nd
// instance of it, so stores are fully coalesced even when one splat covers thousands of tiles.
//
// Sort: least-significant-digit radix sort over the key bits actually in use (31 depth bits + the tile-id bits),
// in an even number of <= 8-bit passes so the result lands back in the caller's buffers. Each pass is
// upsweep (per-CTA digit histograms) -> one-CTA exclusive scan (digit-major) -> downsweep. The downsweep ranks a
// 4096-key tile stably with warp match-any (rank = peers below the lane + running per-warp digit count), scatters it
// into shared memory in digit order and writes runs of equal digits to HBM, which keeps the global stores coalesced.
// No pass waits on another CTA, so there are no spin loops.
#include "common.cuh"

namespace omnigs {
namespace {

typedef unsigned long long u64;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

// Exclusive scan over the CTA of a 32-bit value; `scratch` holds >= blockDim/32 words. Returns the CTA total in *total.
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
        if (lane < nwarps) scratch[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    T base = warp > 0 ? scratch[warp - 1] : T(0);
    T tot = scratch[nwarps - 1];
    __syncthreads();
    *total = tot;
    return base + x - v;
}

struct SplatPos {
    float px, py;
    int radius;
};

// Splats whose centre is not a finite point of [0, W] x [0, H] (which the projection never produces) are treated as
// culled, so no tile index outside the image can arise from malformed input.
__device__ __forceinline__ SplatPos load_pos(const float4* __restrict__ sp, size_t i, int tiles_x, int tiles_y,
                                             int tile) {
    const float4 a = __ldg(sp + 3 * i);
    const float4 c = __ldg(sp + 3 * i + 2);
    SplatPos p;
    p.px = a.x;
    p.py = a.y;
    p.radius = __float_as_int(c.z);
    const bool inside = a.x >= 0.f && a.x <= (float)(tiles_x * tile) && a.y >= 0.f && a.y <= (float)(tiles_y * tile);
    if (!inside || p.radius > kMaxRadius) p.radius = 0;
    return p;
}

__global__ void __launch_bounds__(kBinThreads)
bin_count_kernel(int64_t total_splats, const float4* __restrict__ splats, int tiles_x, int tiles_y, int tile,
                 unsigned* __restrict__ block_sums) {
    __shared__ unsigned scratch[32];
    const int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    unsigned cnt = 0;
    if (i < total_splats) {
        const SplatPos p = load_pos(splats, (size_t)i, tiles_x, tiles_y, tile);
        if (p.radius > 0) {
            const Rect r = splat_rect(p.px, p.py, p.radius, tiles_x, tiles_y, tile);
            cnt = (unsigned)(r.nx * r.ny);
        }
    }
    unsigned tot;
    block_exclusive_scan<unsigned>(cnt, scratch, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the per-CTA sums in 64 bits; total to the header and to offsets[total_splats].
__global__ void __launch_bounds__(1024)
bin_scan_kernel(int nblocks, const unsigned* __restrict__ block_sums, u64* __restrict__ block_offsets,
                WsHeader* __restrict__ hdr, uint32_t* __restrict__ offsets, int64_t total_splats, u64 capacity) {
    __shared__ u64 scratch[32];
    const int per = (nblocks + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    u64 local = 0;
    for (int b = b0; b < min(b0 + per, nblocks); ++b) local += block_sums[b];
    u64 tot;
    u64 run = block_exclusive_scan<u64>(local, scratch, &tot);
    for (int b = b0; b < min(b0 + per, nblocks); ++b) {
        block_offsets[b] = run;
        run += block_sums[b];
    }
    if (threadIdx.x == 0) {
        hdr->count = tot;
        offsets[total_splats] = (uint32_t)(tot < 0xffffffffull ? tot : 0xffffffffull);
        if (tot > capacity) hdr->error |= kErrCapacity;
    }
}

__global__ void __launch_bounds__(kBinThreads)
bin_emit_kernel(int64_t total_splats, int n, const float4* __restrict__ splats, int tiles_x, int tiles_y, int tile,
                const u64* __restrict__ block_offsets, uint32_t* __restrict__ offsets, u64* __restrict__ keys,
                uint32_t* __restrict__ values, u64 capacity) {
    __shared__ unsigned scratch[32];
    const int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    const int tiles = tiles_x * tiles_y;
    unsigned cnt = 0;
    Rect r = {0, 1, 0, 0};
    unsigned dbits = 0;
    u64 tile_base = 0;
    if (i < total_splats) {
        const SplatPos p = load_pos(splats, (size_t)i, tiles_x, tiles_y, tile);
        if (p.radius > 0) {
            r = splat_rect(p.px, p.py, p.radius, tiles_x, tiles_y, tile);
            cnt = (unsigned)(r.nx * r.ny);
            dbits = __float_as_uint(__ldg(reinterpret_cast<const float*>(splats + 3 * i + 2) + 1)) & 0x7fffffffu;
            tile_base = (u64)(i / n) * (u64)tiles;
        }
    }
    unsigned blk_total;
    const unsigned local = block_exclusive_scan<unsigned>(cnt, scratch, &blk_total);
    const u64 off = block_offsets[blockIdx.x] + local;
    if (i < total_splats) offsets[i] = (uint32_t)(off < 0xffffffffull ? off : 0xffffffffull);

    // warp-cooperative emission over the warp's contiguous range
    const unsigned lane = lane_id();
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += y;
    }
    const unsigned excl = incl - cnt;
    const unsigned wtotal = __shfl_sync(0xffffffffu, incl, 31);
    const u64 woff = __shfl_sync(0xffffffffu, off, 0);
    for (unsigned base = 0; base < wtotal; base += 32) {
        const unsigned e = base + lane;
        // owner lane: largest j with excl_j <= e (lanes with cnt = 0 share excl with the next lane; the largest
        // such j has cnt > 0 whenever e < wtotal)
        int j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const unsigned ex = __shfl_sync(0xffffffffu, excl, j + step);
            if (j + step < 32 && ex <= e) j += step;
        }
        const unsigned k = e - __shfl_sync(0xffffffffu, excl, j);
        const int x0 = __shfl_sync(0xffffffffu, r.x0, j);
        const int nx = __shfl_sync(0xffffffffu, r.nx, j);
        const int y0 = __shfl_sync(0xffffffffu, r.y0, j);
        const unsigned db = __shfl_sync(0xffffffffu, dbits, j);
        const u64 tb = __shfl_sync(0xffffffffu, tile_base, j);
        const unsigned vg = (unsigned)(__shfl_sync(0xffffffffu, (unsigned long long)i, j));
        if (e < wtotal) {
            const int row = (int)(k / (unsigned)nx);
            const int col = (int)(k - (unsigned)row * (unsigned)nx);
            int tx = (x0 + col) % tiles_x;
            tx += tx < 0 ? tiles_x : 0;
            const int ty = y0 + row;
            const u64 idx = woff + e;
            if (idx < capacity) {
                keys[idx] = ((tb + (u64)(ty * tiles_x + tx)) << 31) | (u64)db;
                values[idx] = vg;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------ radix sort

struct TileSpan {
    u64 begin, end;  // tile indices of this CTA
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
sort_upsweep_kernel(const u64* __restrict__ keys, const WsHeader* __restrict__ hdr, u64 capacity, int shift,
                    int dbits, unsigned* __restrict__ hist, int G) {
    __shared__ unsigned s_hist[kSortThreads / 32][kSortRadixMax];
    const unsigned R = 1u << dbits, mask = R - 1;
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    for (unsigned d = lane; d < kSortRadixMax; d += 32) s_hist[warp][d] = 0;
    __syncwarp();
    const u64 cnt = min(hdr->count, capacity);
    const TileSpan span = cta_tiles(cnt, G);
    for (u64 t = span.begin; t < span.end; ++t) {
        const u64 base = t * kSortTile + warp * (kSortItems * 32) + lane;
#pragma unroll 4
        for (int j = 0; j < kSortItems; ++j) {
            const u64 idx = base + (u64)j * 32;
            if (idx < cnt) {
                const unsigned d = (unsigned)(__ldg(keys + idx) >> shift) & mask;
                atomicAdd(&s_hist[warp][d], 1u);
            }
        }
    }
    __syncthreads();
    for (unsigned d = threadIdx.x; d < R; d += blockDim.x) {
        unsigned s = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) s += s_hist[w][d];
        hist[(size_t)d * G + blockIdx.x] = s;
    }
}

// One CTA: exclusive scan over the digit-major histogram [R * G].
__global__ void __launch_bounds__(1024) sort_scan_kernel(unsigned* __restrict__ hist, int total) {
    __shared__ unsigned scratch[32];
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, total);
    unsigned local = 0;
    for (int b = b0; b < b1; ++b) local += hist[b];
    unsigned tot;
    unsigned run = block_exclusive_scan<unsigned>(local, scratch, &tot);
    for (int b = b0; b < b1; ++b) {
        const unsigned c = hist[b];
        hist[b] = run;
        run += c;
    }
}

constexpr int kWarps = kSortThreads / 32;
constexpr int kHistRow = kSortRadixMax + 1;  // + one bucket for the padding keys past the end

size_t downsweep_smem() {
    return sizeof(u64) * kSortTile + sizeof(unsigned) * kSortTile + sizeof(unsigned) * kWarps * kHistRow +
           sizeof(unsigned) * (3 * kSortRadixMax + 32);
}

__global__ void __launch_bounds__(kSortThreads)
sort_downsweep_kernel(const u64* __restrict__ keys_in, const unsigned* __restrict__ vals_in, u64* __restrict__ keys_out,
                      unsigned* __restrict__ vals_out, const WsHeader* __restrict__ hdr, u64 capacity, int shift,
                      int dbits, const unsigned* __restrict__ hist, int G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64* s_keys = reinterpret_cast<u64*>(smem_raw);
    unsigned* s_vals = reinterpret_cast<unsigned*>(s_keys + kSortTile);
    unsigned* s_whist = s_vals + kSortTile;
    unsigned* s_start = s_whist + kWarps * kHistRow;
    unsigned* s_tot = s_start + kSortRadixMax;
    unsigned* s_gbase = s_tot + kSortRadixMax;
    unsigned* s_scratch = s_gbase + kSortRadixMax;

    const unsigned R = 1u << dbits, mask = R - 1;
    const unsigned tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const unsigned lt_mask = (1u << lane) - 1u;
    const u64 cnt = min(hdr->count, capacity);
    const TileSpan span = cta_tiles(cnt, G);
    if (tid < R) s_gbase[tid] = hist[(size_t)tid * G + blockIdx.x];
    unsigned* my_hist = s_whist + warp * kHistRow;

    for (u64 t = span.begin; t < span.end; ++t) {
        for (unsigned d = lane; d < (unsigned)kHistRow; d += 32) my_hist[d] = 0;
        __syncwarp();
        const u64 base = t * kSortTile + warp * (kSortItems * 32) + lane;
        u64 k[kSortItems];
        unsigned val[kSortItems], dg[kSortItems], rk[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const u64 idx = base + (u64)j * 32;
            const bool ok = idx < cnt;
            k[j] = ok ? __ldg(keys_in + idx) : 0ull;
            val[j] = ok ? __ldg(vals_in + idx) : 0u;
            dg[j] = ok ? ((unsigned)(k[j] >> shift) & mask) : R;
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
            const unsigned before = my_hist[dg[j]];
            __syncwarp();
            if (lane == (unsigned)(__ffs(peers) - 1)) my_hist[dg[j]] = before + __popc(peers);
            __syncwarp();
            rk[j] = before + __popc(peers & lt_mask);
        }
        __syncthreads();
        if (tid < R) {
            unsigned acc = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const unsigned c = s_whist[w * kHistRow + tid];
                s_whist[w * kHistRow + tid] = acc;
                acc += c;
            }
            s_tot[tid] = acc;
        }
        __syncthreads();
        unsigned tile_total;
        const unsigned ex = block_exclusive_scan<unsigned>(tid < R ? s_tot[tid] : 0u, s_scratch, &tile_total);
        if (tid < R) s_start[tid] = ex;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            if (dg[j] < R) {
                const unsigned pos = s_start[dg[j]] + my_hist[dg[j]] + rk[j];
                s_keys[pos] = k[j];
                s_vals[pos] = val[j];
            }
        }
        __syncthreads();
        const unsigned nvalid = (unsigned)min((u64)kSortTile, cnt - t * kSortTile);
        for (unsigned i = tid; i < nvalid; i += kSortThreads) {
            const u64 key = s_keys[i];
            const unsigned d = (unsigned)(key >> shift) & mask;
            const unsigned gpos = s_gbase[d] + (i - s_start[d]);
            keys_out[gpos] = key;
            vals_out[gpos] = s_vals[i];
        }
        __syncthreads();
        if (tid < R) s_gbase[tid] += s_tot[tid];
        __syncthreads();
    }
}

__global__ void ranges_kernel(const u64* __restrict__ keys, const WsHeader* __restrict__ hdr, u64 capacity,
                              u64 ntiles, uint32_t* __restrict__ ranges) {
    const u64 cnt = min(hdr->count, capacity);
    for (u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x; s < cnt; s += (u64)gridDim.x * blockDim.x) {
        const u64 t = __ldg(keys + s) >> 31;
        if (t >= ntiles) continue;  // cannot happen for keys written by bin_emit
        if (s == 0 || (__ldg(keys + s - 1) >> 31) != t) ranges[2 * t] = (uint32_t)s;
        if (s + 1 == cnt || (__ldg(keys + s + 1) >> 31) != t) ranges[2 * t + 1] = (uint32_t)(s + 1);
    }
}

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

}  // namespace

SortPlan sort_plan(const omnigs_config& cfg) {
    const uint64_t tiles = (uint64_t)(cfg.width / cfg.tile) * (uint64_t)(cfg.height / cfg.tile) * (uint64_t)cfg.num_views;
    SortPlan p;
    p.bits = 31 + ceil_log2(tiles);
    p.passes = (p.bits + 7) / 8;
    if (p.passes % 2) ++p.passes;
    p.digit_bits = (p.bits + p.passes - 1) / p.passes;
    return p;
}

cudaError_t launch_bin(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats, uint32_t* offsets,
                       uint64_t* keys, uint32_t* values, int64_t capacity, const WsLayout& L, char* ws,
                       cudaStream_t stream) {
    const int64_t total = n * cfg.num_views;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), stream);
    if (e != cudaSuccess) return e;
    if (total == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint32_t), stream);
    const int tx = cfg.width / cfg.tile, ty = cfg.height / cfg.tile;
    const float4* sp = reinterpret_cast<const float4*>(splats);
    unsigned* bsums = reinterpret_cast<unsigned*>(ws + L.block_sums);
    u64* boffs = reinterpret_cast<u64*>(ws + L.block_offsets);
    {
        ProfScope prof("bin_count", stream);
        bin_count_kernel<<<L.bin_blocks, kBinThreads, 0, stream>>>(total, sp, tx, ty, cfg.tile, bsums);
    }
    {
        ProfScope prof("bin_scan", stream);
        bin_scan_kernel<<<1, 1024, 0, stream>>>(L.bin_blocks, bsums, boffs, hdr, offsets, total, (u64)capacity);
    }
    {
        ProfScope prof("bin_emit", stream);
        bin_emit_kernel<<<L.bin_blocks, kBinThreads, 0, stream>>>(total, (int)n, sp, tx, ty, cfg.tile, boffs, offsets,
                                                                   reinterpret_cast<u64*>(keys), values, (u64)capacity);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort(const omnigs_config& cfg, int64_t capacity, uint64_t* keys, uint32_t* values,
                        uint32_t* ranges, const WsLayout& L, char* ws, cudaStream_t stream) {
    const uint64_t ntiles = (uint64_t)(cfg.width / cfg.tile) * (cfg.height / cfg.tile) * cfg.num_views;
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * ntiles, stream);
    if (e != cudaSuccess) return e;
    if (capacity == 0) return cudaSuccess;
    const WsHeader* hdr = reinterpret_cast<const WsHeader*>(ws + L.header);
    u64* alt_k = reinterpret_cast<u64*>(ws + L.alt_keys);
    unsigned* alt_v = reinterpret_cast<unsigned*>(ws + L.alt_values);
    unsigned* hist = reinterpret_cast<unsigned*>(ws + L.hist);
    const SortPlan plan = sort_plan(cfg);
    const int G = L.sort_blocks;
    const size_t smem = downsweep_smem();
    e = cudaFuncSetAttribute(sort_downsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    u64* src_k = reinterpret_cast<u64*>(keys);
    unsigned* src_v = values;
    u64* dst_k = alt_k;
    unsigned* dst_v = alt_v;
    for (int p = 0; p < plan.passes; ++p) {
        const int shift = p * plan.digit_bits;
        const int db = min(plan.digit_bits, plan.bits - shift);
        if (db <= 0) break;  // cannot happen: passes * digit_bits covers bits, and passes is the minimum even count
        {
            ProfScope prof("sort_upsweep", stream);
            sort_upsweep_kernel<<<G, kSortThreads, 0, stream>>>(src_k, hdr, (u64)capacity, shift, db, hist, G);
        }
        {
            ProfScope prof("sort_scan", stream);
            sort_scan_kernel<<<1, 1024, 0, stream>>>(hist, (1 << db) * G);
        }
        {
            ProfScope prof("sort_downsweep", stream);
            sort_downsweep_kernel<<<G, kSortThreads, smem, stream>>>(src_k, src_v, dst_k, dst_v, hdr, (u64)capacity,
                                                                      shift, db, hist, G);
        }
        u64* tk = src_k; src_k = dst_k; dst_k = tk;
        unsigned* tv = src_v; src_v = dst_v; dst_v = tv;
    }
    {
        ProfScope prof("tile_ranges", stream);
        const int blocks = num_sms() * 8;
        ranges_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<const u64*>(keys), hdr, (u64)capacity, ntiles,
                                                  ranges);
    }
    return cudaGetLastError();
}

}  // namespace omnigs
