// Tile binning ("one instance per influence", Sec. 3.3) and the ordering of every tile's list by t_r (Sec. 3.3).
//
// The order produced is that of a stable sort of (view * TILES + tile, t_r) keys, i.e. a two-digit radix sort whose
// most significant digit is the tile. The tile digit is resolved by counting instead of by key passes over HBM:
//   1. tile_count: CTAs walk chunks of 2048 splats of one view, enumerate their instances warp-cooperatively,
//      count them per tile in shared memory and add the counts to the global per-tile counts (one atomic per touched
//      tile and chunk instead of one per instance);
//   2. scan_*: an exclusive scan of the counts gives each tile's [start, end) range (the ranges the blend kernels
//      read) and a write cursor per tile; the 64-bit total is checked against the capacity;
//   3. bin_emit: the same walk reserves one block of slots per touched tile and chunk, then writes every instance
//      (t_r bits, splat index) into it;
//   4. segment_sort: one CTA per tile sorts its segment in shared memory by the t_r bits that vary within it (LSD,
//      8-bit digits, stable ranking with warp match-any), then orders runs of equal t_r by splat index, which gives
//      exactly the stable-sort order whatever order the atomics left; segments larger than shared memory are sorted
//      in chunks and merged along merge paths.
// HBM traffic is ~8 B written by the emit and 8 B read + 8 B written by the segment sort per instance, instead of
// ~32 B per instance per pass of a device-wide radix sort. There are no inter-CTA waits.
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
    float px, py;
    int radius;
};

// Splats whose centre is not a point of [0, W] x [0, H] (which the projection never produces) are treated as culled,
// so malformed input cannot produce a tile index outside the image.
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

// ------------------------------------------------------------------------------------------- instance walk

// Splats are processed in chunks of kChunk consecutive splats of one view. The warps of a CTA take 32 splats at a
// time and enumerate their instances together (one per lane per round, owner found by a binary search over the
// warp's exclusive prefix of counts), calling fn(local_tile, depth_bits, splat_index) for each.
constexpr int kChunk = 2048;
constexpr int kBinCtaThreads = 512;
constexpr int kAggTiles = 16384;  // tiles per view up to which per-tile counts are aggregated in shared memory

struct ChunkSpan {
    int v;
    int64_t begin, end;  // splat indices v * n + g
};

__device__ __forceinline__ ChunkSpan chunk_span(int64_t c, int n, int chunks_per_view) {
    ChunkSpan cs;
    cs.v = (int)(c / chunks_per_view);
    const int64_t g0 = (c - (int64_t)cs.v * chunks_per_view) * kChunk;
    cs.begin = (int64_t)cs.v * n + g0;
    cs.end = (int64_t)cs.v * n + min((int64_t)n, g0 + kChunk);
    return cs;
}

template <typename Fn>
__device__ __forceinline__ void for_each_instance(const ChunkSpan& cs, const float4* __restrict__ splats, int tiles_x,
                                                  int tiles_y, int tile, Fn&& fn) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t g0 = cs.begin + (int64_t)warp * 32; g0 < cs.end; g0 += (int64_t)nwarps * 32) {
        const int64_t i = g0 + lane;
        unsigned cnt = 0, dbits = 0;
        Rect r = {0, 1, 0, 0};
        if (i < cs.end) {
            const SplatPos p = load_pos(splats, (size_t)i, tiles_x, tiles_y, tile);
            if (p.radius > 0) {
                r = splat_rect(p.px, p.py, p.radius, tiles_x, tiles_y, tile);
                cnt = (unsigned)(r.nx * r.ny);
                dbits = __float_as_uint(__ldg(reinterpret_cast<const float*>(splats + 3 * i + 2) + 1));
            }
        }
        unsigned incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        const unsigned excl = incl - cnt;
        const unsigned wtotal = __shfl_sync(0xffffffffu, incl, 31);
        for (unsigned base = 0; base < wtotal; base += 32) {
            const unsigned e = base + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const unsigned ex = __shfl_sync(0xffffffffu, excl, (j + step) & 31);
                if (j + step < 32 && ex <= e) j += step;
            }
            const unsigned k = e - __shfl_sync(0xffffffffu, excl, j);
            const int x0 = __shfl_sync(0xffffffffu, r.x0, j);
            const int nx = __shfl_sync(0xffffffffu, r.nx, j);
            const int y0 = __shfl_sync(0xffffffffu, r.y0, j);
            const unsigned db = __shfl_sync(0xffffffffu, dbits, j);
            if (e < wtotal) {
                const int row = (int)(k / (unsigned)nx);
                const int col = (int)(k - (unsigned)row * (unsigned)nx);
                int tx = (x0 + col) % tiles_x;
                tx += tx < 0 ? tiles_x : 0;
                fn((unsigned)((y0 + row) * tiles_x + tx), db, (unsigned)(g0 + j));
            }
        }
    }
}

// ------------------------------------------------------------------------------------------- 1: tile counts

template <bool kAgg>
__global__ void __launch_bounds__(kBinCtaThreads)
tile_count_kernel(int64_t nchunks, int n, int chunks_per_view, const float4* __restrict__ splats, int tiles_x,
                  int tiles_y, int tile, uint32_t* __restrict__ counts) {
    extern __shared__ unsigned s_cnt[];
    const int tpv = tiles_x * tiles_y;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const ChunkSpan cs = chunk_span(c, n, chunks_per_view);
        uint32_t* vcounts = counts + (size_t)cs.v * tpv;
        if (kAgg) {
            for (int t = threadIdx.x; t < tpv; t += blockDim.x) s_cnt[t] = 0;
            __syncthreads();
            for_each_instance(cs, splats, tiles_x, tiles_y, tile,
                              [&](unsigned t, unsigned, unsigned) { atomicAdd(&s_cnt[t], 1u); });
            __syncthreads();
            for (int t = threadIdx.x; t < tpv; t += blockDim.x)
                if (s_cnt[t]) atomicAdd(vcounts + t, s_cnt[t]);
            __syncthreads();
        } else {
            for_each_instance(cs, splats, tiles_x, tiles_y, tile,
                              [&](unsigned t, unsigned, unsigned) { atomicAdd(vcounts + t, 1u); });
        }
    }
}

// ------------------------------------------------------------------------------------------- 2: scan

constexpr int kScanItems = 16;
constexpr int kScanBlock = kBinThreads * kScanItems;

__global__ void __launch_bounds__(kBinThreads)
scan_reduce_kernel(u64 ntiles, const uint32_t* __restrict__ counts, u64* __restrict__ block_sums) {
    __shared__ u64 scratch[32];
    const u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
    u64 s = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < ntiles) s += counts[base + k];
    u64 tot;
    block_exclusive_scan<u64>(s, scratch, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
scan_blocks_kernel(int nblocks, u64* __restrict__ block_sums, WsHeader* __restrict__ hdr, u64 capacity) {
    __shared__ u64 scratch[32];
    const int per = (nblocks + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nblocks);
    u64 local = 0;
    for (int b = b0; b < b1; ++b) local += block_sums[b];
    u64 tot;
    u64 run = block_exclusive_scan<u64>(local, scratch, &tot);
    for (int b = b0; b < b1; ++b) {
        const u64 c = block_sums[b];
        block_sums[b] = run;  // becomes the exclusive offset of the block
        run += c;
    }
    if (threadIdx.x == 0) {
        hdr->count = tot;
        if (tot > capacity) hdr->error |= kErrCapacity;
    }
}

__global__ void __launch_bounds__(kBinThreads)
scan_write_kernel(u64 ntiles, const uint32_t* __restrict__ counts, const u64* __restrict__ block_offsets,
                  u64 capacity, uint32_t* __restrict__ ranges, uint32_t* __restrict__ cursors) {
    __shared__ u64 scratch[32];
    const u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
    unsigned c[kScanItems];
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        c[k] = base + k < ntiles ? counts[base + k] : 0u;
        s += c[k];
    }
    u64 tot;
    u64 run = block_offsets[blockIdx.x] + block_exclusive_scan<u64>(s, scratch, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < ntiles) {
            const u64 e = run + c[k];
            ranges[2 * (base + k)] = (uint32_t)min(run, capacity);
            ranges[2 * (base + k) + 1] = (uint32_t)min(e, capacity);
            cursors[base + k] = (uint32_t)min(run, capacity);
            run = e;
        }
    }
}

// ------------------------------------------------------------------------------------------- 3: emission

// Each CTA counts its chunk's instances per tile in shared memory, reserves one block of slots per touched tile with
// a single global atomic, then writes every instance (t_r bits, splat index) into its tile's block.
template <bool kAgg>
__global__ void __launch_bounds__(kBinCtaThreads)
bin_emit_kernel(int64_t nchunks, int n, int chunks_per_view, const float4* __restrict__ splats, int tiles_x,
                int tiles_y, int tile, uint32_t* __restrict__ cursors, uint32_t* __restrict__ keys,
                uint32_t* __restrict__ values, uint32_t capacity) {
    extern __shared__ unsigned s_mem[];
    const int tpv = tiles_x * tiles_y;
    unsigned* s_cnt = s_mem;
    unsigned* s_base = s_mem + tpv;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const ChunkSpan cs = chunk_span(c, n, chunks_per_view);
        uint32_t* vcur = cursors + (size_t)cs.v * tpv;
        auto put = [&](unsigned pos, unsigned db, unsigned vg) {
            if (pos < capacity) {
                keys[pos] = db;
                values[pos] = vg;
            }
        };
        if (kAgg) {
            for (int t = threadIdx.x; t < tpv; t += blockDim.x) s_cnt[t] = 0;
            __syncthreads();
            for_each_instance(cs, splats, tiles_x, tiles_y, tile,
                              [&](unsigned t, unsigned, unsigned) { atomicAdd(&s_cnt[t], 1u); });
            __syncthreads();
            for (int t = threadIdx.x; t < tpv; t += blockDim.x) {
                const unsigned k = s_cnt[t];
                s_base[t] = k ? atomicAdd(vcur + t, k) : 0u;
                s_cnt[t] = 0;
            }
            __syncthreads();
            for_each_instance(cs, splats, tiles_x, tiles_y, tile, [&](unsigned t, unsigned db, unsigned vg) {
                put(s_base[t] + atomicAdd(&s_cnt[t], 1u), db, vg);
            });
            __syncthreads();
        } else {
            for_each_instance(cs, splats, tiles_x, tiles_y, tile,
                              [&](unsigned t, unsigned db, unsigned vg) { put(atomicAdd(vcur + t, 1u), db, vg); });
        }
    }
}

// ------------------------------------------------------------------------------------------- 4: segment sort

// Stable LSD radix sort of one tile's (t_r bits, splat) pairs, NT threads x ITEMS pairs, keys held in registers
// between passes. Element e = warp * ITEMS * 32 + j * 32 + lane lives in register j of that lane, so the order of
// (warp, j, lane) is the element order. Per pass: every warp ranks its items with match-any (rank = peers below the
// lane + running per-warp count of the digit), one CTA scan over the digit-major [digit][warp] counts gives every
// (digit, warp) its output offset, the items are scattered to shared memory and read back in element order.
constexpr int kRadix = 256;

// Counter of (digit d, warp w), digit-major with the warp index XOR-swizzled by the digit, so that lanes ranking
// different digits hit different banks while one digit's NW counters stay contiguous for the scan.
template <int NW>
__device__ __forceinline__ unsigned cnt_index(unsigned d, unsigned w) { return d * NW + (w ^ (d & (NW - 1))); }

template <int NT, int ITEMS>
struct TileSortSmem {
    static constexpr int NW = NT / 32;
    unsigned keys[NT * ITEMS];
    unsigned vals[NT * ITEMS];
    unsigned cnt[(kRadix + 1) * NW];  // [digit][warp]; digit kRadix collects the padding past the end
    unsigned scratch[32];
    unsigned red[2];
    unsigned flag;
};

template <int NT, int ITEMS>
__device__ void tile_sort(uint32_t* __restrict__ gk, uint32_t* __restrict__ gv, int n, TileSortSmem<NT, ITEMS>& S) {
    constexpr int NW = NT / 32;
    constexpr int PER = (kRadix * NW) / NT;  // scan entries per thread
    const unsigned tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned key[ITEMS], val[ITEMS];
    unsigned kand = 0xffffffffu, kor = 0u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int e = (warp * ITEMS + j) * 32 + lane;
        const bool ok = e < n;
        key[j] = ok ? gk[e] : 0xffffffffu;
        val[j] = ok ? gv[e] : 0u;
        if (ok) {
            kand &= key[j];
            kor |= key[j];
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        kand &= __shfl_xor_sync(0xffffffffu, kand, o);
        kor |= __shfl_xor_sync(0xffffffffu, kor, o);
    }
    if (tid == 0) {
        S.red[0] = 0xffffffffu;
        S.red[1] = 0u;
        S.flag = 0u;
    }
    __syncthreads();
    if (lane == 0) {
        atomicAnd(&S.red[0], kand);
        atomicOr(&S.red[1], kor);
    }
    __syncthreads();
    const unsigned diff = S.red[1] & ~S.red[0];
    const int nbits = diff ? 32 - __clz(diff) : 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        for (int i = tid; i < (kRadix + 1) * NW; i += NT) S.cnt[i] = 0;
        __syncthreads();
        unsigned rk[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int e = (warp * ITEMS + j) * 32 + lane;
            const unsigned d = e < n ? (key[j] >> shift) & 0xffu : (unsigned)kRadix;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            unsigned* c = &S.cnt[cnt_index<NW>(d, warp)];
            const unsigned before = *c;
            __syncwarp();
            if (lane == (unsigned)(__ffs(peers) - 1)) *c = before + __popc(peers);
            __syncwarp();
            rk[j] = before + __popc(peers & lt);
        }
        __syncthreads();
        // exclusive scan over the digit-major counts of the kRadix real digits
        {
            unsigned loc[PER], sum = 0;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const unsigned idx = tid * PER + q;  // logical digit-major position
                loc[q] = S.cnt[cnt_index<NW>(idx / NW, idx % NW)];
                sum += loc[q];
            }
            unsigned tot;
            unsigned run = block_exclusive_scan<unsigned>(sum, S.scratch, &tot);
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const unsigned idx = tid * PER + q;
                S.cnt[cnt_index<NW>(idx / NW, idx % NW)] = run;
                run += loc[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int e = (warp * ITEMS + j) * 32 + lane;
            if (e < n) {
                const unsigned pos = S.cnt[cnt_index<NW>((key[j] >> shift) & 0xffu, warp)] + rk[j];
                S.keys[pos] = key[j];
                S.vals[pos] = val[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int e = (warp * ITEMS + j) * 32 + lane;
            if (e < n) {
                key[j] = S.keys[e];
                val[j] = S.vals[e];
            }
        }
        __syncthreads();
    }
    // equal t_r: order by splat index (a run of equal keys keeps the unspecified bucket order until here)
    bool tie = false;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int e = (warp * ITEMS + j) * 32 + lane;
        const unsigned nxt = __shfl_down_sync(0xffffffffu, key[j], 1);
        if (lane < 31 && e + 1 < n && nxt == key[j]) tie = true;
        if (e < n) S.keys[e] = key[j];  // element order (already there unless no pass ran)
    }
    if (__any_sync(0xffffffffu, tie) && lane == 0) S.flag = 1u;
    __syncthreads();
    // pairs straddling two lanes' registers of different rounds are checked in shared memory
    if (!S.flag) {
        for (int e = tid; e + 1 < n; e += NT)
            if (((e + 1) & 31) == 0 && S.keys[e] == S.keys[e + 1]) S.flag = 1u;
    }
    __syncthreads();
    if (S.flag) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int e = (warp * ITEMS + j) * 32 + lane;
            if (e < n) S.vals[e] = val[j];
        }
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
            if (i > 0 && S.keys[i - 1] == S.keys[i]) continue;      // not a run start
            if (i + 1 >= n || S.keys[i + 1] != S.keys[i]) continue;  // run of length 1
            int e = i + 1;
            while (e < n && S.keys[e] == S.keys[i]) ++e;
            for (int a = i + 1; a < e; ++a) {
                const unsigned x = S.vals[a];
                int b = a - 1;
                while (b >= i && S.vals[b] > x) {
                    S.vals[b + 1] = S.vals[b];
                    --b;
                }
                S.vals[b + 1] = x;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int e = (warp * ITEMS + j) * 32 + lane;
            if (e < n) val[j] = S.vals[e];
        }
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int e = (warp * ITEMS + j) * 32 + lane;
        if (e < n) {
            gk[e] = key[j];
            gv[e] = val[j];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ bool pair_less(unsigned ka, unsigned va, unsigned kb, unsigned vb) {
    return ka < kb || (ka == kb && va < vb);
}

// Merge sorted runs a = [a0, a0 + la) and b = [b0, b0 + lb) of (keys, vals) into (ok, ov) starting at o0, along merge
// paths: thread t produces outputs [t P, (t + 1) P).
__device__ void merge_runs(const unsigned* __restrict__ keys, const unsigned* __restrict__ vals, int64_t a0, int la,
                           int64_t b0, int lb, unsigned* __restrict__ ok, unsigned* __restrict__ ov, int64_t o0) {
    const int total = la + lb;
    const int P = (total + blockDim.x - 1) / blockDim.x;
    const int d0 = min((int)threadIdx.x * P, total), d1 = min(d0 + P, total);
    if (d0 >= d1) return;
    int lo = max(0, d0 - lb), hi = min(d0, la);  // smallest i with b[d0 - 1 - i] < a[i]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int j = d0 - 1 - mid;
        if (pair_less(keys[b0 + j], vals[b0 + j], keys[a0 + mid], vals[a0 + mid])) hi = mid;
        else lo = mid + 1;
    }
    int i = lo, j = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        bool take_a;
        if (i >= la) take_a = false;
        else if (j >= lb) take_a = true;
        else take_a = !pair_less(keys[b0 + j], vals[b0 + j], keys[a0 + i], vals[a0 + i]);
        if (take_a) {
            ok[o0 + d] = keys[a0 + i];
            ov[o0 + d] = vals[a0 + i];
            ++i;
        } else {
            ok[o0 + d] = keys[b0 + j];
            ov[o0 + d] = vals[b0 + j];
            ++j;
        }
    }
}

// One CTA per tile (grid-stride). Segments of up to NT * ITEMS pairs are sorted in registers and shared memory;
// longer ones are sorted in chunks of that size and merged pairwise through the scratch buffers.
template <int NT, int ITEMS>
__global__ void __launch_bounds__(NT, 16 / ITEMS)
segment_sort_kernel(u64 ntiles, const uint32_t* __restrict__ ranges, uint32_t* __restrict__ keys,
                    uint32_t* __restrict__ values, uint32_t* __restrict__ scratch_k, uint32_t* __restrict__ scratch_v,
                    int min_len, int max_len) {
    constexpr int CAP = NT * ITEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSortSmem<NT, ITEMS>& S = *reinterpret_cast<TileSortSmem<NT, ITEMS>*>(smem_raw);
    for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
        const int n = (int)(end - start);
        if (n < min_len || n > max_len || n < 2) continue;
        uint32_t* gk = keys + start;
        uint32_t* gv = values + start;
        for (int c0 = 0; c0 < n; c0 += CAP) tile_sort<NT, ITEMS>(gk + c0, gv + c0, min(CAP, n - c0), S);
        if (n <= CAP) continue;
        uint32_t *sk = keys, *sv = values, *dk = scratch_k, *dv = scratch_v;
        for (int width = CAP; width < n; width *= 2) {
            for (int a0 = 0; a0 < n; a0 += 2 * width) {
                const int la = min(width, n - a0);
                const int lb = max(0, min(width, n - a0 - la));
                merge_runs(sk, sv, (int64_t)start + a0, la, (int64_t)start + a0 + la, lb, dk, dv, (int64_t)start + a0);
            }
            __syncthreads();
            uint32_t* tk = sk; sk = dk; dk = tk;
            uint32_t* tv = sv; sv = dv; dv = tv;
        }
        if (sk != keys) {
            for (int i = threadIdx.x; i < n; i += NT) {
                keys[start + i] = sk[start + i];
                values[start + i] = sv[start + i];
            }
            __syncthreads();
        }
    }
}

constexpr int kSmallNT = 512, kSmallItems = 8;   // lists up to 4096
constexpr int kLargeNT = 512, kLargeItems = 16;  // lists up to 8192 at once, longer ones merged

}  // namespace

cudaError_t launch_bin(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats, uint32_t* keys,
                       uint32_t* values, int64_t capacity, uint32_t* ranges, const WsLayout& L, char* ws,
                       cudaStream_t stream) {
    const int tx = cfg.width / cfg.tile, ty = cfg.height / cfg.tile, tpv = tx * ty;
    const u64 ntiles = (u64)tpv * cfg.num_views;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.tile_counts);
    u64* bsums = reinterpret_cast<u64*>(ws + L.scan_blocks);
    uint32_t* cursors = reinterpret_cast<uint32_t*>(ws + L.cursors);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ntiles, stream);
    if (e != cudaSuccess) return e;
    const float4* sp = reinterpret_cast<const float4*>(splats);
    const int chunks_per_view = (int)((n + kChunk - 1) / kChunk);
    const int64_t nchunks = (int64_t)chunks_per_view * cfg.num_views;
    const bool agg = tpv <= kAggTiles;
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(nchunks, 1), (int64_t)num_sms() * 4);
    if (nchunks > 0) {
        ProfScope prof("tile_count", stream);
        const size_t smem = agg ? sizeof(unsigned) * tpv : 0;
        if (agg) {
            e = cudaFuncSetAttribute(tile_count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            tile_count_kernel<true><<<grid, kBinCtaThreads, smem, stream>>>(nchunks, (int)n, chunks_per_view, sp, tx,
                                                                            ty, cfg.tile, counts);
        } else {
            tile_count_kernel<false><<<grid, kBinCtaThreads, 0, stream>>>(nchunks, (int)n, chunks_per_view, sp, tx,
                                                                          ty, cfg.tile, counts);
        }
    }
    const int nb = (int)((ntiles + kScanBlock - 1) / kScanBlock);
    {
        ProfScope prof("tile_scan", stream);
        scan_reduce_kernel<<<nb, kBinThreads, 0, stream>>>(ntiles, counts, bsums);
        scan_blocks_kernel<<<1, 1024, 0, stream>>>(nb, bsums, hdr, (u64)capacity);
        scan_write_kernel<<<nb, kBinThreads, 0, stream>>>(ntiles, counts, bsums, (u64)capacity, ranges, cursors);
    }
    if (nchunks > 0 && capacity > 0) {
        ProfScope prof("bin_emit", stream);
        const size_t smem = agg ? 2 * sizeof(unsigned) * tpv : 0;
        if (agg) {
            e = cudaFuncSetAttribute(bin_emit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            bin_emit_kernel<true><<<grid, kBinCtaThreads, smem, stream>>>(nchunks, (int)n, chunks_per_view, sp, tx,
                                                                          ty, cfg.tile, cursors, keys, values,
                                                                          (uint32_t)capacity);
        } else {
            bin_emit_kernel<false><<<grid, kBinCtaThreads, 0, stream>>>(nchunks, (int)n, chunks_per_view, sp, tx,
                                                                        ty, cfg.tile, cursors, keys, values,
                                                                        (uint32_t)capacity);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_sort(const omnigs_config& cfg, int64_t capacity, uint32_t* keys, uint32_t* values,
                        const uint32_t* ranges, const WsLayout& L, char* ws, cudaStream_t stream) {
    if (capacity == 0) return cudaSuccess;
    const u64 ntiles = (u64)(cfg.width / cfg.tile) * (cfg.height / cfg.tile) * cfg.num_views;
    uint32_t* sk = reinterpret_cast<uint32_t*>(ws + L.alt_keys);
    uint32_t* sv = reinterpret_cast<uint32_t*>(ws + L.alt_values);
    constexpr size_t small_smem = sizeof(TileSortSmem<kSmallNT, kSmallItems>);
    constexpr size_t large_smem = sizeof(TileSortSmem<kLargeNT, kLargeItems>);
    auto ks = segment_sort_kernel<kSmallNT, kSmallItems>;
    auto kl = segment_sort_kernel<kLargeNT, kLargeItems>;
    cudaError_t e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)large_smem);
    if (e != cudaSuccess) return e;
    const u64 max_grid = (u64)num_sms() * 16;
    const unsigned grid = (unsigned)(ntiles < max_grid ? ntiles : max_grid);
    {
        ProfScope prof("segment_sort", stream);
        ks<<<grid, kSmallNT, small_smem, stream>>>(ntiles, ranges, keys, values, sk, sv, 0, kSmallNT * kSmallItems);
    }
    {
        ProfScope prof("segment_sort_large", stream);
        kl<<<grid, kLargeNT, large_smem, stream>>>(ntiles, ranges, keys, values, sk, sv, kSmallNT * kSmallItems + 1,
                                                   0x7fffffff);
    }
    return cudaGetLastError();
}

}  // namespace omnigs
