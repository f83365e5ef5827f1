// Tile binning ("one instance per influence", Sec. 3.3) and the ordering of every tile's list by t_r (Sec. 3.3).
//
// The order produced is that of a stable sort of (view * TILES + tile, t_r) keys, i.e. a two-digit radix sort whose
// most significant digit is the tile. The tile digit is resolved by counting instead of by key passes over HBM:
//   1. tile_count: each splat adds its tile rectangle (one or two pieces across the longitude seam) to a per-view
//      2D difference grid with four atomic adds per piece;
//   2. tile_prefix: a 2D prefix sum of that grid gives the instance count of every tile;
//   3. scan_*: an exclusive scan of the counts gives each tile's [start, end) range (the ranges the blend kernels
//      read) and a write cursor per tile; the 64-bit total is checked against the capacity;
//   4. bin_emit: warp-cooperative emission of every instance (t_r bits, splat index) at cursor[tile]++;
//   5. segment_sort: one CTA per tile sorts its segment in shared memory by the t_r bits that vary within it (LSD,
//      8-bit digits, stable ranking with warp match-any), then orders runs of equal t_r by splat index, which gives
//      exactly the stable-sort order whatever order the atomics left; segments larger than shared memory are sorted
//      in chunks and merged along merge paths.
// HBM traffic is ~8 B written by the emit and 8 B read + 8 B written by the segment sort per instance, instead of
// ~32 B per instance per pass of a device-wide radix sort. There are no inter-CTA waits.
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

// ------------------------------------------------------------------------------------------- 1-3: tile counts

__global__ void __launch_bounds__(kBinThreads)
tile_count_kernel(int64_t total_splats, int n, const float4* __restrict__ splats, int tiles_x, int tiles_y, int tile,
                  int* __restrict__ diff) {
    const int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    if (i >= total_splats) return;
    const SplatPos p = load_pos(splats, (size_t)i, tiles_x, tiles_y, tile);
    if (p.radius <= 0) return;
    const Rect r = splat_rect(p.px, p.py, p.radius, tiles_x, tiles_y, tile);
    if (r.ny <= 0) return;
    const int gx = tiles_x + 1;
    int* g = diff + (size_t)(i / n) * (size_t)(tiles_y + 1) * gx;
    int xa = r.x0 % tiles_x;
    xa += xa < 0 ? tiles_x : 0;
    const int y0 = r.y0, y1 = r.y0 + r.ny;  // rows [y0, y1)
    auto add = [&](int a, int b) {          // columns [a, b)
        atomicAdd(g + y0 * gx + a, 1);
        atomicAdd(g + y0 * gx + b, -1);
        atomicAdd(g + y1 * gx + a, -1);
        atomicAdd(g + y1 * gx + b, 1);
    };
    if (xa + r.nx <= tiles_x) {
        add(xa, xa + r.nx);
    } else {
        add(xa, tiles_x);
        add(0, xa + r.nx - tiles_x);
    }
}

// One CTA per view: 2D inclusive prefix sum of the difference grid, in place (rows, then columns).
__global__ void __launch_bounds__(1024) tile_prefix_kernel(int tiles_x, int tiles_y, int* __restrict__ diff) {
    const int gx = tiles_x + 1, gy = tiles_y + 1;
    int* g = diff + (size_t)blockIdx.x * gx * gy;
    for (int y = threadIdx.x; y < gy; y += blockDim.x) {
        int acc = 0;
        for (int x = 0; x < gx; ++x) {
            acc += g[y * gx + x];
            g[y * gx + x] = acc;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < gx; x += blockDim.x) {
        int acc = 0;
        for (int y = 0; y < gy; ++y) {
            acc += g[y * gx + x];
            g[y * gx + x] = acc;
        }
    }
}

__device__ __forceinline__ unsigned tile_count_at(const int* __restrict__ grid, u64 t, int tiles_x, int tiles_y) {
    const u64 tiles = (u64)tiles_x * tiles_y;
    const u64 v = t / tiles, r = t - v * tiles;
    const int ty = (int)(r / tiles_x), tx = (int)(r - (u64)ty * tiles_x);
    const int c = grid[v * (u64)(tiles_x + 1) * (tiles_y + 1) + (u64)ty * (tiles_x + 1) + tx];
    return c > 0 ? (unsigned)c : 0u;
}

constexpr int kScanItems = 16;
constexpr int kScanBlock = kBinThreads * kScanItems;

__global__ void __launch_bounds__(kBinThreads)
scan_reduce_kernel(u64 ntiles, const int* __restrict__ grid, int tiles_x, int tiles_y, u64* __restrict__ block_sums) {
    __shared__ u64 scratch[32];
    const u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
    u64 s = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < ntiles) s += tile_count_at(grid, base + k, tiles_x, tiles_y);
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
scan_write_kernel(u64 ntiles, const int* __restrict__ grid, int tiles_x, int tiles_y,
                  const u64* __restrict__ block_offsets, u64 capacity, uint32_t* __restrict__ ranges,
                  uint32_t* __restrict__ cursors) {
    __shared__ u64 scratch[32];
    const u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
    unsigned c[kScanItems];
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        c[k] = base + k < ntiles ? tile_count_at(grid, base + k, tiles_x, tiles_y) : 0u;
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

// ------------------------------------------------------------------------------------------- 4: emission

__global__ void __launch_bounds__(kBinThreads)
bin_emit_kernel(int64_t total_splats, int n, const float4* __restrict__ splats, int tiles_x, int tiles_y, int tile,
                uint32_t* __restrict__ cursors, uint32_t* __restrict__ keys, uint32_t* __restrict__ values,
                uint32_t capacity) {
    const int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    const int tiles = tiles_x * tiles_y;
    unsigned cnt = 0, dbits = 0, tbase = 0;
    Rect r = {0, 1, 0, 0};
    if (i < total_splats) {
        const SplatPos p = load_pos(splats, (size_t)i, tiles_x, tiles_y, tile);
        if (p.radius > 0) {
            r = splat_rect(p.px, p.py, p.radius, tiles_x, tiles_y, tile);
            cnt = (unsigned)(r.nx * r.ny);
            dbits = __float_as_uint(__ldg(reinterpret_cast<const float*>(splats + 3 * i + 2) + 1));
            tbase = (unsigned)(i / n) * (unsigned)tiles;
        }
    }
    // the 32 splats of a warp emit their instances together, one per lane per round
    const unsigned lane = lane_id();
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
        int j = 0;  // owner: the largest lane whose exclusive prefix is <= e
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
        const unsigned tb = __shfl_sync(0xffffffffu, tbase, j);
        const unsigned vg = __shfl_sync(0xffffffffu, (unsigned)i, j);
        if (e < wtotal) {
            const int row = (int)(k / (unsigned)nx);
            const int col = (int)(k - (unsigned)row * (unsigned)nx);
            int tx = (x0 + col) % tiles_x;
            tx += tx < 0 ? tiles_x : 0;
            const unsigned t = tb + (unsigned)((y0 + row) * tiles_x + tx);
            const unsigned pos = atomicAdd(cursors + t, 1u);
            if (pos < capacity) {
                keys[pos] = db;
                values[pos] = vg;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------- 5: segment sort

// Stable LSD radix sort of n <= cap (key, value) pairs held in shared memory, over key bits [0, nbits), 8-bit digits.
// (k0, v0) hold the input; the result ends in (k0, v0) or (k1, v1): returns true if it is in (k1, v1).
// whist: [nwarps][kRadix + 1] counters; scratch: >= 32 words.
constexpr int kRadix = 256;

__device__ bool smem_radix_sort(unsigned* k0, unsigned* v0, unsigned* k1, unsigned* v1, int n, int nbits,
                                unsigned* whist, unsigned* s_start, unsigned* scratch) {
    const unsigned tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nwarps = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int per_warp = ((n + nwarps - 1) / nwarps + 31) & ~31;  // contiguous, 32-aligned chunk per warp
    unsigned* my = whist + warp * (kRadix + 1);
    bool flipped = false;
    for (int shift = 0; shift < nbits; shift += 8) {
        for (int d = lane; d <= kRadix; d += 32) my[d] = 0;
        __syncwarp();
        const int w0 = warp * per_warp, w1 = min(w0 + per_warp, n);
        // ranking: per-warp counts in element order
        for (int b = w0; b < w0 + per_warp; b += 32) {
            const int idx = b + lane;
            const unsigned d = idx < w1 ? (k0[idx] >> shift) & 0xffu : (unsigned)kRadix;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const unsigned before = my[d];
            __syncwarp();
            if (lane == (unsigned)(__ffs(peers) - 1)) my[d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: warp prefix and total
        for (int d = tid; d < kRadix; d += blockDim.x) {
            unsigned acc = 0;
            for (unsigned w = 0; w < nwarps; ++w) {
                const unsigned c = whist[w * (kRadix + 1) + d];
                whist[w * (kRadix + 1) + d] = acc;
                acc += c;
            }
            s_start[d] = acc;
        }
        __syncthreads();
        // exclusive scan of the digit totals (kRadix entries over the CTA)
        {
            unsigned tot;
            unsigned v = 0;
            const int per = (kRadix + blockDim.x - 1) / blockDim.x;
            for (int q = 0; q < per; ++q) {
                const int d = tid * per + q;
                if (d < kRadix) v += s_start[d];
            }
            unsigned run = block_exclusive_scan<unsigned>(v, scratch, &tot);
            for (int q = 0; q < per; ++q) {
                const int d = tid * per + q;
                if (d < kRadix) {
                    const unsigned c = s_start[d];
                    s_start[d] = run;
                    run += c;
                }
            }
        }
        __syncthreads();
        // scatter: a second walk over the warp's chunk recomputes the in-warp ranks on top of the warp prefix
        unsigned* wp = my;
        for (int b = w0; b < w0 + per_warp; b += 32) {
            const int idx = b + lane;
            const bool ok = idx < w1;
            const unsigned key = ok ? k0[idx] : 0u;
            const unsigned d = ok ? (key >> shift) & 0xffu : (unsigned)kRadix;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const unsigned before = wp[d];
            __syncwarp();
            if (lane == (unsigned)(__ffs(peers) - 1)) wp[d] = before + __popc(peers);
            __syncwarp();
            if (ok) {
                const unsigned pos = s_start[d] + before + __popc(peers & lt);
                k1[pos] = key;
                v1[pos] = v0[idx];
            }
        }
        __syncthreads();
        unsigned* t;
        t = k0; k0 = k1; k1 = t;
        t = v0; v0 = v1; v1 = t;
        flipped = !flipped;
    }
    return flipped;
}

// Runs of equal keys are put in value order (insertion sort per run; runs are short and rare).
__device__ void order_ties(unsigned* k, unsigned* v, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (i > 0 && k[i - 1] == k[i]) continue;      // not a run start
        if (i + 1 >= n || k[i + 1] != k[i]) continue;  // run of length 1
        int e = i + 1;
        while (e < n && k[e] == k[i]) ++e;
        for (int a = i + 1; a < e; ++a) {
            const unsigned x = v[a];
            int b = a - 1;
            while (b >= i && v[b] > x) {
                v[b + 1] = v[b];
                --b;
            }
            v[b + 1] = x;
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
    // split of diagonal d0: i elements from a, d0 - i from b
    int lo = max(0, d0 - lb), hi = min(d0, la);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;  // take a[mid] before b[d0 - 1 - mid]?
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

struct SegSmem {
    unsigned *k0, *v0, *k1, *v1, *whist, *start, *scratch;
};

__device__ __forceinline__ SegSmem seg_smem(unsigned char* raw, int cap) {
    SegSmem s;
    s.k0 = reinterpret_cast<unsigned*>(raw);
    s.v0 = s.k0 + cap;
    s.k1 = s.v0 + cap;
    s.v1 = s.k1 + cap;
    s.whist = s.v1 + cap;
    s.start = s.whist + (blockDim.x >> 5) * (kRadix + 1);
    s.scratch = s.start + kRadix;
    return s;
}

size_t seg_smem_bytes(int cap, int threads) {
    return sizeof(unsigned) * (4 * (size_t)cap + (threads / 32) * (kRadix + 1) + kRadix + 32 + 8);
}

// Sort the n <= cap pairs at (gk, gv) in shared memory and write them back in (t_r, splat) order.
__device__ void sort_chunk_in_smem(uint32_t* __restrict__ gk, uint32_t* __restrict__ gv, int n, const SegSmem& s,
                                   unsigned* s_red) {
    unsigned lo_and = 0xffffffffu, hi_or = 0u;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned k = gk[i];
        s.k0[i] = k;
        s.v0[i] = gv[i];
        lo_and &= k;
        hi_or |= k;
    }
    // bits that differ between keys: (OR of keys) & ~(AND of keys)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo_and &= __shfl_xor_sync(0xffffffffu, lo_and, o);
        hi_or |= __shfl_xor_sync(0xffffffffu, hi_or, o);
    }
    if (threadIdx.x == 0) { s_red[0] = 0xffffffffu; s_red[1] = 0u; }
    __syncthreads();
    if (lane_id() == 0) { atomicAnd(&s_red[0], lo_and); atomicOr(&s_red[1], hi_or); }
    __syncthreads();
    const unsigned diff = s_red[1] & ~s_red[0];
    const int nbits = diff ? 32 - __clz(diff) : 0;
    const bool flipped = smem_radix_sort(s.k0, s.v0, s.k1, s.v1, n, nbits, s.whist, s.start, s.scratch);
    unsigned* fk = flipped ? s.k1 : s.k0;
    unsigned* fv = flipped ? s.v1 : s.v0;
    order_ties(fk, fv, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        gk[i] = fk[i];
        gv[i] = fv[i];
    }
    __syncthreads();
}

// One CTA per tile (grid-stride over tiles). Segments of up to `cap` pairs are sorted in shared memory; longer ones
// are sorted in chunks of `cap` and merged pairwise through the scratch buffers (same offsets as the segment).
__global__ void segment_sort_kernel(u64 ntiles, const uint32_t* __restrict__ ranges, uint32_t* __restrict__ keys,
                                    uint32_t* __restrict__ values, uint32_t* __restrict__ scratch_k,
                                    uint32_t* __restrict__ scratch_v, int cap, int min_len, int max_len) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_red[2];
    const SegSmem s = seg_smem(smem_raw, cap);
    for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
        const int n = (int)(end - start);
        if (n < min_len || n > max_len || n < 2) continue;
        uint32_t* gk = keys + start;
        uint32_t* gv = values + start;
        for (int c0 = 0; c0 < n; c0 += cap) sort_chunk_in_smem(gk + c0, gv + c0, min(cap, n - c0), s, s_red);
        if (n <= cap) continue;
        uint32_t *sk = keys, *sv = values, *dk = scratch_k, *dv = scratch_v;
        for (int width = cap; width < n; width *= 2) {
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
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                keys[start + i] = sk[start + i];
                values[start + i] = sv[start + i];
            }
            __syncthreads();
        }
    }
}

constexpr int kSegSmallCap = 4096, kSegSmallThreads = 256;
constexpr int kSegLargeCap = 12288, kSegLargeThreads = 512;

}  // namespace

cudaError_t launch_bin(const omnigs_config& cfg, int64_t n, const omnigs_splat* splats, uint32_t* keys,
                       uint32_t* values, int64_t capacity, uint32_t* ranges, const WsLayout& L, char* ws,
                       cudaStream_t stream) {
    const int64_t total = n * cfg.num_views;
    const int tx = cfg.width / cfg.tile, ty = cfg.height / cfg.tile;
    const u64 ntiles = (u64)tx * ty * cfg.num_views;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    int* grid = reinterpret_cast<int*>(ws + L.tile_grid);
    u64* bsums = reinterpret_cast<u64*>(ws + L.scan_blocks);
    uint32_t* cursors = reinterpret_cast<uint32_t*>(ws + L.cursors);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(grid, 0, L.tile_grid_bytes, stream);
    if (e != cudaSuccess) return e;
    const float4* sp = reinterpret_cast<const float4*>(splats);
    if (total > 0) {
        ProfScope prof("tile_count", stream);
        tile_count_kernel<<<(unsigned)((total + kBinThreads - 1) / kBinThreads), kBinThreads, 0, stream>>>(
            total, (int)n, sp, tx, ty, cfg.tile, grid);
    }
    {
        ProfScope prof("tile_prefix", stream);
        tile_prefix_kernel<<<cfg.num_views, 1024, 0, stream>>>(tx, ty, grid);
    }
    const int nb = (int)((ntiles + kScanBlock - 1) / kScanBlock);
    {
        ProfScope prof("tile_scan", stream);
        scan_reduce_kernel<<<nb, kBinThreads, 0, stream>>>(ntiles, grid, tx, ty, bsums);
        scan_blocks_kernel<<<1, 1024, 0, stream>>>(nb, bsums, hdr, (u64)capacity);
        scan_write_kernel<<<nb, kBinThreads, 0, stream>>>(ntiles, grid, tx, ty, bsums, (u64)capacity, ranges, cursors);
    }
    if (total > 0 && capacity > 0) {
        ProfScope prof("bin_emit", stream);
        bin_emit_kernel<<<(unsigned)((total + kBinThreads - 1) / kBinThreads), kBinThreads, 0, stream>>>(
            total, (int)n, sp, tx, ty, cfg.tile, cursors, keys, values, (uint32_t)capacity);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort(const omnigs_config& cfg, int64_t capacity, uint32_t* keys, uint32_t* values,
                        const uint32_t* ranges, const WsLayout& L, char* ws, cudaStream_t stream) {
    if (capacity == 0) return cudaSuccess;
    const u64 ntiles = (u64)(cfg.width / cfg.tile) * (cfg.height / cfg.tile) * cfg.num_views;
    uint32_t* sk = reinterpret_cast<uint32_t*>(ws + L.alt_keys);
    uint32_t* sv = reinterpret_cast<uint32_t*>(ws + L.alt_values);
    const size_t small_smem = seg_smem_bytes(kSegSmallCap, kSegSmallThreads);
    const size_t large_smem = seg_smem_bytes(kSegLargeCap, kSegLargeThreads);
    cudaError_t e = cudaFuncSetAttribute(segment_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)large_smem);
    if (e != cudaSuccess) return e;
    const u64 max_grid = (u64)num_sms() * 64;
    const unsigned grid = (unsigned)(ntiles < max_grid ? ntiles : max_grid);
    {
        ProfScope prof("segment_sort", stream);
        segment_sort_kernel<<<grid, kSegSmallThreads, small_smem, stream>>>(ntiles, ranges, keys, values, sk, sv,
                                                                             kSegSmallCap, 0, kSegSmallCap);
    }
    {
        ProfScope prof("segment_sort_large", stream);
        segment_sort_kernel<<<grid, kSegLargeThreads, large_smem, stream>>>(ntiles, ranges, keys, values, sk, sv,
                                                                             kSegLargeCap, kSegSmallCap + 1, 0x7fffffff);
    }
    return cudaGetLastError();
}

}  // namespace omnigs
