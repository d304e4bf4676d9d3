// sort.cu -- tile-key expansion, device radix sort and tile ranges (a2-a4).
//
// The (tile, depth) order of the instance list is produced in two stable
// sorts instead of one 64-bit sort:
//   1. the visible (view, Gaussian) items are compacted (index order) and
//      radix-sorted by the binary32 bits of their view-space depth;
//   2. each item emits its (tile id, item) instances in that depth order, and
//      the instances are radix-sorted by tile id only.
// Stability makes the result equal to a sort by (tile id, depth bits, item
// index): the unique order of the 64-bit keys (tile << 32 | depth bits).
// Only ceil(log2(total tiles)) bits are sorted over the (large) instance
// list, instead of 32 + that many.
//
// Every kernel reads its item count from device memory, so a whole step can
// be captured in a CUDA graph without a host round trip; grids are sized by
// host-side upper bounds.
#include <algorithm>

#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems; // 4096

constexpr int kRsWarps = 8;
constexpr int kRsThreads = kRsWarps * 32;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems; // 2048
constexpr int kRsMaxGrid = 1024; // row scan: one thread per block of the grid
constexpr int kRsBlocksPerSm = 3; // downsweep occupancy (its launch bound)

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread block.
// Returns the exclusive prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t x, uint32_t *total) {
    __shared__ uint32_t warp_sums[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    uint32_t warp_off = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t s = warp_sums[w];
        if (w < warp) warp_off += s;
        tot += s;
    }
    __syncthreads();
    *total = tot;
    return warp_off + inc - x;
}

__device__ __forceinline__ uint32_t scan_item(const uint32_t *in, const uint32_t *gather,
                                              int flag_only, uint32_t i) {
    const uint32_t v = in[gather ? gather[i] : i];
    return flag_only ? (v != 0u) : v;
}

__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const uint32_t *in, const uint32_t *gather, int flag_only, const uint32_t *n_dev,
                   uint32_t n_host, uint32_t *block_sums) {
    const uint32_t n = n_dev ? *n_dev : n_host;
    const uint32_t begin = blockIdx.x * (uint32_t)kScanTile;
    uint32_t sum = 0;
    if (begin < n) {
        const uint32_t end = min(begin + (uint32_t)kScanTile, n);
        for (uint32_t i = begin + threadIdx.x; i < end; i += kScanThreads)
            sum += scan_item(in, gather, flag_only, i);
    }
    uint32_t tot;
    block_exclusive_scan_256(sum, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Exclusive scan of the block sums by a single block; writes the grand total.
__global__ void __launch_bounds__(kScanThreads)
scan_blocks_kernel(uint32_t *block_sums, uint32_t nb, uint32_t *out_total) {
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += kScanThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < nb ? block_sums[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(x, &tot);
        if (i < nb) block_sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && out_total) *out_total = carry;
}

// The block's tile moves between memory and registers through shared memory:
// loads and stores stay coalesced (consecutive threads, consecutive items)
// while each thread scans kScanItems consecutive items in registers, so one
// block-wide scan of the thread sums gives all the offsets.
constexpr int kScanPitch = kScanItems + 1; // conflict-free blocked reads
__global__ void __launch_bounds__(kScanThreads)
scan_down_kernel(const uint32_t *in, const uint32_t *gather, int flag_only, const uint32_t *n_dev,
                 uint32_t n_host, const uint32_t *block_offsets, uint32_t *out) {
    __shared__ uint32_t tile[kScanThreads * kScanPitch];
    const uint32_t n = n_dev ? *n_dev : n_host;
    const uint32_t begin = blockIdx.x * (uint32_t)kScanTile;
    if (begin >= n) return;
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t r = (uint32_t)(j * kScanThreads + t); // tile-relative item
        tile[(r / kScanItems) * kScanPitch + r % kScanItems] =
            begin + r < n ? scan_item(in, gather, flag_only, begin + r) : 0u;
    }
    __syncthreads();
    uint32_t x[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        x[j] = tile[t * kScanPitch + j];
        sum += x[j];
    }
    uint32_t tot;
    uint32_t run = block_offsets[blockIdx.x] + block_exclusive_scan_256(sum, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        tile[t * kScanPitch + j] = run;
        run += x[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t r = (uint32_t)(j * kScanThreads + t);
        if (begin + r < n) out[begin + r] = tile[(r / kScanItems) * kScanPitch + r % kScanItems];
    }
}

// The whole scan in one block of 1024 threads, for inputs of at most
// kScanSingle items (one launch instead of three).
constexpr int kScanSingle = 1024 * kScanItems;
__global__ void __launch_bounds__(1024)
scan_single_kernel(const uint32_t *in, const uint32_t *gather, int flag_only, const uint32_t *n_dev,
                   uint32_t n_host, uint32_t *out, uint32_t *out_total) {
    __shared__ uint32_t warp_sums[32];
    const uint32_t n = n_dev ? min(*n_dev, n_host) : n_host;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t i0 = threadIdx.x * (uint32_t)kScanItems;
    uint32_t x[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        x[j] = i0 + j < n ? scan_item(in, gather, flag_only, i0 + j) : 0u;
        sum += x[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t ws = warp_sums[lane];
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_sums[lane] = wi - ws;
        if (lane == 31 && out_total) *out_total = wi;
    }
    __syncthreads();
    uint32_t run = warp_sums[warp] + inc - sum;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (i0 + j < n) out[i0 + j] = run;
        run += x[j];
    }
}

// Compaction of the visible items fused into the scan's last step: each
// thread scans the visibility flags of its kScanItems consecutive items and
// writes the (depth bits, item index) pairs of the visible ones at their
// positions (index order).
__global__ void __launch_bounds__(kScanThreads)
compact_down_kernel(const uint32_t *__restrict__ tiles, const uint32_t *__restrict__ zbits, uint32_t n,
                    const uint32_t *__restrict__ block_offsets, uint32_t *__restrict__ keys,
                    uint32_t *__restrict__ vals) {
    __shared__ uint32_t tile[kScanThreads * kScanPitch];
    const uint32_t begin = blockIdx.x * (uint32_t)kScanTile;
    if (begin >= n) return;
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t r = (uint32_t)(j * kScanThreads + t);
        tile[(r / kScanItems) * kScanPitch + r % kScanItems] = begin + r < n && tiles[begin + r] != 0u;
    }
    __syncthreads();
    uint32_t flags = 0, sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t f = tile[t * kScanPitch + j];
        flags |= f << j;
        sum += f;
    }
    uint32_t tot;
    uint32_t run = block_offsets[blockIdx.x] + block_exclusive_scan_256(sum, &tot);
    const uint32_t i0 = begin + (uint32_t)t * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (flags >> j & 1u) {
            keys[run] = zbits[i0 + j];
            vals[run] = i0 + j;
            ++run;
        }
    }
}

// --------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, reduce-then-scan per pass.
// --------------------------------------------------------------------------
__device__ __forceinline__ void rs_chunk(uint32_t n, int G, int b, uint32_t &begin, uint32_t &end) {
    uint32_t per = (n + G - 1) / G;
    per = (per + kRsTile - 1) / kRsTile * kRsTile;
    const uint64_t bb = (uint64_t)b * per;
    begin = bb < n ? (uint32_t)bb : n;
    end = (uint64_t)begin + per < n ? begin + per : n;
}

__global__ void __launch_bounds__(kRsThreads)
radix_upsweep_kernel(const uint32_t *keys, const uint32_t *n_dev, uint32_t n_host, int shift, int G,
                     uint32_t *counts) {
    __shared__ uint32_t hist[kRsWarps][256];
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n = n_dev ? *n_dev : n_host;
    uint32_t begin, end;
    rs_chunk(n, G, blockIdx.x, begin, end);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // kRsItems keys per lane and round, all loaded before the first is counted
    // and the next round's loaded while this one is counted; within an
    // instruction the leaders of a digit's peers hit distinct bins
    uint32_t kn[kRsItems];
    auto load = [&](uint32_t i0) {
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const uint32_t i = i0 + j * 32 + lane;
            kn[j] = i < end ? __ldg(keys + i) : 0u;
        }
    };
    load(begin + warp * (32 * kRsItems));
    for (uint32_t i0 = begin + warp * (32 * kRsItems); i0 < end; i0 += kRsThreads * kRsItems) {
        uint32_t d[kRsItems];
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) d[j] = i0 + j * 32 + lane < end ? (kn[j] >> shift) & 255u : 256u;
        if (i0 + kRsThreads * kRsItems < end) load(i0 + kRsThreads * kRsItems);
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const uint32_t peers = __match_any_sync(0xffffffffu, d[j]);
            if (d[j] < 256u && lane == __ffs(peers) - 1) hist[warp][d[j]] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) s += hist[w][d];
    counts[(size_t)d * G + blockIdx.x] = s;
}

// One block per digit: exclusive scan of the digit's per-block counts, in place.
__global__ void __launch_bounds__(1024)
radix_rowscan_kernel(uint32_t *counts, int G, uint32_t *totals) {
    __shared__ uint32_t warp_sums[32];
    const int d = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t x = t < G ? counts[(size_t)d * G + t] : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t ws = warp_sums[lane];
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_sums[lane] = wi - ws;
        if (lane == 31) totals[d] = wi;
    }
    __syncthreads();
    if (t < G) counts[(size_t)d * G + t] = warp_sums[warp] + inc - x;
}

__global__ void __launch_bounds__(kRsThreads, kRsBlocksPerSm)
radix_downsweep_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                       uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                       const uint32_t *n_dev, uint32_t n_host, int shift, int G, const uint32_t *counts,
                       const uint32_t *totals) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_hist[kRsWarps][256];
    __shared__ uint32_t s_tile[256];
    __shared__ uint32_t s_start[256];          // first position of each digit in the tile
    __shared__ uint32_t s_k[kRsTile], s_v[kRsTile]; // the tile in digit order
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    {
        uint32_t tot;
        const uint32_t dp = block_exclusive_scan_256(totals[t], &tot);
        s_base[t] = dp + counts[(size_t)t * G + blockIdx.x];
    }
    const uint32_t n = n_dev ? *n_dev : n_host;
    uint32_t begin, end;
    rs_chunk(n, G, blockIdx.x, begin, end);
    const uint32_t lt = lanemask_lt();
    // the next tile's keys and values are loaded while this one is ranked
    uint32_t kn[kRsItems], vn[kRsItems];
    auto load = [&](uint32_t tile0) {
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const uint32_t i = tile0 + warp * (kRsItems * 32) + j * 32 + lane;
            kn[j] = i < end ? keys_in[i] : 0u;
            vn[j] = i < end ? vals_in[i] : 0u;
        }
    };
    if (begin < end) load(begin);
    for (uint32_t tile0 = begin; tile0 < end; tile0 += kRsTile) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) s_hist[w][t] = 0;
        uint32_t k[kRsItems], v[kRsItems], rank[kRsItems], d[kRsItems];
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const uint32_t i = tile0 + warp * (kRsItems * 32) + j * 32 + lane;
            k[j] = kn[j];
            v[j] = vn[j];
            d[j] = i < end ? (k[j] >> shift) & 255u : 256u;
        }
        if (tile0 + kRsTile < end) load(tile0 + kRsTile);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const uint32_t peers = __match_any_sync(0xffffffffu, d[j]);
            uint32_t c = 0;
            if (d[j] < 256u) c = s_hist[warp][d[j]];
            rank[j] = c + __popc(peers & lt);
            __syncwarp();
            if (d[j] < 256u && lane == __ffs(peers) - 1) s_hist[warp][d[j]] = c + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t tile_n;
        {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) {
                const uint32_t c = s_hist[w][t];
                s_hist[w][t] = run;
                run += c;
            }
            s_tile[t] = run;
            s_start[t] = block_exclusive_scan_256(run, &tile_n);
        }
        __syncthreads();
        // reorder the tile by digit in shared memory (stable) ...
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            if (d[j] < 256u) {
                const uint32_t lp = s_start[d[j]] + s_hist[warp][d[j]] + rank[j];
                s_k[lp] = k[j];
                s_v[lp] = v[j];
            }
        }
        __syncthreads();
        // ... and write it out: consecutive threads, consecutive addresses within a digit's run
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const uint32_t lp = (uint32_t)(j * kRsThreads + t);
            if (lp < tile_n) {
                const uint32_t key = s_k[lp];
                const uint32_t dg = (key >> shift) & 255u;
                const uint32_t dest = s_base[dg] + (lp - s_start[dg]);
                keys_out[dest] = key;
                vals_out[dest] = s_v[lp];
            }
        }
        __syncthreads();
        s_base[t] += s_tile[t];
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// Instance emission, ranges, debug keys.
// --------------------------------------------------------------------------
// A warp takes 32 consecutive items (in depth order) and writes all their
// instances together: lane r of each round of 32 output positions finds its
// item by a binary search over the warp's exclusive prefix (shuffles), so the
// stores are coalesced and an item that covers many tiles does not hold one
// lane while the others idle.
__global__ void __launch_bounds__(256)
emit_kernel(const ViewSet *__restrict__ vsp, const uint32_t *__restrict__ sorted_idx,
            const uint32_t *__restrict__ offsets, const uint32_t *n_vis_dev, const uint2 *__restrict__ rects,
            uint32_t n_gauss, uint32_t *__restrict__ tile_ids, uint32_t *__restrict__ inst_vals, uint64_t m_cap,
            uint32_t *status) {
    const uint32_t n = *n_vis_dev;
    const int lane = threadIdx.x & 31;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t j0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; j0 < n; j0 += n_warps * 32u) {
        const uint32_t j = j0 + (uint32_t)lane;
        uint32_t idx = 0, cnt = 0, x0 = 0, y0 = 0, w = 1, base = 0, txn = 0;
        uint64_t pos0 = 0;
        if (j < n) {
            idx = sorted_idx[j];
            const uint32_t vi = idx / n_gauss;
            const uint2 rc = rects[idx];
            x0 = rc.x & 0xffffu;
            y0 = rc.y & 0xffffu;
            w = (rc.x >> 16) - x0;
            cnt = w * ((rc.y >> 16) - y0);
            base = vsp->v[vi].tile_base;
            txn = (uint32_t)vsp->v[vi].tiles_x;
            pos0 = offsets[j];
            // instances past the capacity are dropped: the item that straddles it
            // keeps its first ones, so that every position below min(M, m_cap),
            // the count the sort and ranges read, is written by this launch
            if (pos0 + cnt > m_cap) {
                atomicOr(status, kStatusCapacity);
                cnt = pos0 < m_cap ? (uint32_t)(m_cap - pos0) : 0u;
            }
        }
        if (w == 0) w = 1;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - cnt;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t start_lo = __shfl_sync(0xffffffffu, (uint32_t)pos0, 0);
        const uint32_t start_hi = __shfl_sync(0xffffffffu, (uint32_t)(pos0 >> 32), 0);
        const uint64_t start = ((uint64_t)start_hi << 32) | start_lo;
        const float inv_w = 1.f / (float)w;
        for (uint32_t r0 = 0; r0 < total; r0 += 32) {
            const uint32_t r = r0 + (uint32_t)lane;
            // the last lane k whose exclusive prefix is <= r (zero-count lanes share
            // the prefix of the next item and are passed over)
            int k = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, excl, k + step);
                if (e <= r) k += step;
            }
            const uint32_t q = r - __shfl_sync(0xffffffffu, excl, k);
            const uint32_t kw = __shfl_sync(0xffffffffu, w, k);
            const float kinv = __shfl_sync(0xffffffffu, inv_w, k);
            const uint32_t kx0 = __shfl_sync(0xffffffffu, x0, k);
            const uint32_t ky0 = __shfl_sync(0xffffffffu, y0, k);
            const uint32_t kbase = __shfl_sync(0xffffffffu, base, k);
            const uint32_t ktxn = __shfl_sync(0xffffffffu, txn, k);
            const uint32_t kidx = __shfl_sync(0xffffffffu, idx, k);
            if (r < total) {
                // row within the rectangle: q / w, from the float estimate corrected by one
                uint32_t ty = (uint32_t)((float)q * kinv);
                if (ty * kw > q) --ty;
                if ((ty + 1) * kw <= q) ++ty;
                const uint64_t p = start + r;
                tile_ids[p] = kbase + (ky0 + ty) * ktxn + kx0 + (q - ty * kw);
                inst_vals[p] = kidx;
            }
        }
    }
}

__global__ void ranges_kernel(const uint32_t *__restrict__ tile_ids, const uint32_t *m_dev,
                              uint32_t m_cap, uint2 *__restrict__ ranges) {
    const uint32_t m = min(*m_dev, m_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint32_t t = tile_ids[i];
        if (i == 0 || tile_ids[i - 1] != t) ranges[t].x = i;
        if (i == m - 1 || tile_ids[i + 1] != t) ranges[t].y = i + 1;
    }
}

__global__ void clamp_count_kernel(const uint32_t *m_dev, uint32_t m_cap, uint32_t *out) {
    const uint32_t m = *m_dev;
    *out = m < m_cap ? m : m_cap;
}

__global__ void debug_keys_kernel(const uint32_t *tile_ids, const uint32_t *inst_vals,
                                  const uint32_t *zbits, uint32_t n_gauss, uint64_t *keys,
                                  uint32_t *vals, uint32_t m) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint32_t idx = inst_vals[i];
        keys[i] = ((uint64_t)tile_ids[i] << 32) | zbits[idx];
        vals[i] = idx % n_gauss;
    }
}

__global__ void sum_i32_kernel(const int32_t *x, uint32_t n, unsigned long long *out) {
    unsigned long long acc = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += (uint32_t)x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// One resident wave of the downsweep (kRsBlocksPerSm blocks per SM), each
// block taking an equal run of whole tiles, so no block waits for a second
// wave behind the others.
int rs_grid(int64_t n_max) {
    int64_t g = (n_max + kRsTile - 1) / kRsTile;
    const int64_t wave = (int64_t)device_sm_count() * kRsBlocksPerSm;
    if (g < 1) g = 1;
    if (g > wave) g = wave;
    if (g > kRsMaxGrid) g = kRsMaxGrid;
    return (int)g;
}

int grid_stride_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = device_sm_count() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

} // namespace

size_t scan_tmp_words(int64_t n_max) { return (size_t)((n_max + kScanTile - 1) / kScanTile) + 1; }

void launch_scan(const uint32_t *in, const uint32_t *gather, int flag_only, uint32_t *out,
                 uint32_t *out_total, const uint32_t *n_dev, int64_t n_max, uint32_t *tmp,
                 cudaStream_t s) {
    const uint32_t nb = (uint32_t)((n_max + kScanTile - 1) / kScanTile);
    if (nb == 0) {
        if (out_total) cudaMemsetAsync(out_total, 0, sizeof(uint32_t), s);
        return;
    }
    if (n_max <= kScanSingle) {
        scan_single_kernel<<<1, 1024, 0, s>>>(in, gather, flag_only, n_dev, (uint32_t)n_max, out, out_total);
        return;
    }
    scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(in, gather, flag_only, n_dev, (uint32_t)n_max, tmp);
    scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(tmp, nb, out_total);
    scan_down_kernel<<<nb, kScanThreads, 0, s>>>(in, gather, flag_only, n_dev, (uint32_t)n_max, tmp, out);
}

void launch_compact_scan(const uint32_t *tiles, const uint32_t *zbits, uint32_t *keys, uint32_t *vals,
                         uint32_t *out_total, int64_t n, uint32_t *tmp, cudaStream_t s) {
    const uint32_t nb = (uint32_t)((n + kScanTile - 1) / kScanTile);
    if (nb == 0) {
        cudaMemsetAsync(out_total, 0, sizeof(uint32_t), s);
        return;
    }
    scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(tiles, nullptr, 1, nullptr, (uint32_t)n, tmp);
    scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(tmp, nb, out_total);
    compact_down_kernel<<<nb, kScanThreads, 0, s>>>(tiles, zbits, (uint32_t)n, tmp, keys, vals);
}

size_t radix_tmp_words(int64_t n_max) { return (size_t)256 * rs_grid(n_max) + 256; }

int launch_radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *n_dev, int64_t n_max, int bits, uint32_t *tmp,
                      cudaStream_t s) {
    if (n_max <= 0 || bits <= 0) return 0;
    const int G = rs_grid(n_max);
    uint32_t *counts = tmp;
    uint32_t *totals = tmp + (size_t)256 * G;
    const int passes = std::min((bits + 7) / 8, 4);
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        radix_upsweep_kernel<<<G, kRsThreads, 0, s>>>(ki, n_dev, (uint32_t)n_max, shift, G, counts);
        radix_rowscan_kernel<<<256, 1024, 0, s>>>(counts, G, totals);
        radix_downsweep_kernel<<<G, kRsThreads, 0, s>>>(ki, vi, ko, vo, n_dev, (uint32_t)n_max, shift, G, counts,
                                                        totals);
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    return passes & 1; // 1: the sorted pairs are in keys_alt / vals_alt
}

void launch_emit(const ViewSet *vs, const uint32_t *sorted_idx, const uint32_t *offsets,
                 const uint32_t *n_vis_dev, const uint2 *rects, int n_gauss, uint32_t *tile_ids,
                 uint32_t *inst_vals, int64_t m_cap, int64_t n_max, uint32_t *status,
                 cudaStream_t s) {
    if (n_max <= 0) return;
    emit_kernel<<<grid_stride_blocks(n_max, 256), 256, 0, s>>>(vs, sorted_idx, offsets, n_vis_dev, rects,
                                                                (uint32_t)n_gauss, tile_ids, inst_vals,
                                                                (uint64_t)m_cap, status);
}

void launch_ranges(const uint32_t *tile_ids, const uint32_t *m_dev, int64_t m_cap,
                   uint2 *ranges, uint32_t total_tiles, cudaStream_t s) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, s);
    if (m_cap <= 0) return;
    ranges_kernel<<<grid_stride_blocks(m_cap, 256), 256, 0, s>>>(tile_ids, m_dev, (uint32_t)m_cap, ranges);
}

void launch_clamp_count(const uint32_t *m_dev, int64_t m_cap, uint32_t *out, cudaStream_t s) {
    clamp_count_kernel<<<1, 1, 0, s>>>(m_dev, (uint32_t)(m_cap < 0xffffffffLL ? m_cap : 0xffffffffLL), out);
}

void launch_sum_i32(const int32_t *x, uint32_t n, unsigned long long *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (n == 0) return;
    sum_i32_kernel<<<grid_stride_blocks(n, 256), 256, 0, s>>>(x, n, out);
}

void launch_debug_keys(const uint32_t *tile_ids, const uint32_t *inst_vals, const uint32_t *zbits,
                       int n_gauss, uint64_t *keys, uint32_t *vals, int64_t m, cudaStream_t s) {
    if (m <= 0) return;
    debug_keys_kernel<<<grid_stride_blocks(m, 256), 256, 0, s>>>(tile_ids, inst_vals, zbits,
                                                                  (uint32_t)n_gauss, keys, vals, (uint32_t)m);
}

} // namespace lvigs
