// composite.cu -- front-to-back alpha compositing (a5) and its reverse (a6).
//
// Work unit: one 8x8 block of pixels per warp, two vertically adjacent pixels
// per lane.  The kernels are persistent: a GPU-filling grid of warps takes
// work items from a global counter (one atomicAdd per item; no warp ever
// waits on another).
//
// List-parallel compositing.  A tile's depth-sorted instance list is cut into
// chunks of L entries; every (tile, chunk, 8x8 block) is an independent work
// item, so the tens of thousands of Gaussians that pile up in a tile of a
// coarse pyramid level are composited by many warps at once instead of one.
//   phase 1  each item walks its chunk (Eq. (3)-(6)): alpha = min(0.99,
//            o exp(power)), skipped below 1/255, stop before a Gaussian that
//            would take the transmittance below 1e-4.  A one-chunk tile is
//            final here.  For a longer list the walk starts from T = 1 and
//            stores the chunk's local sums (colour, depth, T, last contributor,
//            whether the local T hit the stop, which implies the global stop
//            lies at or before that Gaussian).  Items run chunk-major (all
//            first chunks, then all second chunks, ...) and a pixel whose local
//            stop is published for an earlier chunk (a per-pixel atomicMin) is
//            skipped by later chunks: they cannot contribute to it.  A list of
//            a few chunks (how many follows the work per warp) is instead one
//            item, walked whole with the true transmittance: final here, its
//            chunks' slots written in the backward's form, no phase 2.
//   phase 2  per pixel the chunks are combined in order: C += T C_k,
//            T *= T_k, until the chunk whose end would cross 1e-4 (2a); that
//            chunk is walked again from the true T to find the exact stop, one
//            (tile, chunk, block) item per warp (2b); then every chunk gets the
//            transmittance at its end and the normalised sums of everything
//            composited after it (all terms non-negative, so no cancellation),
//            the state the backward walk of that chunk starts from (2c).
// Within a walk the list is consumed in batches of 32*BM: each lane gathers
// records and tests them against the block with the conservative box of the
// region where alpha can reach 1/255 (half-extents from preprocessing); the
// hits are compacted into shared memory with a ballot, in list order.  Culled
// Gaussians fail the 1/255 test at every pixel of the block, so results equal
// those of walking the whole list.
//
// The backward pass walks each chunk in reverse from the pixel's last
// contributor, recovering the transmittance by division (T_i = T_{i+1} /
// (1 - alpha_i)); no per-Gaussian state is stored.  dL/dalpha needs only the
// dot product of the upstream gradients with the sums of what lies behind a
// Gaussian, so one running scalar per pixel replaces those five sums.  Each
// lane sums over its two pixels ten terms: five moments of dL/dpower (times
// dx, dy, dx^2, dx dy, dy^2; the conic enters once per Gaussian, in the
// backward preprocess), o dL/dopacity, and the colour and depth weights.  The
// warp reduce-scatters the ten sums with 12 shuffles, and the ten lanes that
// end with a total add it to the Gaussian's gradient record with one atomic
// instruction.
#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr int PB = 8;  // warp pixel block is PB x PB
constexpr int PPT = 2; // pixels per lane (rows 2r, 2r+1 of the block)
constexpr int kWarpsPerCta = 4;
constexpr int kFields = 6; // per (pixel, chunk) slot and checkpoint
constexpr int kSub = 8;    // checkpoint groups per chunk: after each eighth (the last is the chunk's end)
// Lists of 2 .. w chunks are walked whole by one forward warp (the true
// transmittance throughout, so its stops are exact and no combine is needed),
// which writes each chunk's slot in the form the backward starts from; longer
// lists are walked chunk-parallel and combined.  Such an item must not
// outlast the rest of the work: w is the chunk count of about 1.25 times the
// average walk per resident warp (instances x blocks per tile / warps), at
// most kWholeMax, computed alike by every kernel from the instance count.
constexpr uint32_t kWholeMax = 8;
__device__ __forceinline__ uint32_t whole_max(const ChunkPlan &cp) {
    const uint64_t per_warp = (uint64_t)(*cp.n_inst) * (uint64_t)cp.nb / (uint64_t)(cp.warps ? cp.warps : 1u);
    const uint64_t w = per_warp * 5 / (4 * (uint64_t)cp.L);
    return w < kWholeMax ? (uint32_t)w : kWholeMax;
}
__device__ __forceinline__ bool whole_list(uint32_t nch, uint32_t wmax) { return nch >= 2 && nch <= wmax; }

// Can record (a, b, c) reach alpha >= 1/255 anywhere in the block
// [x0, x0+7] x [y0, y0+7]?  First the conservative box of that region
// (half-extents from preprocessing), then the ellipse itself: the largest
// base-2 exponent e2 = a2 dx^2 + b2 dx dy + c2 dy^2 over the block (concave,
// so either 0 at the centre or on one of the four edges, where the best
// offset along the edge is a clamped closed form) plus log2(o) against
// log2(1/255).
// The comparison keeps a slack of 0.05 plus 2e-6 of the largest term any
// pixel of the block can have, far above the rounding of both this bound
// and the per-pixel exponent, so a culled Gaussian fails the 1/255 test at
// every pixel of the block.
__device__ __forceinline__ bool meets(const float4 a, const float4 b, const float4 c, float x0, float y0) {
    const float ex = b.w, ey = c.w;
    if (!(a.x + ex >= x0 && a.x - ex <= x0 + (PB - 1) && a.y + ey >= y0 && a.y - ey <= y0 + (PB - 1)))
        return false;
    // dx = u - px over [X0, X1], dy = v - py over [Y0, Y1]
    const float X1 = a.x - x0, X0 = X1 - (float)(PB - 1);
    const float Y1 = a.y - y0, Y0 = Y1 - (float)(PB - 1);
    if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return true;
    const float a2 = a.z, b2 = a.w, c2 = b.x; // a2, c2 < 0
    const float ka = __fdividef(-0.5f * b2, a2), kc = __fdividef(-0.5f * b2, c2);
    float best = -INFINITY;
    {
        const float dx0 = fminf(fmaxf(ka * Y0, X0), X1), dx1 = fminf(fmaxf(ka * Y1, X0), X1);
        best = fmaxf(best, fmaf(dx0, fmaf(a2, dx0, b2 * Y0), c2 * Y0 * Y0));
        best = fmaxf(best, fmaf(dx1, fmaf(a2, dx1, b2 * Y1), c2 * Y1 * Y1));
        const float dy0 = fminf(fmaxf(kc * X0, Y0), Y1), dy1 = fminf(fmaxf(kc * X1, Y0), Y1);
        best = fmaxf(best, fmaf(dy0, fmaf(c2, dy0, b2 * X0), a2 * X0 * X0));
        best = fmaxf(best, fmaf(dy1, fmaf(c2, dy1, b2 * X1), a2 * X1 * X1));
    }
    const float mx = fmaxf(fabsf(X0), fabsf(X1)), my = fmaxf(fabsf(Y0), fabsf(Y1));
    const float big = fmaf(-a2, mx * mx, fmaf(fabsf(b2), mx * my, -c2 * my * my));
    return best + b.y + fmaf(2e-6f, big, 0.05f) >= kLog2AlphaMin; // b.y = log2(o)
}

template <int TW, int TH>
struct Geometry {
    static constexpr int WX = TW / PB, WY = TH / PB;
    static constexpr int NB = WX * WY; // 8x8 blocks per tile
    static constexpr int TPX = TW * TH;
    static_assert(TW % PB == 0 && TH % PB == 0, "tile is a whole number of 8x8 blocks");
};

// Pixel coordinates of a lane in block `blk` of the tile with local index lt.
template <int TW, int TH>
struct BlockPix {
    int px, py0; // image coordinates of the lane's pixels (px, py0) and (px, py0 + 1)
    int lp0;     // tile-local index of the first pixel (the second is lp0 + TW)
    float fx0, fy0;
    __device__ __forceinline__ BlockPix(const ViewDesc &V, uint32_t lt, int blk, int lane) {
        using Gm = Geometry<TW, TH>;
        const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
        const int lx = (blk % Gm::WX) * PB + (lane & 7), ly = (blk / Gm::WX) * PB + (lane >> 3) * PPT;
        px = tx * TW + lx;
        py0 = ty * TH + ly;
        lp0 = ly * TW + lx;
        fx0 = (float)(tx * TW + (blk % Gm::WX) * PB);
        fy0 = (float)(ty * TH + (blk / Gm::WX) * PB);
    }
};

struct Smem {
    float4 *A, *B, *C;
    int *Pos;
    uint32_t *Idx;
};

// Gather list entries [base, min(base + 32*BM, hi)) and compact the ones whose
// alpha box meets the block into shared memory (list order).  Returns the count.
template <int BM, bool WITH_IDX>
__device__ __forceinline__ int gather_cull(const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs,
                                           uint32_t rg_x, uint32_t base, uint32_t hi, float fx0, float fy0,
                                           const Smem &sm, int lane) {
    const uint32_t ltmask = (1u << lane) - 1u;
    int n = 0;
#pragma unroll
    for (int q = 0; q < BM; ++q) {
        const uint32_t i = base + q * 32 + lane;
        GRec r;
        uint32_t idx = 0;
        bool hit = false;
        if (i < hi) {
            idx = inst_vals[i];
            r = recs[idx];
            hit = meets(r.a, r.b, r.c, fx0, fy0);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int slot = n + __popc(m & ltmask);
            sm.A[slot] = r.a;
            sm.B[slot] = r.b;
            sm.C[slot] = r.c;
            sm.Pos[slot] = (int)(i - rg_x);
            if (WITH_IDX) sm.Idx[slot] = idx;
        }
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

// Where a walk stores its checkpoints: the (pixel, chunk) slot's groups.
struct Checkpoints {
    float *g0;    // group 0, field 0 of the slot (null: no checkpoints)
    int every;    // list entries between checkpoints
    int tpx, lp0, tw;
};

// Front-to-back walk of list entries [lo, hi) for the lane's pixels, from the
// state passed in.  Pixels with done[k] set are left alone; stopped[k] is set
// when the pixel stops (the transmittance test) inside this walk.  With
// CKPT the state after every `every` entries (except at hi) is stored; with
// START a pixel takes no entry before list position start[k].
template <int BM, bool CKPT, bool START>
__device__ __forceinline__ void fwd_walk(const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs,
                                         uint32_t rg_x, uint32_t lo, uint32_t hi, float fpx, int py0, float fx0,
                                         float fy0, const Smem &sm, int lane, float T[PPT], float C0[PPT],
                                         float C1[PPT], float C2[PPT], float D[PPT], int last[PPT], bool done[PPT],
                                         bool stopped[PPT], const Checkpoints &ck, const int start[PPT]) {
    constexpr int B = 32 * BM;
    bool tdone = done[0] && done[1];
    // checkpoints lie at lo + (m + 1) * every < hi; next_ck is the next to store
    const int n_ck = (CKPT && ck.g0 && hi > lo) ? min(kSub - 1, (int)((hi - lo - 1) / (uint32_t)ck.every)) : 0;
    int next_ck = 0;
    auto store_ck = [&](int m) {
        float *g = ck.g0 + (size_t)m * kFields * ck.tpx;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int lp = ck.lp0 + k * ck.tw;
            g[0 * ck.tpx + lp] = C0[k];
            g[1 * ck.tpx + lp] = C1[k];
            g[2 * ck.tpx + lp] = C2[k];
            g[3 * ck.tpx + lp] = D[k];
            g[4 * ck.tpx + lp] = T[k];
            g[5 * ck.tpx + lp] = __int_as_float(last[k] | (stopped[k] ? (int)0x80000000 : 0));
        }
    };
    // Without START a finished pixel is skipped by raising its alpha threshold
    // above any alpha (one test instead of two per evaluation); the re-walk
    // with START keeps the separate test, which its register budget prefers.
    float thr[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) thr[k] = (!START && done[k]) ? 1e30f : kLog2AlphaMin;
    for (uint32_t base = lo; base < hi; base += B) {
        if (__all_sync(0xffffffffu, tdone)) {
            // every pixel is finished: the remaining checkpoints hold the final state
            for (; next_ck < n_ck; ++next_ck) store_ck(next_ck);
            break;
        }
        if (START) {
            // skip the batches before the earliest position an unfinished pixel
            // still needs (pixels that resume further on leave gaps)
            int need = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (!done[k]) need = min(need, start[k]);
            need = __reduce_min_sync(0xffffffffu, need);
            const uint32_t at = rg_x + (uint32_t)need;
            if (at >= base + B) base = lo + (at - lo) / B * B;
            if (base >= hi) break;
        }
        const int n = gather_cull<BM, false>(inst_vals, recs, rg_x, base, hi, fx0, fy0, sm, lane);
        for (int q = 0; q < n && !tdone; ++q) {
            const float4 a = sm.A[q];
            const float4 b = sm.B[q];
            const float dx = a.x - fpx;
            const float a2dx = __fmul_rn(a.z, dx);
            int qpos = 0;
            if (START) qpos = sm.Pos[q];
            // the 1/255 tests of both pixels first (e2 = log2(o G); no test of a
            // positive power: the conic is positive definite, so one is rounding
            // at the centre)
            float e2[PPT];
            bool take[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float dy = a.y - (float)(py0 + k);
                e2[k] = gauss_exponent2(a2dx, a.w, b.x, b.y, dx, dy);
                take[k] = e2[k] >= (START ? kLog2AlphaMin : thr[k]); // alpha >= 1/255, pixel not finished
                if (START) take[k] = take[k] && !done[k] && qpos >= start[k];
            }
            if (!(take[0] || take[1])) continue;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (!take[k]) continue;
                const float alpha = fminf(kAlphaMax, exp2_approx(e2[k]));
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                if (Tn < kTMin) {
                    done[k] = true;
                    stopped[k] = true;
                    thr[k] = 1e30f;
                    tdone = done[0] && done[1];
                    continue;
                }
                const float4 c = sm.C[q];
                const float w = alpha * T[k];
                C0[k] = fmaf(c.x, w, C0[k]);
                C1[k] = fmaf(c.y, w, C1[k]);
                C2[k] = fmaf(c.z, w, C2[k]);
                D[k] = fmaf(b.z, w, D[k]);
                T[k] = Tn;
                last[k] = sm.Pos[q] + 1;
            }
        }
        __syncwarp();
        if (CKPT && next_ck < n_ck && base + B - lo == (uint32_t)(next_ck + 1) * (uint32_t)ck.every)
            store_ck(next_ck++);
    }
}

__device__ __forceinline__ void write_final(const ViewDesc &V, const ViewImages &out, int vi, float *final_T,
                                            int32_t *n_contrib, int px, int py, float T, float C0, float C1,
                                            float C2, float D, int last) {
    if (px < V.W && py < V.H) {
        const size_t HW = (size_t)V.W * V.H;
        const size_t p = (size_t)py * V.W + px;
        out.rgb[vi][p] = C0;
        out.rgb[vi][HW + p] = C1;
        out.rgb[vi][2 * HW + p] = C2;
        out.depth[vi][p] = D;
        out.alpha[vi][p] = 1.f - T;
        final_T[V.pix_base + p] = T;
        n_contrib[V.pix_base + p] = last;
    }
}

// Field of checkpoint group `sub` of a (pixel, chunk) slot; slot_field is the
// chunk's end (the last group), the only one the combine and backward state use.
__device__ __forceinline__ float *slot_group(const ChunkPlan &cp, uint32_t slot, int sub, int field, int tpx) {
    return cp.part + (((size_t)slot * kSub + sub) * kFields + field) * (size_t)tpx;
}
__device__ __forceinline__ float *slot_field(const ChunkPlan &cp, uint32_t slot, int field, int tpx) {
    return slot_group(cp, slot, kSub - 1, field, tpx);
}

__device__ __forceinline__ uint32_t take_item(uint32_t *queue, int lane) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(queue, 1u);
    return __shfl_sync(0xffffffffu, item, 0);
}

// Phase 1: (tile, chunk, block) items.  (Six CTAs per SM: the register cap
// that gives beats the occupancy the unconstrained allocation leaves.)
template <int TW, int TH, int BM>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 6)
composite_fwd_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                     const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs, ViewImages out,
                     float *__restrict__ final_T, int32_t *__restrict__ n_contrib, ChunkPlan cp,
                     uint32_t *__restrict__ queue) {
    using Gm = Geometry<TW, TH>;
    constexpr int B = 32 * BM;
    __shared__ float4 sA[kWarpsPerCta][B], sB[kWarpsPerCta][B], sC[kWarpsPerCta][B];
    __shared__ int sP[kWarpsPerCta][B];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Smem sm{sA[w], sB[w], sC[w], sP[w], nullptr};
    const uint32_t n_items = min(*cp.n_fwd, cp.pair_cap) * Gm::NB;
    const uint32_t wmax = whole_max(cp);
    for (;;) {
        const uint32_t item = take_item(queue, lane);
        if (item >= n_items) break;
        const uint32_t pair = cp.pair_order ? cp.pair_order[item / Gm::NB] : item / Gm::NB;
        const int blk = (int)(item % Gm::NB);
        if (pair >= cp.pair_cap) continue;
        const uint32_t gt = cp.pair_tile[pair];
        if (gt >= vsp->total_tiles) continue; // never written (capacity overflow, latched)
        const uint32_t nch = cp.n_chunks[gt];
        const uint32_t k = pair - cp.chunk_base[gt];
        if (k >= nch) continue;
        const bool whole = whole_list(nch, wmax);
        if (whole && (k != 0 || cp.part_base[gt] + nch > cp.slot_cap)) continue; // (overflow latched)
        const int vi = view_of_tile(*vsp, gt);
        const ViewDesc &V = vsp->v[vi];
        const BlockPix<TW, TH> bp(V, gt - V.tile_base, blk, lane);
        const uint2 rg = ranges[gt];
        float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT];
        int last[PPT];
        bool done[PPT], stopped[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            T[j] = 1.f;
            C0[j] = C1[j] = C2[j] = D[j] = 0.f;
            last[j] = 0;
            done[j] = !(bp.px < V.W && bp.py0 + j < V.H);
            stopped[j] = false;
            // a pixel known to stop in an earlier chunk needs nothing from this one
            if (!done[j] && nch > 1 && !whole) {
                const size_t gp = V.pix_base + (size_t)(bp.py0 + j) * V.W + bp.px;
                if (__ldcg(cp.stop_at + gp) < k) done[j] = true;
            }
        }
        // one chunk, or every chunk of a list walked whole (from the true
        // state: the transmittance runs on, the sums restart per chunk)
        const uint32_t k_end = whole ? nch : k + 1;
        for (uint32_t kk = k; kk < k_end; ++kk) {
            const uint32_t lo = rg.x + kk * (uint32_t)cp.L;
            const uint32_t hi = (nch <= 1 || kk + 1 == nch) ? rg.y : min(rg.y, lo + (uint32_t)cp.L);
            Checkpoints ck{nullptr, cp.L / kSub, Gm::TPX, bp.lp0, TW};
            if (nch > 1 && !whole && cp.part_base[gt] + k < cp.slot_cap)
                ck.g0 = slot_group(cp, cp.part_base[gt] + k, 0, 0, Gm::TPX);
            // (a list walked whole parks the chunk's starting transmittance in
            // the slot field it will fill, rather than in registers)
            if (whole) {
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    slot_field(cp, cp.part_base[gt] + kk, 4, Gm::TPX)[bp.lp0 + j * TW] = T[j];
                    C0[j] = C1[j] = C2[j] = D[j] = 0.f;
                }
            }
            fwd_walk<BM, true, false>(inst_vals, recs, rg.x, lo, hi, (float)bp.px, bp.py0, bp.fx0, bp.fy0, sm, lane,
                                      T, C0, C1, C2, D, last, done, stopped, ck, nullptr);
            if (whole) {
                // the chunk's contribution, the transmittance it removes and the
                // one at its end: the state its backward walk starts from, once
                // the sums of what lies behind are added in (combine_state)
                const uint32_t slot = cp.part_base[gt] + kk;
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const int lp = bp.lp0 + j * TW;
                    slot_field(cp, slot, 0, Gm::TPX)[lp] = C0[j];
                    slot_field(cp, slot, 1, Gm::TPX)[lp] = C1[j];
                    slot_field(cp, slot, 2, Gm::TPX)[lp] = C2[j];
                    slot_field(cp, slot, 3, Gm::TPX)[lp] = D[j];
                    float *f4 = slot_field(cp, slot, 4, Gm::TPX) + lp;
                    *f4 = *f4 - T[j];
                    slot_field(cp, slot, 5, Gm::TPX)[lp] = T[j];
                }
            }
        }
        if (nch > 1 && !whole) {
#pragma unroll
            for (int j = 0; j < PPT; ++j)
                if (stopped[j]) atomicMin(cp.stop_at + V.pix_base + (size_t)(bp.py0 + j) * V.W + bp.px, k);
        }
        if (nch <= 1) {
#pragma unroll
            for (int j = 0; j < PPT; ++j)
                write_final(V, out, vi, final_T, n_contrib, bp.px, bp.py0 + j, T[j], C0[j], C1[j], C2[j], D[j],
                            last[j]);
        } else if (whole) {
            // colour and depth: the chunks' contributions in order (this
            // thread's own stores, read back)
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int lp = bp.lp0 + j * TW;
                float S0 = 0.f, S1 = 0.f, S2 = 0.f, SD = 0.f;
                for (uint32_t kk = 0; kk < nch; ++kk) {
                    const uint32_t slot = cp.part_base[gt] + kk;
                    S0 += slot_field(cp, slot, 0, Gm::TPX)[lp];
                    S1 += slot_field(cp, slot, 1, Gm::TPX)[lp];
                    S2 += slot_field(cp, slot, 2, Gm::TPX)[lp];
                    SD += slot_field(cp, slot, 3, Gm::TPX)[lp];
                }
                write_final(V, out, vi, final_T, n_contrib, bp.px, bp.py0 + j, T[j], S0, S1, S2, SD, last[j]);
            }
        } else {
            const uint32_t slot = cp.part_base[gt] + k;
            if (slot >= cp.slot_cap) continue; // capacity overflow is latched by the planner
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int lp = bp.lp0 + j * TW;
                slot_field(cp, slot, 0, Gm::TPX)[lp] = C0[j];
                slot_field(cp, slot, 1, Gm::TPX)[lp] = C1[j];
                slot_field(cp, slot, 2, Gm::TPX)[lp] = C2[j];
                slot_field(cp, slot, 3, Gm::TPX)[lp] = D[j];
                slot_field(cp, slot, 4, Gm::TPX)[lp] = T[j];
                slot_field(cp, slot, 5, Gm::TPX)[lp] =
                    __int_as_float(last[j] | (stopped[j] ? (int)0x80000000 : 0));
            }
        }
    }
}

// Per-pixel state between the combine kernels (multi-chunk tiles only): stop
// chunk (or -1) and the eighth of it where the walk resumes; transmittance
// and colour / depth at the chunk's start; the state at the resume point.
struct PixState {
    int stop, sub;
    float Tin, C0, C1, C2, D;
    float Tc, Cc0, Cc1, Cc2, Dc;
    int lastc;
    int pad;
};

// Phase 2a: per pixel, combine chunks in order up to the one whose end would
// cross the 1e-4 stop (or whose walk stopped locally).  Pixels that never stop
// are final here.
template <int TW, int TH>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
combine_scan_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges, ViewImages out,
                    float *__restrict__ final_T, int32_t *__restrict__ n_contrib, ChunkPlan cp,
                    PixState *__restrict__ ps, uint32_t total_tiles) {
    using Gm = Geometry<TW, TH>;
    constexpr int TPX = Gm::TPX;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * kWarpsPerCta + w;
    if (item >= total_tiles * Gm::NB) return;
    const uint32_t gt = item / Gm::NB;
    const int blk = (int)(item % Gm::NB);
    const uint32_t nch = cp.n_chunks[gt];
    if (nch <= 1 || whole_list(nch, whole_max(cp))) return; // final after phase 1
    const uint32_t s0 = cp.part_base[gt];
    if (s0 + nch > cp.slot_cap) return; // capacity overflow is latched by the planner
    const int vi = view_of_tile(*vsp, gt);
    const ViewDesc &V = vsp->v[vi];
    const BlockPix<TW, TH> bp(V, gt - V.tile_base, blk, lane);
    // the lane's two pixels are combined together (twice the loads in flight);
    // the six fields of chunk k + 1 are loaded while chunk k is combined
    bool act[PPT];
    float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT], f[PPT][6];
    int last[PPT], stop[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        act[j] = bp.px < V.W && bp.py0 + j < V.H;
        T[j] = 1.f;
        C0[j] = C1[j] = C2[j] = D[j] = 0.f;
        last[j] = 0;
        stop[j] = -1;
#pragma unroll
        for (int q = 0; q < 6; ++q) f[j][q] = act[j] ? slot_field(cp, s0, q, TPX)[bp.lp0 + j * TW] : 0.f;
    }
    for (uint32_t k = 0; k < nch && (act[0] || act[1]); ++k) {
        float g[PPT][6];
#pragma unroll
        for (int j = 0; j < PPT; ++j)
#pragma unroll
            for (int q = 0; q < 6; ++q)
                g[j][q] = (act[j] && k + 1 < nch) ? slot_field(cp, s0 + k + 1, q, TPX)[bp.lp0 + j * TW] : 0.f;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            if (!act[j]) continue;
            const float Tk = f[j][4];
            const int lk = __float_as_int(f[j][5]);
            const float Tn = __fmul_rn(T[j], Tk);
            if ((lk & (int)0x80000000) || Tn < kTMin) {
                stop[j] = (int)k;
                act[j] = false;
                continue;
            }
            C0[j] = fmaf(T[j], f[j][0], C0[j]);
            C1[j] = fmaf(T[j], f[j][1], C1[j]);
            C2[j] = fmaf(T[j], f[j][2], C2[j]);
            D[j] = fmaf(T[j], f[j][3], D[j]);
            T[j] = Tn;
            if (lk) last[j] = lk;
#pragma unroll
            for (int q = 0; q < 6; ++q) f[j][q] = g[j][q];
        }
    }
    // the block's stop chunks, each once, to the list of the exact walks
    {
        int v0 = stop[0], v1 = stop[1];
        for (;;) {
            const int cand = v0 >= 0 ? v0 : v1;
            const uint32_t m = __ballot_sync(0xffffffffu, cand >= 0);
            if (!m) break;
            const int v = __shfl_sync(0xffffffffu, cand, __ffs(m) - 1);
            if (lane == 0) {
                const uint32_t pos = atomicAdd(cp.n_stop, 1u);
                const uint32_t cap = cp.pair_cap * (uint32_t)Gm::NB;
                if (pos < cap) cp.stop_items[pos] = (cp.chunk_base[gt] + (uint32_t)v) * Gm::NB + (uint32_t)blk;
            }
            if (v0 == v) v0 = -1;
            if (v1 == v) v1 = -1;
        }
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int py = bp.py0 + j;
        if (!(bp.px < V.W && py < V.H)) continue;
        const int lp = bp.lp0 + j * TW;
        const size_t gp = V.pix_base + (size_t)py * V.W + bp.px;
        PixState st{stop[j], 0, T[j], C0[j], C1[j], C2[j], D[j], T[j], C0[j], C1[j], C2[j], D[j], last[j], 0};
        if (stop[j] >= 0) {
            // the part of the stop chunk that holds the stop: the first checkpoint
            // whose transmittance is (within 1%) below the limit, or whose local walk
            // had stopped; the walk resumes from the checkpoint before it.  The
            // checkpoints' transmittances and flags are loaded together first.
            const uint2 rg = ranges[gt];
            const int64_t rest = (int64_t)rg.y - (int64_t)rg.x - (int64_t)stop[j] * cp.L;
            const int clen = (int)(rest < cp.L ? rest : cp.L);
            const int every = cp.L / kSub;
            const uint32_t sl = s0 + (uint32_t)stop[j];
            float Tm[kSub - 1];
            int lm[kSub - 1];
#pragma unroll
            for (int m = 0; m < kSub - 1; ++m) {
                const bool written = (m + 1) * every < clen; // else past the chunk's end
                Tm[m] = written ? slot_group(cp, sl, m, 4, TPX)[lp] : 0.f;
                lm[m] = written ? __float_as_int(slot_group(cp, sl, m, 5, TPX)[lp]) : 0;
            }
            int m = 0;
#pragma unroll
            for (int mm = 0; mm < kSub - 1; ++mm) {
                if (m != mm) break;
                if ((mm + 1) * every >= clen) break;
                if ((lm[mm] & (int)0x80000000) || __fmul_rn(T[j], Tm[mm]) < 1.01f * kTMin) break;
                m = mm + 1;
            }
            if (m > 0) {
                // (selected with constant indices, so the arrays stay in registers)
                float tsel = 0.f;
                int lsel = 0;
#pragma unroll
                for (int mm = 0; mm < kSub - 1; ++mm)
                    if (mm == m - 1) {
                        tsel = Tm[mm];
                        lsel = lm[mm];
                    }
                st.Tc = __fmul_rn(T[j], tsel);
                st.Cc0 = fmaf(T[j], slot_group(cp, sl, m - 1, 0, TPX)[lp], C0[j]);
                st.Cc1 = fmaf(T[j], slot_group(cp, sl, m - 1, 1, TPX)[lp], C1[j]);
                st.Cc2 = fmaf(T[j], slot_group(cp, sl, m - 1, 2, TPX)[lp], C2[j]);
                st.Dc = fmaf(T[j], slot_group(cp, sl, m - 1, 3, TPX)[lp], D[j]);
                if (lsel) st.lastc = lsel;
            }
            st.sub = m;
        }
        ps[gp] = st;
        if (stop[j] < 0) write_final(V, out, vi, final_T, n_contrib, bp.px, py, T[j], C0[j], C1[j], C2[j], D[j], last[j]);
    }
}

// Phase 2b: exact walk of each stop chunk from the true transmittance, one
// (tile, chunk, block) item per warp, for the pixels that stop in that chunk.
// Writes their final values and the chunk's contribution (backward state).
// The items are the ones phase 2a listed (a block with a pixel stopping in
// that chunk), so no warp visits a chunk only to find nothing to do.
template <int TW, int TH, int BM>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 6)
combine_walk_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                    const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs, ViewImages out,
                    float *__restrict__ final_T, int32_t *__restrict__ n_contrib, ChunkPlan cp,
                    const PixState *__restrict__ ps, uint32_t *__restrict__ queue) {
    using Gm = Geometry<TW, TH>;
    constexpr int B = 32 * BM;
    constexpr int TPX = Gm::TPX;
    __shared__ float4 sA[kWarpsPerCta][B], sB[kWarpsPerCta][B], sC[kWarpsPerCta][B];
    __shared__ int sP[kWarpsPerCta][B];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Smem sm{sA[w], sB[w], sC[w], sP[w], nullptr};
    const uint32_t n_items = min(*cp.n_stop, cp.pair_cap * (uint32_t)Gm::NB);
    for (;;) {
        const uint32_t idx = take_item(queue, lane);
        if (idx >= n_items) break;
        const uint32_t item = cp.stop_items[idx];
        const uint32_t pair = item / Gm::NB;
        const int blk = (int)(item % Gm::NB);
        if (pair >= cp.pair_cap) continue;
        const uint32_t gt = cp.pair_tile[pair];
        if (gt >= vsp->total_tiles) continue;
        const uint32_t nch = cp.n_chunks[gt];
        const uint32_t k = pair - cp.chunk_base[gt];
        if (nch <= 1 || k >= nch || cp.part_base[gt] + nch > cp.slot_cap) continue;
        const int vi = view_of_tile(*vsp, gt);
        const ViewDesc &V = vsp->v[vi];
        const BlockPix<TW, TH> bp(V, gt - V.tile_base, blk, lane);
        float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT], Tin[PPT], b0[PPT], b1[PPT], b2[PPT], bd[PPT];
        int last[PPT], start[PPT];
        bool done[PPT], stopped[PPT];
        bool any = false;
        int first = 0x7fffffff; // earliest resume position of the lane's pixels (list-relative)
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            done[j] = true;
            stopped[j] = false;
            T[j] = Tin[j] = 1.f;
            C0[j] = C1[j] = C2[j] = D[j] = 0.f;
            b0[j] = b1[j] = b2[j] = bd[j] = 0.f;
            last[j] = 0;
            start[j] = 0;
            const int py = bp.py0 + j;
            if (bp.px < V.W && py < V.H) {
                const PixState st = ps[V.pix_base + (size_t)py * V.W + bp.px];
                if (st.stop == (int)k) {
                    done[j] = false;
                    any = true;
                    Tin[j] = st.Tin;
                    b0[j] = st.C0;
                    b1[j] = st.C1;
                    b2[j] = st.C2;
                    bd[j] = st.D;
                    T[j] = st.Tc;
                    C0[j] = st.Cc0;
                    C1[j] = st.Cc1;
                    C2[j] = st.Cc2;
                    D[j] = st.Dc;
                    last[j] = st.lastc;
                    start[j] = (int)(k * (uint32_t)cp.L) + st.sub * (cp.L / kSub);
                    first = min(first, start[j]);
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        first = __reduce_min_sync(0xffffffffu, first);
        const uint2 rg = ranges[gt];
        const uint32_t lo = rg.x + (uint32_t)first;
        const uint32_t hi = min(rg.y, rg.x + k * (uint32_t)cp.L + (uint32_t)cp.L);
        const Checkpoints no_ck{nullptr, 1, Gm::TPX, 0, TW};
        fwd_walk<BM, false, true>(inst_vals, recs, rg.x, lo, hi, (float)bp.px, bp.py0, bp.fx0, bp.fy0, sm, lane, T, C0,
                                  C1, C2, D, last, done, stopped, no_ck, start);
        const uint32_t slot = cp.part_base[gt] + k;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int py = bp.py0 + j;
            if (!(bp.px < V.W && py < V.H)) continue;
            if (ps[V.pix_base + (size_t)py * V.W + bp.px].stop != (int)k) continue;
            write_final(V, out, vi, final_T, n_contrib, bp.px, py, T[j], C0[j], C1[j], C2[j], D[j], last[j]);
            const int lp = bp.lp0 + j * TW;
            slot_field(cp, slot, 0, TPX)[lp] = C0[j] - b0[j];
            slot_field(cp, slot, 1, TPX)[lp] = C1[j] - b1[j];
            slot_field(cp, slot, 2, TPX)[lp] = C2[j] - b2[j];
            slot_field(cp, slot, 3, TPX)[lp] = D[j] - bd[j];
            slot_field(cp, slot, 4, TPX)[lp] = Tin[j] - T[j];
            slot_field(cp, slot, 5, TPX)[lp] = T[j];
        }
    }
}

// Phase 2c: per chunk, the transmittance at its end and the normalised sums of
// everything composited after it: the state the backward walk of the chunk
// starts from.  All summed terms are non-negative (no cancellation).
template <int TW, int TH>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
combine_state_kernel(const ViewSet *__restrict__ vsp, ChunkPlan cp, const PixState *__restrict__ ps,
                     uint32_t total_tiles) {
    using Gm = Geometry<TW, TH>;
    constexpr int TPX = Gm::TPX;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * kWarpsPerCta + w;
    if (item >= total_tiles * Gm::NB) return;
    const uint32_t gt = item / Gm::NB;
    const int blk = (int)(item % Gm::NB);
    const uint32_t nch = cp.n_chunks[gt];
    if (nch <= 1) return;
    // a list walked whole left every chunk's slot in the form pass 2 reads
    const bool whole = whole_list(nch, whole_max(cp));
    const uint32_t s0 = cp.part_base[gt];
    if (s0 + nch > cp.slot_cap) return;
    const int vi = view_of_tile(*vsp, gt);
    const ViewDesc &V = vsp->v[vi];
    const BlockPix<TW, TH> bp(V, gt - V.tile_base, blk, lane);
    // Each slot before the stop chunk becomes (its contribution, T at its end);
    // the stop chunk's slot was written by the exact walk.  Then, from the last
    // chunk back, every slot gets the normalised sums of what lies after it.
    // The lane's two pixels run together, and both loops load the next chunk's
    // fields while handling the current one.
    bool in[PPT];
    int lp[PPT];
    uint32_t top[PPT], n_fwd[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int py = bp.py0 + j;
        in[j] = bp.px < V.W && py < V.H;
        lp[j] = bp.lp0 + j * TW;
        const int stop = (in[j] && !whole) ? ps[V.pix_base + (size_t)py * V.W + bp.px].stop : -1;
        top[j] = stop >= 0 ? (uint32_t)stop : nch - 1;
        n_fwd[j] = (!in[j] || whole) ? 0u : (stop < 0 ? top[j] + 1 : top[j]);
    }
    {
        float t[PPT] = {1.f, 1.f}, h[PPT][5];
#pragma unroll
        for (int j = 0; j < PPT; ++j)
#pragma unroll
            for (int q = 0; q < 5; ++q) h[j][q] = n_fwd[j] > 0 ? slot_field(cp, s0, q, TPX)[lp[j]] : 0.f;
        const uint32_t n_max = max(n_fwd[0], n_fwd[1]);
        for (uint32_t k = 0; k < n_max; ++k) {
            float nx[PPT][5];
#pragma unroll
            for (int j = 0; j < PPT; ++j)
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    nx[j][q] = k + 1 < n_fwd[j] ? slot_field(cp, s0 + k + 1, q, TPX)[lp[j]] : 0.f;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                if (k >= n_fwd[j]) continue;
                const float tend = __fmul_rn(t[j], h[j][4]);
#pragma unroll
                for (int q = 0; q < 4; ++q) slot_field(cp, s0 + k, q, TPX)[lp[j]] = h[j][q] * t[j];
                slot_field(cp, s0 + k, 4, TPX)[lp[j]] = t[j] - tend;
                slot_field(cp, s0 + k, 5, TPX)[lp[j]] = tend;
                t[j] = tend;
#pragma unroll
                for (int q = 0; q < 5; ++q) h[j][q] = nx[j][q];
            }
        }
    }
    {
        float acc[PPT][5], h[PPT][6];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[j][q] = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) h[j][q] = in[j] ? slot_field(cp, s0 + top[j], q, TPX)[lp[j]] : 0.f;
        }
        // k runs from the larger top down; pixel j joins at its own top
        for (int k = (int)max(top[0], top[1]); k >= 0; --k) {
            float nx[PPT][6];
#pragma unroll
            for (int j = 0; j < PPT; ++j)
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    nx[j][q] = (in[j] && k > 0 && k <= (int)top[j]) ? slot_field(cp, s0 + k - 1, q, TPX)[lp[j]] : 0.f;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                if (!in[j] || k > (int)top[j]) continue;
                const float tend = h[j][5];
                const float inv = tend > 0.f ? 1.f / tend : 0.f;
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    slot_field(cp, s0 + k, q, TPX)[lp[j]] = acc[j][q] * inv;
                    acc[j][q] += h[j][q];
                }
#pragma unroll
                for (int q = 0; q < 6; ++q) h[j][q] = nx[j][q];
            }
        }
    }
}

// Reduce-scatter of 10 per-lane values over the warp with 12 shuffles.  On
// return, lane L holds the warp total of value index idx(L) when valid(L):
// idx = 5*b4 + (3*b3 + 2*b2 + b1) over the lane bits, valid for b0 = 0 and
// (b3 = 0: b2 b1 in {00, 01, 10}; b3 = 1: b2 b1 in {00, 01}).
__device__ __forceinline__ float reduce_scatter10(const float v[10], int lane, int &idx, bool &valid) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float u[6];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float keep = b4 ? v[5 + i] : v[i];
        const float send = b4 ? v[i] : v[5 + i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    u[5] = 0.f;
    float w[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float keep = b3 ? u[3 + i] : u[i];
        const float send = b3 ? u[i] : u[3 + i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    w[3] = 0.f;
    float x[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b2 ? w[2 + i] : w[i];
        const float send = b2 ? w[i] : w[2 + i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const float keep = b1 ? x[1] : x[0];
    const float send = b1 ? x[0] : x[1];
    float y = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    const int pos = (b3 ? 3 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
    idx = (b4 ? 5 : 0) + pos;
    valid = !(lane & 1) && (b3 ? pos <= 4 : pos <= 2);
    return y;
}

// float offset in GGrad of reduced value index: five moments, dop, dr dg db, dz
__device__ __forceinline__ int grad_offset(int idx) { return idx < 6 ? idx : (idx < 9 ? idx + 2 : 6); }

template <int TW, int TH, int BM>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 6)
composite_bwd_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                     const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs, ViewGrads G,
                     const float *__restrict__ final_T, const int32_t *__restrict__ n_contrib,
                     GGrad *__restrict__ g2d, ChunkPlan cp, uint32_t *__restrict__ queue) {
    using Gm = Geometry<TW, TH>;
    constexpr int B = 32 * BM;
    constexpr int NACC = 10;
    __shared__ float4 sA[kWarpsPerCta][B], sB[kWarpsPerCta][B], sC[kWarpsPerCta][B];
    __shared__ int sP[kWarpsPerCta][B];
    __shared__ uint32_t sI[kWarpsPerCta][B];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Smem sm{sA[w], sB[w], sC[w], sP[w], sI[w]};
    const uint32_t n_items = min(*cp.n_pairs, cp.pair_cap) * Gm::NB;
    for (;;) {
        const uint32_t item = take_item(queue, lane);
        if (item >= n_items) break;
        const uint32_t pair = cp.pair_order ? cp.pair_order[item / Gm::NB] : item / Gm::NB;
        const int blk = (int)(item % Gm::NB);
        if (pair >= cp.pair_cap) continue;
        const uint32_t gt = cp.pair_tile[pair];
        if (gt >= vsp->total_tiles) continue; // never written (capacity overflow, latched)
        const uint32_t nch = cp.n_chunks[gt];
        const uint32_t k = pair - cp.chunk_base[gt];
        if (k >= nch || (nch > 1 && cp.part_base[gt] + k >= cp.slot_cap)) continue;
        const int vi = view_of_tile(*vsp, gt);
        const ViewDesc &V = vsp->v[vi];
        const BlockPix<TW, TH> bp(V, gt - V.tile_base, blk, lane);
        const uint2 rg = ranges[gt];
        const size_t HW = (size_t)V.W * V.H;
        const float fpx = (float)bp.px;

        // Per pixel: T, the upstream gradients, and Q = sum over the colour, depth
        // and visibility channels x of g_x S_x, where S_x is the normalised sum of
        // what is composited behind the current Gaussian.  dL/dalpha_i only ever
        // needs that dot product, so one running scalar replaces the five sums:
        // dL/dalpha_i = T_i (cg_i - Q), Q <- alpha_i cg_i + (1 - alpha_i) Q, with
        // cg_i = c_i . g_C + z_i g_D + g_V.
        float T[PPT], gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], gA[PPT], Q[PPT];
        int last[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int py = bp.py0 + j;
            T[j] = 1.f;
            gC0[j] = gC1[j] = gC2[j] = gD[j] = gA[j] = Q[j] = 0.f;
            last[j] = 0;
            if (bp.px < V.W && py < V.H) {
                const size_t p = (size_t)py * V.W + bp.px;
                last[j] = n_contrib[V.pix_base + p];
                gC0[j] = G.d_rgb[vi][p];
                gC1[j] = G.d_rgb[vi][HW + p];
                gC2[j] = G.d_rgb[vi][2 * HW + p];
                gD[j] = G.d_depth[vi] ? G.d_depth[vi][p] : 0.f;
                gA[j] = G.d_alpha[vi] ? G.d_alpha[vi][p] : 0.f;
                if (nch <= 1) {
                    T[j] = final_T[V.pix_base + p];
                } else if (k * (uint32_t)cp.L < (uint32_t)last[j]) {
                    const uint32_t slot = cp.part_base[gt] + k;
                    const int lp = bp.lp0 + j * TW;
                    Q[j] = slot_field(cp, slot, 0, Gm::TPX)[lp] * gC0[j] + slot_field(cp, slot, 1, Gm::TPX)[lp] * gC1[j] +
                           slot_field(cp, slot, 2, Gm::TPX)[lp] * gC2[j] + slot_field(cp, slot, 3, Gm::TPX)[lp] * gD[j] +
                           slot_field(cp, slot, 4, Gm::TPX)[lp] * gA[j];
                    T[j] = slot_field(cp, slot, 5, Gm::TPX)[lp];
                }
            }
        }
        const int warp_last = __reduce_max_sync(0xffffffffu, max(last[0], last[1]));
        const uint32_t lo_chunk = rg.x + k * (uint32_t)cp.L;
        const uint32_t end = min(nch <= 1 ? rg.y : min(rg.y, lo_chunk + (uint32_t)cp.L), rg.x + (uint32_t)warp_last);

        for (uint32_t hi = end; hi > lo_chunk;) {
            const uint32_t lo = hi - lo_chunk > (uint32_t)B ? hi - B : lo_chunk;
            const int n = gather_cull<BM, true>(inst_vals, recs, rg.x, lo, hi, bp.fx0, bp.fy0, sm, lane);
            for (int q = n - 1; q >= 0; --q) {
                const float4 a = sm.A[q];
                const float4 b = sm.B[q];
                const int pos = sm.Pos[q];
                const float dx = a.x - fpx;
                const float a2dx = __fmul_rn(a.z, dx);
                // the 1/255 tests of both pixels first: a Gaussian that no pixel
                // of the block takes costs the warp nothing more
                float e2[PPT];
                bool take[PPT];
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const float dy = a.y - (float)(bp.py0 + j);
                    e2[j] = gauss_exponent2(a2dx, a.w, b.x, b.y, dx, dy); // log2(o G), as forward
                    take[j] = pos < last[j] && e2[j] >= kLog2AlphaMin;
                }
                if (!__any_sync(0xffffffffu, take[0] || take[1])) continue;
                const float4 c = sm.C[q];
                // v: sums over the lane's pixels of dp dx, dp dy, dp dx^2, dp dx dy,
                // dp dy^2 (dp = dL/dpower), o dL/do, and w g_R, w g_G, w g_B, w g_D;
                // the conic is applied per Gaussian in the chain rule that follows
                float v[NACC];
#pragma unroll
                for (int m = 0; m < NACC; ++m) v[m] = 0.f;
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    if (!take[j]) continue;
                    const float dy = a.y - (float)(bp.py0 + j);
                    const float oG = exp2_approx(e2[j]);
                    const float alpha = fminf(kAlphaMax, oG);
                    T[j] = __fdividef(T[j], 1.f - alpha);
                    const float wgt = alpha * T[j];
                    const float cg = fmaf(c.x, gC0[j], fmaf(c.y, gC1[j], fmaf(c.z, gC2[j], fmaf(b.z, gD[j], gA[j]))));
                    const float dLda = T[j] * (cg - Q[j]);
                    Q[j] = fmaf(alpha, cg - Q[j], Q[j]);
                    v[6] = fmaf(wgt, gC0[j], v[6]);
                    v[7] = fmaf(wgt, gC1[j], v[7]);
                    v[8] = fmaf(wgt, gC2[j], v[8]);
                    v[9] = fmaf(wgt, gD[j], v[9]);
                    if (oG < kAlphaMax) {
                        const float dp = dLda * alpha;
                        const float dpx = dp * dx, dpy = dp * dy;
                        v[5] = fmaf(dLda, oG, v[5]); // o dL/do
                        v[0] += dpx;
                        v[1] += dpy;
                        v[2] = fmaf(dpx, dx, v[2]);
                        v[3] = fmaf(dpx, dy, v[3]);
                        v[4] = fmaf(dpy, dy, v[4]);
                    }
                }
                int vidx;
                bool valid;
                const float tot = reduce_scatter10(v, lane, vidx, valid);
                if (valid && tot != 0.f) atomicAdd((float *)(g2d + sm.Idx[q]) + grad_offset(vidx), tot);
            }
            __syncwarp();
            hi = lo;
        }
    }
}

// List-parallel plan: per tile the number of chunks (an empty tile still has
// one; a list of up to 1.5 L entries stays one chunk: the combine of two
// chunks costs more than the longer item), its first pair and, for a multi-chunk tile, its first slot (exclusive
// scans over the tiles), the tile of every pair, and the forward work order:
// pairs by chunk index, all first chunks (in tile order), then all second
// chunks, ... (chunks from the 255th on share the last bucket).  Within a
// later bucket the order is that of arrival, which only schedules work: no
// result depends on it.
//
// Two launches over the tiles, one thread per tile.  The first counts and
// publishes per-block sums and bucket counts; the block that finishes last (a
// ticket taken after a fence, no waiting) turns them into block bases and
// bucket start positions.  The second places every pair.
//
// aux (zeroed before the first launch): [0, 256) bucket counts, then start
// positions, then cursors; [256] the ticket; from 257 two words per block:
// the block's sums, then its bases.
constexpr int kPlanThreads = 256;
constexpr uint32_t kOrderBuckets = 256;
constexpr int kAuxTicket = 256, kAuxBlocks = 257;

// Exclusive scan of two values over a kPlanThreads block: prefixes returned in
// a, b; block totals in ta, tb (every thread).
__device__ __forceinline__ void block_scan2(uint32_t &a, uint32_t &b, uint32_t &ta, uint32_t &tb) {
    __shared__ uint32_t sa[kPlanThreads / 32], sb[kPlanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ya;
            ib += yb;
        }
    }
    if (lane == 31) {
        sa[wid] = ia;
        sb[wid] = ib;
    }
    __syncthreads();
    uint32_t wa = 0, wb = 0;
    ta = tb = 0;
#pragma unroll
    for (int j = 0; j < kPlanThreads / 32; ++j) {
        if (j < wid) {
            wa += sa[j];
            wb += sb[j];
        }
        ta += sa[j];
        tb += sb[j];
    }
    __syncthreads(); // sa, sb reusable
    a = wa + ia - a;
    b = wb + ib - b;
}

// In the last block: exclusive scan of the 256 bucket counts in aux, in
// place (written by other blocks' atomics: read from L2); *total (if given)
// receives their sum.
__device__ __forceinline__ void bucket_starts(uint32_t *aux, uint32_t *total = nullptr) {
    __shared__ uint32_t sv[kOrderBuckets];
    for (uint32_t i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) sv[i] = __ldcg(aux + i);
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        constexpr int per = kOrderBuckets / 32;
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < per; ++j) sum += sv[lane * per + j];
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int j = 0; j < per; ++j) {
            const uint32_t v = sv[lane * per + j];
            aux[lane * per + j] = run;
            run += v;
        }
        if (total && lane == 31) *total = inc;
    }
}

// True in every thread of the block that finished last (after its own
// published results); the other blocks' writes are then visible to it.
__device__ __forceinline__ bool last_block(uint32_t *ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__global__ void __launch_bounds__(kPlanThreads)
plan_count_kernel(const uint2 *__restrict__ ranges, uint32_t n_tiles, uint32_t L, uint32_t *__restrict__ n_chunks,
                  uint32_t *__restrict__ aux, uint32_t *__restrict__ counters, ChunkPlan cp) {
    __shared__ uint32_t hist[kOrderBuckets];
    const int tid = threadIdx.x;
    const uint32_t wmax = whole_max(cp);
    for (uint32_t i = tid; i < kOrderBuckets; i += kPlanThreads) hist[i] = 0;
    __syncthreads();
    const uint32_t t = blockIdx.x * kPlanThreads + tid;
    uint32_t c = 0;
    if (t < n_tiles) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x;
        c = len > L + L / 2 ? (len + L - 1) / L : 1u; // up to 1.5 chunks stay one item
        n_chunks[t] = c;
        // forward order: bucket 0 the lists one warp walks whole (the longest
        // items, first), 1 the first chunks of the others, k + 1 the k-th later
        // chunks of the lists walked chunk-parallel
        if (whole_list(c, wmax)) {
            atomicAdd(&hist[0], 1u);
        } else {
            atomicAdd(&hist[1], 1u);
            const uint32_t kc = min(c, kOrderBuckets - 2);
            for (uint32_t k = 1; k < kc; ++k) atomicAdd(&hist[k + 1], 1u);
            if (c > kc) atomicAdd(&hist[kOrderBuckets - 1], c - kc);
        }
    }
    uint32_t a = c, b = c > 1 ? c : 0u, ta, tb;
    block_scan2(a, b, ta, tb); // (synchronises: hist is complete)
    for (uint32_t i = tid; i < kOrderBuckets; i += kPlanThreads)
        if (hist[i]) atomicAdd(aux + i, hist[i]);
    if (tid == 0) {
        aux[kAuxBlocks + 2 * blockIdx.x] = ta;
        aux[kAuxBlocks + 2 * blockIdx.x + 1] = tb;
    }
    if (!last_block(aux + kAuxTicket)) return;
    // block bases (exclusive scan of the block sums), in chunks of the block size
    uint32_t carry_a = 0, carry_b = 0;
    for (uint32_t b0 = 0; b0 < gridDim.x; b0 += kPlanThreads) {
        const uint32_t j = b0 + tid;
        uint32_t sa = 0, sb = 0;
        if (j < gridDim.x) {
            sa = __ldcg(aux + kAuxBlocks + 2 * j);
            sb = __ldcg(aux + kAuxBlocks + 2 * j + 1);
        }
        uint32_t ea = sa, eb = sb, tot_a, tot_b;
        block_scan2(ea, eb, tot_a, tot_b);
        if (j < gridDim.x) {
            aux[kAuxBlocks + 2 * j] = carry_a + ea;
            aux[kAuxBlocks + 2 * j + 1] = carry_b + eb;
        }
        carry_a += tot_a;
        carry_b += tot_b;
    }
    if (tid == 0) {
        counters[4] = carry_a; // pairs
        counters[5] = carry_b; // slots
    }
    __syncthreads();
    bucket_starts(aux, counters + 7); // the forward's items (pairs in its order)
}

__global__ void __launch_bounds__(kPlanThreads)
plan_place_kernel(uint32_t n_tiles, const uint32_t *__restrict__ n_chunks, uint32_t *__restrict__ chunk_base,
                  uint32_t *__restrict__ part_base, uint32_t *__restrict__ pair_tile, uint32_t pair_cap,
                  uint32_t slot_cap, uint32_t *__restrict__ order, uint32_t *__restrict__ aux, uint32_t *status,
                  ChunkPlan cp) {
    const uint32_t t = blockIdx.x * kPlanThreads + threadIdx.x;
    const uint32_t c = t < n_tiles ? n_chunks[t] : 0u;
    uint32_t cb = c, pb = c > 1 ? c : 0u, ta, tb;
    block_scan2(cb, pb, ta, tb);
    bool ok = t < n_tiles;
    if (ok) {
        cb += aux[kAuxBlocks + 2 * blockIdx.x];
        pb += aux[kAuxBlocks + 2 * blockIdx.x + 1];
        chunk_base[t] = cb;
        part_base[t] = pb;
        if (c > 1 && pb + c > slot_cap) atomicOr(status, kStatusCapacity);
        if (cb + c > pair_cap) {
            atomicOr(status, kStatusCapacity);
            ok = false;
        }
    }
    if (ok)
        for (uint32_t k = 0; k < c; ++k) pair_tile[cb + k] = t;
    // one atomic per warp and bucket (the lanes of one bucket take consecutive
    // positions): first chunks by whether the list is walked whole, then the
    // later chunks of the chunk-parallel lists by index
    const bool whole = ok && whole_list(c, whole_max(cp));
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (uint32_t b = 0; b < 2; ++b) {
        const bool mine = ok && (b == 0 ? whole : !whole);
        const uint32_t m = __ballot_sync(0xffffffffu, mine);
        if (!m) continue;
        uint32_t base = 0;
        if (lane == (uint32_t)(__ffs(m) - 1)) base = atomicAdd(aux + b, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (mine) {
            const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
            if (pos < pair_cap) order[pos] = cb;
        }
    }
    const uint32_t kc = (ok && !whole) ? c : 0u;
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, kc);
    for (uint32_t k = 1; k < kmax; ++k) {
        const uint32_t m = __ballot_sync(0xffffffffu, k < kc);
        uint32_t base = 0;
        if (lane == (uint32_t)(__ffs(m) - 1))
            base = atomicAdd(aux + min(k + 1, kOrderBuckets - 1), (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (k < kc) {
            const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
            if (pos < pair_cap) order[pos] = cb + k;
        }
    }
}

// Backward work order from the 8-bit keys: pos = next free position of the
// pair's bucket (start positions in aux from the keys kernel).
__global__ void bucket_place_kernel(const uint32_t *__restrict__ keys, const uint32_t *n_dev, uint32_t cap,
                                    uint32_t *__restrict__ aux, uint32_t *__restrict__ order) {
    const uint32_t n = min(*n_dev, cap);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    // whole warps iterate (the ones past n idle), so the lanes with one key
    // take consecutive positions with one atomic
    for (uint32_t p0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); p0 < n; p0 += stride) {
        const uint32_t p = p0 + lane;
        const uint32_t key = p < n ? (keys[p] & (kOrderBuckets - 1)) : kOrderBuckets;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int lead = __ffs(peers) - 1;
        uint32_t base = 0;
        if (key < kOrderBuckets && (int)lane == lead) base = atomicAdd(aux + key, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, lead);
        if (key < kOrderBuckets) {
            const uint32_t pos = base + __popc(peers & ((1u << lane) - 1u));
            if (pos < n) order[pos] = p;
        }
    }
}

// Backward work order: (tile, chunk) pairs by decreasing expected walk, the
// part of the chunk before the tile's furthest last contributor; the longest
// items start first, which keeps the tail of the persistent kernel short.
// One warp per pair; key = (L - walk) scaled to 0..254 (0 first), 255 for
// pairs of no tile: 8 bits, one bucket pass.
template <int TW, int TH>
__global__ void bwd_pair_keys_kernel(const ViewSet *__restrict__ vsp, ChunkPlan cp,
                                     const int32_t *__restrict__ n_contrib, uint32_t *__restrict__ keys,
                                     uint32_t *__restrict__ aux) {
    using Gm = Geometry<TW, TH>;
    __shared__ uint32_t hist[kOrderBuckets];
    for (uint32_t i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint32_t n = min(*cp.n_pairs, cp.pair_cap);
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nw) {
        const uint32_t t = cp.pair_tile[p];
        uint32_t key = 255u;
        if (t < vsp->total_tiles) {
            const uint32_t k = p - cp.chunk_base[t];
            const ViewDesc &V = vsp->v[view_of_tile(*vsp, t)];
            const uint32_t lt = t - V.tile_base;
            const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
            int mx = 0;
            for (int i = lane; i < Gm::TPX; i += 32) {
                const int px = tx * TW + i % TW, py = ty * TH + i / TW;
                if (px < V.W && py < V.H) mx = max(mx, n_contrib[V.pix_base + (size_t)py * V.W + px]);
            }
            mx = __reduce_max_sync(0xffffffffu, mx);
            const int64_t walk = (int64_t)mx - (int64_t)k * cp.L;
            const uint32_t rest = (uint32_t)cp.L - (uint32_t)(walk < 0 ? 0 : (walk > cp.L ? cp.L : walk));
            key = (uint32_t)(((uint64_t)rest * 254u) / (uint32_t)cp.L);
        }
        if (lane == 0) {
            keys[p] = key;
            atomicAdd(&hist[key], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
        if (hist[i]) atomicAdd(aux + i, hist[i]);
    if (last_block(aux + kAuxTicket)) bucket_starts(aux);
}

template <typename K>
unsigned persistent_grid(K kernel, uint64_t max_items) {
    const int sms = device_sm_count();
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarpsPerCta * 32, 0);
    if (per_sm < 1) per_sm = 1;
    const uint64_t want = (uint64_t)sms * per_sm;
    const uint64_t need = (max_items + kWarpsPerCta - 1) / kWarpsPerCta;
    return (unsigned)(want < need ? want : (need > 0 ? need : 1));
}

template <int TW, int TH, int BM>
void fwd_launch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib, const ChunkPlan &cp,
                uint32_t *queue, void *pix_state, int part, cudaStream_t s) {
    using Gm = Geometry<TW, TH>;
    PixState *ps = (PixState *)pix_state;
    const uint64_t max_items = (uint64_t)cp.pair_cap * Gm::NB;
    const uint64_t tw = (uint64_t)vs.total_tiles * Gm::NB;
    const unsigned grid_tiles = (unsigned)((tw + kWarpsPerCta - 1) / kWarpsPerCta);
    if (part & kFwdWalk) {
        cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
        composite_fwd_kernel<TW, TH, BM><<<persistent_grid(composite_fwd_kernel<TW, TH, BM>, max_items),
                                           kWarpsPerCta * 32, 0, s>>>(vsd, ranges, inst_vals, recs, out, final_T,
                                                                      n_contrib, cp, queue);
    }
    if (part & kFwdCombine) {
        cudaMemsetAsync(cp.n_stop, 0, sizeof(uint32_t), s);
        combine_scan_kernel<TW, TH><<<grid_tiles, kWarpsPerCta * 32, 0, s>>>(vsd, ranges, out, final_T, n_contrib, cp,
                                                                            ps, vs.total_tiles);
        cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
        combine_walk_kernel<TW, TH, BM><<<persistent_grid(combine_walk_kernel<TW, TH, BM>, max_items),
                                          kWarpsPerCta * 32, 0, s>>>(vsd, ranges, inst_vals, recs, out, final_T,
                                                                     n_contrib, cp, ps, queue);
    }
    if (part & kFwdBackwardState)
        combine_state_kernel<TW, TH><<<grid_tiles, kWarpsPerCta * 32, 0, s>>>(vsd, cp, ps, vs.total_tiles);
}

template <int TW, int TH, int BM>
void bwd_launch(const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals, const GRec *recs,
                const ViewGrads &g, const float *final_T, const int32_t *n_contrib, GGrad *g2d, const ChunkPlan &cp,
                uint32_t *queue, cudaStream_t s) {
    using Gm = Geometry<TW, TH>;
    cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
    const uint64_t max_items = (uint64_t)cp.pair_cap * Gm::NB;
    composite_bwd_kernel<TW, TH, BM><<<persistent_grid(composite_bwd_kernel<TW, TH, BM>, max_items),
                                       kWarpsPerCta * 32, 0, s>>>(vsd, ranges, inst_vals, recs, g, final_T,
                                                                  n_contrib, g2d, cp, queue);
}

template <int BM>
void fwd_dispatch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                  const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib, const ChunkPlan &cp,
                  uint32_t *queue, void *pix_state, int part, cudaStream_t s) {
    if (vs.tile_w == 16 && vs.tile_h == 16)
        fwd_launch<16, 16, BM>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, cp, queue, pix_state, part, s);
    else if (vs.tile_w == 8 && vs.tile_h == 8)
        fwd_launch<8, 8, BM>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, cp, queue, pix_state, part, s);
    else if (vs.tile_w == 32 && vs.tile_h == 16)
        fwd_launch<32, 16, BM>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, cp, queue, pix_state, part, s);
}

template <int BM>
void bwd_dispatch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                  const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib, GGrad *g2d,
                  const ChunkPlan &cp, uint32_t *queue, cudaStream_t s) {
    if (vs.tile_w == 16 && vs.tile_h == 16)
        bwd_launch<16, 16, BM>(vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, cp, queue, s);
    else if (vs.tile_w == 8 && vs.tile_h == 8)
        bwd_launch<8, 8, BM>(vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, cp, queue, s);
    else if (vs.tile_w == 32 && vs.tile_h == 16)
        bwd_launch<32, 16, BM>(vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, cp, queue, s);
}

} // namespace

size_t plan_aux_bytes(uint32_t n_tiles) {
    return sizeof(uint32_t) * (kAuxBlocks + 2 * (size_t)((n_tiles + kPlanThreads - 1) / kPlanThreads));
}

void launch_plan(const ChunkPlan &cp, const uint2 *ranges, uint32_t n_tiles, uint32_t *counters, uint32_t *order,
                 uint32_t *aux, uint32_t *status, cudaStream_t s) {
    if (n_tiles == 0) {
        cudaMemsetAsync(counters + 4, 0, 2 * sizeof(uint32_t), s);
        cudaMemsetAsync(counters + 7, 0, sizeof(uint32_t), s);
        return;
    }
    const unsigned nb = (n_tiles + kPlanThreads - 1) / kPlanThreads;
    cudaMemsetAsync(aux, 0, sizeof(uint32_t) * kAuxBlocks, s);
    plan_count_kernel<<<nb, kPlanThreads, 0, s>>>(ranges, n_tiles, (uint32_t)cp.L, (uint32_t *)cp.n_chunks, aux,
                                                  counters, cp);
    plan_place_kernel<<<nb, kPlanThreads, 0, s>>>(n_tiles, cp.n_chunks, (uint32_t *)cp.chunk_base,
                                                  (uint32_t *)cp.part_base, (uint32_t *)cp.pair_tile, cp.pair_cap,
                                                  cp.slot_cap, order, aux, status, cp);
}

void launch_bucket_place(const uint32_t *keys, const uint32_t *n_dev, uint32_t cap, uint32_t *aux, uint32_t *order,
                         cudaStream_t s) {
    if (cap == 0) return;
    int blocks = (int)((cap + 255) / 256);
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    bucket_place_kernel<<<blocks, 256, 0, s>>>(keys, n_dev, cap, aux, order);
}

void launch_bwd_pair_keys(const ViewSet &vs, const ViewSet *vsd, const ChunkPlan &cp, const int32_t *n_contrib,
                          uint32_t *keys, uint32_t *aux, cudaStream_t s) {
    if (cp.pair_cap == 0) return;
    cudaMemsetAsync(aux, 0, sizeof(uint32_t) * kAuxBlocks, s);
    uint64_t blocks = ((uint64_t)cp.pair_cap * 32 + 255) / 256;
    if (blocks > (uint64_t)device_sm_count() * 16) blocks = (uint64_t)device_sm_count() * 16;
    if (vs.tile_w == 16 && vs.tile_h == 16)
        bwd_pair_keys_kernel<16, 16><<<(unsigned)blocks, 256, 0, s>>>(vsd, cp, n_contrib, keys, aux);
    else if (vs.tile_w == 8 && vs.tile_h == 8)
        bwd_pair_keys_kernel<8, 8><<<(unsigned)blocks, 256, 0, s>>>(vsd, cp, n_contrib, keys, aux);
    else if (vs.tile_w == 32 && vs.tile_h == 16)
        bwd_pair_keys_kernel<32, 16><<<(unsigned)blocks, 256, 0, s>>>(vsd, cp, n_contrib, keys, aux);
}

size_t chunk_slot_bytes(int tile_w, int tile_h) {
    return (size_t)kFields * kSub * tile_w * tile_h * sizeof(float);
}

size_t pix_state_bytes() { return sizeof(PixState); }

void launch_composite_fwd(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib,
                          const ChunkPlan &cp, uint32_t *queue, void *pix_state, cudaStream_t s, int bm, int part) {
    if (vs.total_tiles == 0) return;
    if (bm == 1) fwd_dispatch<1>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, cp, queue, pix_state, part, s);
    else fwd_dispatch<2>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, cp, queue, pix_state, part, s);
}

void launch_composite_bwd(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib,
                          GGrad *g2d, const ChunkPlan &cp, uint32_t *queue, cudaStream_t s, int bm) {
    if (vs.total_tiles == 0) return;
    if (bm == 1) bwd_dispatch<1>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, cp, queue, s);
    else bwd_dispatch<2>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, cp, queue, s);
}

} // namespace lvigs
