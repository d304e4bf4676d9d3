// composite.cu -- front-to-back alpha compositing (a5) and its reverse (a6).
//
// Work unit: one warp per 8x8 block of pixels, two vertically adjacent pixels
// per lane.  A CTA holds the (tile_w/8) x (tile_h/8) warps of one (view,
// tile); every warp walks the tile's depth-sorted instance list on its own
// (no block-wide barrier), so a warp whose pixels saturate early, or that few
// Gaussians reach, never waits for its neighbours.
//
// The list is consumed in batches of 32*BM instances.  Each lane gathers
// records and tests them against the warp's 8x8 block using the conservative
// box of the region where alpha can reach 1/255 (half-extents precomputed by
// preprocessing); the hits are compacted into the warp's shared-memory slice
// with a ballot, in list order.  Culled Gaussians would fail the 1/255 test at
// every pixel of the block, so results are exactly those of walking the whole
// list.  Per pixel (Eq. (3)-(6)): alpha = min(0.99, o exp(power)), skipped
// below 1/255, and the pixel stops before a Gaussian that would take the
// transmittance below 1e-4.
//
// The backward pass walks the same list in reverse from the warp's last
// contributor, recovering the transmittance by division (T_i = T_{i+1} /
// (1 - alpha_i)) so no per-Gaussian state is stored.  Each lane sums its two
// pixels' ten screen-space gradient terms, the warp reduce-scatters the ten
// sums with 12 shuffles, and the ten lanes that end with a total add it to
// the Gaussian's gradient record with one atomic instruction.
#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr int PB = 8;  // warp pixel block is PB x PB
constexpr int PPT = 2; // pixels per lane (rows 2r, 2r+1 of the block)

// does the alpha box of record (a, b, c) meet the block [x0, x0+7] x [y0, y0+7]?
__device__ __forceinline__ bool meets(const float4 a, const float4 b, const float4 c, float x0, float y0) {
    const float ex = b.w, ey = c.w;
    return a.x + ex >= x0 && a.x - ex <= x0 + (PB - 1) && a.y + ey >= y0 && a.y - ey <= y0 + (PB - 1);
}

template <int TW, int TH>
struct Geometry {
    static constexpr int WX = TW / PB, WY = TH / PB;
    static constexpr int NW = WX * WY;
    static constexpr int NT = NW * 32;
    static_assert(TW % PB == 0 && TH % PB == 0, "tile is a whole number of 8x8 blocks");
};

template <int TW, int TH, int BM>
__global__ void __launch_bounds__(Geometry<TW, TH>::NT)
composite_fwd_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                     const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs,
                     ViewImages out, float *__restrict__ final_T, int32_t *__restrict__ n_contrib) {
    using Gm = Geometry<TW, TH>;
    constexpr int B = 32 * BM;
    __shared__ float4 s_a[Gm::NW][B], s_b[Gm::NW][B], s_c[Gm::NW][B];
    __shared__ int s_pos[Gm::NW][B];
    const uint32_t gt = blockIdx.x;
    const int vi = view_of_tile(*vsp, gt);
    const ViewDesc &V = vsp->v[vi];
    const uint32_t lt = gt - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx0 = tx * TW + (warp % Gm::WX) * PB, by0 = ty * TH + (warp / Gm::WX) * PB;
    const int px = bx0 + (lane & 7), py0 = by0 + (lane >> 3) * PPT;
    const float fpx = (float)px, fx0 = (float)bx0, fy0 = (float)by0;
    const uint2 rg = ranges[gt];
    const uint32_t ltmask = (1u << lane) - 1u;
    float4 *A = s_a[warp], *Bv = s_b[warp], *Cv = s_c[warp];
    int *Pos = s_pos[warp];

    float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT];
    int last[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = D[k] = 0.f;
        last[k] = 0;
        done[k] = !(px < V.W && py0 + k < V.H);
    }
    bool tdone = done[0] && done[1];
    for (uint32_t base = rg.x; base < rg.y; base += B) {
        if (__all_sync(0xffffffffu, tdone)) break;
        // gather and compact the Gaussians whose alpha box meets this block
        int n = 0;
#pragma unroll
        for (int q = 0; q < BM; ++q) {
            const uint32_t i = base + q * 32 + lane;
            GRec r;
            bool hit = false;
            if (i < rg.y) {
                r = recs[inst_vals[i]];
                hit = meets(r.a, r.b, r.c, fx0, fy0);
            }
            const uint32_t m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int slot = n + __popc(m & ltmask);
                A[slot] = r.a;
                Bv[slot] = r.b;
                Cv[slot] = r.c;
                Pos[slot] = (int)(i - rg.x);
            }
            n += __popc(m);
        }
        __syncwarp();
        for (int q = 0; q < n && !tdone; ++q) {
            const float4 a = A[q];
            const float4 b = Bv[q];
            const float dx = a.x - fpx;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (done[k]) continue;
                const float dy = a.y - (float)(py0 + k);
                const float power = gauss_power(a.z, a.w, b.x, dx, dy);
                if (power > 0.f) continue;
                const float alpha = fminf(kAlphaMax, __fmul_rn(b.y, __expf(power)));
                if (alpha < kAlphaMin) continue;
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                if (Tn < kTMin) {
                    done[k] = true;
                    continue;
                }
                const float4 c = Cv[q];
                const float w = alpha * T[k];
                C0[k] = fmaf(c.x, w, C0[k]);
                C1[k] = fmaf(c.y, w, C1[k]);
                C2[k] = fmaf(c.z, w, C2[k]);
                D[k] = fmaf(b.z, w, D[k]);
                T[k] = Tn;
                last[k] = Pos[q] + 1;
            }
            tdone = done[0] && done[1];
        }
        __syncwarp();
    }
    const size_t HW = (size_t)V.W * V.H;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int py = py0 + k;
        if (px < V.W && py < V.H) {
            const size_t p = (size_t)py * V.W + px;
            out.rgb[vi][p] = C0[k];
            out.rgb[vi][HW + p] = C1[k];
            out.rgb[vi][2 * HW + p] = C2[k];
            out.depth[vi][p] = D[k];
            out.alpha[vi][p] = 1.f - T[k];
            final_T[V.pix_base + p] = T[k];
            n_contrib[V.pix_base + p] = last[k];
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

// float offset in GGrad of reduced value index: du dv dA dB dC dop dr dg db dz
__device__ __forceinline__ int grad_offset(int idx) {
    return idx < 6 ? idx : (idx < 9 ? idx + 2 : 6);
}

template <int TW, int TH, int BM>
__global__ void __launch_bounds__(Geometry<TW, TH>::NT)
composite_bwd_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                     const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs,
                     ViewGrads G, const float *__restrict__ final_T,
                     const int32_t *__restrict__ n_contrib, GGrad *__restrict__ g2d) {
    using Gm = Geometry<TW, TH>;
    constexpr int B = 32 * BM;
    constexpr int NACC = 10;
    __shared__ float4 s_a[Gm::NW][B], s_b[Gm::NW][B], s_c[Gm::NW][B];
    __shared__ int s_pos[Gm::NW][B];
    __shared__ uint32_t s_idx[Gm::NW][B];
    const uint32_t gt = blockIdx.x;
    const int vi = view_of_tile(*vsp, gt);
    const ViewDesc &V = vsp->v[vi];
    const uint32_t lt = gt - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx0 = tx * TW + (warp % Gm::WX) * PB, by0 = ty * TH + (warp / Gm::WX) * PB;
    const int px = bx0 + (lane & 7), py0 = by0 + (lane >> 3) * PPT;
    const float fpx = (float)px, fx0 = (float)bx0, fy0 = (float)by0;
    const uint2 rg = ranges[gt];
    const uint32_t ltmask = (1u << lane) - 1u;
    const size_t HW = (size_t)V.W * V.H;
    float4 *A = s_a[warp], *Bv = s_b[warp], *Cv = s_c[warp];
    int *Pos = s_pos[warp];
    uint32_t *Idx = s_idx[warp];

    float T[PPT], gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], gA[PPT];
    float S0[PPT], S1[PPT], S2[PPT], SD[PPT], SA[PPT];
    int last[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int py = py0 + k;
        T[k] = 1.f;
        gC0[k] = gC1[k] = gC2[k] = gD[k] = gA[k] = 0.f;
        S0[k] = S1[k] = S2[k] = SD[k] = SA[k] = 0.f;
        last[k] = 0;
        if (px < V.W && py < V.H) {
            const size_t p = (size_t)py * V.W + px;
            T[k] = final_T[V.pix_base + p];
            last[k] = n_contrib[V.pix_base + p];
            gC0[k] = G.d_rgb[vi][p];
            gC1[k] = G.d_rgb[vi][HW + p];
            gC2[k] = G.d_rgb[vi][2 * HW + p];
            gD[k] = G.d_depth[vi] ? G.d_depth[vi][p] : 0.f;
            gA[k] = G.d_alpha[vi] ? G.d_alpha[vi][p] : 0.f;
        }
    }
    const int warp_last = __reduce_max_sync(0xffffffffu, max(last[0], last[1]));
    const uint32_t end = rg.x + (uint32_t)warp_last;

    for (uint32_t hi = end; hi > rg.x;) {
        const uint32_t lo = hi - rg.x > (uint32_t)B ? hi - B : rg.x;
        int n = 0;
#pragma unroll
        for (int q = 0; q < BM; ++q) {
            const uint32_t i = lo + q * 32 + lane;
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
                A[slot] = r.a;
                Bv[slot] = r.b;
                Cv[slot] = r.c;
                Pos[slot] = (int)(i - rg.x);
                Idx[slot] = idx;
            }
            n += __popc(m);
        }
        __syncwarp();
        for (int q = n - 1; q >= 0; --q) {
            const float4 a = A[q];
            const float4 b = Bv[q];
            const float4 c = Cv[q];
            const int pos = Pos[q];
            const float dx = a.x - fpx;
            float v[NACC];
#pragma unroll
            for (int m = 0; m < NACC; ++m) v[m] = 0.f;
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (pos >= last[k]) continue;
                const float dy = a.y - (float)(py0 + k);
                const float power = gauss_power(a.z, a.w, b.x, dx, dy);
                if (power > 0.f) continue;
                const float G_ = __expf(power);
                const float oG = __fmul_rn(b.y, G_);
                const float alpha = fminf(kAlphaMax, oG);
                if (alpha < kAlphaMin) continue;
                any = true;
                const float one_m = 1.f - alpha;
                T[k] = __fdividef(T[k], one_m);
                const float w = alpha * T[k];
                const float dLda = T[k] * ((c.x - S0[k]) * gC0[k] + (c.y - S1[k]) * gC1[k] +
                                           (c.z - S2[k]) * gC2[k] + (b.z - SD[k]) * gD[k] + (1.f - SA[k]) * gA[k]);
                S0[k] = fmaf(alpha, c.x - S0[k], S0[k]);
                S1[k] = fmaf(alpha, c.y - S1[k], S1[k]);
                S2[k] = fmaf(alpha, c.z - S2[k], S2[k]);
                SD[k] = fmaf(alpha, b.z - SD[k], SD[k]);
                SA[k] = fmaf(alpha, 1.f - SA[k], SA[k]);
                v[6] = fmaf(w, gC0[k], v[6]);
                v[7] = fmaf(w, gC1[k], v[7]);
                v[8] = fmaf(w, gC2[k], v[8]);
                v[9] = fmaf(w, gD[k], v[9]);
                if (oG < kAlphaMax) {
                    const float dpow = dLda * alpha;
                    v[5] = fmaf(dLda, G_, v[5]);
                    v[0] -= dpow * (a.z * dx + a.w * dy);
                    v[1] -= dpow * (b.x * dy + a.w * dx);
                    v[2] -= 0.5f * dpow * dx * dx;
                    v[3] -= dpow * dx * dy;
                    v[4] -= 0.5f * dpow * dy * dy;
                }
            }
            if (__any_sync(0xffffffffu, any)) {
                int vidx;
                bool valid;
                const float tot = reduce_scatter10(v, lane, vidx, valid);
                if (valid && tot != 0.f) atomicAdd((float *)(g2d + Idx[q]) + grad_offset(vidx), tot);
            }
        }
        __syncwarp();
        hi = lo;
    }
}

template <int TW, int TH, int BM>
void fwd_launch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib, cudaStream_t s) {
    composite_fwd_kernel<TW, TH, BM><<<vs.total_tiles, Geometry<TW, TH>::NT, 0, s>>>(vsd, ranges, inst_vals, recs, out,
                                                                                   final_T, n_contrib);
}

template <int TW, int TH, int BM>
void bwd_launch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib,
                GGrad *g2d, cudaStream_t s) {
    composite_bwd_kernel<TW, TH, BM><<<vs.total_tiles, Geometry<TW, TH>::NT, 0, s>>>(vsd, ranges, inst_vals, recs, g,
                                                                                   final_T, n_contrib, g2d);
}

template <int BM>
void fwd_dispatch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                  const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib, cudaStream_t s) {
    if (vs.tile_w == 16 && vs.tile_h == 16) fwd_launch<16, 16, BM>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
    else if (vs.tile_w == 8 && vs.tile_h == 8) fwd_launch<8, 8, BM>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
    else if (vs.tile_w == 32 && vs.tile_h == 16) fwd_launch<32, 16, BM>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
}

template <int BM>
void bwd_dispatch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                  const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib, GGrad *g2d,
                  cudaStream_t s) {
    if (vs.tile_w == 16 && vs.tile_h == 16) bwd_launch<16, 16, BM>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
    else if (vs.tile_w == 8 && vs.tile_h == 8) bwd_launch<8, 8, BM>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
    else if (vs.tile_w == 32 && vs.tile_h == 16) bwd_launch<32, 16, BM>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
}

} // namespace

void launch_composite_fwd(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib,
                          cudaStream_t s, int bm) {
    if (vs.total_tiles == 0) return;
    if (bm == 1) fwd_dispatch<1>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
    else fwd_dispatch<2>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
}

void launch_composite_bwd(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib,
                          GGrad *g2d, cudaStream_t s, int bm) {
    if (vs.total_tiles == 0) return;
    if (bm == 1) bwd_dispatch<1>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
    else bwd_dispatch<2>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
}

} // namespace lvigs
