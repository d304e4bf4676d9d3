// composite.cu -- front-to-back alpha compositing (a5) and its reverse (a6).
//
// One CTA per (view, pixel tile), one thread per pixel.  The tile's
// depth-sorted instance list is consumed in rounds: each thread gathers one
// Gaussian record (48 B) into shared memory, then every thread walks the
// round against its pixel (Eq. (3)-(6)): alpha = min(0.99, o exp(power)),
// skipped below 1/255, and the pixel stops before a Gaussian that would take
// the transmittance below 1e-4.  The CTA leaves the list once every pixel
// has stopped.
//
// The backward pass walks the same list in reverse from the last contributor
// of the tile, recovering the transmittance by division (T_i = T_{i+1} /
// (1 - alpha_i)) so no per-Gaussian state is stored, and reduces each
// Gaussian's ten screen-space gradient terms across the warp with shuffles,
// across the CTA in shared memory, and then into global memory with one
// vector atomic per float4.
#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH)
composite_fwd_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                     const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs,
                     ViewImages out, float *__restrict__ final_T, int32_t *__restrict__ n_contrib) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_a[NT], s_b[NT], s_c[NT];
    const uint32_t gt = blockIdx.x;
    const int vi = view_of_tile(*vsp, gt);
    const ViewDesc &V = vsp->v[vi];
    const uint32_t lt = gt - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const bool inside = px < V.W && py < V.H;
    const uint2 rg = ranges[gt];
    const float fpx = (float)px, fpy = (float)py;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    int last = 0;
    bool done = !inside;
    for (uint32_t base = rg.x; base < rg.y; base += NT) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t i = base + t;
        if (i < rg.y) {
            const GRec r = recs[inst_vals[i]];
            s_a[t] = r.a;
            s_b[t] = r.b;
            s_c[t] = r.c;
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)NT, rg.y - base);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                const float dx = a.x - fpx, dy = a.y - fpy;
                const float power = gauss_power(a.z, a.w, b.x, dx, dy);
                if (power > 0.f) continue;
                const float alpha = fminf(kAlphaMax, __fmul_rn(b.y, __expf(power)));
                if (alpha < kAlphaMin) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                if (Tn < kTMin) {
                    done = true;
                    break;
                }
                const float4 c = s_c[j];
                const float w = alpha * T;
                C0 = fmaf(c.x, w, C0);
                C1 = fmaf(c.y, w, C1);
                C2 = fmaf(c.z, w, C2);
                D = fmaf(b.z, w, D);
                T = Tn;
                last = (int)(base - rg.x) + j + 1;
            }
        }
    }
    if (inside) {
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

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH)
composite_bwd_kernel(const ViewSet *__restrict__ vsp, const uint2 *__restrict__ ranges,
                     const uint32_t *__restrict__ inst_vals, const GRec *__restrict__ recs,
                     ViewGrads G, const float *__restrict__ final_T,
                     const int32_t *__restrict__ n_contrib, GGrad *__restrict__ g2d) {
    constexpr int NT = TW * TH;
    constexpr int NACC = 10;
    __shared__ float4 s_a[NT], s_b[NT], s_c[NT];
    __shared__ uint32_t s_idx[NT];
    __shared__ float s_acc[NT * NACC];
    __shared__ int s_last;
    const uint32_t gt = blockIdx.x;
    const int vi = view_of_tile(*vsp, gt);
    const ViewDesc &V = vsp->v[vi];
    const uint32_t lt = gt - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const int t = threadIdx.x, lane = t & 31;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const bool inside = px < V.W && py < V.H;
    const uint2 rg = ranges[gt];
    const float fpx = (float)px, fpy = (float)py;

    float T = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f;
    int last = 0;
    if (inside) {
        const size_t HW = (size_t)V.W * V.H;
        const size_t p = (size_t)py * V.W + px;
        T = final_T[V.pix_base + p];
        last = n_contrib[V.pix_base + p];
        gC0 = G.d_rgb[vi][p];
        gC1 = G.d_rgb[vi][HW + p];
        gC2 = G.d_rgb[vi][2 * HW + p];
        gD = G.d_depth[vi] ? G.d_depth[vi][p] : 0.f;
        gA = G.d_alpha[vi] ? G.d_alpha[vi][p] : 0.f;
    }
    if (t == 0) s_last = 0;
#pragma unroll
    for (int k = 0; k < NACC; ++k) s_acc[t * NACC + k] = 0.f;
    __syncthreads();
    if (last > 0) atomicMax(&s_last, last);
    __syncthreads();
    const uint32_t end = rg.x + (uint32_t)s_last;

    // suffix sums S of Eq. (3)-(5) behind the current Gaussian, normalised
    float S0 = 0.f, S1 = 0.f, S2 = 0.f, SD = 0.f, SA = 0.f;
    for (uint32_t hi = end; hi > rg.x;) {
        const uint32_t lo = hi - rg.x > (uint32_t)NT ? hi - NT : rg.x;
        const uint32_t i = lo + t;
        if (i < hi) {
            const uint32_t idx = inst_vals[i];
            const GRec r = recs[idx];
            s_idx[t] = idx;
            s_a[t] = r.a;
            s_b[t] = r.b;
            s_c[t] = r.c;
        }
        __syncthreads();
        const int cnt = (int)(hi - lo);
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = (int)(lo - rg.x) + j;
            bool contrib = pos < last;
            float alpha = 0.f, G_ = 0.f, dx = 0.f, dy = 0.f;
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            if (contrib) {
                dx = a.x - fpx;
                dy = a.y - fpy;
                const float power = gauss_power(a.z, a.w, b.x, dx, dy);
                contrib = power <= 0.f;
                if (contrib) {
                    G_ = __expf(power);
                    alpha = fminf(kAlphaMax, __fmul_rn(b.y, G_));
                    contrib = alpha >= kAlphaMin;
                }
            }
            float v[NACC];
#pragma unroll
            for (int k = 0; k < NACC; ++k) v[k] = 0.f;
            if (contrib) {
                const float4 c = s_c[j];
                const float one_m = 1.f - alpha;
                T = T / one_m;
                const float w = alpha * T;
                const float dLda = T * ((c.x - S0) * gC0 + (c.y - S1) * gC1 + (c.z - S2) * gC2 +
                                        (b.z - SD) * gD + (1.f - SA) * gA);
                S0 = alpha * c.x + one_m * S0;
                S1 = alpha * c.y + one_m * S1;
                S2 = alpha * c.z + one_m * S2;
                SD = alpha * b.z + one_m * SD;
                SA = alpha + one_m * SA;
                v[6] = w * gC0;
                v[7] = w * gC1;
                v[8] = w * gC2;
                v[9] = w * gD;
                if (b.y * G_ < kAlphaMax) {
                    const float dpow = dLda * alpha;
                    v[5] = dLda * G_;
                    v[0] = -dpow * (a.z * dx + a.w * dy);
                    v[1] = -dpow * (b.x * dy + a.w * dx);
                    v[2] = -0.5f * dpow * dx * dx;
                    v[3] = -dpow * dx * dy;
                    v[4] = -0.5f * dpow * dy * dy;
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int k = 0; k < NACC; ++k) v[k] = warp_sum(v[k]);
                if (lane == 0) {
#pragma unroll
                    for (int k = 0; k < NACC; ++k) atomicAdd(&s_acc[j * NACC + k], v[k]);
                }
            }
        }
        __syncthreads();
        if (t < cnt) {
            float *acc = &s_acc[t * NACC];
            bool nz = false;
#pragma unroll
            for (int k = 0; k < NACC; ++k) nz |= acc[k] != 0.f;
            if (nz) {
                GGrad *dst = g2d + s_idx[t];
                atomicAdd(&dst->g0, make_float4(acc[0], acc[1], acc[2], acc[3]));
                atomicAdd(&dst->g1, make_float4(acc[4], acc[5], acc[9], 0.f));
                atomicAdd(&dst->g2, make_float4(acc[6], acc[7], acc[8], 0.f));
#pragma unroll
                for (int k = 0; k < NACC; ++k) acc[k] = 0.f;
            }
        }
        __syncthreads();
        hi = lo;
    }
}

template <int TW, int TH>
void fwd_launch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib,
                cudaStream_t s) {
    composite_fwd_kernel<TW, TH><<<vs.total_tiles, TW * TH, 0, s>>>(vsd, ranges, inst_vals, recs, out,
                                                                     final_T, n_contrib);
}

template <int TW, int TH>
void bwd_launch(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib,
                GGrad *g2d, cudaStream_t s) {
    composite_bwd_kernel<TW, TH><<<vs.total_tiles, TW * TH, 0, s>>>(vsd, ranges, inst_vals, recs, g,
                                                                     final_T, n_contrib, g2d);
}

} // namespace

void launch_composite_fwd(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewImages &out, float *final_T,
                          int32_t *n_contrib, cudaStream_t s) {
    if (vs.total_tiles == 0) return;
    if (vs.tile_w == 16 && vs.tile_h == 16)
        fwd_launch<16, 16>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
    else if (vs.tile_w == 8 && vs.tile_h == 8)
        fwd_launch<8, 8>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
    else if (vs.tile_w == 32 && vs.tile_h == 16)
        fwd_launch<32, 16>(vs, vsd, ranges, inst_vals, recs, out, final_T, n_contrib, s);
}

void launch_composite_bwd(const ViewSet &vs, const ViewSet *vsd, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewGrads &g, const float *final_T,
                          const int32_t *n_contrib, GGrad *g2d, cudaStream_t s) {
    if (vs.total_tiles == 0) return;
    if (vs.tile_w == 16 && vs.tile_h == 16)
        bwd_launch<16, 16>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
    else if (vs.tile_w == 8 && vs.tile_h == 8)
        bwd_launch<8, 8>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
    else if (vs.tile_w == 32 && vs.tile_h == 16)
        bwd_launch<32, 16>(vs, vsd, ranges, inst_vals, recs, g, final_T, n_contrib, g2d, s);
}

} // namespace lvigs
