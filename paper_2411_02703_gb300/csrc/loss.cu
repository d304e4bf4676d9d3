// loss.cu -- fused mapping loss (a8) and image pyramid (a9).
//
// L = (1 - lambda) L1 + lambda (1 - mean SSIM) + lambda_d L_d   (Eq. 10-12)
//
// Pass 1, one CTA per 32x32 pixel tile (of every view of the call): stages
// the rendered and target images of the tile plus a 5-pixel halo in shared
// memory, forms the five windowed moments of each channel with a separable
// 11-tap Gaussian (sigma 1.5, zero padding), and writes per pixel the three
// partial derivatives of SSIM with respect to the moments (mu_x, E[x^2],
// E[xy]); it also reduces the L1, SSIM and LiDAR-depth sums of the tile.
// Each thread filters a run of four outputs from a 14-sample window held in
// registers (rows in the horizontal pass, columns in the vertical one), so a
// staged sample is read from shared memory about 3.5 times instead of 11.
// The next channel's tile is copied in (cp.async) while the current one's
// vertical pass runs.
// A one-block-per-view kernel sums the tile partials in a fixed order
// (deterministic) into the four loss terms.
// Pass 2 applies the adjoint window to those derivative maps and adds the
// L1 and depth terms, giving dL/drgb and dL/ddepth.
#include <cmath>

#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

constexpr int LT = kLossTile;     // 32
constexpr int HALO = 5;           // (11 - 1) / 2
constexpr int LS = LT + 2 * HALO; // 42
constexpr int RUN = 4;            // outputs per thread and pass
constexpr int WIN = RUN + 2 * HALO; // 14 samples feed a run
constexpr int kThreads = 256;
constexpr int kRowTasks = LS * (LT / RUN); // horizontal: 42 rows x 8 runs
static_assert(LT * LT / RUN == kThreads, "one vertical run per thread");

struct Window {
    float w[11];
};

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

__device__ __forceinline__ void loss_tile_of(const LossViews &lv, uint32_t b, int &vi, int &tx, int &ty) {
    vi = 0;
    for (int i = 1; i < lv.n_views; ++i)
        if (lv.tile_base[i] <= b) vi = i;
    const uint32_t lt = b - lv.tile_base[vi];
    const int tiles_x = (lv.W[vi] + LT - 1) / LT;
    tx = (int)(lt % (uint32_t)tiles_x);
    ty = (int)(lt / (uint32_t)tiles_x);
}

__device__ __forceinline__ double block_sum_d(double v, double *red) {
    // 256 threads
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) s += red[w];
    return s;
}

// Stage a tile of `img` (plus halo) into dst[LS][LS+1] asynchronously
// (cp.async, 4 bytes per element, zero-filled outside the image): the copies
// land while the block goes on computing; cp_async_wait<0> and a barrier make
// them visible.
constexpr int kStageIt = (LS * LS + kThreads - 1) / kThreads;
__device__ __forceinline__ void stage_async(const float *__restrict__ img, int W, int H, int tx, int ty,
                                            float (*dst)[LS + 1]) {
#pragma unroll
    for (int j = 0; j < kStageIt; ++j) {
        const int i = threadIdx.x + j * kThreads;
        if (i < LS * LS) {
            const int r = i / LS, c = i - r * LS;
            const int gx = tx * LT + c - HALO, gy = ty * LT + r - HALO;
            const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const float *src = ok ? img + (size_t)gy * W + gx : img;
            const uint32_t d = (uint32_t)__cvta_generic_to_shared(&dst[r][c]);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0));
        }
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__global__ void __launch_bounds__(kThreads, 4)
loss_pass1_kernel(LossViews lv, Window win, float *__restrict__ gmaps, double *__restrict__ partials) {
    __shared__ float sx[LS][LS + 1], sy[LS][LS + 1];
    __shared__ float sh[5][LS][LT + 1];
    __shared__ double red[8];
    int vi, tx, ty;
    loss_tile_of(lv, blockIdx.x, vi, tx, ty);
    const int W = lv.W[vi], H = lv.H[vi];
    const size_t HW = (size_t)W * H;
    const int t = threadIdx.x;
    // this thread's vertical run: column vc, rows vr .. vr + 3 of the tile
    const int vc = t % LT, vr = (t / LT) * RUN;
    const int px = tx * LT + vc;
    const float lam = lv.lambda_ssim;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    // a thread's own sums (at most 12 terms each) in binary32, the block's in binary64
    float l1 = 0.f, ssim = 0.f, dsum = 0.f, dcnt = 0.f;
    float *G = gmaps + lv.gmap_base[vi];

    // the next channel is copied in while the current one's vertical pass runs
    if (lam != 0.f) {
        stage_async(lv.rgb[vi], W, H, tx, ty, sx);
        stage_async(lv.gt[vi], W, H, tx, ty, sy);
        cp_async_commit();
    }
    for (int ch = 0; ch < 3; ++ch) {
        const float *x = lv.rgb[vi] + ch * HW;
        const float *y = lv.gt[vi] + ch * HW;
        if (lam == 0.f) {
#pragma unroll
            for (int o = 0; o < RUN; ++o) {
                const int py = ty * LT + vr + o;
                if (px < W && py < H) l1 += fabsf(x[(size_t)py * W + px] - y[(size_t)py * W + px]);
            }
            continue;
        }
        cp_async_wait<0>();
        __syncthreads();
        // L1 from the staged samples (zero outside the image on both sides)
#pragma unroll
        for (int o = 0; o < RUN; ++o) l1 += fabsf(sx[HALO + vr + o][HALO + vc] - sy[HALO + vr + o][HALO + vc]);
        // horizontal pass: runs of four outputs along the staged rows
        for (int task = t; task < kRowTasks; task += kThreads) {
            const int r = task / (LT / RUN), c0 = (task % (LT / RUN)) * RUN;
            float a[WIN], b[WIN];
#pragma unroll
            for (int i = 0; i < WIN; ++i) {
                a[i] = sx[r][c0 + i];
                b[i] = sy[r][c0 + i];
            }
            float m1[RUN], m2[RUN], m11[RUN], m22[RUN], m12[RUN];
#pragma unroll
            for (int o = 0; o < RUN; ++o) m1[o] = m2[o] = m11[o] = m22[o] = m12[o] = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float w = win.w[k];
#pragma unroll
                for (int o = 0; o < RUN; ++o) {
                    const float wa = w * a[o + k], wb = w * b[o + k];
                    m1[o] += wa;
                    m2[o] += wb;
                    m11[o] = fmaf(wa, a[o + k], m11[o]);
                    m22[o] = fmaf(wb, b[o + k], m22[o]);
                    m12[o] = fmaf(wa, b[o + k], m12[o]);
                }
            }
#pragma unroll
            for (int o = 0; o < RUN; ++o) {
                sh[0][r][c0 + o] = m1[o];
                sh[1][r][c0 + o] = m2[o];
                sh[2][r][c0 + o] = m11[o];
                sh[3][r][c0 + o] = m22[o];
                sh[4][r][c0 + o] = m12[o];
            }
        }
        __syncthreads();
        // sx, sy are free now: copy the next channel in
        if (ch + 1 < 3) {
            stage_async(x + HW, W, H, tx, ty, sx);
            stage_async(y + HW, W, H, tx, ty, sy);
            cp_async_commit();
        }
        // vertical pass: this thread's run of four pixels
        float mom[5][RUN];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            float v[WIN];
#pragma unroll
            for (int i = 0; i < WIN; ++i) v[i] = sh[m][vr + i][vc];
#pragma unroll
            for (int o = 0; o < RUN; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 11; ++k) acc = fmaf(win.w[k], v[o + k], acc);
                mom[m][o] = acc;
            }
        }
#pragma unroll
        for (int o = 0; o < RUN; ++o) {
            const int py = ty * LT + vr + o;
            if (!(px < W && py < H)) continue;
            const size_t p = (size_t)py * W + px;
            const float mx = mom[0][o], my = mom[1][o], mxx = mom[2][o], myy = mom[3][o], mxy = mom[4][o];
            const float vx = mxx - mx * mx, vy = myy - my * my, cxy = mxy - mx * my;
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * cxy + C2;
            const float B1 = mx * mx + my * my + C1, B2 = vx + vy + C2;
            const float rB1 = __frcp_rn(B1), rB2 = __frcp_rn(B2);
            const float inv = rB1 * rB2;
            const float S = A1 * A2 * inv;
            ssim += S;
            // dS/d mu_x, dS/d E[x^2], dS/d E[xy]
            const float d1 = 2.f * my * (A2 - A1) * inv - S * (2.f * mx) * (rB1 - rB2);
            const float d2 = -S * rB2;
            const float d12 = 2.f * A1 * inv;
            G[(0 * 3 + ch) * HW + p] = d1;
            G[(1 * 3 + ch) * HW + p] = d2;
            G[(2 * 3 + ch) * HW + p] = d12;
        }
    }
    if (lv.lidar[vi]) {
#pragma unroll
        for (int o = 0; o < RUN; ++o) {
            const int py = ty * LT + vr + o;
            if (!(px < W && py < H)) continue;
            const size_t p = (size_t)py * W + px;
            const float L = lv.lidar[vi][p];
            if (L > 0.f) {
                dsum += fabsf(lv.depth[vi][p] - L);
                dcnt += 1.f;
            }
        }
    }
    const double s0 = block_sum_d(l1, red);
    const double s1 = block_sum_d(ssim, red);
    const double s2 = block_sum_d(dsum, red);
    const double s3 = block_sum_d(dcnt, red);
    if (t == 0) {
        double *o = partials + 4 * (size_t)blockIdx.x;
        o[0] = s0;
        o[1] = s1;
        o[2] = s2;
        o[3] = s3;
    }
}

// One block per view: fixed-order sum of the tile partials.
__global__ void __launch_bounds__(256)
loss_reduce_kernel(LossViews lv, const double *__restrict__ partials, double *__restrict__ nvalid_out) {
    __shared__ double red[4][256];
    const int vi = blockIdx.x;
    const uint32_t b0 = lv.tile_base[vi];
    const uint32_t b1 = vi + 1 < lv.n_views ? lv.tile_base[vi + 1] : lv.total_tiles;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint32_t b = b0 + threadIdx.x; b < b1; b += 256)
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] += partials[4 * (size_t)b + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double P3 = 3.0 * lv.W[vi] * lv.H[vi];
        const double lam = lv.lambda_ssim, lamd = lv.lambda_depth;
        const double l1 = red[0][0] / P3;
        const double ssim = lam != 0.0 ? red[1][0] / P3 : 1.0;
        const double nv = red[3][0];
        const double ld = nv > 0 ? red[2][0] / nv : 0.0;
        double *o = lv.loss_out[vi];
        if (o) {
            o[0] = (1.0 - lam) * l1 + (lam != 0.0 ? lam * (1.0 - ssim) : 0.0) + lamd * ld;
            o[1] = l1;
            o[2] = ssim;
            o[3] = ld;
        }
        nvalid_out[vi] = nv;
    }
}

__global__ void __launch_bounds__(kThreads, 4)
loss_pass2_kernel(LossViews lv, Window win, const float *__restrict__ gmaps,
                  const double *__restrict__ nvalid) {
    __shared__ float sg[3][LS][LS + 1];
    __shared__ float sh[3][LS][LT + 1];
    int vi, tx, ty;
    loss_tile_of(lv, blockIdx.x, vi, tx, ty);
    const int W = lv.W[vi], H = lv.H[vi];
    const size_t HW = (size_t)W * H;
    const int t = threadIdx.x;
    const int vc = t % LT, vr = (t / LT) * RUN;
    const int px = tx * LT + vc;
    const float lam = lv.lambda_ssim;
    const float k1 = (1.f - lam) / (float)(3.0 * HW);
    const float k2 = -lam / (float)(3.0 * HW);
    const float *G = gmaps + lv.gmap_base[vi];
    float *drgb = lv.d_rgb[vi];

    for (int ch = 0; ch < 3; ++ch) {
        const float *x = lv.rgb[vi] + ch * HW;
        const float *y = lv.gt[vi] + ch * HW;
        float s1[RUN], s2[RUN], s12[RUN];
#pragma unroll
        for (int o = 0; o < RUN; ++o) s1[o] = s2[o] = s12[o] = 0.f;
        if (lam != 0.f) {
            if (ch == 0) {
#pragma unroll
                for (int m = 0; m < 3; ++m) stage_async(G + (size_t)(m * 3) * HW, W, H, tx, ty, sg[m]);
                cp_async_commit();
            }
            cp_async_wait<0>();
            __syncthreads();
            for (int task = t; task < kRowTasks; task += kThreads) {
                const int r = task / (LT / RUN), c0 = (task % (LT / RUN)) * RUN;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    float a[WIN];
#pragma unroll
                    for (int i = 0; i < WIN; ++i) a[i] = sg[m][r][c0 + i];
#pragma unroll
                    for (int o = 0; o < RUN; ++o) {
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < 11; ++k) acc = fmaf(win.w[k], a[o + k], acc);
                        sh[m][r][c0 + o] = acc;
                    }
                }
            }
            __syncthreads();
            // sg is free now: copy the next channel's maps in during the vertical pass
            if (ch + 1 < 3) {
#pragma unroll
                for (int m = 0; m < 3; ++m) stage_async(G + (size_t)(m * 3 + ch + 1) * HW, W, H, tx, ty, sg[m]);
                cp_async_commit();
            }
            float *outs[3] = {s1, s2, s12};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                float v[WIN];
#pragma unroll
                for (int i = 0; i < WIN; ++i) v[i] = sh[m][vr + i][vc];
#pragma unroll
                for (int o = 0; o < RUN; ++o) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < 11; ++k) acc = fmaf(win.w[k], v[o + k], acc);
                    outs[m][o] = acc;
                }
            }
        }
        if (drgb) {
#pragma unroll
            for (int o = 0; o < RUN; ++o) {
                const int py = ty * LT + vr + o;
                if (!(px < W && py < H)) continue;
                const size_t p = (size_t)py * W + px;
                const float xv = x[p], yv = y[p];
                drgb[ch * HW + p] = k1 * sgnf(xv - yv) + k2 * (s1[o] + 2.f * xv * s2[o] + yv * s12[o]);
            }
        }
    }
    if (lv.d_depth[vi]) {
        const double nv = lv.lidar[vi] ? nvalid[vi] : 0.0;
        const float gs = nv > 0 ? lv.lambda_depth / (float)nv : 0.f; // times a sign: exact
#pragma unroll
        for (int o = 0; o < RUN; ++o) {
            const int py = ty * LT + vr + o;
            if (!(px < W && py < H)) continue;
            const size_t p = (size_t)py * W + px;
            float g = 0.f;
            if (gs != 0.f) {
                const float L = lv.lidar[vi][p];
                if (L > 0.f) g = gs * sgnf(lv.depth[vi][p] - L);
            }
            lv.d_depth[vi][p] = g;
        }
    }
}

__global__ void pyramid_down_kernel(int W, int H, const float *__restrict__ rgb,
                                    const float *__restrict__ depth, float *__restrict__ rgb_out,
                                    float *__restrict__ depth_out) {
    const int W2 = W / 2, H2 = H / 2;
    const int n = W2 * H2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = i % W2, y = i / W2;
        const size_t q00 = (size_t)(2 * y) * W + 2 * x, q10 = q00 + W;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float *s = rgb + (size_t)ch * W * H;
            rgb_out[(size_t)ch * n + i] = 0.25f * ((s[q00] + s[q00 + 1]) + (s[q10] + s[q10 + 1]));
        }
        if (depth) {
            const float d[4] = {depth[q00], depth[q00 + 1], depth[q10], depth[q10 + 1]};
            float sum = 0.f;
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (d[k] > 0.f) {
                    sum += d[k];
                    ++cnt;
                }
            depth_out[i] = cnt ? sum / (float)cnt : 0.f;
        }
    }
}

// The pyramid level `L` value of pixel (x, y), evaluated from level 0 with the
// arithmetic of L successive pyramid_down_kernel passes (same operations in
// the same order, so the result is bit-identical).
template <int L>
__device__ __forceinline__ float pyr_rgb(const float *__restrict__ s, int W0, int x, int y) {
    if constexpr (L == 0) {
        return s[(size_t)y * W0 + x];
    } else {
        return 0.25f * ((pyr_rgb<L - 1>(s, W0, 2 * x, 2 * y) + pyr_rgb<L - 1>(s, W0, 2 * x + 1, 2 * y)) +
                        (pyr_rgb<L - 1>(s, W0, 2 * x, 2 * y + 1) + pyr_rgb<L - 1>(s, W0, 2 * x + 1, 2 * y + 1)));
    }
}

template <int L>
__device__ __forceinline__ float pyr_depth(const float *__restrict__ d, int W0, int x, int y) {
    if constexpr (L == 0) {
        return d[(size_t)y * W0 + x];
    } else {
        const float v[4] = {pyr_depth<L - 1>(d, W0, 2 * x, 2 * y), pyr_depth<L - 1>(d, W0, 2 * x + 1, 2 * y),
                            pyr_depth<L - 1>(d, W0, 2 * x, 2 * y + 1), pyr_depth<L - 1>(d, W0, 2 * x + 1, 2 * y + 1)};
        float sum = 0.f;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (v[k] > 0.f) {
                sum += v[k];
                ++cnt;
            }
        return cnt ? sum / (float)cnt : 0.f;
    }
}

// Every listed view's target at pyramid level L, straight from level 0, in
// one launch (one instantiation per level keeps the register use of the
// shallow levels low).
template <int L>
__global__ void pyramid_views_kernel(PyrViews pv) {
    const uint32_t total = pv.base[pv.n];
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < pv.n && pv.base[v + 1] <= t) ++v;
        const int W0 = pv.W[v], H0 = pv.H[v];
        const int Wl = W0 >> L;
        const uint32_t i = t - pv.base[v];
        const int x = (int)(i % (uint32_t)Wl), y = (int)(i / (uint32_t)Wl);
        const size_t n = (size_t)Wl * (H0 >> L);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            pv.rgb_out[v][(size_t)ch * n + i] = pyr_rgb<L>(pv.rgb[v] + (size_t)ch * W0 * H0, W0, x, y);
        if (pv.depth[v]) pv.depth_out[v][i] = pyr_depth<L>(pv.depth[v], W0, x, y);
    }
}

Window make_window() {
    Window w;
    double g[11], s = 0.0;
    for (int i = 0; i < 11; ++i) {
        g[i] = std::exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    for (int i = 0; i < 11; ++i) w.w[i] = (float)(g[i] / s);
    return w;
}

} // namespace

// Workspace: derivative maps (9 floats per pixel), their per-view bases,
// tile partials (4 doubles per tile), per-view valid counts.
size_t loss_tmp_bytes(const LossViews &lv) {
    size_t pix = 0;
    for (int v = 0; v < lv.n_views; ++v) pix += (size_t)lv.W[v] * lv.H[v];
    return pix * 9 * sizeof(float) + 256 + (size_t)lv.total_tiles * 4 * sizeof(double) +
           kMaxViews * sizeof(double) + 256;
}

void launch_loss(const LossViews &lv_in, void *tmp, cudaStream_t s) {
    if (lv_in.total_tiles == 0) return;
    LossViews lv = lv_in;
    size_t pix = 0;
    for (int v = 0; v < lv.n_views; ++v) {
        lv.gmap_base[v] = pix * 9;
        pix += (size_t)lv.W[v] * lv.H[v];
    }
    char *base = (char *)tmp;
    float *gmaps = (float *)base;
    size_t off = (pix * 9 * sizeof(float) + 255) / 256 * 256;
    double *partials = (double *)(base + off);
    off += (size_t)lv.total_tiles * 4 * sizeof(double);
    double *nvalid = (double *)(base + off);
    const Window win = make_window();
    loss_pass1_kernel<<<lv.total_tiles, kThreads, 0, s>>>(lv, win, gmaps, partials);
    loss_reduce_kernel<<<lv.n_views, 256, 0, s>>>(lv, partials, nvalid);
    loss_pass2_kernel<<<lv.total_tiles, kThreads, 0, s>>>(lv, win, gmaps, nvalid);
}

void launch_pyramid_down(int W, int H, const float *rgb, const float *depth, float *rgb_out,
                         float *depth_out, cudaStream_t s) {
    const int n = (W / 2) * (H / 2);
    if (n <= 0) return;
    int blocks = (n + 255) / 256;
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    pyramid_down_kernel<<<blocks, 256, 0, s>>>(W, H, rgb, depth, rgb_out, depth_out);
}

void launch_pyramid_views(const PyrViews &pv, int level, cudaStream_t s) {
    const uint32_t total = pv.n > 0 ? pv.base[pv.n] : 0;
    if (total == 0) return;
    int blocks = (int)((total + 255) / 256);
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    switch (level) {
    case 1: pyramid_views_kernel<1><<<blocks, 256, 0, s>>>(pv); break;
    case 2: pyramid_views_kernel<2><<<blocks, 256, 0, s>>>(pv); break;
    case 3: pyramid_views_kernel<3><<<blocks, 256, 0, s>>>(pv); break;
    case 4: pyramid_views_kernel<4><<<blocks, 256, 0, s>>>(pv); break;
    default: break;
    }
}

} // namespace lvigs
