// map.cu -- map maintenance around the differentiable path: the optimiser
// step over every Gaussian parameter, initialisation of new Gaussians from
// colourised LiDAR points with the cumulative-opacity filter on additions,
// and pruning of Gaussians below the prunable opacity (Sec. III-C, III-E).
//
// Adam: one launch over the five parameter buffers, each element read once
// (parameter, gradient, two moments) and written once: HBM-bound, 28 B per
// parameter float (32 B when the gradient is cleared as well).
//
// Initialisation: the centre is the point; the isotropic scale comes from the
// mean squared distance to the three nearest other new points.  The neighbour
// search is exact: points are bucketed in a uniform grid (radix sort by cell)
// and every query scans cubic shells of cells around its own until its third
// distance is inside the scanned radius.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

__device__ __forceinline__ float adam_one(float p, float g, float &m, float &v, float lr, const AdamArgs &A) {
    m = fmaf(A.b1, m, A.omb1 * g);
    v = fmaf(A.b2, v, A.omb2 * (g * g));
    const float denom = sqrtf(v) * A.inv_sqrt_bc2 + A.eps;
    return p - (lr * A.inv_bc1) * m / denom;
}

__device__ __forceinline__ float seg_lr(const AdamSeg &S, int64_t e) {
    if (S.sh_k <= 0) return S.lr;
    return ((e / 3) % S.sh_k) == 0 ? S.lr : S.lr_rest;
}

// Grid-stride over the concatenation of the segments in units of 4 floats.
__global__ void __launch_bounds__(256) adam_kernel(AdamArgs A) {
    const int64_t total = A.unit_base[kAdamSegs];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < total;
         u += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
#pragma unroll
        for (int j = 1; j < kAdamSegs; ++j)
            if (u >= A.unit_base[j]) s = j;
        const AdamSeg &S = A.seg[s];
        const int64_t e0 = (u - A.unit_base[s]) * 4;
        if (S.vec && e0 + 4 <= S.len) {
            float4 p = *(const float4 *)(S.p + e0), g = *(const float4 *)(S.g + e0);
            float4 m = *(const float4 *)(S.m + e0), v = *(const float4 *)(S.v + e0);
            p.x = adam_one(p.x, g.x, m.x, v.x, seg_lr(S, e0), A);
            p.y = adam_one(p.y, g.y, m.y, v.y, seg_lr(S, e0 + 1), A);
            p.z = adam_one(p.z, g.z, m.z, v.z, seg_lr(S, e0 + 2), A);
            p.w = adam_one(p.w, g.w, m.w, v.w, seg_lr(S, e0 + 3), A);
            *(float4 *)(S.p + e0) = p;
            *(float4 *)(S.m + e0) = m;
            *(float4 *)(S.v + e0) = v;
            if (A.zero_grads) *(float4 *)(S.g + e0) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            for (int64_t e = e0; e < e0 + 4 && e < S.len; ++e) {
                float m = S.m[e], v = S.v[e];
                S.p[e] = adam_one(S.p[e], S.g[e], m, v, seg_lr(S, e), A);
                S.m[e] = m;
                S.v[e] = v;
                if (A.zero_grads) S.g[e] = 0.f;
            }
        }
    }
}

// Keep flag of every point (1 = keep) under the cumulative-opacity filter.
// Projection in binary32, one rounding per operation, in this order:
// x_c = ((R00 x + R01 y) + R02 z) + t0 (likewise y_c, z_c); u = (fx x_c) / z_c
// + cx; px = floor(u + 0.5).  Points behind the near plane or outside the
// image are kept.
__global__ void filter_kernel(const float *__restrict__ pts, int64_t k, PointCamera C, const float *__restrict__ alpha,
                              float tau, int literal, uint32_t *__restrict__ keep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(C.R[0], x), __fmul_rn(C.R[1], y)), __fmul_rn(C.R[2], z)), C.t[0]);
        const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(C.R[3], x), __fmul_rn(C.R[4], y)), __fmul_rn(C.R[5], z)), C.t[1]);
        const float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(C.R[6], x), __fmul_rn(C.R[7], y)), __fmul_rn(C.R[8], z)), C.t[2]);
        uint32_t kp = 1;
        if (zc > C.near) {
            const float u = __fadd_rn(__fdiv_rn(__fmul_rn(C.fx, xc), zc), C.cx);
            const float v = __fadd_rn(__fdiv_rn(__fmul_rn(C.fy, yc), zc), C.cy);
            const float fu = floorf(__fadd_rn(u, 0.5f)), fv = floorf(__fadd_rn(v, 0.5f));
            if (fu >= 0.f && fu < (float)C.W && fv >= 0.f && fv < (float)C.H) {
                const float a = alpha[(size_t)fv * C.W + (size_t)fu];
                const bool drop = literal ? (a <= tau) : (__fsub_rn(1.f, a) <= tau);
                kp = drop ? 0u : 1u;
            }
        }
        keep[i] = kp;
    }
}

// Kept points (and colours) to consecutive rows, in their original order.
__global__ void gather_points_kernel(const float *__restrict__ pts, const float *__restrict__ col, int64_t k,
                                     const uint32_t *__restrict__ keep, const uint32_t *__restrict__ offs,
                                     float *__restrict__ pts_out, float *__restrict__ col_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[i]) continue;
        const int64_t o = offs[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pts_out[3 * o + c] = pts[3 * i + c];
            col_out[3 * o + c] = col[3 * i + c];
        }
    }
}

// Ordered-integer image of a float, so that atomicMin / atomicMax on it order
// like the floats (finite values).
__device__ __forceinline__ int ord_of(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}

__global__ void bbox_init_kernel(int *box) {
    if (threadIdx.x < 6) box[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : INT_MIN;
}

// k bounds the points; when count is given, only the first *count are taken.
__global__ void bbox_kernel(const float *__restrict__ pts, int64_t k, const uint32_t *__restrict__ count,
                            int *__restrict__ box) {
    if (count) k = min(k, (int64_t)*count);
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int o = ord_of(pts[3 * i + c]);
            lo[c] = min(lo[c], o);
            hi[c] = max(hi[c], o);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = __reduce_min_sync(0xffffffffu, lo[c]);
        hi[c] = __reduce_max_sync(0xffffffffu, hi[c]);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMin(box + c, lo[c]);
            atomicMax(box + 3 + c, hi[c]);
        }
    }
}

__device__ __forceinline__ int cell_coord(float x, float o, float inv_h, int D) {
    const int c = (int)floorf((x - o) * inv_h);
    return c < 0 ? 0 : (c >= D ? D - 1 : c);
}

__global__ void cell_keys_kernel(const float *__restrict__ pts, int64_t k, KnnGrid G, uint32_t *__restrict__ keys,
                                 uint32_t *__restrict__ vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int cx = cell_coord(pts[3 * i], G.o[0], G.inv_h, G.D[0]);
        const int cy = cell_coord(pts[3 * i + 1], G.o[1], G.inv_h, G.D[1]);
        const int cz = cell_coord(pts[3 * i + 2], G.o[2], G.inv_h, G.D[2]);
        keys[i] = ((uint32_t)cz * (uint32_t)G.D[1] + (uint32_t)cy) * (uint32_t)G.D[0] + (uint32_t)cx;
        vals[i] = (uint32_t)i;
    }
}

__device__ __forceinline__ void push3(float d, float best[3], int &cnt) {
    if (cnt < 3) ++cnt;
    if (d < best[2]) {
        if (d < best[1]) {
            best[2] = best[1];
            if (d < best[0]) {
                best[1] = best[0];
                best[0] = d;
            } else {
                best[1] = d;
            }
        } else {
            best[2] = d;
        }
    }
}

// Points in cell order, with the position of each in the input as .w bits.
__global__ void gather_sorted_kernel(const float *__restrict__ pts, int64_t k, const uint32_t *__restrict__ order,
                                     float4 *__restrict__ spts) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = order[j];
        spts[j] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __uint_as_float(i));
    }
}

// Lane-parallel scan of the points of the cells in x-row [x0, x1] of (cy, cz):
// the lanes read the row's cell ranges together (the cells of a row are
// consecutive ids, so their points are one run of the sorted order), then
// split the run; each lane keeps its own three smallest squared distances.
__device__ __forceinline__ void scan_row_warp(const float4 *__restrict__ spts, const uint2 *__restrict__ cells,
                                              const KnnGrid &G, int cy, int cz, int x0, int x1, uint32_t self,
                                              float qx, float qy, float qz, float best[3], int &cnt, int lane) {
    x0 = max(x0, 0);
    x1 = min(x1, G.D[0] - 1);
    if (cy < 0 || cy >= G.D[1] || cz < 0 || cz >= G.D[2] || x0 > x1) return;
    const uint32_t row = ((uint32_t)cz * (uint32_t)G.D[1] + (uint32_t)cy) * (uint32_t)G.D[0];
    uint32_t start = 0xffffffffu, end = 0;
    for (int xb = x0; xb <= x1; xb += 32) {
        const int x = xb + lane;
        uint2 r = make_uint2(0, 0);
        if (x <= x1) r = cells[row + x];
        const unsigned nz = __ballot_sync(0xffffffffu, r.y > r.x);
        if (nz) {
            const uint32_t first = __shfl_sync(0xffffffffu, r.x, __ffs(nz) - 1);
            const uint32_t last = __shfl_sync(0xffffffffu, r.y, 31 - __clz(nz));
            if (start == 0xffffffffu) start = first;
            end = last;
        }
    }
    if (start == 0xffffffffu) return;
    for (uint32_t j = start + lane; j < end; j += 32) {
        if (j == self) continue;
        const float4 p = spts[j];
        const float dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
        push3(dx * dx + dy * dy + dz * dz, best, cnt);
    }
}

// The warp's three smallest of the lanes' lists (as a multiset, ascending)
// and how many candidates the warp has seen, capped at 3.
__device__ __forceinline__ void warp_top3(const float best[3], int cnt, int lane, float top[3], int &tot) {
    int head = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float mine = head == 0 ? best[0] : (head == 1 ? best[1] : (head == 2 ? best[2] : INFINITY));
        float m = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        top[q] = m;
        const unsigned own = __ballot_sync(0xffffffffu, mine == m && head < 3);
        if (own && lane == __ffs(own) - 1) ++head;
    }
    int c = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    tot = min(c, 3);
}

// One warp per point, in cell order (neighbouring warps scan the same cells).
// After the shells up to r are scanned, every point within r*h of the query
// has been seen (same cell arithmetic for all points; 0.99 absorbs the
// binary32 rounding of the cell coordinates), so the search stops once the
// wanted neighbours are all within that radius.
__global__ void __launch_bounds__(256, 4) knn_kernel(const float4 *__restrict__ spts, int64_t k, KnnGrid G,
                                                  const uint2 *__restrict__ cells, float min_dist2,
                                                  float *__restrict__ log_scales_out) {
    const int lane = threadIdx.x & 31;
    const int want = (int)(k - 1 < 3 ? k - 1 : 3);
    const int rmax = max(G.D[0], max(G.D[1], G.D[2]));
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); j < k; j += warps) {
        const float4 q = spts[j];
        const int cx = cell_coord(q.x, G.o[0], G.inv_h, G.D[0]);
        const int cy = cell_coord(q.y, G.o[1], G.inv_h, G.D[1]);
        const int cz = cell_coord(q.z, G.o[2], G.inv_h, G.D[2]);
        float best[3] = {INFINITY, INFINITY, INFINITY};
        float top[3] = {INFINITY, INFINITY, INFINITY};
        int cnt = 0;
        const uint32_t self = (uint32_t)j;
        if (want > 0) {
            for (int r = 0; r <= rmax; ++r) {
                for (int dz = -r; dz <= r; ++dz) {
                    const bool zface = (dz == -r || dz == r);
                    for (int dy = -r; dy <= r; ++dy) {
                        if (zface || dy == -r || dy == r) {
                            scan_row_warp(spts, cells, G, cy + dy, cz + dz, cx - r, cx + r, self, q.x, q.y, q.z,
                                          best, cnt, lane);
                        } else {
                            scan_row_warp(spts, cells, G, cy + dy, cz + dz, cx - r, cx - r, self, q.x, q.y, q.z,
                                          best, cnt, lane);
                            if (r > 0)
                                scan_row_warp(spts, cells, G, cy + dy, cz + dz, cx + r, cx + r, self, q.x, q.y, q.z,
                                              best, cnt, lane);
                        }
                    }
                }
                int tot;
                warp_top3(best, cnt, lane, top, tot);
                const float rad = 0.99f * (float)r * G.h;
                const float worst = want == 1 ? top[0] : (want == 2 ? top[1] : top[2]);
                if (tot >= want && worst <= rad * rad) break;
            }
        }
        if (lane == 0) {
            float mean = 0.f;
            if (want > 0) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    if (t < want) acc += top[t];
                mean = acc / (float)want;
            }
            log_scales_out[__float_as_uint(q.w)] = 0.5f * logf(fmaxf(mean, min_dist2));
        }
    }
}

// Rows [n0, n0 + k) of the parameter buffers from the kept points.
__global__ void init_rows_kernel(const float *__restrict__ pts, const float *__restrict__ col,
                                 const float *__restrict__ log_s, int64_t k, int64_t n0, ParamBufs P, ParamBufs M,
                                 ParamBufs V, int K, float opacity_logit, float inv_c0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = n0 + i;
        const float ls = log_s[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P.means[3 * r + c] = pts[3 * i + c];
            P.log_scales[3 * r + c] = ls;
        }
        P.quats[4 * r] = 1.f;
        P.quats[4 * r + 1] = 0.f;
        P.quats[4 * r + 2] = 0.f;
        P.quats[4 * r + 3] = 0.f;
        P.opacity_logits[r] = opacity_logit;
        float *sh = P.sh + (size_t)r * K * 3;
        for (int c = 0; c < 3; ++c) sh[c] = (col[3 * i + c] - 0.5f) * inv_c0;
        for (int e = 3; e < K * 3; ++e) sh[e] = 0.f;
        const ParamBufs *st[2] = {&M, &V};
        for (int q = 0; q < 2; ++q) {
            const ParamBufs &S = *st[q];
            if (!S.means) continue;
            for (int c = 0; c < 3; ++c) {
                S.means[3 * r + c] = 0.f;
                S.log_scales[3 * r + c] = 0.f;
            }
            for (int c = 0; c < 4; ++c) S.quats[4 * r + c] = 0.f;
            S.opacity_logits[r] = 0.f;
            for (int e = 0; e < K * 3; ++e) S.sh[(size_t)r * K * 3 + e] = 0.f;
        }
    }
}

__global__ void set_u32_kernel(uint32_t *p, uint32_t v) { *p = v; }

__global__ void prune_flags_kernel(const float *__restrict__ logits, int64_t n, float thr, uint32_t *__restrict__ keep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keep[i] = logits[i] >= thr ? 1u : 0u;
}

// Pruning, first pass: the kept rows of every buffer (blockIdx.y picks the
// buffer) to consecutive rows of its scratch segment.  Rows are taken in
// chunks of kPruneRows whose keep flags and destinations are staged in shared
// memory; an element's row comes from a product with 1/w, corrected to the
// exact quotient.  Nothing is done when every row is kept (offs[n] == n).
constexpr int kPruneRows = 256;
__global__ void __launch_bounds__(256) prune_compact_kernel(PruneArgs A) {
    __shared__ uint32_t s_keep[kPruneRows], s_offs[kPruneRows];
    const int64_t n = A.n;
    if ((int64_t)A.offs[n] == n) return;
    const PruneSeg S = A.seg[blockIdx.y];
    const uint32_t w = (uint32_t)S.w;
    const float inv_w = 1.f / (float)w;
    for (int64_t r0 = (int64_t)blockIdx.x * kPruneRows; r0 < n; r0 += (int64_t)gridDim.x * kPruneRows) {
        const uint32_t rows = (uint32_t)min((int64_t)kPruneRows, n - r0);
        __syncthreads(); // the previous chunk's flags are no longer read
        for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) {
            s_keep[i] = A.keep[r0 + i];
            s_offs[i] = A.offs[r0 + i];
        }
        __syncthreads();
        const float *src = S.buf + r0 * w;
        for (uint32_t e = threadIdx.x; e < rows * w; e += blockDim.x) {
            uint32_t r = __float2uint_rz(((float)e + 0.5f) * inv_w);
            if (r * w > e) --r;
            else if ((r + 1) * w <= e) ++r;
            if (s_keep[r]) S.tmp[(int64_t)s_offs[r] * w + (e - r * w)] = src[e];
        }
    }
}

// Second pass: the first offs[n] rows of each scratch segment back over the
// buffer (float4 where the buffer allows it; the segments are 16-byte aligned).
__global__ void __launch_bounds__(256) prune_copy_back_kernel(PruneArgs A) {
    const int64_t n = A.n;
    const int64_t kept = A.offs[n];
    if (kept == n) return;
    const PruneSeg S = A.seg[blockIdx.y];
    const int64_t len = kept * S.w;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (S.vec) {
        const int64_t units = len >> 2;
        for (int64_t u = t0; u < units; u += stride)
            ((float4 *)S.buf)[u] = ((const float4 *)S.tmp)[u];
        for (int64_t e = (units << 2) + t0; e < len; e += stride) S.buf[e] = S.tmp[e];
    } else {
        for (int64_t e = t0; e < len; e += stride) S.buf[e] = S.tmp[e];
    }
}

int blocks_for(int64_t n, int threads, int per_sm = 8) {
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

} // namespace

void launch_adam(const AdamArgs &A, cudaStream_t s) {
    if (A.unit_base[kAdamSegs] == 0) return;
    adam_kernel<<<blocks_for(A.unit_base[kAdamSegs], 256, 16), 256, 0, s>>>(A);
}

void launch_point_filter(const float *pts, int64_t k, const PointCamera &C, const float *alpha, float tau, int literal,
                         uint32_t *keep, cudaStream_t s) {
    if (k <= 0) return;
    filter_kernel<<<blocks_for(k, 256), 256, 0, s>>>(pts, k, C, alpha, tau, literal, keep);
}

void launch_gather_points(const float *pts, const float *col, int64_t k, const uint32_t *keep, const uint32_t *offs,
                          float *pts_out, float *col_out, cudaStream_t s) {
    if (k <= 0) return;
    gather_points_kernel<<<blocks_for(k, 256), 256, 0, s>>>(pts, col, k, keep, offs, pts_out, col_out);
}

void launch_bbox(const float *pts, int64_t k, const uint32_t *count, int *box, cudaStream_t s) {
    bbox_init_kernel<<<1, 32, 0, s>>>(box);
    if (k <= 0) return;
    bbox_kernel<<<blocks_for(k, 256), 256, 0, s>>>(pts, k, count, box);
}

float ord_to_float(int o) {
    const int b = o >= 0 ? o : (o ^ 0x7fffffff);
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

void launch_cell_keys(const float *pts, int64_t k, const KnnGrid &G, uint32_t *keys, uint32_t *vals, cudaStream_t s) {
    if (k <= 0) return;
    cell_keys_kernel<<<blocks_for(k, 256), 256, 0, s>>>(pts, k, G, keys, vals);
}

void launch_knn(const float *pts, int64_t k, const KnnGrid &G, const uint2 *cells, const uint32_t *order,
                float4 *spts, float min_dist2, float *log_scales_out, cudaStream_t s) {
    if (k <= 0) return;
    gather_sorted_kernel<<<blocks_for(k, 256), 256, 0, s>>>(pts, k, order, spts);
    knn_kernel<<<blocks_for(k * 32, 256), 256, 0, s>>>(spts, k, G, cells, min_dist2, log_scales_out);
}

void launch_init_rows(const float *pts, const float *col, const float *log_s, int64_t k, int64_t n0,
                      const ParamBufs &P, const ParamBufs &M, const ParamBufs &V, int K, float opacity_logit,
                      float inv_c0, cudaStream_t s) {
    if (k <= 0) return;
    init_rows_kernel<<<blocks_for(k, 128), 128, 0, s>>>(pts, col, log_s, k, n0, P, M, V, K, opacity_logit, inv_c0);
}

void launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t s) { set_u32_kernel<<<1, 1, 0, s>>>(p, v); }

void launch_prune_flags(const float *logits, int64_t n, float thr, uint32_t *keep, cudaStream_t s) {
    if (n <= 0) return;
    prune_flags_kernel<<<blocks_for(n, 256), 256, 0, s>>>(logits, n, thr, keep);
}

void launch_prune_compact(const PruneArgs &A, cudaStream_t s) {
    if (A.n <= 0 || A.nseg <= 0) return;
    // a full grid for every buffer: the SH buffers hold most of the bytes and
    // need many loads in flight; the blocks of the small ones finish early
    const int sms = device_sm_count();
    const int64_t chunks = (A.n + kPruneRows - 1) / kPruneRows;
    const int gx1 = (int)std::min<int64_t>(chunks, (int64_t)sms * 8);
    prune_compact_kernel<<<dim3(gx1, A.nseg), 256, 0, s>>>(A);
    prune_copy_back_kernel<<<dim3(sms * 8, A.nseg), 256, 0, s>>>(A);
}

} // namespace lvigs
