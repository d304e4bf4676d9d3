// lvigs_internal.cuh -- device-side structures shared by the kernels of the
// GB300 Gaussian-splatting hot path.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lvigs {

constexpr int kMaxViews = 32;

// Status bits latched on the device and read back by lvigs_sync_status.
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// One view at its pyramid level, as the kernels see it.
struct ViewDesc {
    float R[9];         // world -> camera rotation, row-major (Q_iw of Eq. 7)
    float t[3];         // world -> camera translation (T_iw of Eq. 7)
    float fx, fy, cx, cy;
    float limx, limy;   // Jacobian clamp: 1.3 * tan(half field of view)
    float campos[3];    // camera centre in world coordinates (SH view direction)
    int W, H;
    int tiles_x, tiles_y;
    uint32_t tile_base; // first global tile id of this view
    uint32_t pix_base;  // first pixel of this view in packed per-pixel buffers
};

struct ViewSet {
    int n_views;
    int tile_w, tile_h;
    uint32_t total_tiles;
    uint32_t total_pixels;
    ViewDesc v[kMaxViews];
};

// Per-view image pointers (device).
struct ViewImages {
    float *rgb[kMaxViews];
    float *depth[kMaxViews];
    float *alpha[kMaxViews];
};

struct ViewGrads {
    const float *d_rgb[kMaxViews];
    const float *d_depth[kMaxViews];
    const float *d_alpha[kMaxViews]; // may be null
};

// Gaussian parameters (device, SoA, caller-owned).
struct GaussParams {
    const float *means, *log_scales, *quats, *opacity_logits, *sh;
    int n;
    int sh_degree;
    int sh_stride_k;
};

struct ParamGrads {
    float *d_means, *d_log_scales, *d_quats, *d_opacity_logits, *d_sh;
    int accumulate;
};

// Screen-space record of one (view, Gaussian), written by preprocessing and
// gathered by the compositing kernels: a = (u, v, a2, b2), b = (c2, lo, z, ex),
// c = (r, g, b, ey).  With the conic [[A, B], [B, C]], the Gaussian's exponent
// at offset (dx, dy) = (u - px, v - py) is power = -(A dx^2 + C dy^2)/2
// - B dx dy; the record holds it in base 2, a2 = -A log2(e) / 2,
// b2 = -B log2(e), c2 = -C log2(e) / 2, together with lo = log2(opacity), so
// that o exp(power) = 2^(a2 dx^2 + b2 dx dy + c2 dy^2 + lo): the 1/255 test is
// a test of that exponent, taken before the exponential.  (ex, ey) are the
// half-extents of a box that holds every pixel where alpha can reach 1/255.
struct __align__(16) GRec {
    float4 a, b, c;
};

// Screen-space gradient sums of one (view, Gaussian) over its pixels, with
// dp = dL/dpower and (dx, dy) = (u - px, v - py):
// g0 = (sum dp dx, sum dp dy, sum dp dx^2, sum dp dx dy),
// g1 = (sum dp dy^2, dL/dopacity, dL/dz, -), g2 = (dL/dr, dL/dg, dL/db, clamp
// word).  The clamp word is the bit pattern kClampKnown | (bit c set when colour
// channel c was clamped at 0) when forward preprocessing cleared the record,
// else 0 (the backward preprocessing then re-evaluates the colour).
// Since power = -(A dx^2 + C dy^2)/2 - B dx dy, the conic gradients follow per
// Gaussian: dL/du = -(A m_x + B m_y), dL/dv = -(C m_y + B m_x),
// dL/dA = -m_xx / 2, dL/dB = -m_xy, dL/dC = -m_yy / 2.
struct __align__(16) GGrad {
    float4 g0, g1, g2;
};
constexpr uint32_t kClampKnown = 0x40000000u;

__host__ __device__ inline int view_of_tile(const ViewSet &vs, uint32_t gt) {
    int v = 0;
#pragma unroll 1
    for (int i = 1; i < vs.n_views; ++i)
        if (vs.v[i].tile_base <= gt) v = i;
    return v;
}

// Alpha of Eq. (6) at pixel offset (dx, dy) = (u - px, v - py).  Written with
// explicit rounding so the forward and backward kernels take identical
// branches on the 0.99 / (1/255) tests.
// log2(o exp(power)) at offset (dx, dy) from the record's coefficients,
// given a2dx = a2 * dx (shared by the pixels of a column) and lo = log2(o):
// dx (a2 dx + b2 dy) + ((c2 dy) dy + lo), explicitly rounded so every kernel
// gets the same bits.
__device__ __forceinline__ float gauss_exponent2(float a2dx, float b2, float c2, float lo, float dx, float dy) {
    return __fmaf_rn(dx, __fmaf_rn(b2, dy, a2dx), __fmaf_rn(__fmul_rn(c2, dy), dy, lo));
}

// log2(1/255): alpha = min(0.99, 2^e) reaches 1/255 exactly when e >= this
constexpr float kLog2AlphaMin = -7.99435343685885793770f;

// 2^x by the hardware approximation (relative error about 2^-22).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

} // namespace lvigs

// May a kernel write through p?  Device or managed memory, or page-locked
// host memory (mapped into the device's address space).  Host-only query.
inline bool kernel_writable(const void *p) {
    cudaPointerAttributes pa{};
    const cudaError_t e = cudaPointerGetAttributes(&pa, p);
    cudaGetLastError();
    return e == cudaSuccess &&
           (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged || pa.type == cudaMemoryTypeHost);
}

// Streaming multiprocessors of the current device (queried once per device):
// grid-stride kernels cap their grids at a multiple of it.
inline int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 1;
    }
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        cache[dev] = v;
    }
    return cache[dev];
}

// Kernel launchers (defined in the .cu files, called from the host API).
namespace lvigs {

// ViewSet pointers passed to kernels are DEVICE copies; the host copy (by
// reference) is only used to size grids.
// Table and constants of the key stage's binary32 exponential.
struct ExpKeyTable {
    float hi[32], lo[32]; // 2^(j/32) = hi + lo
    float inv_step;       // 32 / ln 2
    float c1, c2, c3;     // ln2 / 32 = c1 + c2 + c3 (c1, c2: 12 significant bits)
};
// y[i] = (float)exp((double)x[i]) as the key stage evaluates it (parity hook).
void launch_exp_key(const float *x, float *y, int64_t n, cudaStream_t s);

// g2d_init (may be null): the per-pair gradient records of the backward, cleared
// here for every pair that has tiles, with its colour clamp word.
void launch_preprocess_fwd(const GaussParams &P, const ViewSet *vs_dev, GRec *recs, uint32_t *tiles,
                           uint32_t *zbits, uint2 *rects, GGrad *g2d_init, cudaStream_t s);
void launch_preprocess_bwd(const GaussParams &P, const ViewSet *vs_dev, const uint32_t *tiles,
                           const GGrad *g2d, const ParamGrads &G, cudaStream_t s);

// Device-wide exclusive scan of n items (n read from the device when n_dev is
// non-null, else n_host).  in[i] is gathered as in[gather[i]] when gather is
// non-null; with flag_only the item is (in[i] != 0).  Writes out[i] and, at
// out_total, the total.  tmp needs scan_tmp_words(n_host) uint32 words.
size_t scan_tmp_words(int64_t n_max);
void launch_scan(const uint32_t *in, const uint32_t *gather, int flag_only, uint32_t *out,
                 uint32_t *out_total, const uint32_t *n_dev, int64_t n_max, uint32_t *tmp,
                 cudaStream_t s);

// Compaction of the visible (tiles > 0) items in index order: keys = zbits[i],
// vals = i; out_total receives their count.  tmp as for launch_scan.
void launch_compact_scan(const uint32_t *tiles, const uint32_t *zbits, uint32_t *keys, uint32_t *vals,
                         uint32_t *out_total, int64_t n, uint32_t *tmp, cudaStream_t s);

// LSD radix sort of (key, value) pairs over bits [0, bits).  Stable.
// n read from the device (n_dev), or n_max when n_dev is null.  Returns 1 when
// the result ends in the alt buffers.
size_t radix_tmp_words(int64_t n_max);
int launch_radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                       const uint32_t *n_dev, int64_t n_max, int bits, uint32_t *tmp,
                       cudaStream_t s);

void launch_emit(const ViewSet *vs_dev, const uint32_t *sorted_idx, const uint32_t *offsets,
                 const uint32_t *n_vis_dev, const uint2 *rects, int n_gauss, uint32_t *tile_ids,
                 uint32_t *inst_vals, int64_t m_cap, int64_t n_max, uint32_t *status,
                 cudaStream_t s);
void launch_ranges(const uint32_t *tile_ids, const uint32_t *m_dev, int64_t m_cap,
                   uint2 *ranges, uint32_t total_tiles, cudaStream_t s);
void launch_sum_i32(const int32_t *x, uint32_t n, unsigned long long *out, cudaStream_t s);
void launch_clamp_count(const uint32_t *m_dev, int64_t m_cap, uint32_t *out, cudaStream_t s);
void launch_debug_keys(const uint32_t *tile_ids, const uint32_t *inst_vals, const uint32_t *zbits,
                       int n_gauss, uint64_t *keys, uint32_t *vals, int64_t m, cudaStream_t s);

// List-parallel compositing plan (device arrays, built after the tile ranges):
// each tile's list is cut into chunks of L entries; (tile, chunk) pairs are
// numbered tile by tile; tiles with more than one chunk own `n_chunks` slots
// of per-pixel partial state.
struct ChunkPlan {
    int L;
    const uint32_t *n_chunks;   // [tiles]
    const uint32_t *chunk_base; // [tiles] first pair of the tile
    const uint32_t *part_base;  // [tiles] first slot of a multi-chunk tile
    const uint32_t *pair_tile;  // [pair_cap] tile of each pair
    const uint32_t *n_pairs;    // device count of pairs
    const uint32_t *n_fwd;      // device count of the forward's items (pairs in its order)
    const uint32_t *n_inst;     // device count of the instances in the lists
    int nb;                     // 8x8 blocks per tile
    uint32_t warps;             // warps the compositing kernels keep resident
    float *part;                // [slot_cap] slots: 8 checkpoint groups of 6 x tile_w x tile_h floats
    uint32_t pair_cap, slot_cap;
    const uint32_t *pair_order; // [pair_cap] work order (chunk-major), or null
    uint32_t *stop_at;          // [total pixels] first chunk with a local stop (reset to ~0)
    uint32_t *stop_items;       // [pair_cap * 8x8 blocks per tile] (pair, block) items with a stop
    uint32_t *n_stop;           // device count of stop_items
};
// The plan from the tile ranges: n_chunks, chunk_base, part_base and
// pair_tile of cp, counters[4] = pairs, counters[5] = slots, and the
// chunk-major forward work order in `order`; capacity overflow is latched.
// aux: plan_aux_bytes(n_tiles) of scratch.
size_t plan_aux_bytes(uint32_t n_tiles);
void launch_plan(const ChunkPlan &cp, const uint2 *ranges, uint32_t n_tiles, uint32_t *counters, uint32_t *order,
                 uint32_t *aux, uint32_t *status, cudaStream_t s);
// order[0, n) = the pairs by the 8-bit keys of launch_bwd_pair_keys (n =
// min(*n_dev, cap)), with the bucket starts it left in aux.
void launch_bucket_place(const uint32_t *keys, const uint32_t *n_dev, uint32_t cap, uint32_t *aux, uint32_t *order,
                         cudaStream_t s);
size_t chunk_slot_bytes(int tile_w, int tile_h);
// Keys of the backward work order (8 bits: L - expected walk of each pair).
void launch_bwd_pair_keys(const ViewSet &vs, const ViewSet *vsd, const ChunkPlan &cp, const int32_t *n_contrib,
                          uint32_t *keys, uint32_t *aux, cudaStream_t s);

// Compositing: persistent warps, one (tile, chunk, 8x8 block) per work item;
// each stages 32 * bm Gaussians per round (bm = 1 or 2).  `queue` is one device
// word (the work counter; reset by the launcher).
// pix_state: pix_state_bytes() per pixel of the view set (forward scratch).
// `part` of launch_composite_fwd: any of the bits below, in this order: the
// chunk walks (phase 1), the combine and exact stop walks (the images are
// final after it), the state each backward chunk walk starts from.
constexpr int kFwdWalk = 1, kFwdCombine = 2, kFwdBackwardState = 4;
size_t pix_state_bytes();
void launch_composite_fwd(const ViewSet &vs, const ViewSet *vs_dev, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewImages &out, float *final_T, int32_t *n_contrib,
                          const ChunkPlan &cp, uint32_t *queue, void *pix_state, cudaStream_t s, int bm,
                          int part);
void launch_composite_bwd(const ViewSet &vs, const ViewSet *vs_dev, const uint2 *ranges, const uint32_t *inst_vals,
                          const GRec *recs, const ViewGrads &g, const float *final_T, const int32_t *n_contrib,
                          GGrad *g2d, const ChunkPlan &cp, uint32_t *queue, cudaStream_t s, int bm);

// Loss (Eq. 10-12) over one or more views (packed per view through the arrays).
// The loss kernels work on square tiles of kLossTile pixels.
constexpr int kLossTile = 32;
inline uint32_t loss_tile_count(int W, int H) {
    return (uint32_t)(((W + kLossTile - 1) / kLossTile) * ((H + kLossTile - 1) / kLossTile));
}
struct LossViews {
    int n_views;
    int W[kMaxViews], H[kMaxViews];
    uint32_t tile_base[kMaxViews]; // first loss tile of each view
    uint32_t total_tiles;
    const float *rgb[kMaxViews];
    const float *depth[kMaxViews];
    const float *gt[kMaxViews];
    const float *lidar[kMaxViews];
    float *d_rgb[kMaxViews];
    float *d_depth[kMaxViews];
    double *loss_out[kMaxViews];
    float lambda_ssim, lambda_depth;
    size_t gmap_base[kMaxViews]; // filled by launch_loss
};
size_t loss_tmp_bytes(const LossViews &lv);
void launch_loss(const LossViews &lv, void *tmp, cudaStream_t s);

void launch_pyramid_down(int W, int H, const float *rgb, const float *depth, float *rgb_out,
                         float *depth_out, cudaStream_t s);

// Targets of several views at one pyramid level (1..4) in one launch,
// bit-identical to repeated launch_pyramid_down.  W, H: level-0 size; base:
// prefix of the output pixel counts.
struct PyrViews {
    int n;
    int W[kMaxViews], H[kMaxViews];
    const float *rgb[kMaxViews];
    const float *depth[kMaxViews]; // may be null
    float *rgb_out[kMaxViews];
    float *depth_out[kMaxViews];
    uint32_t base[kMaxViews + 1];
};
void launch_pyramid_views(const PyrViews &pv, int level, cudaStream_t s);

// ---- map maintenance (map.cu) ----
// Five parameter-shaped buffers (layouts of the Gaussian parameters).
struct ParamBufs {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
};

constexpr int kAdamSegs = 5;
struct AdamSeg {
    float *p, *g, *m, *v;
    int64_t len;     // floats
    float lr, lr_rest; // lr_rest: SH coefficients other than band 0
    int sh_k;        // coefficients per Gaussian for the SH segment, 0 otherwise
    int vec;         // all four pointers 16-byte aligned
};
struct AdamArgs {
    AdamSeg seg[kAdamSegs];
    int64_t unit_base[kAdamSegs + 1]; // prefix of ceil(len / 4)
    float b1, b2, omb1, omb2, eps; // omb = 1 - b, formed in double
    float inv_bc1, inv_sqrt_bc2;   // 1 / (1 - b1^t), 1 / sqrt(1 - b2^t)
    int zero_grads;
};
void launch_adam(const AdamArgs &A, cudaStream_t s);

// Level camera for the point filter.
struct PointCamera {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int W, H;
    float near;
};
void launch_point_filter(const float *pts, int64_t k, const PointCamera &C, const float *alpha, float tau, int literal,
                         uint32_t *keep, cudaStream_t s);
void launch_gather_points(const float *pts, const float *col, int64_t k, const uint32_t *keep, const uint32_t *offs,
                          float *pts_out, float *col_out, cudaStream_t s);
// box: 6 ints, ordered-integer images of (min xyz, max xyz); ord_to_float decodes them.
// With count (device, may be null) only the first *count of the k points are taken.
void launch_bbox(const float *pts, int64_t k, const uint32_t *count, int *box, cudaStream_t s);
float ord_to_float(int o);

// Uniform grid of the neighbour search: origin o, cell size h, D cells per axis.
struct KnnGrid {
    float o[3];
    float h, inv_h;
    int D[3];
};
void launch_cell_keys(const float *pts, int64_t k, const KnnGrid &G, uint32_t *keys, uint32_t *vals, cudaStream_t s);
// spts: k float4 of scratch (the points in cell order).
void launch_knn(const float *pts, int64_t k, const KnnGrid &G, const uint2 *cells, const uint32_t *order,
                float4 *spts, float min_dist2, float *log_scales_out, cudaStream_t s);
void launch_init_rows(const float *pts, const float *col, const float *log_s, int64_t k, int64_t n0,
                      const ParamBufs &P, const ParamBufs &M, const ParamBufs &V, int K, float opacity_logit,
                      float inv_c0, cudaStream_t s);
void launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t s);
void launch_prune_flags(const float *logits, int64_t n, float thr, uint32_t *keep, cudaStream_t s);
// Pruning of up to three sets of the five parameter buffers at once: kept
// rows (keep[r] = 1) move to row offs[r]; the kept count offs[n] is read on
// the device.  tmp: a scratch segment per buffer (n * w floats, 16-byte aligned).
constexpr int kPruneSegs = 15;
struct PruneSeg {
    float *buf, *tmp;
    int w;   // floats per row
    int vec; // buf 16-byte aligned
};
struct PruneArgs {
    PruneSeg seg[kPruneSegs];
    int nseg;
    int64_t n;
    const uint32_t *keep, *offs;
};
void launch_prune_compact(const PruneArgs &A, cudaStream_t s);

} // namespace lvigs
