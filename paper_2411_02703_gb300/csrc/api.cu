// api.cu -- the C ABI of include/lvigs.h: contexts and their workspace, the
// plain single-view path (render / loss / backward), the batched path that
// replays one CUDA graph per step, and the parity hooks.
//
// Host arithmetic that feeds the tile keys (the pyramid-level intrinsics and
// the Jacobian clamp limits) is plain binary32 C++ compiled with
// -ffp-contract=off, one rounding per operation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lvigs.h"
#include "lvigs_internal.cuh"

using namespace lvigs;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Tile lists longer than this are composited by several warps in parallel.
constexpr int kChunkLen = 1024;
// Pinned staging copies of the view descriptors.
constexpr int kVsRing = 8;

struct RenderState {
    DevBuf recs, tiles, zbits, rects;
    DevBuf inst_a_t, inst_a_v, inst_b_t, inst_b_v;
    DevBuf ranges, final_T, n_contrib, vs_dev, counters;
    DevBuf n_chunks, chunk_base, part_base, pair_tile, part; // list-parallel plan
    DevBuf pair_k, pair_v, pair_v2, stop_at, plan_aux;       // work orders, stop record
    DevBuf stop_items;                                       // forward stop walks
    DevBuf pix_state;                                                 // forward combine scratch
    uint32_t pair_cap = 0, slot_cap = 0;
    ViewSet vs{};
    GaussParams P{};
    int64_t m = 0;      // instances of the last eager build
    int64_t m_cap = 0;  // instance capacity
    int sorted_in_b = 0;
    bool valid = false;
    uint32_t generation = 0;

    const uint32_t *sorted_tiles() const { return (const uint32_t *)(sorted_in_b ? inst_b_t.p : inst_a_t.p); }
    ChunkPlan plan() const {
        ChunkPlan cp;
        cp.L = kChunkLen;
        cp.n_chunks = (const uint32_t *)n_chunks.p;
        cp.chunk_base = (const uint32_t *)chunk_base.p;
        cp.part_base = (const uint32_t *)part_base.p;
        cp.pair_tile = (const uint32_t *)pair_tile.p;
        cp.n_pairs = (const uint32_t *)counters.p + 4;
        cp.n_fwd = (const uint32_t *)counters.p + 7;
        cp.n_inst = (const uint32_t *)counters.p + 2;
        cp.nb = (vs.tile_w / 8) * (vs.tile_h / 8);
        cp.warps = (uint32_t)device_sm_count() * 24; // six 4-warp CTAs per SM
        cp.part = (float *)part.p;
        cp.pair_cap = pair_cap;
        cp.slot_cap = slot_cap;
        cp.pair_order = (const uint32_t *)pair_v.p;
        cp.stop_at = (uint32_t *)stop_at.p;
        cp.stop_items = (uint32_t *)stop_items.p;
        cp.n_stop = (uint32_t *)counters.p + 6;
        return cp;
    }
    const uint32_t *sorted_vals() const { return (const uint32_t *)(sorted_in_b ? inst_b_v.p : inst_a_v.p); }
};

struct BatchKey {
    std::vector<uint64_t> k;
    bool operator==(const BatchKey &o) const { return k == o.k; }
};

} // namespace

struct lvigs_ctx {
    lvigs_config cfg{};
    int bm = 2; // Gaussians staged per compositing round = bm x threads
    int device = 0;
    std::string err;
    size_t bytes_in_use = 0;
    uint64_t ws_epoch = 0;
    bool capturing = false;
    bool capture_short = false;

    // shared temporaries (one stream at a time per context)
    DevBuf pos, ck, cv, ck2, cv2, scan_tmp, radix_tmp, status, g2d, loss_tmp, stats;
    uint32_t *host_counters = nullptr; // pinned [8]
    uint32_t *host_status = nullptr;   // pinned [1]

    std::vector<RenderState *> slots;

    // batched path
    RenderState batch;
    DevBuf gt_stage[kMaxViews], lidar_stage[kMaxViews];
    DevBuf pyr_rgb[kMaxViews][LVIGS_MAX_LEVEL + 1], pyr_depth[kMaxViews][LVIGS_MAX_LEVEL + 1];
    DevBuf img_rgb, img_depth, img_alpha, d_rgb, d_depth;
    double *host_losses = nullptr;       // pinned [kMaxViews * 4]
    uint32_t *host_batch_counters = nullptr; // pinned [4]
    // pinned staging copies of the view descriptors, used in turn: an upload
    // waits only for the one kVsRing uploads earlier
    ViewSet *vs_staging = nullptr;       // pinned [kVsRing]
    cudaEvent_t vs_event[kVsRing] = {};
    int vs_next = 0;
    cudaEvent_t step_event = nullptr;
    // instance capacity of the largest plain render sized so far (the size a
    // render that does not wait starts from)
    int64_t render_m_cap = 0;
    bool step_pending = false;
    cudaStream_t cap_stream = nullptr;
    // second stream of the batched step: the target pyramid, and the backward's
    // start state and work order, run beside the main chain (graph branches)
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev[4] = {};
    // one graph for steps with their own targets, one per staging slot
    cudaGraphExec_t graph_exec[1 + LVIGS_STAGE_SLOTS] = {};
    BatchKey graph_key[1 + LVIGS_STAGE_SLOTS];
    BatchKey sized_shape; // the step shape the instance capacity was last sized for
    bool graph_ok[1 + LVIGS_STAGE_SLOTS] = {};
    int kernels_per_step = 0;
    // targets staged by lvigs_stage_targets: per slot the buffers, whether the
    // LiDAR maps were staged, the sizes, and the copy-done / last-read events
    DevBuf stg_gt[LVIGS_STAGE_SLOTS][kMaxViews], stg_li[LVIGS_STAGE_SLOTS][kMaxViews];
    bool stg_has_li[LVIGS_STAGE_SLOTS] = {};
    int stg_views[LVIGS_STAGE_SLOTS] = {};
    int stg_w[LVIGS_STAGE_SLOTS][kMaxViews] = {}, stg_h[LVIGS_STAGE_SLOTS][kMaxViews] = {};
    cudaEvent_t stg_ready[LVIGS_STAGE_SLOTS] = {}, stg_read[LVIGS_STAGE_SLOTS] = {};

    // map maintenance (append / prune) scratch, kept apart from the step's
    // buffers so that growing it does not invalidate the step's graph
    DevBuf mp_pts, mp_col, mp_keep, mp_offs, mp_keys, mp_vals, mp_keys2, mp_vals2, mp_scan, mp_radix, mp_cells,
        mp_logs, mp_small, mp_tmp, mp_spts;

    // opt-in per-phase device timing of eagerly enqueued work
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    double prof_ms[LVIGS_N_PHASES] = {};
    int64_t prof_calls[LVIGS_N_PHASES] = {};
};

namespace {

lvigs_status fail(lvigs_ctx *c, lvigs_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

lvigs_status cuda_fail(lvigs_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, LVIGS_ERR_CUDA, m);
}

#define LV_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);             \
    } while (0)

// Grow a buffer to at least `bytes`.  While a graph is being captured no
// allocation is allowed: a short buffer marks the capture as unusable.
lvigs_status ensure(lvigs_ctx *ctx, DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return LVIGS_OK;
    if (ctx->capturing) {
        ctx->capture_short = true;
        return LVIGS_ERR_CAPACITY;
    }
    size_t want = bytes + bytes / 8;
    want = (want + 255) / 256 * 256;
    const size_t after = ctx->bytes_in_use - b.bytes + want;
    if (ctx->cfg.max_workspace_bytes && after > ctx->cfg.max_workspace_bytes)
        return fail(ctx, LVIGS_ERR_CAPACITY, "workspace cap exceeded");
    if (b.p) {
        cudaFree(b.p);
        ctx->bytes_in_use -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LVIGS_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b.p = p;
    b.bytes = want;
    ctx->bytes_in_use += want;
    ++ctx->ws_epoch;
    return LVIGS_OK;
}

void release(lvigs_ctx *ctx, DevBuf &b) {
    if (b.p) {
        cudaFree(b.p);
        ctx->bytes_in_use -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

void release_state(lvigs_ctx *ctx, RenderState &s) {
    DevBuf *all[] = {&s.recs, &s.tiles, &s.zbits, &s.rects, &s.inst_a_t, &s.inst_a_v, &s.inst_b_t,
                     &s.inst_b_v, &s.ranges, &s.final_T, &s.n_contrib, &s.vs_dev, &s.counters,
                     &s.n_chunks, &s.chunk_base, &s.part_base, &s.pair_tile, &s.part,
                     &s.pair_k, &s.pair_v, &s.pair_v2, &s.stop_at, &s.plan_aux, &s.stop_items,
                     &s.pix_state};
    for (DevBuf *b : all) release(ctx, *b);
    s.valid = false;
    s.m_cap = 0;
}

// Records device time of one phase while profiling is on and nothing is captured.
struct Phase {
    lvigs_ctx *ctx;
    int phase;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEvent_t take() {
        cudaEvent_t e;
        if (!ctx->ev_pool.empty()) {
            e = ctx->ev_pool.back();
            ctx->ev_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    Phase(lvigs_ctx *c, int ph, cudaStream_t st) : ctx(c), phase(ph), s(st) {
        if (ctx->prof && !ctx->capturing) {
            e0 = take();
            e1 = take();
            if (e0) cudaEventRecord(e0, s);
        }
    }
    ~Phase() {
        if (e0 && e1) {
            cudaEventRecord(e1, s);
            ctx->prof_pending.push_back({phase, {e0, e1}});
        }
    }
};

#define LV_TRY(expr)                                 \
    do {                                             \
        lvigs_status st_ = (expr);                   \
        if (st_ != LVIGS_OK) return st_;             \
    } while (0)

// (Powers of two only: key preprocessing divides by the tile size as a
// product with its exact reciprocal.)
bool tile_supported(int w, int h) {
    return (w == 16 && h == 16) || (w == 8 && h == 8) || (w == 32 && h == 16);
}

// Level-l camera (Sec. III-D): the level halves the image l times; with pixels
// sampled at integer coordinates a level-l pixel's block centre gives the
// principal point (c + 0.5) / 2^l - 0.5.  Binary32, one rounding per op.
ViewDesc make_view(const lvigs_camera &c, int level, int tw, int th) {
    ViewDesc v{};
    float scale = 1.0f;
    for (int i = 0; i < level; ++i) scale = scale * 0.5f;
    for (int i = 0; i < 9; ++i) v.R[i] = c.R[i];
    for (int i = 0; i < 3; ++i) v.t[i] = c.t[i];
    v.fx = c.fx * scale;
    v.fy = c.fy * scale;
    v.cx = (c.cx + 0.5f) * scale - 0.5f;
    v.cy = (c.cy + 0.5f) * scale - 0.5f;
    v.W = c.width >> level;
    v.H = c.height >> level;
    v.limx = 1.3f * ((0.5f * (float)v.W) / v.fx);
    v.limy = 1.3f * ((0.5f * (float)v.H) / v.fy);
    for (int i = 0; i < 3; ++i)
        v.campos[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
    v.tiles_x = (v.W + tw - 1) / tw;
    v.tiles_y = (v.H + th - 1) / th;
    return v;
}

lvigs_status check_gauss(lvigs_ctx *ctx, const lvigs_gaussians *g) {
    if (!g) return fail(ctx, LVIGS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0 || g->n >= (int64_t)1 << 31) return fail(ctx, LVIGS_ERR_INVALID_ARG, "n out of range");
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ctx, LVIGS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (g->sh_stride_k < (g->sh_degree + 1) * (g->sh_degree + 1))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "sh_stride_k < (sh_degree+1)^2");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL parameter pointer");
    return LVIGS_OK;
}

lvigs_status check_camera(lvigs_ctx *ctx, const lvigs_camera *cam, int level) {
    if (!cam) return fail(ctx, LVIGS_ERR_INVALID_ARG, "camera is NULL");
    if (level < 0 || level > LVIGS_MAX_LEVEL) return fail(ctx, LVIGS_ERR_INVALID_ARG, "level out of range");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 16384 || cam->height > 16384)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "image size out of range");
    if ((cam->width >> level) < 1 || (cam->height >> level) < 1)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "level too deep for the image");
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(ctx, LVIGS_ERR_INVALID_ARG, "focal length must be > 0");
    return LVIGS_OK;
}

GaussParams to_params(const lvigs_gaussians *g) {
    GaussParams P;
    P.means = g->means;
    P.log_scales = g->log_scales;
    P.quats = g->quats;
    P.opacity_logits = g->opacity_logits;
    P.sh = g->sh;
    P.n = (int)g->n;
    P.sh_degree = g->sh_degree;
    P.sh_stride_k = g->sh_stride_k;
    return P;
}

int key_bits(uint32_t total_tiles) {
    int b = 1;
    while (b < 32 && ((uint64_t)1 << b) < total_tiles) ++b;
    return b;
}

// Capacities of the list-parallel plan for m_cap instances: at most
// tiles + m_cap / L pairs, and a multi-chunk tile of n > L entries owns at most
// 2 n / L slots.
lvigs_status ensure_plan(lvigs_ctx *ctx, RenderState &st) {
    const uint64_t pairs = (uint64_t)st.vs.total_tiles + (uint64_t)st.m_cap / kChunkLen + 1;
    const uint64_t slots = 2 * ((uint64_t)st.m_cap / kChunkLen) + 1;
    if (pairs > 0xffffffffull || slots > 0xffffffffull) return fail(ctx, LVIGS_ERR_CAPACITY, "plan too large");
    LV_TRY(ensure(ctx, st.pair_tile, (size_t)pairs * 4));
    LV_TRY(ensure(ctx, st.pair_k, (size_t)pairs * 4));
    LV_TRY(ensure(ctx, st.pair_v, (size_t)pairs * 4));
    LV_TRY(ensure(ctx, st.pair_v2, (size_t)pairs * 4));
    LV_TRY(ensure(ctx, st.stop_at, (size_t)st.vs.total_pixels * 4));
    LV_TRY(ensure(ctx, st.plan_aux, plan_aux_bytes(st.vs.total_tiles)));
    LV_TRY(ensure(ctx, st.stop_items, (size_t)pairs * (st.vs.tile_w / 8) * (st.vs.tile_h / 8) * 4));
    LV_TRY(ensure(ctx, st.pix_state, (size_t)st.vs.total_pixels * pix_state_bytes()));
    LV_TRY(ensure(ctx, st.part, (size_t)slots * chunk_slot_bytes(st.vs.tile_w, st.vs.tile_h)));
    st.pair_cap = (uint32_t)pairs;
    st.slot_cap = (uint32_t)slots;
    return LVIGS_OK;
}

// a1-a4 for the views of `st`: preprocess, compact, depth sort, scan,
// emit, tile sort, ranges.  In eager mode the call waits once to learn the
// instance count and grows the instance buffers; otherwise it relies on
// st.m_cap (overflow is latched in the status word).
lvigs_status build_lists(lvigs_ctx *ctx, RenderState &st, cudaStream_t s, bool eager, double headroom,
                         GGrad *g2d_init = nullptr) {
    const int64_t N = st.P.n;
    const int64_t VN = N * st.vs.n_views;
    LV_TRY(ensure(ctx, st.recs, (size_t)VN * sizeof(GRec)));
    LV_TRY(ensure(ctx, st.tiles, (size_t)VN * 4));
    LV_TRY(ensure(ctx, st.zbits, (size_t)VN * 4));
    LV_TRY(ensure(ctx, st.rects, (size_t)VN * 8));
    LV_TRY(ensure(ctx, st.counters, 32));
    LV_TRY(ensure(ctx, st.ranges, (size_t)st.vs.total_tiles * sizeof(uint2)));
    LV_TRY(ensure(ctx, st.n_chunks, (size_t)st.vs.total_tiles * 4));
    LV_TRY(ensure(ctx, st.chunk_base, (size_t)st.vs.total_tiles * 4));
    LV_TRY(ensure(ctx, st.part_base, (size_t)st.vs.total_tiles * 4));
    LV_TRY(ensure(ctx, ctx->pos, (size_t)VN * 4));
    LV_TRY(ensure(ctx, ctx->ck, (size_t)VN * 4));
    LV_TRY(ensure(ctx, ctx->cv, (size_t)VN * 4));
    LV_TRY(ensure(ctx, ctx->ck2, (size_t)VN * 4));
    LV_TRY(ensure(ctx, ctx->cv2, (size_t)VN * 4));
    const int64_t scan_n = VN > (int64_t)st.vs.total_tiles ? VN : (int64_t)st.vs.total_tiles;
    LV_TRY(ensure(ctx, ctx->scan_tmp, scan_tmp_words(scan_n) * 4));
    LV_TRY(ensure(ctx, ctx->radix_tmp, radix_tmp_words((int64_t)1 << 40) * 4));
    LV_TRY(ensure(ctx, ctx->status, 16));
    if (!eager) {
        LV_TRY(ensure(ctx, st.inst_a_t, (size_t)st.m_cap * 4));
        LV_TRY(ensure(ctx, st.inst_a_v, (size_t)st.m_cap * 4));
        LV_TRY(ensure(ctx, st.inst_b_t, (size_t)st.m_cap * 4));
        LV_TRY(ensure(ctx, st.inst_b_v, (size_t)st.m_cap * 4));
        LV_TRY(ensure_plan(ctx, st));
    }
    // [0] visible, [1] instances, [2] clamped instances, [3] work queue, [4] pairs, [5] slots
    uint32_t *cnt = (uint32_t *)st.counters.p;
    const ViewSet *vsd = (const ViewSet *)st.vs_dev.p;

    {
        Phase ph(ctx, LVIGS_PHASE_PREPROCESS, s);
        launch_preprocess_fwd(st.P, vsd, (GRec *)st.recs.p, (uint32_t *)st.tiles.p, (uint32_t *)st.zbits.p,
                              (uint2 *)st.rects.p, g2d_init, s);
    }
    {
        Phase ph(ctx, LVIGS_PHASE_COMPACT, s);
        launch_compact_scan((const uint32_t *)st.tiles.p, (const uint32_t *)st.zbits.p, (uint32_t *)ctx->ck.p,
                            (uint32_t *)ctx->cv.p, cnt + 0, VN, (uint32_t *)ctx->scan_tmp.p, s);
    }
    int r;
    {
        // depth keys of visible Gaussians are positive floats: 31 significant bits
        Phase ph(ctx, LVIGS_PHASE_DEPTH_SORT, s);
        r = launch_radix_sort((uint32_t *)ctx->ck.p, (uint32_t *)ctx->cv.p, (uint32_t *)ctx->ck2.p,
                              (uint32_t *)ctx->cv2.p, cnt + 0, VN, 31, (uint32_t *)ctx->radix_tmp.p, s);
    }
    const uint32_t *sorted_idx = (const uint32_t *)(r ? ctx->cv2.p : ctx->cv.p);
    {
        Phase ph(ctx, LVIGS_PHASE_OFFSETS, s);
        launch_scan((const uint32_t *)st.tiles.p, sorted_idx, 0, (uint32_t *)ctx->pos.p, cnt + 1, cnt + 0, VN,
                    (uint32_t *)ctx->scan_tmp.p, s);
    }
    if (eager) {
        LV_CUDA(cudaMemcpyAsync(ctx->host_counters, cnt, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        st.m = ctx->host_counters[1];
        const int64_t need = (int64_t)((double)st.m * headroom) + 1024;
        if (st.m_cap < st.m || st.m_cap < need / 2 || st.m_cap == 0) st.m_cap = need;
        if (st.m_cap > 0xfffffff0LL) return fail(ctx, LVIGS_ERR_CAPACITY, "more than 2^32 instances");
        LV_TRY(ensure(ctx, st.inst_a_t, (size_t)st.m_cap * 4));
        LV_TRY(ensure(ctx, st.inst_a_v, (size_t)st.m_cap * 4));
        LV_TRY(ensure(ctx, st.inst_b_t, (size_t)st.m_cap * 4));
        LV_TRY(ensure(ctx, st.inst_b_v, (size_t)st.m_cap * 4));
        LV_TRY(ensure_plan(ctx, st));
    }
    {
        Phase ph(ctx, LVIGS_PHASE_EMIT, s);
        launch_emit(vsd, sorted_idx, (const uint32_t *)ctx->pos.p, cnt + 0, (const uint2 *)st.rects.p, (int)N,
                    (uint32_t *)st.inst_a_t.p, (uint32_t *)st.inst_a_v.p, st.m_cap, VN, (uint32_t *)ctx->status.p, s);
        launch_clamp_count(cnt + 1, st.m_cap, cnt + 2, s);
    }
    {
        Phase ph(ctx, LVIGS_PHASE_TILE_SORT, s);
        st.sorted_in_b = launch_radix_sort((uint32_t *)st.inst_a_t.p, (uint32_t *)st.inst_a_v.p,
                                           (uint32_t *)st.inst_b_t.p, (uint32_t *)st.inst_b_v.p, cnt + 2, st.m_cap,
                                           key_bits(st.vs.total_tiles), (uint32_t *)ctx->radix_tmp.p, s);
    }
    {
        Phase ph(ctx, LVIGS_PHASE_RANGES, s);
        launch_ranges(st.sorted_tiles(), cnt + 2, st.m_cap, (uint2 *)st.ranges.p, st.vs.total_tiles, s);
        // list-parallel plan: chunks per tile, pair and slot numbering, the
        // chunk-major work order; and the per-pixel stop record
        launch_plan(st.plan(), (const uint2 *)st.ranges.p, st.vs.total_tiles, cnt, (uint32_t *)st.pair_v.p,
                    (uint32_t *)st.plan_aux.p, (uint32_t *)ctx->status.p, s);
        LV_CUDA(cudaMemsetAsync(st.stop_at.p, 0xff, (size_t)st.vs.total_pixels * 4, s));
    }
    return LVIGS_OK;
}

// The backward's work order: the plan's pairs by decreasing expected walk (in
// its own buffer; the forward's order stays as it was).
ChunkPlan backward_plan(RenderState &st, cudaStream_t s) {
    ChunkPlan cp = st.plan();
    uint32_t *cnt = (uint32_t *)st.counters.p;
    launch_bwd_pair_keys(st.vs, (const ViewSet *)st.vs_dev.p, cp, (const int32_t *)st.n_contrib.p,
                         (uint32_t *)st.pair_k.p, (uint32_t *)st.plan_aux.p, s);
    launch_bucket_place((const uint32_t *)st.pair_k.p, cnt + 4, st.pair_cap, (uint32_t *)st.plan_aux.p,
                        (uint32_t *)st.pair_v2.p, s);
    cp.pair_order = (const uint32_t *)st.pair_v2.p;
    return cp;
}

lvigs_status upload_viewset(lvigs_ctx *ctx, RenderState &st, cudaStream_t s) {
    LV_TRY(ensure(ctx, st.vs_dev, sizeof(ViewSet)));
    // a pinned staging copy is reused once its previous upload has landed
    const int k = ctx->vs_next;
    ctx->vs_next = (k + 1) % kVsRing;
    LV_CUDA(cudaEventSynchronize(ctx->vs_event[k]));
    std::memcpy(ctx->vs_staging + k, &st.vs, sizeof(ViewSet));
    LV_CUDA(cudaMemcpyAsync(st.vs_dev.p, ctx->vs_staging + k, sizeof(ViewSet), cudaMemcpyHostToDevice, s));
    LV_CUDA(cudaEventRecord(ctx->vs_event[k], s));
    return LVIGS_OK;
}

int slot_index(const lvigs_ctx *ctx, int handle, RenderState **out) {
    const int idx = handle & 0xfff;
    const uint32_t gen = (uint32_t)handle >> 12;
    if (handle < 0 || idx >= (int)ctx->slots.size()) return -1;
    RenderState *s = ctx->slots[idx];
    if (!s->valid || (s->generation & 0x7ffff) != gen) return -1;
    *out = s;
    return idx;
}

} // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *lvigs_version(void) { return "lvigs-gb300 0.1 (sm_103a)"; }

void lvigs_config_default(lvigs_config *cfg) {
    if (!cfg) return;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->batch_depth = 0;
    cfg->max_workspace_bytes = 0;
}

lvigs_status lvigs_create(lvigs_ctx **out, const lvigs_config *cfg) {
    if (!out) return LVIGS_ERR_INVALID_ARG;
    *out = nullptr;
    lvigs_config c;
    lvigs_config_default(&c);
    if (cfg) c = *cfg;
    if (!tile_supported(c.tile_w, c.tile_h)) return LVIGS_ERR_INVALID_ARG;
    // compositing warps stage 32 (bm = 1) or 64 (bm = 2) Gaussians per round
    int bm = 2;
    if (c.batch_depth == 32) bm = 1;
    else if (c.batch_depth != 0 && c.batch_depth != 64) return LVIGS_ERR_INVALID_ARG;
    lvigs_ctx *ctx = new lvigs_ctx();
    ctx->cfg = c;
    ctx->bm = bm;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->host_counters, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->host_status, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->host_losses, kMaxViews * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->host_batch_counters, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->vs_staging, kVsRing * sizeof(ViewSet));
    for (int k = 0; k < kVsRing && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&ctx->vs_event[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->step_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&ctx->side_ev[k], cudaEventDisableTiming);
    for (int k = 0; k < LVIGS_STAGE_SLOTS && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&ctx->stg_ready[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->stg_read[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        lvigs_destroy(ctx);
        return LVIGS_ERR_CUDA;
    }
    if (ensure(ctx, ctx->status, 16) != LVIGS_OK) {
        lvigs_destroy(ctx);
        return LVIGS_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(ctx->status.p, 0, 16);
    *out = ctx;
    return LVIGS_OK;
}

void lvigs_destroy(lvigs_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    for (RenderState *s : ctx->slots) {
        release_state(ctx, *s);
        delete s;
    }
    release_state(ctx, ctx->batch);
    DevBuf *shared[] = {&ctx->pos, &ctx->ck, &ctx->cv, &ctx->ck2, &ctx->cv2, &ctx->scan_tmp, &ctx->radix_tmp,
                        &ctx->status, &ctx->g2d, &ctx->loss_tmp, &ctx->stats, &ctx->img_rgb, &ctx->img_depth,
                        &ctx->img_alpha, &ctx->d_rgb, &ctx->d_depth, &ctx->mp_pts,
                        &ctx->mp_col, &ctx->mp_keep, &ctx->mp_offs, &ctx->mp_keys, &ctx->mp_vals, &ctx->mp_keys2,
                        &ctx->mp_vals2, &ctx->mp_scan, &ctx->mp_radix, &ctx->mp_cells, &ctx->mp_logs,
                        &ctx->mp_small, &ctx->mp_tmp, &ctx->mp_spts};
    for (DevBuf *b : shared) release(ctx, *b);
    for (int v = 0; v < kMaxViews; ++v) {
        release(ctx, ctx->gt_stage[v]);
        release(ctx, ctx->lidar_stage[v]);
        for (int k = 0; k < LVIGS_STAGE_SLOTS; ++k) {
            release(ctx, ctx->stg_gt[k][v]);
            release(ctx, ctx->stg_li[k][v]);
        }
        for (int l = 0; l <= LVIGS_MAX_LEVEL; ++l) {
            release(ctx, ctx->pyr_rgb[v][l]);
            release(ctx, ctx->pyr_depth[v][l]);
        }
    }
    for (cudaGraphExec_t ge : ctx->graph_exec)
        if (ge) cudaGraphExecDestroy(ge);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (cudaEvent_t ev : ctx->side_ev)
        if (ev) cudaEventDestroy(ev);
    for (int k = 0; k < LVIGS_STAGE_SLOTS; ++k) {
        if (ctx->stg_ready[k]) cudaEventDestroy(ctx->stg_ready[k]);
        if (ctx->stg_read[k]) cudaEventDestroy(ctx->stg_read[k]);
    }
    for (auto &pe : ctx->prof_pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t ev : ctx->vs_event)
        if (ev) cudaEventDestroy(ev);
    if (ctx->step_event) cudaEventDestroy(ctx->step_event);
    if (ctx->host_counters) cudaFreeHost(ctx->host_counters);
    if (ctx->host_status) cudaFreeHost(ctx->host_status);
    if (ctx->host_losses) cudaFreeHost(ctx->host_losses);
    if (ctx->host_batch_counters) cudaFreeHost(ctx->host_batch_counters);
    if (ctx->vs_staging) cudaFreeHost(ctx->vs_staging);
    delete ctx;
}

lvigs_status lvigs_level_size(const lvigs_camera *cam, int level, int *width, int *height) {
    if (!cam || !width || !height || level < 0 || level > LVIGS_MAX_LEVEL) return LVIGS_ERR_INVALID_ARG;
    *width = cam->width >> level;
    *height = cam->height >> level;
    return LVIGS_OK;
}

} // extern "C"

namespace {

// lvigs_render (wait: size the instance lists from the device's count) and
// lvigs_render_async (no wait: size them from the context's earlier renders).
lvigs_status render_view(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_camera *cam, int level,
                         const lvigs_image_out *out, int *view_slot, void *stream, bool wait) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    LV_TRY(check_gauss(ctx, g));
    LV_TRY(check_camera(ctx, cam, level));
    if (!out || !out->rgb || !out->depth || !out->alpha || !view_slot)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    // pick a free slot
    int idx = -1;
    for (size_t i = 0; i < ctx->slots.size(); ++i)
        if (!ctx->slots[i]->valid) {
            idx = (int)i;
            break;
        }
    if (idx < 0) {
        if (ctx->slots.size() >= 4096) return fail(ctx, LVIGS_ERR_CAPACITY, "too many live view slots");
        ctx->slots.push_back(new RenderState());
        idx = (int)ctx->slots.size() - 1;
    }
    RenderState &st = *ctx->slots[idx];
    st.P = to_params(g);
    std::memset(&st.vs, 0, sizeof(ViewSet));
    st.vs.n_views = 1;
    st.vs.tile_w = ctx->cfg.tile_w;
    st.vs.tile_h = ctx->cfg.tile_h;
    st.vs.v[0] = make_view(*cam, level, ctx->cfg.tile_w, ctx->cfg.tile_h);
    st.vs.v[0].tile_base = 0;
    st.vs.v[0].pix_base = 0;
    st.vs.total_tiles = (uint32_t)(st.vs.v[0].tiles_x * st.vs.v[0].tiles_y);
    st.vs.total_pixels = (uint32_t)(st.vs.v[0].W * st.vs.v[0].H);
    LV_TRY(upload_viewset(ctx, st, s));
    LV_TRY(ensure(ctx, st.final_T, (size_t)st.vs.total_pixels * 4));
    LV_TRY(ensure(ctx, st.n_contrib, (size_t)st.vs.total_pixels * 4));
    if (!wait && st.m_cap < ctx->render_m_cap) st.m_cap = ctx->render_m_cap;
    const bool eager = wait || st.m_cap == 0;
    LV_TRY(build_lists(ctx, st, s, eager, 1.0));
    if (eager && st.m_cap > ctx->render_m_cap) ctx->render_m_cap = st.m_cap;
    ViewImages im{};
    im.rgb[0] = out->rgb;
    im.depth[0] = out->depth;
    im.alpha[0] = out->alpha;
    for (int part = 1; part <= 2; ++part) {
        Phase ph(ctx, part == 1 ? LVIGS_PHASE_COMPOSITE_FWD : LVIGS_PHASE_COMBINE, s);
        launch_composite_fwd(st.vs, (const ViewSet *)st.vs_dev.p, (const uint2 *)st.ranges.p, st.sorted_vals(),
                             (const GRec *)st.recs.p, im, (float *)st.final_T.p, (int32_t *)st.n_contrib.p, st.plan(),
                             (uint32_t *)st.counters.p + 3, st.pix_state.p, s, ctx->bm,
                             part == 1 ? kFwdWalk : kFwdCombine | kFwdBackwardState);
    }
    LV_CUDA(cudaGetLastError());
    st.valid = true;
    st.generation = (st.generation + 1) & 0x7ffff;
    *view_slot = (int)((st.generation << 12) | (uint32_t)idx);
    return LVIGS_OK;
}

} // namespace

extern "C" {

lvigs_status lvigs_render(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_camera *cam, int level,
                          const lvigs_image_out *out, int *view_slot, void *stream) {
    return render_view(ctx, g, cam, level, out, view_slot, stream, true);
}

lvigs_status lvigs_render_async(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_camera *cam, int level,
                                const lvigs_image_out *out, int *view_slot, void *stream) {
    return render_view(ctx, g, cam, level, out, view_slot, stream, false);
}

lvigs_status lvigs_backward(lvigs_ctx *ctx, int view_slot, const float *dL_drgb, const float *dL_ddepth,
                            const float *dL_dalpha, const lvigs_grads *grads, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    RenderState *st = nullptr;
    if (slot_index(ctx, view_slot, &st) < 0) return fail(ctx, LVIGS_ERR_STATE, "stale or unknown view slot");
    if (!grads || (st->P.n > 0 && (!grads->d_means || !grads->d_log_scales || !grads->d_quats ||
                                   !grads->d_opacity_logits || !grads->d_sh)))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL gradient output");
    if (!dL_drgb) return fail(ctx, LVIGS_ERR_INVALID_ARG, "dL_drgb is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t VN = (int64_t)st->P.n * st->vs.n_views;
    LV_TRY(ensure(ctx, ctx->g2d, (size_t)VN * sizeof(GGrad)));
    if (VN > 0) LV_CUDA(cudaMemsetAsync(ctx->g2d.p, 0, (size_t)VN * sizeof(GGrad), s));
    ViewGrads vg{};
    vg.d_rgb[0] = dL_drgb;
    vg.d_depth[0] = dL_ddepth;
    vg.d_alpha[0] = dL_dalpha;
    {
        Phase ph(ctx, LVIGS_PHASE_COMPOSITE_BWD, s);
        const ChunkPlan bp = backward_plan(*st, s);
        launch_composite_bwd(st->vs, (const ViewSet *)st->vs_dev.p, (const uint2 *)st->ranges.p, st->sorted_vals(),
                             (const GRec *)st->recs.p, vg, (const float *)st->final_T.p,
                             (const int32_t *)st->n_contrib.p, (GGrad *)ctx->g2d.p, bp,
                             (uint32_t *)st->counters.p + 3, s, ctx->bm);
    }
    ParamGrads G{grads->d_means, grads->d_log_scales, grads->d_quats, grads->d_opacity_logits, grads->d_sh,
                 grads->accumulate};
    {
        Phase ph(ctx, LVIGS_PHASE_PREPROCESS_BWD, s);
        launch_preprocess_bwd(st->P, (const ViewSet *)st->vs_dev.p, (const uint32_t *)st->tiles.p,
                              (const GGrad *)ctx->g2d.p, G, s);
    }
    LV_CUDA(cudaGetLastError());
    return LVIGS_OK;
}

lvigs_status lvigs_loss(lvigs_ctx *ctx, int width, int height, const float *rgb, const float *depth,
                        const float *gt_rgb, const float *lidar_depth, float lambda_ssim, float lambda_depth,
                        double *loss_out, float *d_rgb, float *d_depth, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    if (width <= 0 || height <= 0 || !rgb || !gt_rgb || !loss_out)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "bad loss arguments");
    if (lidar_depth && !depth) return fail(ctx, LVIGS_ERR_INVALID_ARG, "lidar_depth given without depth");
    if (!(lambda_ssim >= 0.f && lambda_ssim <= 1.f)) return fail(ctx, LVIGS_ERR_INVALID_ARG, "lambda_ssim outside [0,1]");
    if (!kernel_writable(loss_out))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "loss_out must be device or page-locked host memory");
    LossViews lv{};
    lv.n_views = 1;
    lv.W[0] = width;
    lv.H[0] = height;
    lv.tile_base[0] = 0;
    lv.total_tiles = loss_tile_count(width, height);
    lv.rgb[0] = rgb;
    lv.depth[0] = depth;
    lv.gt[0] = gt_rgb;
    lv.lidar[0] = lidar_depth;
    lv.d_rgb[0] = d_rgb;
    lv.d_depth[0] = d_depth;
    lv.loss_out[0] = loss_out;
    lv.lambda_ssim = lambda_ssim;
    lv.lambda_depth = lambda_depth;
    LV_TRY(ensure(ctx, ctx->loss_tmp, loss_tmp_bytes(lv)));
    {
        Phase ph(ctx, LVIGS_PHASE_LOSS, (cudaStream_t)stream);
        launch_loss(lv, ctx->loss_tmp.p, (cudaStream_t)stream);
    }
    LV_CUDA(cudaGetLastError());
    return LVIGS_OK;
}

lvigs_status lvigs_pyramid_down(int width, int height, const float *rgb, const float *depth, float *rgb_out,
                                float *depth_out, void *stream) {
    if (width < 2 || height < 2 || !rgb || !rgb_out || (depth && !depth_out)) return LVIGS_ERR_INVALID_ARG;
    launch_pyramid_down(width, height, rgb, depth, rgb_out, depth_out, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LVIGS_OK : LVIGS_ERR_CUDA;
}

lvigs_status lvigs_debug_keys(lvigs_ctx *ctx, int view_slot, uint64_t *keys, uint32_t *vals, int64_t m_cap,
                              int64_t *m, void *stream) {
    if (!ctx || !m) return LVIGS_ERR_INVALID_ARG;
    RenderState *st = nullptr;
    if (slot_index(ctx, view_slot, &st) < 0) return fail(ctx, LVIGS_ERR_STATE, "stale or unknown view slot");
    *m = st->m;
    if (!keys) return LVIGS_OK;
    if (!vals || m_cap < st->m) return fail(ctx, LVIGS_ERR_INVALID_ARG, "key buffer too small");
    launch_debug_keys(st->sorted_tiles(), st->sorted_vals(), (const uint32_t *)st->zbits.p, st->P.n, keys, vals,
                      st->m, (cudaStream_t)stream);
    LV_CUDA(cudaGetLastError());
    return LVIGS_OK;
}

lvigs_status lvigs_debug_exp_key(const float *x, float *y, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return LVIGS_ERR_INVALID_ARG;
    launch_exp_key(x, y, n, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LVIGS_OK : LVIGS_ERR_CUDA;
}

lvigs_status lvigs_debug_state(lvigs_ctx *ctx, int view_slot, uint32_t *ranges, int32_t *n_contrib,
                               float *final_T, int *n_tiles, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    RenderState *st = nullptr;
    if (slot_index(ctx, view_slot, &st) < 0) return fail(ctx, LVIGS_ERR_STATE, "stale or unknown view slot");
    if (n_tiles) *n_tiles = (int)st->vs.total_tiles;
    cudaStream_t s = (cudaStream_t)stream;
    if (ranges)
        LV_CUDA(cudaMemcpyAsync(ranges, st->ranges.p, sizeof(uint2) * st->vs.total_tiles, cudaMemcpyDeviceToDevice, s));
    if (n_contrib)
        LV_CUDA(cudaMemcpyAsync(n_contrib, st->n_contrib.p, 4 * (size_t)st->vs.total_pixels, cudaMemcpyDeviceToDevice, s));
    if (final_T)
        LV_CUDA(cudaMemcpyAsync(final_T, st->final_T.p, 4 * (size_t)st->vs.total_pixels, cudaMemcpyDeviceToDevice, s));
    return LVIGS_OK;
}

lvigs_status lvigs_sync_status(lvigs_ctx *ctx, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    LV_CUDA(cudaMemcpyAsync(ctx->host_status, ctx->status.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const uint32_t st = *ctx->host_status;
    if (st) LV_CUDA(cudaMemsetAsync(ctx->status.p, 0, sizeof(uint32_t), s));
    LV_CUDA(cudaStreamSynchronize(s));
    if (st & kStatusTimeout) return fail(ctx, LVIGS_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & kStatusCapacity) return fail(ctx, LVIGS_ERR_CAPACITY, "instance capacity exceeded on the device");
    return LVIGS_OK;
}

lvigs_status lvigs_release_view(lvigs_ctx *ctx, int view_slot) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    RenderState *st = nullptr;
    if (slot_index(ctx, view_slot, &st) < 0) return fail(ctx, LVIGS_ERR_STATE, "stale or unknown view slot");
    st->valid = false;
    return LVIGS_OK;
}

const char *lvigs_last_error(const lvigs_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

lvigs_status lvigs_step_stats(lvigs_ctx *ctx, int64_t *out, void *stream) {
    if (!ctx || !out) return LVIGS_ERR_INVALID_ARG;
    RenderState &st = ctx->batch;
    cudaStream_t s = (cudaStream_t)stream;
    out[0] = out[1] = out[2] = out[3] = 0;
    if (!st.counters.p || !st.n_contrib.p) return LVIGS_OK;
    LV_TRY(ensure(ctx, ctx->stats, 16));
    launch_sum_i32((const int32_t *)st.n_contrib.p, st.vs.total_pixels, (unsigned long long *)ctx->stats.p, s);
    LV_CUDA(cudaMemcpyAsync(ctx->host_counters, st.counters.p, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    unsigned long long sum = 0;
    LV_CUDA(cudaMemcpyAsync(&sum, ctx->stats.p, sizeof(sum), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    out[0] = ctx->host_counters[0];
    out[1] = ctx->host_counters[1];
    out[2] = (int64_t)sum;
    out[3] = st.vs.total_pixels;
    return LVIGS_OK;
}

lvigs_status lvigs_profile_enable(lvigs_ctx *ctx, int enable) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    ctx->prof = enable != 0;
    return LVIGS_OK;
}

lvigs_status lvigs_profile_read(lvigs_ctx *ctx, double *ms, int64_t *calls, int *kernels_per_step) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    for (auto &pe : ctx->prof_pending) {
        cudaEvent_t e0 = pe.second.first, e1 = pe.second.second;
        float t = 0.f;
        LV_CUDA(cudaEventSynchronize(e1));
        LV_CUDA(cudaEventElapsedTime(&t, e0, e1));
        ctx->prof_ms[pe.first] += t;
        ctx->prof_calls[pe.first] += 1;
        ctx->ev_pool.push_back(e0);
        ctx->ev_pool.push_back(e1);
    }
    ctx->prof_pending.clear();
    for (int i = 0; i < LVIGS_N_PHASES; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (calls) calls[i] = ctx->prof_calls[i];
        ctx->prof_ms[i] = 0.0;
        ctx->prof_calls[i] = 0;
    }
    if (kernels_per_step) *kernels_per_step = ctx->kernels_per_step;
    return LVIGS_OK;
}

} // extern "C"

// ===========================================================================
// Batched step
// ===========================================================================
namespace {

// Everything of one batched step, enqueued on `s`.  eager: may allocate and
// waits once to size the instance list; otherwise no allocation and no wait
// (capture-safe).
lvigs_status batched_body(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_batch *b, const lvigs_grads *gr,
                          cudaStream_t s, bool eager) {
    RenderState &st = ctx->batch;
    const int V = b->n_views;
    const bool staged = (b->flags & LVIGS_STEP_STAGED_TARGETS) != 0;
    const bool host_tg = !staged && (b->flags & LVIGS_STEP_HOST_TARGETS) != 0;
    // 1. targets at each view's level (Sec. III-D)
    const float *gt_l[kMaxViews];
    const float *li_l[kMaxViews];
    PyrViews pv[LVIGS_MAX_LEVEL + 1] = {};
    for (int v = 0; v < V; ++v) {
        const lvigs_camera &c = b->cameras[v];
        const size_t P0 = (size_t)c.width * c.height;
        const float *gsrc = nullptr, *lsrc = nullptr;
        if (staged) {
            gsrc = (const float *)ctx->stg_gt[b->staged_slot][v].p;
            lsrc = ctx->stg_has_li[b->staged_slot] ? (const float *)ctx->stg_li[b->staged_slot][v].p : nullptr;
        } else {
            gsrc = b->gt_rgb[v];
            lsrc = b->lidar_depth ? b->lidar_depth[v] : nullptr;
        }
        if (host_tg) {
            LV_TRY(ensure(ctx, ctx->gt_stage[v], 3 * P0 * 4));
            LV_CUDA(cudaMemcpyAsync(ctx->gt_stage[v].p, gsrc, 3 * P0 * 4, cudaMemcpyHostToDevice, s));
            gsrc = (const float *)ctx->gt_stage[v].p;
            if (lsrc) {
                LV_TRY(ensure(ctx, ctx->lidar_stage[v], P0 * 4));
                LV_CUDA(cudaMemcpyAsync(ctx->lidar_stage[v].p, lsrc, P0 * 4, cudaMemcpyHostToDevice, s));
                lsrc = (const float *)ctx->lidar_stage[v].p;
            }
        }
        const int l = b->levels[v];
        if (l > 0) {
            const int W2 = c.width >> l, H2 = c.height >> l;
            LV_TRY(ensure(ctx, ctx->pyr_rgb[v][l], 3 * (size_t)W2 * H2 * 4));
            if (lsrc) LV_TRY(ensure(ctx, ctx->pyr_depth[v][l], (size_t)W2 * H2 * 4));
            PyrViews &q = pv[l];
            const int j = q.n++;
            q.W[j] = c.width;
            q.H[j] = c.height;
            q.rgb[j] = gsrc;
            q.depth[j] = lsrc;
            q.rgb_out[j] = (float *)ctx->pyr_rgb[v][l].p;
            q.depth_out[j] = lsrc ? (float *)ctx->pyr_depth[v][l].p : nullptr;
            q.base[j + 1] = q.base[j] + (uint32_t)W2 * (uint32_t)H2;
            gsrc = q.rgb_out[j];
            if (lsrc) lsrc = q.depth_out[j];
        }
        gt_l[v] = gsrc;
        li_l[v] = lsrc;
    }
    // The side stream takes the pyramid (needed by the loss only) and later the
    // backward's start state and work order (needed by the backward only).
    // With the phase profiler on, everything runs in order on `s`.
    const bool par = !ctx->prof;
    cudaStream_t ss = par ? ctx->side : s;
    if (par) {
        LV_CUDA(cudaEventRecord(ctx->side_ev[0], s));
        LV_CUDA(cudaStreamWaitEvent(ss, ctx->side_ev[0], 0));
    }
    {
        Phase ph(ctx, LVIGS_PHASE_PYRAMID, ss);
        for (int l = 1; l <= LVIGS_MAX_LEVEL; ++l) launch_pyramid_views(pv[l], l, ss);
    }
    if (par) LV_CUDA(cudaEventRecord(ctx->side_ev[1], ss));
    // 2. a1-a4 over all views at once; preprocessing also clears the gradient
    // records of the pairs the backward will read (forward and backward of one
    // call, so nothing else writes them in between)
    const int64_t VN = (int64_t)st.P.n * V;
    LV_TRY(ensure(ctx, ctx->g2d, (size_t)VN * sizeof(GGrad)));
    LV_TRY(build_lists(ctx, st, s, eager, 1.3, (GGrad *)ctx->g2d.p));
    // 3. a5 into the caller's images or the internal ones
    const size_t TP = st.vs.total_pixels;
    LV_TRY(ensure(ctx, st.final_T, TP * 4));
    LV_TRY(ensure(ctx, st.n_contrib, TP * 4));
    LV_TRY(ensure(ctx, ctx->img_rgb, 3 * TP * 4));
    LV_TRY(ensure(ctx, ctx->img_depth, TP * 4));
    LV_TRY(ensure(ctx, ctx->img_alpha, TP * 4));
    LV_TRY(ensure(ctx, ctx->d_rgb, 3 * TP * 4));
    LV_TRY(ensure(ctx, ctx->d_depth, TP * 4));
    ViewImages im{};
    ViewGrads vg{};
    LossViews lv{};
    lv.n_views = V;
    uint32_t ltiles = 0;
    for (int v = 0; v < V; ++v) {
        const ViewDesc &d = st.vs.v[v];
        const size_t pb = d.pix_base;
        im.rgb[v] = b->rgb_out && b->rgb_out[v] ? b->rgb_out[v] : (float *)ctx->img_rgb.p + 3 * pb;
        im.depth[v] = b->depth_out && b->depth_out[v] ? b->depth_out[v] : (float *)ctx->img_depth.p + pb;
        im.alpha[v] = b->alpha_out && b->alpha_out[v] ? b->alpha_out[v] : (float *)ctx->img_alpha.p + pb;
        vg.d_rgb[v] = (float *)ctx->d_rgb.p + 3 * pb;
        vg.d_depth[v] = (float *)ctx->d_depth.p + pb;
        vg.d_alpha[v] = nullptr;
        lv.W[v] = d.W;
        lv.H[v] = d.H;
        lv.tile_base[v] = ltiles;
        ltiles += loss_tile_count(d.W, d.H);
        lv.rgb[v] = im.rgb[v];
        lv.depth[v] = im.depth[v];
        lv.gt[v] = gt_l[v];
        lv.lidar[v] = li_l[v];
        lv.d_rgb[v] = (float *)vg.d_rgb[v];
        lv.d_depth[v] = (float *)vg.d_depth[v];
        // the loss kernel writes each view's terms where they are read: the
        // caller's buffer (device, or pinned host with HOST_LOSS_ASYNC) or the
        // context's pinned host copy (HOST_LOSS); no copy engine is involved
        lv.loss_out[v] = ((b->flags & LVIGS_STEP_HOST_LOSS) ? ctx->host_losses : b->losses) + 4 * v;
    }
    lv.total_tiles = ltiles;
    lv.lambda_ssim = b->lambda_ssim;
    lv.lambda_depth = b->lambda_depth;
    LV_TRY(ensure(ctx, ctx->loss_tmp, loss_tmp_bytes(lv)));
    const ViewSet *vsd = (const ViewSet *)st.vs_dev.p;
    for (int part = 1; part <= 2; ++part) {
        Phase ph(ctx, part == 1 ? LVIGS_PHASE_COMPOSITE_FWD : LVIGS_PHASE_COMBINE, s);
        const int what = part == 1 ? kFwdWalk : (par ? kFwdCombine : kFwdCombine | kFwdBackwardState);
        launch_composite_fwd(st.vs, vsd, (const uint2 *)st.ranges.p, st.sorted_vals(), (const GRec *)st.recs.p, im,
                             (float *)st.final_T.p, (int32_t *)st.n_contrib.p, st.plan(), (uint32_t *)st.counters.p + 3,
                             st.pix_state.p, s, ctx->bm, what);
    }
    // the images are final: the backward's start state and work order beside the loss
    ChunkPlan bp{};
    if (par) {
        LV_CUDA(cudaEventRecord(ctx->side_ev[2], s));
        LV_CUDA(cudaStreamWaitEvent(ss, ctx->side_ev[2], 0));
        launch_composite_fwd(st.vs, vsd, (const uint2 *)st.ranges.p, st.sorted_vals(), (const GRec *)st.recs.p, im,
                             (float *)st.final_T.p, (int32_t *)st.n_contrib.p, st.plan(), (uint32_t *)st.counters.p + 3,
                             st.pix_state.p, ss, ctx->bm, kFwdBackwardState);
        bp = backward_plan(st, ss);
        LV_CUDA(cudaEventRecord(ctx->side_ev[3], ss));
        LV_CUDA(cudaStreamWaitEvent(s, ctx->side_ev[1], 0)); // the pyramid, for the loss
    }
    // 4. a8: loss and its image gradients for every view
    {
        Phase ph(ctx, LVIGS_PHASE_LOSS, s);
        launch_loss(lv, ctx->loss_tmp.p, s);
    }
    // 5. a6 + a7
    if (par) LV_CUDA(cudaStreamWaitEvent(s, ctx->side_ev[3], 0));
    {
        Phase ph(ctx, LVIGS_PHASE_COMPOSITE_BWD, s);
        if (!par) bp = backward_plan(st, s);
        launch_composite_bwd(st.vs, vsd, (const uint2 *)st.ranges.p, st.sorted_vals(), (const GRec *)st.recs.p, vg,
                             (const float *)st.final_T.p, (const int32_t *)st.n_contrib.p, (GGrad *)ctx->g2d.p, bp,
                             (uint32_t *)st.counters.p + 3, s, ctx->bm);
    }
    ParamGrads G{gr->d_means, gr->d_log_scales, gr->d_quats, gr->d_opacity_logits, gr->d_sh, gr->accumulate};
    {
        Phase ph(ctx, LVIGS_PHASE_PREPROCESS_BWD, s);
        launch_preprocess_bwd(st.P, vsd, (const uint32_t *)st.tiles.p, (const GGrad *)ctx->g2d.p, G, s);
    }
    // instance count of this step, for the capacity check of the next one
    LV_CUDA(cudaMemcpyAsync(ctx->host_batch_counters, st.counters.p, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return LVIGS_OK;
}

// What the instance count mostly depends on besides the poses: the Gaussian
// count and each view's size and level.  A step with a shape the capacity was
// not sized for runs eagerly (it waits once to size the lists) before a graph
// of that shape is captured.
BatchKey shape_key(const lvigs_gaussians *g, const lvigs_batch *b) {
    BatchKey k;
    k.k.push_back((uint64_t)g->n);
    k.k.push_back((uint64_t)b->n_views);
    for (int v = 0; v < b->n_views; ++v) {
        k.k.push_back((uint64_t)b->cameras[v].width << 32 | (uint32_t)b->cameras[v].height);
        k.k.push_back((uint64_t)b->levels[v]);
    }
    return k;
}

BatchKey make_key(const lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_batch *b, const lvigs_grads *gr) {
    BatchKey k;
    auto add = [&](uint64_t x) { k.k.push_back(x); };
    auto addp = [&](const void *p) { k.k.push_back((uint64_t)(uintptr_t)p); };
    auto addf = [&](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        k.k.push_back(u);
    };
    add(ctx->ws_epoch);
    add((uint64_t)ctx->batch.m_cap);
    add((uint64_t)ctx->cfg.tile_w);
    add((uint64_t)ctx->cfg.tile_h);
    add((uint64_t)ctx->bm);
    add((uint64_t)g->n);
    add((uint64_t)g->sh_degree);
    add((uint64_t)g->sh_stride_k);
    addp(g->means);
    addp(g->log_scales);
    addp(g->quats);
    addp(g->opacity_logits);
    addp(g->sh);
    addp(gr->d_means);
    addp(gr->d_log_scales);
    addp(gr->d_quats);
    addp(gr->d_opacity_logits);
    addp(gr->d_sh);
    add((uint64_t)gr->accumulate);
    add((uint64_t)b->n_views);
    add((uint64_t)b->flags);
    addf(b->lambda_ssim);
    addf(b->lambda_depth);
    addp(b->losses);
    const bool staged = (b->flags & LVIGS_STEP_STAGED_TARGETS) != 0;
    if (staged) add((uint64_t)b->staged_slot);
    for (int v = 0; v < b->n_views; ++v) {
        add((uint64_t)b->cameras[v].width);
        add((uint64_t)b->cameras[v].height);
        add((uint64_t)b->levels[v]);
        if (staged) {
            addp(ctx->stg_gt[b->staged_slot][v].p);
            addp(ctx->stg_has_li[b->staged_slot] ? ctx->stg_li[b->staged_slot][v].p : nullptr);
        } else {
            addp(b->gt_rgb[v]);
            addp(b->lidar_depth ? b->lidar_depth[v] : nullptr);
        }
        addp(b->rgb_out ? b->rgb_out[v] : nullptr);
        addp(b->depth_out ? b->depth_out[v] : nullptr);
        addp(b->alpha_out ? b->alpha_out[v] : nullptr);
    }
    return k;
}

} // namespace

extern "C" lvigs_status lvigs_train_step_batched(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_batch *b,
                                                 const lvigs_grads *gr, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    LV_TRY(check_gauss(ctx, g));
    const bool staged = b && (b->flags & LVIGS_STEP_STAGED_TARGETS) != 0;
    if (!b || b->n_views < 1 || b->n_views > kMaxViews || !b->cameras || !b->levels || (!staged && !b->gt_rgb) ||
        !b->losses)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "bad batch description");
    if (staged && (b->staged_slot < 0 || b->staged_slot >= LVIGS_STAGE_SLOTS ||
                   ctx->stg_views[b->staged_slot] != b->n_views))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "staged slot does not hold this step's targets");
    if (!(b->flags & LVIGS_STEP_HOST_LOSS)) {
        // the loss kernel writes b->losses itself: it must be device memory, or
        // page-locked host memory with HOST_LOSS_ASYNC
        cudaPointerAttributes pa{};
        const cudaError_t pe = cudaPointerGetAttributes(&pa, b->losses);
        cudaGetLastError();
        const bool host_async = (b->flags & LVIGS_STEP_HOST_LOSS_ASYNC) != 0;
        const bool ok = pe == cudaSuccess && (host_async ? pa.type == cudaMemoryTypeHost
                                                         : (pa.type == cudaMemoryTypeDevice ||
                                                            pa.type == cudaMemoryTypeManaged));
        if (!ok)
            return fail(ctx, LVIGS_ERR_INVALID_ARG,
                        host_async ? "losses must be page-locked host memory" : "losses must be device memory");
    }
    if (!gr || (g->n > 0 && (!gr->d_means || !gr->d_log_scales || !gr->d_quats || !gr->d_opacity_logits ||
                             !gr->d_sh)))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL gradient output");
    if (!(b->lambda_ssim >= 0.f && b->lambda_ssim <= 1.f))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "lambda_ssim outside [0,1]");
    if ((uint64_t)g->n * (uint64_t)b->n_views >= 0xffffffffull)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "n * n_views must be below 2^32");
    for (int v = 0; v < b->n_views; ++v) {
        LV_TRY(check_camera(ctx, &b->cameras[v], b->levels[v]));
        if (staged) {
            if (ctx->stg_w[b->staged_slot][v] != b->cameras[v].width ||
                ctx->stg_h[b->staged_slot][v] != b->cameras[v].height)
                return fail(ctx, LVIGS_ERR_INVALID_ARG, "staged target size differs from the camera");
        } else if (!b->gt_rgb[v]) {
            return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL target image");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    RenderState &st = ctx->batch;
    // view set (cameras may change every step without a new graph)
    std::memset(&st.vs, 0, sizeof(ViewSet));
    st.vs.n_views = b->n_views;
    st.vs.tile_w = ctx->cfg.tile_w;
    st.vs.tile_h = ctx->cfg.tile_h;
    uint32_t tb = 0, pb = 0;
    for (int v = 0; v < b->n_views; ++v) {
        ViewDesc d = make_view(b->cameras[v], b->levels[v], ctx->cfg.tile_w, ctx->cfg.tile_h);
        d.tile_base = tb;
        d.pix_base = pb;
        tb += (uint32_t)(d.tiles_x * d.tiles_y);
        pb += (uint32_t)(d.W * d.H);
        st.vs.v[v] = d;
    }
    st.vs.total_tiles = tb;
    st.vs.total_pixels = pb;
    st.P = to_params(g);
    LV_TRY(upload_viewset(ctx, st, s));

    // capacity check of the previous step (non-blocking unless it has finished)
    bool grow = false;
    if (ctx->step_pending && cudaEventQuery(ctx->step_event) == cudaSuccess) {
        ctx->step_pending = false;
        if ((int64_t)ctx->host_batch_counters[1] > st.m_cap) grow = true;
    }
    cudaGetLastError();

    const bool use_graph = !(b->flags & LVIGS_STEP_NO_GRAPH);
    BatchKey key = make_key(ctx, g, b, gr);
    const int gi = staged ? 1 + b->staged_slot : 0; // which cached graph
    if (staged) LV_CUDA(cudaStreamWaitEvent(s, ctx->stg_ready[b->staged_slot], 0));
    const BatchKey shape = shape_key(g, b);
    if (!use_graph || grow || st.m_cap == 0 || !(shape == ctx->sized_shape)) {
        // eager step: sizes the instance capacity (waits once on the stream)
        LV_TRY(batched_body(ctx, g, b, gr, s, true));
        ctx->sized_shape = shape;
    } else {
        if (!ctx->graph_ok[gi] || !(key == ctx->graph_key[gi])) {
            if (ctx->graph_exec[gi]) {
                cudaGraphExecDestroy(ctx->graph_exec[gi]);
                ctx->graph_exec[gi] = nullptr;
            }
            ctx->graph_ok[gi] = false;
            // the capture stream waits for nothing; the graph is launched on `s`
            ctx->capturing = true;
            ctx->capture_short = false;
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            lvigs_status bs = LVIGS_OK;
            if (e == cudaSuccess) bs = batched_body(ctx, g, b, gr, ctx->cap_stream, false);
            cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
            ctx->capturing = false;
            if (e == cudaSuccess && e2 == cudaSuccess && bs == LVIGS_OK && !ctx->capture_short) {
                size_t nn = 0;
                if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
                    std::vector<cudaGraphNode_t> nodes(nn);
                    cudaGraphGetNodes(graph, nodes.data(), &nn);
                    int kc = 0;
                    for (auto nd : nodes) {
                        cudaGraphNodeType ty;
                        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kc;
                    }
                    ctx->kernels_per_step = kc;
                }
                e = cudaGraphInstantiate(&ctx->graph_exec[gi], graph, 0);
                if (e == cudaSuccess) {
                    ctx->graph_ok[gi] = true;
                    ctx->graph_key[gi] = key;
                }
            }
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
        }
        if (ctx->graph_ok[gi]) {
            LV_CUDA(cudaGraphLaunch(ctx->graph_exec[gi], s));
        } else {
            LV_TRY(batched_body(ctx, g, b, gr, s, true));
        }
    }
    LV_CUDA(cudaEventRecord(ctx->step_event, s));
    if (staged) LV_CUDA(cudaEventRecord(ctx->stg_read[b->staged_slot], s)); // the slot may be refilled after this
    ctx->step_pending = true;
    if (b->flags & LVIGS_STEP_HOST_LOSS) {
        LV_CUDA(cudaStreamSynchronize(s));
        std::memcpy(b->losses, ctx->host_losses, (size_t)b->n_views * 4 * sizeof(double));
    }
    LV_CUDA(cudaGetLastError());
    return LVIGS_OK;
}

// Targets of a later batched step copied in from pinned host memory on a
// second stream (double-buffered slots), so that the copy overlaps the step
// before it.
extern "C" lvigs_status lvigs_stage_targets(lvigs_ctx *ctx, int slot, int n_views, const lvigs_camera *cameras,
                                            const float *const *gt_rgb, const float *const *lidar_depth,
                                            void *copy_stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    if (slot < 0 || slot >= LVIGS_STAGE_SLOTS || n_views < 1 || n_views > kMaxViews || !cameras || !gt_rgb)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "bad staging request");
    if (ctx->capturing) return fail(ctx, LVIGS_ERR_STATE, "staging during a graph capture");
    for (int v = 0; v < n_views; ++v) {
        if (cameras[v].width <= 0 || cameras[v].height <= 0 || !gt_rgb[v] || (lidar_depth && !lidar_depth[v]))
            return fail(ctx, LVIGS_ERR_INVALID_ARG, "bad staged view");
    }
    cudaStream_t cs = (cudaStream_t)copy_stream;
    // the previous reader of the slot must be done before it is overwritten
    // (a buffer that grows is reallocated, which waits for the device)
    LV_CUDA(cudaStreamWaitEvent(cs, ctx->stg_read[slot], 0));
    for (int v = 0; v < n_views; ++v) {
        const size_t P0 = (size_t)cameras[v].width * cameras[v].height;
        LV_TRY(ensure(ctx, ctx->stg_gt[slot][v], 3 * P0 * 4));
        LV_CUDA(cudaMemcpyAsync(ctx->stg_gt[slot][v].p, gt_rgb[v], 3 * P0 * 4, cudaMemcpyHostToDevice, cs));
        if (lidar_depth) {
            LV_TRY(ensure(ctx, ctx->stg_li[slot][v], P0 * 4));
            LV_CUDA(cudaMemcpyAsync(ctx->stg_li[slot][v].p, lidar_depth[v], P0 * 4, cudaMemcpyHostToDevice, cs));
        }
        ctx->stg_w[slot][v] = cameras[v].width;
        ctx->stg_h[slot][v] = cameras[v].height;
    }
    ctx->stg_views[slot] = n_views;
    ctx->stg_has_li[slot] = lidar_depth != nullptr;
    LV_CUDA(cudaEventRecord(ctx->stg_ready[slot], cs));
    return LVIGS_OK;
}

// ===========================================================================
// Autotuner (a10): tile size and compositing batch depth by measurement
// ===========================================================================
extern "C" lvigs_status lvigs_autotune_batched(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_batch *b,
                                               const lvigs_grads *gr, int trials, void *stream,
                                               lvigs_config *chosen, double *ms_out) {
    if (!ctx || !b || !gr || trials < 1) return ctx ? fail(ctx, LVIGS_ERR_INVALID_ARG, "bad autotune arguments")
                                                    : LVIGS_ERR_INVALID_ARG;
    struct Cand {
        int tw, th, bm;
    };
    const Cand cands[] = {{16, 16, 2}, {16, 16, 1}, {8, 8, 2}, {8, 8, 1}, {32, 16, 2}, {32, 16, 1}};
    const int nc = (int)(sizeof(cands) / sizeof(cands[0]));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LV_CUDA(cudaEventCreate(&e0));
    LV_CUDA(cudaEventCreate(&e1));
    const lvigs_config saved = ctx->cfg;
    const int saved_bm = ctx->bm;
    double best = 1e30;
    int best_i = -1;
    lvigs_batch bb = *b;
    bb.flags &= ~(LVIGS_STEP_HOST_LOSS | LVIGS_STEP_NO_GRAPH);
    lvigs_status st = LVIGS_OK;
    for (int i = 0; i < nc && st == LVIGS_OK; ++i) {
        ctx->cfg.tile_w = cands[i].tw;
        ctx->cfg.tile_h = cands[i].th;
        ctx->bm = cands[i].bm;
        ctx->batch.m_cap = 0; // size the instance list again for this tile size
        ctx->step_pending = false;
        // one eager step sizes the workspace, one more captures the graph
        for (int w = 0; w < 2 && st == LVIGS_OK; ++w) st = lvigs_train_step_batched(ctx, g, &bb, gr, stream);
        if (st != LVIGS_OK) break;
        cudaEventRecord(e0, s);
        for (int t = 0; t < trials && st == LVIGS_OK; ++t) st = lvigs_train_step_batched(ctx, g, &bb, gr, stream);
        cudaEventRecord(e1, s);
        if (st != LVIGS_OK) break;
        LV_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / trials;
        if (ms_out) ms_out[i] = per;
        if (per < best) {
            best = per;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LVIGS_OK || best_i < 0) {
        ctx->cfg = saved;
        ctx->bm = saved_bm;
        ctx->batch.m_cap = 0;
        return st != LVIGS_OK ? st : fail(ctx, LVIGS_ERR_STATE, "autotune measured nothing");
    }
    ctx->cfg.tile_w = cands[best_i].tw;
    ctx->cfg.tile_h = cands[best_i].th;
    ctx->bm = cands[best_i].bm;
    ctx->cfg.batch_depth = 32 * cands[best_i].bm;
    ctx->batch.m_cap = 0;
    ctx->step_pending = false;
    // view slots rendered with another tile size stay valid (they keep their own view set)
    if (chosen) *chosen = ctx->cfg;
    return LVIGS_OK;
}

// ---------------------------------------------------------------------------
// Map maintenance: Adam, expansion from colourised LiDAR points, pruning.
// ---------------------------------------------------------------------------

void lvigs_adam_config_default(lvigs_adam_config *c) {
    if (!c) return;
    c->lr_means = 1.6e-4f;
    c->lr_log_scales = 5e-3f;
    c->lr_quats = 1e-3f;
    c->lr_opacity = 5e-2f;
    c->lr_sh_dc = 2.5e-3f;
    c->lr_sh_rest = 2.5e-3f / 20.0f;
    c->beta1 = 0.9;
    c->beta2 = 0.999;
    c->eps = 1e-15;
}

namespace {

bool bufs_complete(const lvigs_param_buffers *b) {
    return b && b->means && b->log_scales && b->quats && b->opacity_logits && b->sh;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

} // namespace

lvigs_status lvigs_adam_step(const lvigs_param_buffers *params, const lvigs_grads *grads,
                             const lvigs_param_buffers *exp_avg, const lvigs_param_buffers *exp_avg_sq, int64_t n,
                             int sh_stride_k, int64_t step, const lvigs_adam_config *cfg_in, int zero_grads,
                             void *stream) {
    if (n < 0 || sh_stride_k < 1 || step < 1) return LVIGS_ERR_INVALID_ARG;
    lvigs_adam_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else lvigs_adam_config_default(&cfg);
    if (!(cfg.beta1 >= 0.0 && cfg.beta1 < 1.0) || !(cfg.beta2 >= 0.0 && cfg.beta2 < 1.0) || !(cfg.eps >= 0.0))
        return LVIGS_ERR_INVALID_ARG;
    if (n == 0) return LVIGS_OK;
    if (!bufs_complete(params) || !bufs_complete(exp_avg) || !bufs_complete(exp_avg_sq) || !grads ||
        !grads->d_means || !grads->d_log_scales || !grads->d_quats || !grads->d_opacity_logits || !grads->d_sh)
        return LVIGS_ERR_INVALID_ARG;
    AdamArgs A{};
    float *P[5] = {params->means, params->log_scales, params->quats, params->opacity_logits, params->sh};
    float *G[5] = {grads->d_means, grads->d_log_scales, grads->d_quats, grads->d_opacity_logits, grads->d_sh};
    float *M[5] = {exp_avg->means, exp_avg->log_scales, exp_avg->quats, exp_avg->opacity_logits, exp_avg->sh};
    float *V[5] = {exp_avg_sq->means, exp_avg_sq->log_scales, exp_avg_sq->quats, exp_avg_sq->opacity_logits,
                   exp_avg_sq->sh};
    const int64_t width[5] = {3, 3, 4, 1, 3 * (int64_t)sh_stride_k};
    const float lr[5] = {cfg.lr_means, cfg.lr_log_scales, cfg.lr_quats, cfg.lr_opacity, cfg.lr_sh_dc};
    A.unit_base[0] = 0;
    for (int s = 0; s < kAdamSegs; ++s) {
        AdamSeg &S = A.seg[s];
        S.p = P[s];
        S.g = G[s];
        S.m = M[s];
        S.v = V[s];
        S.len = n * width[s];
        S.lr = lr[s];
        S.lr_rest = s == 4 ? cfg.lr_sh_rest : lr[s];
        S.sh_k = s == 4 ? sh_stride_k : 0;
        S.vec = aligned16(S.p) && aligned16(S.g) && aligned16(S.m) && aligned16(S.v);
        A.unit_base[s + 1] = A.unit_base[s] + (S.len + 3) / 4;
    }
    A.b1 = (float)cfg.beta1;
    A.b2 = (float)cfg.beta2;
    A.omb1 = (float)(1.0 - cfg.beta1);
    A.omb2 = (float)(1.0 - cfg.beta2);
    A.eps = (float)cfg.eps;
    A.inv_bc1 = (float)(1.0 / (1.0 - std::pow(cfg.beta1, (double)step)));
    A.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(1.0 - std::pow(cfg.beta2, (double)step)));
    A.zero_grads = zero_grads ? 1 : 0;
    launch_adam(A, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LVIGS_OK : LVIGS_ERR_CUDA;
}

void lvigs_init_config_default(lvigs_init_config *c) {
    if (!c) return;
    c->init_opacity = 0.1f;
    c->min_dist2 = 1e-7f;
    c->tau_alpha = 0.5f;
    c->filter_literal = 0;
}

namespace {

// Uniform grid for k points in the box [lo, hi]: about one point per cell of
// the box's volume, at most 16384 cells per axis (so the binary32 cell
// coordinates stay within 1% of a cell of exact) and 2^24 cells in total.
KnnGrid make_grid(const float lo[3], const float hi[3], int64_t k) {
    double ext[3], emax = 0.0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = (double)hi[a] - (double)lo[a];
        emax = std::max(emax, ext[a]);
    }
    const double floor_ext = std::max(emax * 1e-3, 1e-6);
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= std::max(ext[a], floor_ext);
    double h = std::cbrt(vol / (double)std::max<int64_t>(k, 1));
    h = std::max(h, std::max(emax / 16000.0, 1e-6));
    KnnGrid G{};
    for (;;) {
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) {
            G.D[a] = (int)std::floor(ext[a] / h) + 1;
            cells *= G.D[a];
        }
        if (cells <= (double)(1 << 24) && G.D[0] <= 16384 && G.D[1] <= 16384 && G.D[2] <= 16384) break;
        h *= 1.25;
    }
    for (int a = 0; a < 3; ++a) G.o[a] = lo[a];
    G.h = (float)h;
    G.inv_h = (float)(1.0 / h);
    return G;
}

} // namespace

lvigs_status lvigs_append_gaussians(lvigs_ctx *ctx, const float *points, const float *colours, int64_t k,
                                    const lvigs_camera *cam, int level, const float *alpha,
                                    const lvigs_init_config *cfg_in, const lvigs_param_buffers *params,
                                    const lvigs_param_buffers *exp_avg, const lvigs_param_buffers *exp_avg_sq,
                                    int64_t n, int64_t capacity, int sh_stride_k, int64_t *n_out, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    if (!n_out || n < 0 || k < 0 || sh_stride_k < 1 || capacity < 0)
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "bad append arguments");
    if (k > 0 && (!points || !colours)) return fail(ctx, LVIGS_ERR_INVALID_ARG, "points / colours are NULL");
    if (!bufs_complete(params)) return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL parameter buffer");
    if ((exp_avg && !bufs_complete(exp_avg)) || (exp_avg_sq && !bufs_complete(exp_avg_sq)))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "incomplete Adam state buffers");
    if (n + k > capacity) return fail(ctx, LVIGS_ERR_CAPACITY, "n + k exceeds the parameter capacity");
    if (k >= ((int64_t)1 << 31) || n + k >= ((int64_t)1 << 31))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "too many Gaussians");
    lvigs_init_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else lvigs_init_config_default(&cfg);
    if (!(cfg.init_opacity > 0.f && cfg.init_opacity < 1.f) || !(cfg.min_dist2 > 0.f))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "init_opacity must be in (0,1) and min_dist2 > 0");
    if (alpha) LV_TRY(check_camera(ctx, cam, level));
    cudaStream_t s = (cudaStream_t)stream;
    *n_out = n;
    if (k == 0) return LVIGS_OK;

    const float *src_pts = points, *src_col = colours;
    LV_TRY(ensure(ctx, ctx->mp_small, 64));
    uint32_t *small = (uint32_t *)ctx->mp_small.p; // [0] count, [2..8) box
    int *box = (int *)(small + 2);
    const uint32_t *dev_count = nullptr;
    if (alpha) {
        const ViewDesc v = make_view(*cam, level, 16, 16);
        PointCamera C{};
        for (int i = 0; i < 9; ++i) C.R[i] = v.R[i];
        for (int i = 0; i < 3; ++i) C.t[i] = v.t[i];
        C.fx = v.fx;
        C.fy = v.fy;
        C.cx = v.cx;
        C.cy = v.cy;
        C.W = v.W;
        C.H = v.H;
        C.near = 0.2f;
        LV_TRY(ensure(ctx, ctx->mp_keep, (size_t)k * 4));
        LV_TRY(ensure(ctx, ctx->mp_offs, (size_t)(k + 1) * 4));
        LV_TRY(ensure(ctx, ctx->mp_scan, scan_tmp_words(k) * 4));
        LV_TRY(ensure(ctx, ctx->mp_pts, (size_t)k * 12));
        LV_TRY(ensure(ctx, ctx->mp_col, (size_t)k * 12));
        uint32_t *keep = (uint32_t *)ctx->mp_keep.p, *offs = (uint32_t *)ctx->mp_offs.p;
        launch_point_filter(points, k, C, alpha, cfg.tau_alpha, cfg.filter_literal, keep, s);
        launch_scan(keep, nullptr, 1, offs, offs + k, nullptr, k, (uint32_t *)ctx->mp_scan.p, s);
        launch_gather_points(points, colours, k, keep, offs, (float *)ctx->mp_pts.p, (float *)ctx->mp_col.p, s);
        src_pts = (const float *)ctx->mp_pts.p;
        src_col = (const float *)ctx->mp_col.p;
        dev_count = offs + k;
    }

    // bounding box of the kept points -> grid; one wait reads the count and the box
    launch_bbox(src_pts, k, dev_count, box, s);
    LV_CUDA(cudaMemcpyAsync(ctx->host_counters, box, 24, cudaMemcpyDeviceToHost, s));
    if (dev_count) LV_CUDA(cudaMemcpyAsync(ctx->host_counters + 6, dev_count, 4, cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const int64_t kk = dev_count ? (int64_t)ctx->host_counters[6] : k;
    if (kk == 0) return LVIGS_OK;
    int hbox[6];
    std::memcpy(hbox, ctx->host_counters, 24);
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = ord_to_float(hbox[a]);
        hi[a] = ord_to_float(hbox[3 + a]);
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]))
            return fail(ctx, LVIGS_ERR_INVALID_ARG, "non-finite point coordinates");
    }
    const KnnGrid G = make_grid(lo, hi, kk);
    const uint32_t n_cells = (uint32_t)G.D[0] * (uint32_t)G.D[1] * (uint32_t)G.D[2];
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)n_cells) ++bits;

    LV_TRY(ensure(ctx, ctx->mp_keys, (size_t)kk * 4));
    LV_TRY(ensure(ctx, ctx->mp_vals, (size_t)kk * 4));
    LV_TRY(ensure(ctx, ctx->mp_keys2, (size_t)kk * 4));
    LV_TRY(ensure(ctx, ctx->mp_vals2, (size_t)kk * 4));
    LV_TRY(ensure(ctx, ctx->mp_radix, radix_tmp_words(kk) * 4));
    LV_TRY(ensure(ctx, ctx->mp_cells, (size_t)n_cells * sizeof(uint2)));
    LV_TRY(ensure(ctx, ctx->mp_logs, (size_t)kk * 4));
    LV_TRY(ensure(ctx, ctx->mp_spts, (size_t)kk * sizeof(float4)));
    uint32_t *keys = (uint32_t *)ctx->mp_keys.p, *vals = (uint32_t *)ctx->mp_vals.p;
    uint32_t *keys2 = (uint32_t *)ctx->mp_keys2.p, *vals2 = (uint32_t *)ctx->mp_vals2.p;
    launch_cell_keys(src_pts, kk, G, keys, vals, s);
    const int alt = launch_radix_sort(keys, vals, keys2, vals2, nullptr, kk, bits, (uint32_t *)ctx->mp_radix.p, s);
    const uint32_t *skeys = alt ? keys2 : keys, *svals = alt ? vals2 : vals;
    launch_set_u32(small, (uint32_t)kk, s);
    launch_ranges(skeys, small, kk, (uint2 *)ctx->mp_cells.p, n_cells, s);
    launch_knn(src_pts, kk, G, (const uint2 *)ctx->mp_cells.p, svals, (float4 *)ctx->mp_spts.p, cfg.min_dist2,
               (float *)ctx->mp_logs.p, s);

    const ParamBufs P{params->means, params->log_scales, params->quats, params->opacity_logits, params->sh};
    ParamBufs Mb{}, Vb{};
    if (exp_avg) Mb = {exp_avg->means, exp_avg->log_scales, exp_avg->quats, exp_avg->opacity_logits, exp_avg->sh};
    if (exp_avg_sq)
        Vb = {exp_avg_sq->means, exp_avg_sq->log_scales, exp_avg_sq->quats, exp_avg_sq->opacity_logits,
              exp_avg_sq->sh};
    const double o = (double)cfg.init_opacity;
    const float logit = (float)std::log(o / (1.0 - o));
    const float inv_c0 = (float)(2.0 * std::sqrt(3.14159265358979323846));
    launch_init_rows(src_pts, src_col, (const float *)ctx->mp_logs.p, kk, n, P, Mb, Vb, sh_stride_k, logit, inv_c0, s);
    LV_CUDA(cudaGetLastError());
    *n_out = n + kk;
    return LVIGS_OK;
}

lvigs_status lvigs_prune_gaussians(lvigs_ctx *ctx, float min_opacity, const lvigs_param_buffers *params,
                                   const lvigs_param_buffers *exp_avg, const lvigs_param_buffers *exp_avg_sq,
                                   int64_t n, int sh_stride_k, int64_t *n_out, void *stream) {
    if (!ctx) return LVIGS_ERR_INVALID_ARG;
    if (!n_out || n < 0 || n >= ((int64_t)1 << 31) || sh_stride_k < 1 || !(min_opacity > 0.f && min_opacity < 1.f))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "bad prune arguments");
    if (!bufs_complete(params)) return fail(ctx, LVIGS_ERR_INVALID_ARG, "NULL parameter buffer");
    if ((exp_avg && !bufs_complete(exp_avg)) || (exp_avg_sq && !bufs_complete(exp_avg_sq)))
        return fail(ctx, LVIGS_ERR_INVALID_ARG, "incomplete Adam state buffers");
    *n_out = n;
    if (n == 0) return LVIGS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const double m = (double)min_opacity;
    const float thr = (float)std::log(m / (1.0 - m));
    LV_TRY(ensure(ctx, ctx->mp_keep, (size_t)n * 4));
    LV_TRY(ensure(ctx, ctx->mp_offs, (size_t)(n + 1) * 4));
    LV_TRY(ensure(ctx, ctx->mp_scan, scan_tmp_words(n) * 4));
    uint32_t *keep = (uint32_t *)ctx->mp_keep.p, *offs = (uint32_t *)ctx->mp_offs.p;
    launch_prune_flags(params->opacity_logits, n, thr, keep, s);
    launch_scan(keep, nullptr, 1, offs, offs + n, nullptr, n, (uint32_t *)ctx->mp_scan.p, s);
    // every buffer compacted through its own scratch segment; the kernels read
    // the kept count on the device, so the only wait is for the count returned
    const int widths[5] = {3, 3, 4, 1, 3 * sh_stride_k};
    PruneArgs A{};
    A.n = n;
    A.keep = keep;
    A.offs = offs;
    size_t words = 0, seg_off[kPruneSegs];
    const lvigs_param_buffers *sets[3] = {params, exp_avg, exp_avg_sq};
    for (const lvigs_param_buffers *b : sets) {
        if (!b) continue;
        float *bufs[5] = {b->means, b->log_scales, b->quats, b->opacity_logits, b->sh};
        for (int f = 0; f < 5; ++f) {
            seg_off[A.nseg] = words;
            PruneSeg &S = A.seg[A.nseg++];
            S.buf = bufs[f];
            S.w = widths[f];
            S.vec = ((uintptr_t)bufs[f] & 15) == 0;
            words += ((size_t)n * widths[f] + 3) & ~(size_t)3; // segments start 16-byte aligned
        }
    }
    LV_TRY(ensure(ctx, ctx->mp_tmp, words * 4));
    for (int i = 0; i < A.nseg; ++i) A.seg[i].tmp = (float *)ctx->mp_tmp.p + seg_off[i];
    launch_prune_compact(A, s);
    LV_CUDA(cudaMemcpyAsync(ctx->host_counters, offs + n, 4, cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const int64_t kept = ctx->host_counters[0];
    LV_CUDA(cudaGetLastError());
    *n_out = kept;
    return LVIGS_OK;
}
