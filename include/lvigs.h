/*
 * lvigs.h -- C ABI of the GB300 (sm_103a) differentiable Gaussian-splatting
 * hot path of LVI-GS (arxiv 2411.02703).
 *
 * The library renders colour, depth and visibility images from a set of 3D
 * Gaussians seen by a pinhole camera at a pyramid level (Sec. III-B,
 * Eq. (2)-(7); Sec. III-D), evaluates the mapping loss (Sec. III-E,
 * Eq. (10)-(12)) and returns the gradient of a loss with respect to every
 * Gaussian parameter (means, log-scales, quaternions, opacity logits and
 * spherical-harmonic coefficients; the parameter set of Sec. III-E).
 *
 * Conventions shared by every entry point
 *   - Every pointer to image, parameter or gradient data is a DEVICE pointer
 *     into memory the caller owns (contiguous, float32, layouts below), unless
 *     a flag says otherwise.  The library owns only its workspace.
 *   - Work is enqueued on the CUDA stream passed as `stream` (a cudaStream_t;
 *     NULL is the legacy default stream) and runs asynchronously.  Argument
 *     errors are returned before anything is enqueued.  Errors found on the
 *     device are latched in the context and returned by lvigs_sync_status().
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - Fixed constants of the method (readings of the paper, which is silent
 *     on them): near plane 0.2, 0.3 px^2 dilation of the projected
 *     covariance, Jacobian clamp at 1.3 x tan(half field of view), radius
 *     ceil(3 sqrt(lambda_max)) with the eigenvalue discriminant floored at
 *     0.1, alpha clamp 0.99, alpha cut-off 1/255, compositing stops before a
 *     Gaussian that would take the transmittance below 1e-4, black
 *     background, view-space z as the depth d_i of Eq. (4), real spherical
 *     harmonics up to degree 3 plus 0.5, clamped at 0.
 *
 * Layouts
 *   means [n,3], log_scales [n,3], quats [n,4] (w,x,y,z; normalised inside),
 *   opacity_logits [n] (opacity = sigmoid), sh [n, sh_stride_k, 3];
 *   images are planar: rgb [3,H,W], depth [H,W], alpha [H,W].
 */
#ifndef LVIGS_H
#define LVIGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LVIGS_MAX_VIEWS 32 /* views per batched call */
#define LVIGS_MAX_LEVEL 4  /* pyramid levels 0..4 */

typedef enum {
    LVIGS_OK = 0,
    LVIGS_ERR_INVALID_ARG = 1,   /* a NULL, size, level or layout outside the contract */
    LVIGS_ERR_OUT_OF_MEMORY = 2, /* workspace allocation failed */
    LVIGS_ERR_CUDA = 3,          /* a CUDA runtime call failed (see lvigs_last_error) */
    LVIGS_ERR_CAPACITY = 4,      /* workspace cap or instance capacity exceeded */
    LVIGS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    LVIGS_ERR_STATE = 6          /* a view slot that is free, stale or of another context */
} lvigs_status;

typedef struct lvigs_ctx lvigs_ctx;

/* Context configuration.  Tile size changes which Gaussians a pixel composites
 * (a pixel composites every Gaussian whose tile rectangle covers its tile), so
 * results depend on it; batch_depth does not change results. */
typedef struct {
    int tile_w, tile_h;         /* 16x16 (default), 8x8 or 32x16 */
    int batch_depth;            /* Gaussians each compositing warp stages per round: 0 (auto), 32 or 64 */
    size_t max_workspace_bytes; /* 0 = no cap; else LVIGS_ERR_CAPACITY beyond it */
} lvigs_config;

/* Gaussian map (device pointers, caller-owned, float32). */
typedef struct {
    const float *means, *log_scales, *quats, *opacity_logits, *sh;
    int64_t n;       /* number of Gaussians, 0 <= n < 2^31 */
    int sh_degree;   /* active SH degree 0..3 (Sec. III-E schedule) */
    int sh_stride_k; /* coefficients per Gaussian in `sh`, >= (sh_degree+1)^2 */
} lvigs_gaussians;

/* Pinhole camera at pyramid level 0.  R, t map world to camera coordinates
 * (x right, y down, z forward): the pose [Q_iw, T_iw] of Eq. (7). */
typedef struct {
    float R[9]; /* row-major */
    float t[3];
    float fx, fy, cx, cy;
    int width, height;
} lvigs_camera;

/* Render outputs (device, caller-owned; sized for the level's W x H). */
typedef struct {
    float *rgb;   /* [3,H,W]  C_p of Eq. (3) */
    float *depth; /* [H,W]    D_p of Eq. (4) */
    float *alpha; /* [H,W]    V_p of Eq. (5) */
} lvigs_image_out;

/* Parameter gradients (device, caller-owned, same layouts as the parameters).
 * accumulate = 0 overwrites, 1 adds to the current contents. */
typedef struct {
    float *d_means, *d_log_scales, *d_quats, *d_opacity_logits, *d_sh;
    int accumulate;
} lvigs_grads;

/* Flags of a batched step. */
#define LVIGS_STEP_HOST_TARGETS 1 /* gt_rgb / lidar_depth are pinned HOST pointers, copied in */
#define LVIGS_STEP_HOST_LOSS 2    /* losses is a HOST pointer; the call waits for the step */
#define LVIGS_STEP_NO_GRAPH 4     /* enqueue kernels directly instead of replaying a CUDA graph */
#define LVIGS_STEP_STAGED_TARGETS 8 /* targets were copied in by lvigs_stage_targets into staged_slot;
                                      gt_rgb / lidar_depth are not read */
#define LVIGS_STEP_HOST_LOSS_ASYNC 16 /* losses is a pinned (page-locked) HOST pointer that the step's
                                        kernels write directly; the call does not wait (order a later
                                        read with an event on the stream) */

/* Staging slots of lvigs_stage_targets (double buffering). */
#define LVIGS_STAGE_SLOTS 2

/* One batched training step over several keyframes at mixed pyramid levels. */
typedef struct {
    int n_views;                     /* 1..LVIGS_MAX_VIEWS */
    const lvigs_camera *cameras;     /* host array [n_views], level-0 cameras */
    const int *levels;               /* host array [n_views], 0..LVIGS_MAX_LEVEL */
    const float *const *gt_rgb;      /* host array of n_views pointers to level-0 [3,H0,W0] */
    const float *const *lidar_depth; /* host array of n_views pointers to level-0 [H0,W0]; 0 = no return */
    float lambda_ssim;               /* lambda of Eq. (11) */
    float lambda_depth;              /* lambda_d of Eq. (10) */
    int flags;                       /* LVIGS_STEP_* */
    double *losses;                  /* [n_views,4]: total, L1, mean SSIM, depth L1 (device memory
                                        unless a HOST_LOSS flag says otherwise) */
    float *const *rgb_out;           /* optional host array of n_views device pointers, or NULL */
    float *const *depth_out;         /* optional, as rgb_out */
    float *const *alpha_out;         /* optional, as rgb_out */
    int staged_slot;                 /* with LVIGS_STEP_STAGED_TARGETS: 0..LVIGS_STAGE_SLOTS-1 */
} lvigs_batch;

/* Copy the level-0 targets of a batched step (Sec. III-D: each keyframe's image
 * and projected LiDAR depth) from pinned HOST memory into the context's
 * staging slot `slot`, on `copy_stream`, so that the copy of the next step's
 * targets runs while the current step computes.  gt_rgb[v] points to
 * [3,H0,W0] float32 and lidar_depth[v] (array may be NULL: no LiDAR term) to
 * [H0,W0] float32 (0 = no return), sizes from cameras[v].  The copy first
 * waits, on copy_stream, for the last batched step that read this slot; a
 * later lvigs_train_step_batched with LVIGS_STEP_STAGED_TARGETS and
 * staged_slot = slot waits for the copy on its own stream and must describe
 * the same number of views and sizes.  The host buffers must stay valid until
 * the copy has completed (e.g. until that step returns with
 * LVIGS_STEP_HOST_LOSS).  Errors: LVIGS_ERR_INVALID_ARG (slot, view count,
 * camera or NULL pointer), LVIGS_ERR_OUT_OF_MEMORY, LVIGS_ERR_CUDA. */
lvigs_status lvigs_stage_targets(lvigs_ctx *ctx, int slot, int n_views, const lvigs_camera *cameras,
                                 const float *const *gt_rgb, const float *const *lidar_depth, void *copy_stream);

/* ----------------------------------------------------------------------- */

/* Library version string (static storage). */
const char *lvigs_version(void);

/* Default configuration (16x16 tiles, automatic batch depth, no cap). */
void lvigs_config_default(lvigs_config *cfg);

/* Create a context on the current CUDA device.  cfg may be NULL (defaults).
 * Returns LVIGS_ERR_INVALID_ARG for an unsupported tile size. */
lvigs_status lvigs_create(lvigs_ctx **out, const lvigs_config *cfg);

/* Destroy a context and free its workspace (synchronises the device). */
void lvigs_destroy(lvigs_ctx *ctx);

/* Image size of pyramid level `level` of a level-0 camera: W >> level, H >> level. */
lvigs_status lvigs_level_size(const lvigs_camera *cam, int level, int *width, int *height);

/* Forward render of one view at pyramid level `level` (Sec. III-B, Eq. (2)-(7);
 * Sec. III-D).  Writes out->rgb/depth/alpha at the level's size and returns
 * in *view_slot a handle of the compositing state kept for lvigs_backward.
 * The parameter buffers must stay unchanged until the backward call.  This
 * call waits once on the stream to learn the number of (tile, Gaussian)
 * instances and size the workspace. */
lvigs_status lvigs_render(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_camera *cam,
                          int level, const lvigs_image_out *out, int *view_slot, void *stream);

/* lvigs_render without the wait: the instance lists are sized from the
 * largest lvigs_render (or earlier no-wait render) of this context instead of
 * the device's count, so the call only enqueues work.  Same arguments,
 * results and slot handle as lvigs_render.  If the view has more (tile,
 * Gaussian) instances than that capacity, the lists are cut at the capacity
 * (the images then miss the dropped instances) and LVIGS_ERR_CAPACITY is
 * latched for lvigs_sync_status: render that view once with lvigs_render,
 * which grows the capacity, and repeat.  A context that has rendered nothing
 * yet waits once, like lvigs_render. */
lvigs_status lvigs_render_async(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_camera *cam,
                                int level, const lvigs_image_out *out, int *view_slot, void *stream);

/* Gradients of a loss with respect to the Gaussian parameters, given the
 * gradients of that loss with respect to the images of `view_slot`
 * (dL_dalpha may be NULL).  Reverse traversal of each pixel's list with the
 * transmittance recovered by division (no per-Gaussian state is stored). */
lvigs_status lvigs_backward(lvigs_ctx *ctx, int view_slot, const float *dL_drgb,
                            const float *dL_ddepth, const float *dL_dalpha,
                            const lvigs_grads *grads, void *stream);

/* Mapping loss of Eq. (10)-(12) for one W x H image:
 *   L = (1 - lambda) L1(rgb, gt) + lambda (1 - mean SSIM) + lambda_d L_d,
 * SSIM with an 11x11 Gaussian window (sigma 1.5), zero padding,
 * C1 = 0.01^2, C2 = 0.03^2, averaged over channels and pixels; L_d is the
 * mean |depth - lidar| over pixels with lidar > 0 (0 if none).
 * loss_out: 4 doubles (total, L1, mean SSIM, L_d) in device memory or
 * page-locked host memory (written by the kernel; LVIGS_ERR_INVALID_ARG for
 * anything else).  d_rgb / d_depth receive dL/drgb and dL/ddepth (either may
 * be NULL to skip gradients). */
lvigs_status lvigs_loss(lvigs_ctx *ctx, int width, int height, const float *rgb,
                        const float *depth, const float *gt_rgb, const float *lidar_depth,
                        float lambda_ssim, float lambda_depth, double *loss_out, float *d_rgb,
                        float *d_depth, void *stream);

/* lvigs_loss for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the loss above.
 *
 * Who cannot allocate: a host whose allocator already owns the device-memory
 * budget (a caching allocator holding the free memory, an embedded process
 * with a fixed memory plan), and a real-time loop such as the tracking thread
 * of a SLAM front end, where cudaMalloc / cudaFree are off limits because
 * cudaFree synchronises the whole device.  lvigs_loss grows its workspace in a
 * context with cudaMalloc; this entry point takes no context and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Its scratch is a fixed 12 MiB array inside the library's device code, held
 * by every GPU that loads the library until the process exits.  Images are
 * limited to LVIGS_LOSS_NOALLOC_MAX_PIXELS pixels (640 x 512) and
 * LVIGS_LOSS_NOALLOC_MAX_SIDE pixels per side; larger ones return
 * LVIGS_ERR_CAPACITY before anything is enqueued.
 *
 * Arguments, layouts and results are those of lvigs_loss, on the current
 * device (`stream` must belong to it).  LVIGS_ERR_INVALID_ARG for the argument
 * errors of lvigs_loss; LVIGS_ERR_CUDA when a CUDA call fails.
 *
 * Set-up: the first call on a device looks up the device address of the
 * scratch array (which may create the device's primary context and load the
 * library's module onto it), so make that first call before any stream
 * capture begins.  The address is kept with the id of the context it came
 * from; after a device reset (cudaDeviceReset, or the primary context released
 * and created again) the next call looks it up again in the new context, so
 * that call is a first call too.
 *
 * Every call on a device shares the one array, and it keeps what the last
 * call left (no call depends on it: each writes everything it reads).  Calls
 * that overlap on the GPU (other streams, other host threads) race on it:
 * order them, for example on one stream. */
#define LVIGS_LOSS_NOALLOC_MAX_PIXELS 327680
#define LVIGS_LOSS_NOALLOC_MAX_SIDE 2048
lvigs_status lvigs_loss_noalloc(int width, int height, const float *rgb, const float *depth,
                                const float *gt_rgb, const float *lidar_depth, float lambda_ssim,
                                float lambda_depth, double *loss_out, float *d_rgb, float *d_depth,
                                void *stream);

/* One pyramid level down (Sec. III-D): rgb 2x2 box mean, depth the mean of
 * the valid (> 0) samples of each 2x2 block (0 if none).  Output size is
 * (width/2) x (height/2). */
lvigs_status lvigs_pyramid_down(int width, int height, const float *rgb, const float *depth,
                                float *rgb_out, float *depth_out, void *stream);

/* Batched training step: every view rendered, its loss evaluated against its
 * level of the target pyramid and differentiated, gradients accumulated over
 * views into `grads`, all in one CUDA graph (unless LVIGS_STEP_NO_GRAPH).
 * Returns after enqueueing (or after the step with LVIGS_STEP_HOST_LOSS).
 * Device-side capacity overflow is reported by lvigs_sync_status; the
 * capacity grows for the next call. */
lvigs_status lvigs_train_step_batched(lvigs_ctx *ctx, const lvigs_gaussians *g,
                                      const lvigs_batch *batch, const lvigs_grads *grads,
                                      void *stream);

/* Autotuner of the batched step (a10): times `trials` graph replays of the
 * step for each candidate (tile 16x16, 8x8, 32x16) x (batch depth 64, 32) and
 * leaves the context configured with the fastest, which is written to
 * *chosen (ms_out, optional, receives the 6 per-step times in that order).
 * The tile size is part of what is computed (a pixel composites the Gaussians
 * whose rectangle covers its tile), so results follow the chosen tile size.
 * The candidate steps write `grads` and `batch->losses` like a normal step. */
lvigs_status lvigs_autotune_batched(lvigs_ctx *ctx, const lvigs_gaussians *g, const lvigs_batch *batch,
                                    const lvigs_grads *grads, int trials, void *stream,
                                    lvigs_config *chosen, double *ms_out);

/* Parity hooks: the sorted 64-bit keys ((tile id << 32) | float bits of depth)
 * and Gaussian indices of `view_slot`.  With keys == NULL only *m is set.
 * keys/vals are device pointers with room for *m entries on input (m_cap). */
lvigs_status lvigs_debug_keys(lvigs_ctx *ctx, int view_slot, uint64_t *keys, uint32_t *vals,
                              int64_t m_cap, int64_t *m, void *stream);

/* Parity hook: per-tile [start, end) of the sorted list (device uint32 [n_tiles,2])
 * and the per-pixel contributor count and final transmittance (device). */
lvigs_status lvigs_debug_state(lvigs_ctx *ctx, int view_slot, uint32_t *ranges, int32_t *n_contrib,
                               float *final_T, int *n_tiles, void *stream);

/* Parity hook: y[i] = exp(x[i]) rounded once to binary32 as the key stage
 * computes the scales (the value of exp in binary64, rounded; Sec. III-E
 * scale activation), for n device floats. */
lvigs_status lvigs_debug_exp_key(const float *x, float *y, int64_t n, void *stream);

/* Wait for `stream` and return any error latched on the device since the
 * last call (capacity overflow, bounded-wait timeout), clearing it. */
lvigs_status lvigs_sync_status(lvigs_ctx *ctx, void *stream);

/* Release a view slot (its state becomes stale). */
lvigs_status lvigs_release_view(lvigs_ctx *ctx, int view_slot);

/* Last error message of the context (static storage of the context). */
const char *lvigs_last_error(const lvigs_ctx *ctx);

/* Opt-in device timing of eagerly enqueued work (not of graph replays):
 * CUDA events around each phase below, on the stream the phase runs on. */
enum {
    LVIGS_PHASE_PREPROCESS = 0,     /* a1 */
    LVIGS_PHASE_COMPACT = 1,        /* visibility scan + compaction */
    LVIGS_PHASE_DEPTH_SORT = 2,     /* a3, depth radix sort of visible Gaussians */
    LVIGS_PHASE_OFFSETS = 3,        /* a2, scan of tiles touched */
    LVIGS_PHASE_EMIT = 4,           /* a2, instance emission */
    LVIGS_PHASE_TILE_SORT = 5,      /* a3, tile-id radix sort of instances */
    LVIGS_PHASE_RANGES = 6,         /* a4 */
    LVIGS_PHASE_COMPOSITE_FWD = 7,  /* a5, per-chunk compositing */
    LVIGS_PHASE_LOSS = 8,           /* a8 */
    LVIGS_PHASE_COMPOSITE_BWD = 9,  /* a6 */
    LVIGS_PHASE_PREPROCESS_BWD = 10,/* a7 */
    LVIGS_PHASE_PYRAMID = 11,       /* a9 */
    LVIGS_PHASE_COMBINE = 12,       /* a5, combine of multi-chunk tile lists */
    LVIGS_N_PHASES = 13
};
lvigs_status lvigs_profile_enable(lvigs_ctx *ctx, int enable);
/* Waits for the recorded phases; writes the summed milliseconds and call
 * counts per phase (arrays of LVIGS_N_PHASES, either may be NULL) and the
 * kernel launches per replay of the batched-step graph, then resets. */
lvigs_status lvigs_profile_read(lvigs_ctx *ctx, double *ms, int64_t *calls, int *kernels_per_step);

/* ----------------------------------------------------------------------- */
/* Map maintenance around the differentiable path: the optimiser step, map  */
/* expansion from colourised LiDAR points and pruning (Sec. III-C, III-E).  */
/* ----------------------------------------------------------------------- */

/* Five parameter-shaped device buffers (caller-owned, mutable) in the layouts
 * of lvigs_gaussians; rows beyond the live count are capacity. */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
} lvigs_param_buffers;

/* Optimiser of the Gaussian parameters.  Sec. III-E names the parameters
 * (position, rotation, scaling, density, SH colour) and the loss but not the
 * optimiser; Adam with per-parameter learning rates is the reading taken.
 * Defaults: lr means 1.6e-4, log-scales 5e-3, quaternions 1e-3, opacity
 * 5e-2, SH band 0 2.5e-3, higher SH bands 1.25e-4; beta1 0.9, beta2 0.999,
 * eps 1e-15. */
typedef struct {
    float lr_means, lr_log_scales, lr_quats, lr_opacity, lr_sh_dc, lr_sh_rest;
    double beta1, beta2, eps; /* double: 1 - beta is formed before rounding to binary32 */
} lvigs_adam_config;

void lvigs_adam_config_default(lvigs_adam_config *cfg);

/* One Adam step over rows [0, n) of every parameter, in one launch:
 *   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
 *   p <- p - lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps),
 * with t = `step` >= 1 the step count after this update.  exp_avg and
 * exp_avg_sq hold m and v (zero before the first step).  zero_grads = 1 also
 * clears the gradient buffers (grads->accumulate is ignored).  cfg may be
 * NULL (defaults).  LVIGS_ERR_INVALID_ARG on a NULL buffer with n > 0, n < 0,
 * sh_stride_k < 1, step < 1 or betas outside [0, 1). */
lvigs_status lvigs_adam_step(const lvigs_param_buffers *params, const lvigs_grads *grads,
                             const lvigs_param_buffers *exp_avg, const lvigs_param_buffers *exp_avg_sq,
                             int64_t n, int sh_stride_k, int64_t step, const lvigs_adam_config *cfg,
                             int zero_grads, void *stream);

/* Initialisation of new Gaussians (Sec. III-E) and the filter on Gaussian
 * additions (Sec. III-C). */
typedef struct {
    float init_opacity;  /* opacity of a new Gaussian (stored as its logit): 0.1 */
    float min_dist2;     /* floor of the mean squared neighbour distance: 1e-7 */
    float tau_alpha;     /* filter threshold tau_alpha: 0.5 */
    int filter_literal;  /* 0 (default): drop a point whose pixel has transparency
                            1 - V_p <= tau_alpha (the map is already opaque there);
                            1: drop when V_p <= tau_alpha, the inequality as printed */
} lvigs_init_config;

void lvigs_init_config_default(lvigs_init_config *cfg);

/* Map expansion: Gaussians for k colourised LiDAR points (device float
 * points [k,3], colours [k,3] in [0,1]) are written at rows
 * [n, n + k_kept) of `params`, in the points' order:
 *   centre = the point; log-scale (all three axes) = 0.5 ln(max(d2, min_dist2))
 *   with d2 the mean squared distance to the 3 nearest other kept points
 *   (fewer if there are fewer; 0 if none); quaternion (1,0,0,0); opacity
 *   logit = ln(o / (1 - o)); SH band 0 = (colour - 0.5) / Y_00 with
 *   Y_00 = 1 / (2 sqrt(pi)), higher bands 0.
 * Filter (when alpha != NULL): each point is projected into `cam` at pyramid
 * level `level` in binary32, one rounding per operation in the order
 * x_c = ((R00 x + R01 y) + R02 z) + t0 (likewise y_c, z_c), u = (fx x_c)/z_c
 * + cx, px = floor(u + 0.5) (likewise v, py); a point with z_c > 0.2 inside
 * the image is dropped per cfg->filter_literal against alpha[py, px] (the
 * V_p image of Eq. (5) at that level, [H_l, W_l]); other points are kept.
 * exp_avg / exp_avg_sq (either may be NULL) get zero rows.  Every buffer must
 * have `capacity` rows; LVIGS_ERR_CAPACITY if n + k > capacity (checked
 * before any work).  *n_out receives n + k_kept; the call waits on `stream`.
 * cfg may be NULL (defaults).  Uses the context's workspace. */
lvigs_status lvigs_append_gaussians(lvigs_ctx *ctx, const float *points, const float *colours, int64_t k,
                                    const lvigs_camera *cam, int level, const float *alpha,
                                    const lvigs_init_config *cfg, const lvigs_param_buffers *params,
                                    const lvigs_param_buffers *exp_avg, const lvigs_param_buffers *exp_avg_sq,
                                    int64_t n, int64_t capacity, int sh_stride_k, int64_t *n_out, void *stream);

/* Pruning (the prunable opacity of Sec. III-C): rows [0, n) whose opacity
 * sigmoid(logit) is below min_opacity are removed from `params` and the Adam
 * state (either may be NULL), keeping the order of the rest.  The test is
 * logit >= (float)ln(m / (1 - m)), computed in double and rounded once.
 * Gradient buffers are not touched: the next backward should overwrite them
 * (accumulate = 0).  *n_out receives the count kept; the call waits on
 * `stream`.  min_opacity in (0, 1). */
lvigs_status lvigs_prune_gaussians(lvigs_ctx *ctx, float min_opacity, const lvigs_param_buffers *params,
                                   const lvigs_param_buffers *exp_avg, const lvigs_param_buffers *exp_avg_sq,
                                   int64_t n, int sh_stride_k, int64_t *n_out, void *stream);

/* Work counts of the last batched step (waits on `stream`): out[0] visible
 * (view, Gaussian) pairs, out[1] (tile, Gaussian) instances, out[2] the sum
 * over pixels of the contributor counts, out[3] pixels rendered. */
lvigs_status lvigs_step_stats(lvigs_ctx *ctx, int64_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LVIGS_H */
