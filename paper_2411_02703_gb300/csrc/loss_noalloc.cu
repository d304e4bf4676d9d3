// loss_noalloc.cu -- lvigs_loss_noalloc: the mapping loss of lvigs_loss for
// callers that must not allocate device memory.
//
// Who needs it: a host that owns the whole device-memory budget (a caching
// allocator that already holds the free memory, an embedded process with a
// fixed memory plan), and a real-time loop (the tracking thread of a SLAM
// front end) in which cudaMalloc / cudaFree are off limits because cudaFree
// synchronises the whole device and cudaMalloc can stall on the driver.
// lvigs_loss cannot serve them: its workspace lives in a context that grows
// it with cudaMalloc on first use.  Here the workspace is a fixed array in
// the library's own device image, created when the module is loaded on a
// device and held by every device that loads the library until the process
// exits.
//
// The kernels are those of lvigs_loss (loss.cu); only where their scratch
// lives differs, so results are identical for identical inputs.
#include <cuda.h>

#include <mutex>

#include "lvigs.h"
#include "lvigs_internal.cuh"

using namespace lvigs;

namespace {

// Worst case of loss_tmp_bytes over images with at most
// LVIGS_LOSS_NOALLOC_MAX_PIXELS pixels and at most LVIGS_LOSS_NOALLOC_MAX_SIDE
// pixels per side is 11,809,056 bytes (164 x 1998: the derivative maps, 9
// floats a pixel, plus 32 bytes for each of 378 32x32 tiles); 12 MiB covers it.
constexpr size_t kScratchBytes = size_t(12) << 20;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; nothing in it has to start at zero
// (each call writes every element it later reads).
static __device__ __align__(256) unsigned char lvigs_loss_scratch[kScratchBytes];

// Device address of lvigs_loss_scratch per device ordinal, with the id of the
// context it was looked up in.  A device reset (or the primary context being
// released and created again) loads the module afresh, possibly elsewhere, so
// the address is valid only while the context that gave it is current.
struct ScratchSlot {
    unsigned long long ctx_id = 0;
    void *addr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_setup_mu;

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the
// library links the runtime only).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

lvigs_status current_context_id(unsigned long long *id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return LVIGS_ERR_CUDA;
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return LVIGS_ERR_CUDA;
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return LVIGS_ERR_CUDA;
    return LVIGS_OK;
}

// With the caller's device current: the device address of the scratch array.
// Host code may not use the symbol itself (it names a host-side shadow, not
// device memory), so the address comes from cudaGetSymbolAddress, once per
// device and context.  That first lookup may create the device's primary
// context and load the module onto it.
lvigs_status scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LVIGS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    ScratchSlot &slot = g_scratch[dev];
    unsigned long long id = 0;
    // no current context yet: the lookup below creates it
    if (current_context_id(&id) == LVIGS_OK && slot.addr && slot.ctx_id == id) {
        *out = slot.addr;
        return LVIGS_OK;
    }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, lvigs_loss_scratch);
    if (e != cudaSuccess || !p) return LVIGS_ERR_CUDA;
    const lvigs_status st = current_context_id(&id);
    if (st != LVIGS_OK) return st;
    slot.addr = p;
    slot.ctx_id = id;
    *out = p;
    return LVIGS_OK;
}

} // namespace

static_assert(kScratchBytes % 256 == 0, "scratch array size");

extern "C" lvigs_status lvigs_loss_noalloc(int width, int height, const float *rgb, const float *depth,
                                           const float *gt_rgb, const float *lidar_depth, float lambda_ssim,
                                           float lambda_depth, double *loss_out, float *d_rgb, float *d_depth,
                                           void *stream) {
    // argument and size checks come first: nothing is enqueued on an error
    if (width <= 0 || height <= 0 || !rgb || !gt_rgb || !loss_out) return LVIGS_ERR_INVALID_ARG;
    if (lidar_depth && !depth) return LVIGS_ERR_INVALID_ARG;
    if (!(lambda_ssim >= 0.f && lambda_ssim <= 1.f)) return LVIGS_ERR_INVALID_ARG;
    if (width > LVIGS_LOSS_NOALLOC_MAX_SIDE || height > LVIGS_LOSS_NOALLOC_MAX_SIDE ||
        (int64_t)width * height > LVIGS_LOSS_NOALLOC_MAX_PIXELS)
        return LVIGS_ERR_CAPACITY;
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
    if (loss_tmp_bytes(lv) > kScratchBytes) return LVIGS_ERR_CAPACITY;
    // the loss kernel writes loss_out itself: device or page-locked host memory
    if (!kernel_writable(loss_out)) return LVIGS_ERR_INVALID_ARG;
    void *scratch = nullptr;
    const lvigs_status st = scratch_address(&scratch);
    if (st != LVIGS_OK) return st;
    launch_loss(lv, scratch, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LVIGS_OK : LVIGS_ERR_CUDA;
}
