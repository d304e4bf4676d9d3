"""Torch-facing wrapper of the C ABI (argument marshalling only).

PyTorch supplies device memory and the current CUDA stream; every step of
the hot path (preprocess, key sort, compositing, loss, backward) runs in
liblvigs.so.  Tensors passed in must be CUDA, float32 and contiguous.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check_tensor(t, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def camera_struct(cam) -> L.Camera:
    """Accepts any object with R (3x3), t (3), fx, fy, cx, cy, W, H."""
    c = L.Camera()
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float32).reshape(9).tolist()]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float32).reshape(3).tolist()]
    c.R[:] = R
    c.t[:] = t
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.W), int(cam.H)
    return c


def gaussians_struct(params, sh_degree=None) -> L.Gaussians:
    for k in PARAM_NAMES:
        _check_tensor(params[k], k)
    n = params["means"].shape[0]
    sh = params["sh"]
    g = L.Gaussians()
    g.means, g.log_scales, g.quats, g.opacity_logits, g.sh = (params[k].data_ptr() for k in PARAM_NAMES)
    g.n = n
    g.sh_degree = int(params.get("sh_degree", 0) if sh_degree is None else sh_degree)
    g.sh_stride_k = sh.shape[1]
    return g


def level_size(cam, level):
    return int(cam.W) >> level, int(cam.H) >> level


LOSS_NOALLOC_MAX_PIXELS = 640 * 512
LOSS_NOALLOC_MAX_SIDE = 2048


def loss_noalloc(rgb, depth, gt, lidar, lambda_ssim, lambda_depth, terms, d_rgb=None, d_depth=None):
    """The mapping loss through lvigs_loss_noalloc, for callers that cannot let
    the library allocate device memory (their allocator owns the budget, or a
    real-time loop where cudaFree would synchronise the device).  Every output
    is a caller-provided tensor: `terms` float64 [4], `d_rgb` [3,H,W] and
    `d_depth` [H,W] (either may be None).  The library's scratch is a fixed
    array on the device, shared by all calls: calls that overlap on the GPU
    race, so order them (for example on one stream)."""
    _check_tensor(rgb, "rgb")
    _check_tensor(gt, "gt", rgb.shape)
    H, W = rgb.shape[1], rgb.shape[2]
    for t, name, shape in ((depth, "depth", (H, W)), (lidar, "lidar", (H, W)), (d_rgb, "d_rgb", rgb.shape),
                           (d_depth, "d_depth", (H, W))):
        if t is not None:
            _check_tensor(t, name, shape)
    if not (terms.is_cuda and terms.dtype == torch.float64 and terms.numel() >= 4 and terms.is_contiguous()):
        raise ValueError("terms must be a contiguous CUDA float64 tensor of 4 elements")
    code = L.load().lvigs_loss_noalloc(W, H, _ptr(rgb), _ptr(depth), _ptr(gt), _ptr(lidar), float(lambda_ssim),
                                       float(lambda_depth), _ptr(terms), _ptr(d_rgb), _ptr(d_depth), _stream())
    if code == 4:
        raise L.LvigsError(code, "lvigs_loss_noalloc",
                           f"{W}x{H} image beyond the fixed scratch: at most {LOSS_NOALLOC_MAX_PIXELS} pixels "
                           f"and {LOSS_NOALLOC_MAX_SIDE} per side")
    L.check(code, "lvigs_loss_noalloc")
    return terms, d_rgb, d_depth


class Context:
    """One library context (workspace, view slots, batched-step graph)."""

    def __init__(self, tile=(16, 16), max_workspace_bytes=0, batch_depth=0):
        self._lib = L.load()
        cfg = L.Config(int(tile[0]), int(tile[1]), int(batch_depth), int(max_workspace_bytes))
        self._h = ctypes.c_void_p()
        L.check(self._lib.lvigs_create(ctypes.byref(self._h), ctypes.byref(cfg)), "lvigs_create")
        self.tile = (int(tile[0]), int(tile[1]))
        self._copy_stream = None  # stream of stage_targets, created on first use

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lvigs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, code, where):
        L.check(code, where, self._h)

    # -- plain path --------------------------------------------------------
    def render(self, params, cam, level=0, sh_degree=None, wait=True):
        """Forward render (a1-a5).  Returns (rgb [3,H,W], depth [H,W], alpha [H,W], slot).

        wait=False calls lvigs_render_async: no wait on the stream, the
        instance lists sized from this context's earlier renders (an overflow
        is reported by sync_status)."""
        g = gaussians_struct(params, sh_degree)
        c = camera_struct(cam)
        W, H = level_size(cam, level)
        dev = params["means"].device
        rgb = torch.empty((3, H, W), device=dev, dtype=torch.float32)
        depth = torch.empty((H, W), device=dev, dtype=torch.float32)
        alpha = torch.empty((H, W), device=dev, dtype=torch.float32)
        out = L.ImageOut(rgb.data_ptr(), depth.data_ptr(), alpha.data_ptr())
        slot = ctypes.c_int()
        fn = self._lib.lvigs_render if wait else self._lib.lvigs_render_async
        self._chk(fn(self._h, ctypes.byref(g), ctypes.byref(c), int(level), ctypes.byref(out), ctypes.byref(slot),
                     _stream()), "lvigs_render" if wait else "lvigs_render_async")
        return rgb, depth, alpha, slot.value

    def backward(self, slot, params, d_rgb, d_depth=None, d_alpha=None, grads=None, accumulate=False):
        """Parameter gradients (a6 + a7) of the render in `slot`."""
        _check_tensor(d_rgb, "d_rgb")
        for t, nm in ((d_depth, "d_depth"), (d_alpha, "d_alpha")):
            if t is not None:
                _check_tensor(t, nm)
        if grads is None:
            grads = {k: torch.zeros_like(params[k]) for k in PARAM_NAMES}
        gs = L.Grads(*(grads[k].data_ptr() for k in PARAM_NAMES), int(bool(accumulate)))
        self._chk(self._lib.lvigs_backward(self._h, int(slot), _ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha),
                                           ctypes.byref(gs), _stream()), "lvigs_backward")
        return grads

    def release(self, slot):
        self._chk(self._lib.lvigs_release_view(self._h, int(slot)), "lvigs_release_view")

    def loss(self, rgb, depth, gt, lidar, lambda_ssim, lambda_depth, grads=True):
        """Mapping loss (a8).  Returns (terms float64 [4] on device, d_rgb, d_depth)."""
        _check_tensor(rgb, "rgb")
        _check_tensor(gt, "gt", rgb.shape)
        H, W = rgb.shape[1], rgb.shape[2]
        if depth is not None:
            _check_tensor(depth, "depth", (H, W))
        if lidar is not None:
            _check_tensor(lidar, "lidar", (H, W))
        terms = torch.zeros(4, device=rgb.device, dtype=torch.float64)
        d_rgb = torch.empty_like(rgb) if grads else None
        d_depth = torch.empty((H, W), device=rgb.device, dtype=torch.float32) if grads and depth is not None else None
        self._chk(self._lib.lvigs_loss(self._h, W, H, _ptr(rgb), _ptr(depth), _ptr(gt), _ptr(lidar),
                                       float(lambda_ssim), float(lambda_depth), _ptr(terms), _ptr(d_rgb),
                                       _ptr(d_depth), _stream()), "lvigs_loss")
        return terms, d_rgb, d_depth

    def pyramid_down(self, rgb, depth=None):
        """One pyramid level down (a9)."""
        _check_tensor(rgb, "rgb")
        H, W = rgb.shape[1], rgb.shape[2]
        r2 = torch.empty((3, H // 2, W // 2), device=rgb.device, dtype=torch.float32)
        d2 = torch.empty((H // 2, W // 2), device=rgb.device, dtype=torch.float32) if depth is not None else None
        if depth is not None:
            _check_tensor(depth, "depth", (H, W))
        L.check(self._lib.lvigs_pyramid_down(W, H, _ptr(rgb), _ptr(depth), _ptr(r2), _ptr(d2), _stream()),
                "lvigs_pyramid_down")
        return r2, d2

    # -- batched path ------------------------------------------------------
    def _batch(self, params, cams, levels, gts, lidars, lambda_ssim, lambda_depth, grads, accumulate, host_targets,
               host_loss, graph, outputs, losses, staged_slot=None):
        V = len(cams)
        g = gaussians_struct(params)
        if grads is None:
            grads = {k: torch.zeros_like(params[k]) for k in PARAM_NAMES}
        gs = L.Grads(*(grads[k].data_ptr() for k in PARAM_NAMES), int(bool(accumulate)))
        keep = []  # ctypes arrays referenced by the Batch struct
        camarr = (L.Camera * V)(*[camera_struct(c) for c in cams])
        lvl = (ctypes.c_int * V)(*[int(x) for x in levels])
        gtp = (ctypes.c_void_p * V)(*([t.data_ptr() for t in gts] if gts is not None else [None] * V))
        lip = (ctypes.c_void_p * V)(*([t.data_ptr() if t is not None else None for t in lidars]
                                      if lidars is not None else [None] * V))
        keep += [camarr, lvl, gtp, lip]
        host_async = False
        if losses is None:
            losses = torch.zeros((V, 4), dtype=torch.float64,
                                 device="cpu" if host_loss else params["means"].device)
        elif not losses.is_cuda and not host_loss:
            # written by the step's kernels through the page-locked mapping; read it
            # after an event recorded behind the step
            if not losses.is_pinned() or losses.dtype != torch.float64 or not losses.is_contiguous():
                raise ValueError("host losses without host_loss=True must be a pinned contiguous float64 tensor")
            host_async = True
        b = L.Batch()
        b.n_views = V
        b.cameras = camarr
        b.levels = lvl
        b.gt_rgb = gtp
        b.lidar_depth = lip
        b.lambda_ssim = float(lambda_ssim)
        b.lambda_depth = float(lambda_depth)
        b.flags = ((L.STEP_HOST_TARGETS if host_targets else 0) | (L.STEP_HOST_LOSS if host_loss else 0)
                   | (0 if graph else L.STEP_NO_GRAPH) | (L.STEP_STAGED_TARGETS if staged_slot is not None else 0)
                   | (L.STEP_HOST_LOSS_ASYNC if host_async else 0))
        b.staged_slot = int(staged_slot) if staged_slot is not None else 0
        b.losses = losses.data_ptr()
        if outputs is not None:
            for i, nm in enumerate(("rgb_out", "depth_out", "alpha_out")):
                arr = (ctypes.c_void_p * V)(*[o[i].data_ptr() for o in outputs])
                keep.append(arr)
                setattr(b, nm, arr)
        return g, b, gs, grads, losses, keep

    def stage_targets(self, cams, gts, lidars, slot):
        """Copy level-0 targets from pinned CPU tensors into staging slot `slot`
        (0 or 1) on the context's copy stream, after the last step that read the
        slot; a later train_step_batched(..., staged_slot=slot) waits for the copy.
        The tensors must stay alive until that step has run."""
        V = len(cams)
        if len(gts) != V or (lidars is not None and len(lidars) != V):
            raise ValueError("one target (and LiDAR map) per camera")
        for i, c in enumerate(cams):
            shapes = [(gts[i], (3, c.H, c.W))] + ([(lidars[i], (c.H, c.W))] if lidars is not None else [])
            for t, shp in shapes:
                if (not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_pinned() or t.dtype != torch.float32
                        or not t.is_contiguous() or tuple(t.shape) != shp):
                    raise ValueError(f"stage_targets takes pinned contiguous float32 CPU tensors of shape {shp}")
        if self._copy_stream is None:
            self._copy_stream = torch.cuda.Stream()
        camarr = (L.Camera * V)(*[camera_struct(c) for c in cams])
        gtp = (ctypes.c_void_p * V)(*[t.data_ptr() for t in gts])
        lip = None if lidars is None else (ctypes.c_void_p * V)(*[t.data_ptr() for t in lidars])
        self._chk(self._lib.lvigs_stage_targets(self._h, int(slot), V, camarr, gtp, lip,
                                                ctypes.c_void_p(self._copy_stream.cuda_stream)),
                  "lvigs_stage_targets")

    def train_step_batched(self, params, cams, levels, gts, lidars, lambda_ssim, lambda_depth, grads=None,
                           accumulate=False, host_targets=False, host_loss=False, graph=True, outputs=None,
                           losses=None, staged_slot=None):
        """One batched step (a10): render, loss and backward of every view.

        gts / lidars are level-0 targets (CUDA tensors, or pinned CPU tensors with
        host_targets=True), or None with staged_slot = the slot a previous
        stage_targets call filled.  losses may be a pinned CPU tensor without
        host_loss: the step's kernels then write it directly and the call
        returns at once (read it after an event recorded behind the step).
        Returns (losses [V,4] float64, grads).
        """
        g, b, gs, grads, losses, keep = self._batch(params, cams, levels, gts, lidars, lambda_ssim, lambda_depth,
                                                    grads, accumulate, host_targets, host_loss, graph, outputs,
                                                    losses, staged_slot)
        self._chk(self._lib.lvigs_train_step_batched(self._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(gs),
                                                     _stream()), "lvigs_train_step_batched")
        del keep
        return losses, grads

    def autotune(self, params, cams, levels, gts, lidars, lambda_ssim, lambda_depth, trials=3, grads=None):
        """Pick tile size and batch depth by timing the batched step; returns
        ((tile_w, tile_h), batch_depth, {candidate: ms per step})."""
        g, b, gs, grads, losses, keep = self._batch(params, cams, levels, gts, lidars, lambda_ssim, lambda_depth,
                                                    grads, False, False, False, True, None, None)
        cfg = L.Config()
        ms = (ctypes.c_double * len(L.AUTOTUNE_CANDIDATES))()
        self._chk(self._lib.lvigs_autotune_batched(self._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(gs),
                                                   int(trials), _stream(), ctypes.byref(cfg), ms),
                  "lvigs_autotune_batched")
        del keep
        self.tile = (cfg.tile_w, cfg.tile_h)
        times = {f"{c[0][0]}x{c[0][1]}/{c[1]}": round(ms[i], 4) for i, c in enumerate(L.AUTOTUNE_CANDIDATES)}
        return self.tile, cfg.batch_depth, times

    # -- parity hooks ------------------------------------------------------
    def debug_keys(self, slot):
        """Sorted 64-bit keys (as int64 bit patterns) and Gaussian indices (int32)."""
        m = ctypes.c_int64()
        self._chk(self._lib.lvigs_debug_keys(self._h, int(slot), None, None, 0, ctypes.byref(m), _stream()),
                  "lvigs_debug_keys")
        n = m.value
        keys = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        vals = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        self._chk(self._lib.lvigs_debug_keys(self._h, int(slot), _ptr(keys), _ptr(vals), n, ctypes.byref(m),
                                             _stream()), "lvigs_debug_keys")
        return keys[:n], vals[:n]

    def debug_state(self, slot, H, W):
        nt = ctypes.c_int()
        self._chk(self._lib.lvigs_debug_state(self._h, int(slot), None, None, None, ctypes.byref(nt), _stream()),
                  "lvigs_debug_state")
        ranges = torch.empty((nt.value, 2), dtype=torch.int32, device="cuda")
        nc = torch.empty((H, W), dtype=torch.int32, device="cuda")
        ft = torch.empty((H, W), dtype=torch.float32, device="cuda")
        self._chk(self._lib.lvigs_debug_state(self._h, int(slot), _ptr(ranges), _ptr(nc), _ptr(ft),
                                              ctypes.byref(nt), _stream()), "lvigs_debug_state")
        return ranges, nc, ft

    def profile(self, enable=True):
        self._chk(self._lib.lvigs_profile_enable(self._h, int(bool(enable))), "lvigs_profile_enable")

    def profile_read(self):
        """{phase: (ms summed, calls)} since the last read, and kernels per graph replay."""
        n = len(L.PHASES)
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_int64 * n)()
        kps = ctypes.c_int()
        self._chk(self._lib.lvigs_profile_read(self._h, ms, calls, ctypes.byref(kps)), "lvigs_profile_read")
        return {L.PHASES[i]: (ms[i], calls[i]) for i in range(n)}, kps.value

    def step_stats(self):
        """(visible pairs, instances, sum of contributor counts, pixels) of the last batched step."""
        out = (ctypes.c_int64 * 4)()
        self._chk(self._lib.lvigs_step_stats(self._h, out, _stream()), "lvigs_step_stats")
        return tuple(int(x) for x in out)

    def sync_status(self):
        self._chk(self._lib.lvigs_sync_status(self._h, _stream()), "lvigs_sync_status")
