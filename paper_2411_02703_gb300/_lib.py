"""ctypes mirror of include/lvigs.h and the loader of liblvigs.so.

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Importing this module builds the library in-tree when it is
missing or stale and raises if that is impossible; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LVIGS_MAX_VIEWS = 32
LVIGS_MAX_LEVEL = 4
STEP_HOST_TARGETS = 1
STEP_HOST_LOSS = 2
STEP_NO_GRAPH = 4
STEP_STAGED_TARGETS = 8
STEP_HOST_LOSS_ASYNC = 16
STAGE_SLOTS = 2

STATUS = {0: "LVIGS_OK", 1: "LVIGS_ERR_INVALID_ARG", 2: "LVIGS_ERR_OUT_OF_MEMORY", 3: "LVIGS_ERR_CUDA",
          4: "LVIGS_ERR_CAPACITY", 5: "LVIGS_ERR_TIMEOUT", 6: "LVIGS_ERR_STATE"}


class LvigsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}" + (f" ({msg})" if msg else ""))


class Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("batch_depth", ctypes.c_int),
                ("max_workspace_bytes", ctypes.c_size_t)]


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("sh_degree", ctypes.c_int), ("sh_stride_k", ctypes.c_int)]


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


class ImageOut(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("alpha", ctypes.c_void_p)]


class Grads(ctypes.Structure):
    _fields_ = [("d_means", ctypes.c_void_p), ("d_log_scales", ctypes.c_void_p), ("d_quats", ctypes.c_void_p),
                ("d_opacity_logits", ctypes.c_void_p), ("d_sh", ctypes.c_void_p), ("accumulate", ctypes.c_int)]


class Batch(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("cameras", ctypes.POINTER(Camera)),
                ("levels", ctypes.POINTER(ctypes.c_int)), ("gt_rgb", ctypes.POINTER(ctypes.c_void_p)),
                ("lidar_depth", ctypes.POINTER(ctypes.c_void_p)), ("lambda_ssim", ctypes.c_float),
                ("lambda_depth", ctypes.c_float), ("flags", ctypes.c_int), ("losses", ctypes.c_void_p),
                ("rgb_out", ctypes.POINTER(ctypes.c_void_p)), ("depth_out", ctypes.POINTER(ctypes.c_void_p)),
                ("alpha_out", ctypes.POINTER(ctypes.c_void_p)), ("staged_slot", ctypes.c_int)]


class ParamBuffers(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class AdamConfig(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_float) for n in ("lr_means", "lr_log_scales", "lr_quats", "lr_opacity", "lr_sh_dc",
                                               "lr_sh_rest")]
                + [(n, ctypes.c_double) for n in ("beta1", "beta2", "eps")])


class InitConfig(ctypes.Structure):
    _fields_ = [("init_opacity", ctypes.c_float), ("min_dist2", ctypes.c_float), ("tau_alpha", ctypes.c_float),
                ("filter_literal", ctypes.c_int)]


# every entry point declared in include/lvigs.h, with its ctypes signature
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "lvigs_version": (ctypes.c_char_p, []),
    "lvigs_config_default": (None, [ctypes.POINTER(Config)]),
    "lvigs_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Config)]),
    "lvigs_destroy": (None, [_P]),
    "lvigs_level_size": (_I, [ctypes.POINTER(Camera), _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lvigs_render": (_I, [_P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), _I, ctypes.POINTER(ImageOut),
                          ctypes.POINTER(_I), _P]),
    "lvigs_render_async": (_I, [_P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), _I,
                                ctypes.POINTER(ImageOut), ctypes.POINTER(_I), _P]),
    "lvigs_backward": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(Grads), _P]),
    "lvigs_loss": (_I, [_P, _I, _I, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]),
    "lvigs_loss_noalloc": (_I, [_I, _I, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]),
    "lvigs_pyramid_down": (_I, [_I, _I, _P, _P, _P, _P, _P]),
    "lvigs_train_step_batched": (_I, [_P, ctypes.POINTER(Gaussians), ctypes.POINTER(Batch), ctypes.POINTER(Grads), _P]),
    "lvigs_stage_targets": (_I, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Camera), ctypes.POINTER(_P),
                                 ctypes.POINTER(_P), _P]),
    "lvigs_debug_keys": (_I, [_P, _I, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _P]),
    "lvigs_debug_state": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(_I), _P]),
    "lvigs_debug_exp_key": (_I, [_P, _P, ctypes.c_int64, _P]),
    "lvigs_sync_status": (_I, [_P, _P]),
    "lvigs_release_view": (_I, [_P, _I]),
    "lvigs_last_error": (ctypes.c_char_p, [_P]),
    "lvigs_step_stats": (_I, [_P, ctypes.POINTER(ctypes.c_int64), _P]),
    "lvigs_autotune_batched": (_I, [_P, ctypes.POINTER(Gaussians), ctypes.POINTER(Batch), ctypes.POINTER(Grads), _I,
                                    _P, ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_double)]),
    "lvigs_adam_config_default": (None, [ctypes.POINTER(AdamConfig)]),
    "lvigs_adam_step": (_I, [ctypes.POINTER(ParamBuffers), ctypes.POINTER(Grads), ctypes.POINTER(ParamBuffers),
                             ctypes.POINTER(ParamBuffers), ctypes.c_int64, _I, ctypes.c_int64,
                             ctypes.POINTER(AdamConfig), _I, _P]),
    "lvigs_init_config_default": (None, [ctypes.POINTER(InitConfig)]),
    "lvigs_append_gaussians": (_I, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(Camera), _I, _P,
                                    ctypes.POINTER(InitConfig), ctypes.POINTER(ParamBuffers),
                                    ctypes.POINTER(ParamBuffers), ctypes.POINTER(ParamBuffers), ctypes.c_int64,
                                    ctypes.c_int64, _I, ctypes.POINTER(ctypes.c_int64), _P]),
    "lvigs_prune_gaussians": (_I, [_P, ctypes.c_float, ctypes.POINTER(ParamBuffers), ctypes.POINTER(ParamBuffers),
                                   ctypes.POINTER(ParamBuffers), ctypes.c_int64, _I,
                                   ctypes.POINTER(ctypes.c_int64), _P]),
    "lvigs_profile_enable": (_I, [_P, _I]),
    "lvigs_profile_read": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(_I)]),
}

AUTOTUNE_CANDIDATES = [((16, 16), 64), ((16, 16), 32), ((8, 8), 64), ((8, 8), 32), ((32, 16), 64), ((32, 16), 32)]

PHASES = ["preprocess", "compact", "depth_sort", "offsets", "emit", "tile_sort", "ranges", "composite_fwd",
          "loss", "composite_bwd", "preprocess_bwd", "pyramid", "combine"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load liblvigs.so (building it in-tree when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"liblvigs.so not found at {path}; run paper_2411_02703_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str, ctx=None):
    if code != 0:
        msg = ""
        if ctx is not None and _lib is not None:
            m = _lib.lvigs_last_error(ctx)
            msg = m.decode() if m else ""
        raise LvigsError(code, where, msg)
