"""Plain, slow CPU oracle of the LVI-GS Gaussian-splatting hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library and never imports it.

The arithmetic lives in ``lvigs_oracle.c`` (binary64, with the tile-key stage
in strict binary32); this module compiles it with gcc and wraps it with ctypes.

What it computes, by the paper's equations (arxiv 2411.02703):
  * Sec. III-B, Eq. (2) Sigma = R S S^T R^T and Eq. (7) the EWA projection
    (a1), the per-tile depth-ordered lists (a2-a4), Eq. (3)-(6) compositing of
    colour, depth and visibility (a5), and their hand-derived gradients
    (a6, a7);
  * Sec. III-E, Eq. (10)-(12), the L1 + SSIM + LiDAR-depth loss (a8);
  * Sec. III-D, the image pyramid (a9).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lvigs_oracle.c")
_LIB = os.path.join(_HERE, "liblvigs_oracle.so")

# -ffp-contract=off keeps every binary32 operation of the key stage separately
# rounded (GCC contracts a*b+c into an FMA by default on AArch64).
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Cam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("W", ctypes.c_int), ("H", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_count_instances.restype = ctypes.c_int64
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def exp_key(x):
    """The key stage's scale exp: (float)exp((double)x) per element (C libm)."""
    xs = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(xs)
    _load().orc_exp_key(_p(xs), _p(y), ctypes.c_int64(xs.size))
    return y


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the following oracle calls (OpenMP)."""
    _load().orc_set_num_threads(ctypes.c_int(int(n)))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


@dataclass
class Camera:
    """Pinhole camera; R, t map world to camera (x right, y down, z forward)."""
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int

    def _c(self) -> _Cam:
        c = _Cam()
        c.R[:] = [float(v) for v in np.asarray(self.R, np.float32).reshape(9)]
        c.t[:] = [float(v) for v in np.asarray(self.t, np.float32).reshape(3)]
        c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (self.fx, self.fy, self.cx, self.cy))
        c.W, c.H = int(self.W), int(self.H)
        return c


def level_camera(cam: Camera, level: int) -> Camera:
    """Camera of pyramid level ``level`` (Sec. III-D), in binary32 like the key stage."""
    out = _Cam()
    src = cam._c()
    _load().orc_level_camera(ctypes.byref(src), ctypes.c_int(level), ctypes.byref(out))
    return Camera(np.array(out.R[:], np.float32).reshape(3, 3), np.array(out.t[:], np.float32),
                  out.fx, out.fy, out.cx, out.cy, out.W, out.H)


def sh_basis(d):
    """Real SH basis (16 values) and its Cartesian gradient at direction d."""
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    _load().orc_sh_basis(ctypes.c_double(d[0]), ctypes.c_double(d[1]), ctypes.c_double(d[2]),
                         _p(Y), _p(dY))
    return Y, dY


def _params(params):
    means = np.ascontiguousarray(params["means"], np.float32)
    n = means.shape[0]
    sh = np.ascontiguousarray(params["sh"], np.float32)
    return (n, means, np.ascontiguousarray(params["log_scales"], np.float32),
            np.ascontiguousarray(params["quats"], np.float32),
            np.ascontiguousarray(params["opacity_logits"], np.float32), sh,
            sh.shape[1], int(params["sh_degree"]))


def preprocess(params, cam: Camera, tile=(16, 16), screen="key"):
    """a1 for one view at the camera's own resolution.

    ``screen`` chooses the screen-space Gaussian the composited values
    describe: ``"key"`` (the default) takes the key stage's binary32 centre and
    depth and the binary64 inverse of its binary32 covariance, the projection
    of Eq. (7) that also decides the tile lists; ``"f64"`` recomputes the
    projection in binary64, a smooth function of the parameters for the
    finite-difference checks of the gradients."""
    if screen not in ("key", "f64"):
        raise ValueError(f"screen must be 'key' or 'f64', not {screen!r}")
    n, means, ls, q, ol, sh, K, deg = _params(params)
    out = dict(z_f=np.zeros(n, np.float32), uv_f=np.zeros((n, 2), np.float32),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               tiles=np.zeros(n, np.uint32), uv=np.zeros((n, 2)), conic=np.zeros((n, 3)),
               opacity=np.zeros(n), rgb=np.zeros((n, 3)), depth=np.zeros(n), conic_f=np.zeros((n, 3)),
               rgb_margin=np.zeros(n))
    c = cam._c()
    rc = _load().orc_preprocess(
        ctypes.c_int64(n), _p(means), _p(ls), _p(q), _p(ol), _p(sh), ctypes.c_int(K),
        ctypes.c_int(deg), ctypes.byref(c), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
        _p(out["z_f"]), _p(out["uv_f"]), _p(out["radius"]), _p(out["rect"]), _p(out["tiles"]),
        _p(out["uv"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]), _p(out["depth"]),
        _p(out["conic_f"]), _p(out["rgb_margin"]), ctypes.c_int(1 if screen == "key" else 0))
    if rc:
        raise ValueError(f"orc_preprocess failed ({rc})")
    out["tiles_x"] = (cam.W + tile[0] - 1) // tile[0]
    out["tiles_y"] = (cam.H + tile[1] - 1) // tile[1]
    return out


def build_keys(pre, tile_base: int = 0):
    """a2 + a3: sorted 64-bit (tile, depth) keys and Gaussian indices."""
    n = pre["tiles"].shape[0]
    m = int(_load().orc_count_instances(ctypes.c_int64(n), _p(pre["tiles"])))
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    rc = _load().orc_build_keys(ctypes.c_int64(n), _p(pre["rect"]), _p(pre["z_f"]),
                                _p(pre["tiles"]), ctypes.c_int(pre["tiles_x"]),
                                ctypes.c_uint32(tile_base), ctypes.c_int64(m), _p(keys), _p(vals))
    if rc:
        raise ValueError(f"orc_build_keys failed ({rc})")
    return keys[:m], vals[:m]


def tile_ranges(keys, n_tiles: int, tile_base: int = 0):
    """a4: [start, end) per tile."""
    r = np.zeros((n_tiles, 2), np.uint32)
    k = np.ascontiguousarray(keys, np.uint64)
    _load().orc_tile_ranges(ctypes.c_int64(k.shape[0]), _p(k), ctypes.c_uint32(tile_base),
                            ctypes.c_int(n_tiles), _p(r))
    return r


def _allowance_inputs(pre):
    uv_f, conic_f = pre.get("uv_f"), pre.get("conic_f")
    if uv_f is None or conic_f is None:
        return None, None
    return np.ascontiguousarray(uv_f, np.float32), np.ascontiguousarray(conic_f, np.float64)


def render(pre, vals, ranges, W, H, tile=(16, 16), sel_tiles=None, close_margin=-np.inf, flip=False):
    """a5: binary64 compositing.  ``sel_tiles`` limits the work to some tiles.

    ``margin`` is, per pixel, the smallest relative distance of any of its
    threshold tests to the threshold, net of the deviation binary32 inputs and
    evaluation may cause (see orc_render).  ``n_close`` counts the tests whose
    margin is at most ``close_margin``; with ``flip`` each of them takes the
    other branch, which gives the other result the same arithmetic may
    legitimately reach."""
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), alpha=np.zeros((H, W)),
               final_T=np.ones((H, W)), n_contrib=np.zeros((H, W), np.int32),
               margin=np.full((H, W), np.inf), signature=np.zeros((H, W), np.uint64),
               n_close=np.zeros((H, W), np.int32))
    sel = None if sel_tiles is None else np.ascontiguousarray(sel_tiles, np.int32)
    if sel is not None and sel.shape[0] == 0:
        return out
    uv_f, conic_f = _allowance_inputs(pre)
    v = np.ascontiguousarray(vals, np.uint32)
    rg = np.ascontiguousarray(ranges, np.uint32)
    rc = _load().orc_render(
        ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
        _p(pre["uv"]), _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]),
        _p(v), _p(rg), ctypes.c_int(0 if sel is None else sel.shape[0]), _p(sel),
        _p(out["rgb"]), _p(out["depth"]), _p(out["alpha"]), _p(out["final_T"]),
        _p(out["n_contrib"]), _p(out["margin"]), _p(out["signature"]),
        _p(uv_f), _p(conic_f), ctypes.c_double(close_margin), ctypes.c_int(1 if flip else 0),
        _p(out["n_close"]))
    if rc:
        raise ValueError(f"orc_render failed ({rc})")
    return out


def loss(img, gt, depth, lidar, lam: float, lam_d: float, grads: bool = True,
         kink_margin: float = -1.0, depth_kink_margin: float = -1.0, flip: bool = False):
    """a8: (loss, l1, mean_ssim, depth_l1), d_img, d_depth, all binary64.

    With ``flip`` an L1 residual within ``kink_margin`` (colour) or
    ``depth_kink_margin`` (depth) of zero takes the other sign in the gradients."""
    img = np.ascontiguousarray(img, np.float64)
    gt = np.ascontiguousarray(gt, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    lidar = np.ascontiguousarray(lidar, np.float64)
    H, W = depth.shape
    terms = np.zeros(4)
    d_img = np.zeros_like(img) if grads else None
    d_depth = np.zeros_like(depth) if grads else None
    rc = _load().orc_loss(ctypes.c_int(W), ctypes.c_int(H), _p(img), _p(gt), _p(depth), _p(lidar),
                          ctypes.c_double(lam), ctypes.c_double(lam_d), _p(terms), _p(d_img),
                          _p(d_depth), ctypes.c_double(kink_margin), ctypes.c_double(depth_kink_margin),
                          ctypes.c_int(1 if flip else 0))
    if rc:
        raise ValueError(f"orc_loss failed ({rc})")
    return terms, d_img, d_depth


def backward_render(pre, vals, ranges, W, H, d_rgb, d_depth, d_alpha=None, tile=(16, 16),
                    close_margin=-np.inf, flip=False):
    """a6: per-Gaussian (du, dv, dA, dB, dC, dopacity, drgb[3], ddepth), over the
    walk of ``render`` with the same ``close_margin`` / ``flip``."""
    n = pre["tiles"].shape[0]
    g2 = np.zeros((n, 10))
    d_rgb = np.ascontiguousarray(d_rgb, np.float64)
    d_depth = np.ascontiguousarray(d_depth, np.float64)
    d_alpha = None if d_alpha is None else np.ascontiguousarray(d_alpha, np.float64)
    rc = _load().orc_backward_render(
        ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(tile[0]), ctypes.c_int(tile[1]),
        ctypes.c_int64(n), _p(pre["uv"]), _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]),
        _p(pre["depth"]), _p(np.ascontiguousarray(vals, np.uint32)),
        _p(np.ascontiguousarray(ranges, np.uint32)), _p(d_rgb), _p(d_depth), _p(d_alpha), _p(g2),
        *(_p(a) for a in _allowance_inputs(pre)), ctypes.c_double(close_margin),
        ctypes.c_int(1 if flip else 0))
    if rc:
        raise ValueError(f"orc_backward_render failed ({rc})")
    return g2


def zero_grads(params):
    n = params["means"].shape[0]
    K = params["sh"].shape[1]
    return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)))


def backward_preprocess(params, cam: Camera, pre, grad2d, grads=None):
    """a7: accumulate parameter gradients of one view into ``grads``."""
    n, means, ls, q, ol, sh, K, deg = _params(params)
    if grads is None:
        grads = zero_grads(params)
    c = cam._c()
    rc = _load().orc_backward_preprocess(
        ctypes.c_int64(n), _p(means), _p(ls), _p(q), _p(ol), _p(sh), ctypes.c_int(K),
        ctypes.c_int(deg), ctypes.byref(c), _p(pre["tiles"]),
        _p(np.ascontiguousarray(grad2d, np.float64)), _p(grads["means"]),
        _p(grads["log_scales"]), _p(grads["quats"]), _p(grads["opacity_logits"]), _p(grads["sh"]))
    if rc:
        raise ValueError(f"orc_backward_preprocess failed ({rc})")
    return grads


def pyramid_down(rgb, depth):
    """a9: one level down (2x2 box mean; valid-mean depth)."""
    rgb = np.ascontiguousarray(rgb, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    H, W = depth.shape
    ro = np.zeros((3, H // 2, W // 2))
    do = np.zeros((H // 2, W // 2))
    _load().orc_pyramid_down(ctypes.c_int(W), ctypes.c_int(H), _p(rgb), _p(depth), _p(ro), _p(do))
    return ro, do


def pyramid(rgb, depth, level: int):
    for _ in range(level):
        rgb, depth = pyramid_down(rgb, depth)
    return np.asarray(rgb, np.float64), np.asarray(depth, np.float64)


def render_view(params, cam0: Camera, level: int = 0, tile=(16, 16), sel_tiles=None, screen="key",
                close_margin=-np.inf, flip=False):
    """a1-a5 for one view at pyramid level ``level`` (``screen``: see
    ``preprocess``; ``close_margin``, ``flip``: see ``render``)."""
    cam = level_camera(cam0, level)
    pre = preprocess(params, cam, tile, screen)
    keys, vals = build_keys(pre)
    n_tiles = pre["tiles_x"] * pre["tiles_y"]
    ranges = tile_ranges(keys, n_tiles)
    img = render(pre, vals, ranges, cam.W, cam.H, tile, sel_tiles, close_margin, flip)
    return dict(cam=cam, pre=pre, keys=keys, vals=vals, ranges=ranges, **img)


def train_step(params, cams, levels, gts, lidars, lam, lam_d, tile=(16, 16), screen="key",
               close_margin=-np.inf, flip=False, kink_margin=-1.0, depth_kink_margin=-1.0):
    """One hot-path pass over several views: render, loss and gradients.

    ``gts`` / ``lidars`` are level-0 targets; each view's targets are brought
    to its level with ``pyramid``.  Returns per-view loss terms, renders and
    the parameter gradients summed over views.
    """
    grads = zero_grads(params)
    out = []
    for cam0, lvl, gt0, li0 in zip(cams, levels, gts, lidars):
        r = render_view(params, cam0, lvl, tile, screen=screen, close_margin=close_margin, flip=flip)
        gt, li = pyramid(gt0, li0, lvl)
        terms, d_img, d_depth = loss(r["rgb"], gt, r["depth"], li, lam, lam_d, True,
                                     kink_margin, depth_kink_margin, flip)
        g2 = backward_render(r["pre"], r["vals"], r["ranges"], r["cam"].W, r["cam"].H,
                             d_img, d_depth, None, tile, close_margin, flip)
        backward_preprocess(params, r["cam"], r["pre"], g2, grads)
        out.append(dict(terms=terms, render=r, grad2d=g2, gt=gt, lidar=li))
    return out, grads
