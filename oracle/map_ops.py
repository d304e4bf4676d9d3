"""Plain CPU oracle of the map-maintenance steps around the rendering path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this module.  It
shares no code with the CUDA library and never imports it.

Each function is the plain definition, in float64 unless a decision has to be
taken in binary32 on both sides (stated where it happens):

  * ``adam_step``  -- the Adam update (Kingma & Ba, Algorithm 1, with the bias
    corrections folded into the step size and the denominator) applied to the
    parameter set the paper optimises (Sec. III-E: position, rotation,
    scaling, density and SH colour);
  * ``init_gaussians`` -- Gaussians initialised from colourised LiDAR points
    (Sec. III-E): centre = point, isotropic scale from the mean squared
    distance to the three nearest other points (floored), identity rotation,
    opacity through the inverse sigmoid, SH degree-0 coefficient from the
    point colour, higher bands zero;
  * ``visibility_keep`` -- the cumulative-opacity filter on Gaussian additions
    (Sec. III-C): a point is dropped when the rendered map at its pixel is
    already opaque, i.e. its transparency 1 - V_p is at most tau_alpha;
  * ``prune_keep`` -- removal of Gaussians whose opacity fell below a
    prunable threshold (Sec. III-C).
"""
from __future__ import annotations

import math

import numpy as np

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")

# degree-0 real spherical harmonic, 1 / (2 sqrt(pi))
SH_C0 = 0.5 / math.sqrt(math.pi)

ADAM_DEFAULTS = dict(lr_means=1.6e-4, lr_log_scales=5e-3, lr_quats=1e-3, lr_opacity=5e-2, lr_sh_dc=2.5e-3,
                     lr_sh_rest=2.5e-3 / 20.0, beta1=0.9, beta2=0.999, eps=1e-15)


def _lr_tensor(key, shape, cfg):
    """Learning rate of every element of parameter ``key`` (SH: band 0 vs the rest)."""
    if key == "sh":
        lr = np.full(shape, cfg["lr_sh_rest"], np.float64)
        lr[:, 0, :] = cfg["lr_sh_dc"]
        return lr
    name = {"means": "lr_means", "log_scales": "lr_log_scales", "quats": "lr_quats",
            "opacity_logits": "lr_opacity"}[key]
    return np.full(shape, cfg[name], np.float64)


def adam_step(params, grads, exp_avg, exp_avg_sq, step, cfg=None):
    """One Adam step at step count ``step`` (>= 1, the count after this update).

    m_t = b1 m + (1 - b1) g,  v_t = b2 v + (1 - b2) g^2,
    p  <- p - lr m_t / (1 - b1^t) / (sqrt(v_t / (1 - b2^t)) + eps).
    Returns new (params, exp_avg, exp_avg_sq) dicts in float64."""
    cfg = dict(ADAM_DEFAULTS, **(cfg or {}))
    b1, b2, eps = cfg["beta1"], cfg["beta2"], cfg["eps"]
    bc1 = 1.0 - b1 ** step
    bc2 = 1.0 - b2 ** step
    P, M, V = {}, {}, {}
    for k in PARAM_KEYS:
        if k not in params:
            continue
        g = np.asarray(grads[k], np.float64)
        m = b1 * np.asarray(exp_avg[k], np.float64) + (1.0 - b1) * g
        v = b2 * np.asarray(exp_avg_sq[k], np.float64) + (1.0 - b2) * g * g
        lr = _lr_tensor(k, g.shape, cfg)
        P[k] = np.asarray(params[k], np.float64) - lr * (m / bc1) / (np.sqrt(v / bc2) + eps)
        M[k], V[k] = m, v
    return P, M, V


def knn_mean_dist2(points, k=3):
    """Mean squared distance of every point to its ``k`` nearest OTHER points
    (a duplicate counts at distance 0); with fewer than k others, the mean over
    the others; with none, 0.  The neighbour search is scipy's kd-tree."""
    from scipy.spatial import cKDTree

    pts = np.asarray(points, np.float64)
    n = pts.shape[0]
    if n <= 1:
        return np.zeros(n)
    kk = min(k, n - 1)
    d, _ = cKDTree(pts).query(pts, k=kk + 1)
    d = np.asarray(d).reshape(n, kk + 1)
    # the query point itself is among the results at distance 0: drop one zero
    d2 = np.sort(d * d, axis=1)[:, 1:]
    return d2.mean(axis=1)


def init_gaussians(points, colours, sh_stride_k=16, init_opacity=0.1, min_dist2=1e-7, knn=3):
    """Gaussians of colourised LiDAR points (Sec. III-E).  Returns float64 arrays."""
    pts = np.asarray(points, np.float64)
    col = np.asarray(colours, np.float64)
    n = pts.shape[0]
    d2 = np.maximum(knn_mean_dist2(pts, knn), min_dist2)
    log_s = 0.5 * np.log(d2)
    sh = np.zeros((n, sh_stride_k, 3))
    sh[:, 0, :] = (col - 0.5) / SH_C0
    quats = np.zeros((n, 4))
    quats[:, 0] = 1.0
    return {
        "means": pts.copy(),
        "log_scales": np.repeat(log_s[:, None], 3, axis=1),
        "quats": quats,
        "opacity_logits": np.full(n, math.log(init_opacity / (1.0 - init_opacity))),
        "sh": sh,
    }


def point_pixels(points, cam, near=0.2):
    """Pixel of every point in camera ``cam`` (a level camera), in binary32 with
    one rounding per operation in this order:
        x_c = ((R00 x + R01 y) + R02 z) + t0   (likewise y_c, z_c)
        u = (fx x_c) / z_c + cx,  px = floor(u + 0.5)   (likewise v, py)
    Returns (px, py, inside) where inside = z_c > near and the pixel lies in
    the image.  numpy rounds every float32 operation separately."""
    f = np.float32
    p = np.asarray(points, f)
    R = np.asarray(cam.R, f).reshape(3, 3)
    t = np.asarray(cam.t, f).reshape(3)
    xc = ((R[0, 0] * p[:, 0] + R[0, 1] * p[:, 1]) + R[0, 2] * p[:, 2]) + t[0]
    yc = ((R[1, 0] * p[:, 0] + R[1, 1] * p[:, 1]) + R[1, 2] * p[:, 2]) + t[1]
    zc = ((R[2, 0] * p[:, 0] + R[2, 1] * p[:, 1]) + R[2, 2] * p[:, 2]) + t[2]
    front = zc > f(near)
    zs = np.where(front, zc, f(1.0))
    u = (f(cam.fx) * xc) / zs + f(cam.cx)
    v = (f(cam.fy) * yc) / zs + f(cam.cy)
    fu = np.floor(u + f(0.5))
    fv = np.floor(v + f(0.5))
    inside = front & (fu >= 0) & (fu < cam.W) & (fv >= 0) & (fv < cam.H)
    px = np.where(inside, fu, 0).astype(np.int64)
    py = np.where(inside, fv, 0).astype(np.int64)
    return px, py, inside


def visibility_keep(points, cam, alpha, tau_alpha=0.5, literal=False, near=0.2):
    """Keep mask of the Gaussian-addition filter (Sec. III-C).

    Default reading: the filter keeps additions where the map is still
    transparent; a point whose pixel has transparency 1 - V_p <= tau_alpha is
    dropped (both in binary32).  ``literal=True`` applies the printed inequality
    to V_p itself: dropped when V_p <= tau_alpha.  Points behind the near plane
    or outside the image are kept (the keyframe says nothing about them)."""
    f = np.float32
    px, py, inside = point_pixels(points, cam, near)
    a = np.asarray(alpha, f)[py, px]
    if literal:
        drop = a <= f(tau_alpha)
    else:
        drop = (f(1.0) - a) <= f(tau_alpha)
    return ~(inside & drop)


def prune_keep(opacity_logits, min_opacity=0.005):
    """Keep mask: opacity sigmoid(logit) >= min_opacity.  Sigmoid is monotone,
    so the test is taken on the logit against logit(min_opacity) rounded once to
    binary32 (the decision precision of both sides)."""
    thr = np.float32(math.log(min_opacity / (1.0 - min_opacity)))
    return np.asarray(opacity_logits, np.float32) >= thr


def compact_rows(arrays, keep):
    """Rows of every array where ``keep`` holds, in their original order."""
    idx = np.nonzero(keep)[0]
    return {k: np.asarray(v)[idx] for k, v in arrays.items()}
