"""Seeded synthetic inputs for the Gaussian-splatting hot path.

The paper's data (FAST-LIVO and R3LIVE sequences, 640x512 images) are not
available, so every workload is synthetic.  This module only draws inputs:
Gaussian parameters (from a simulated LiDAR sweep for the large workloads),
camera poses, target images and sparse LiDAR depth targets.  It holds none
of the rendering, loss or gradient arithmetic, and both the CUDA tests and
the oracle tests draw their inputs from it.

All arrays are float32 numpy arrays in the layouts the library takes:
means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z, not normalised),
opacity_logits [N], sh [N,K,3] with K = (max degree + 1)^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20241105


@dataclass
class CameraSpec:
    """World->camera rotation R (row-major 3x3), translation t, level-0 pinhole."""
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int


def _rng(seed):
    return np.random.default_rng(seed)


def random_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True).astype(np.float32)
    return q.astype(np.float32)


def identity_camera(W, H, f, cx=None, cy=None):
    return CameraSpec(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), float(f), float(f),
                      float(W / 2 if cx is None else cx), float(H / 2 if cy is None else cy), W, H)


def small_scene(seed=BASE_SEED + 1, n=2000, W=160, H=120, f=150.0, xy=4.0, z=(2.0, 10.0),
                sh_degree=0, sh_max_degree=None, log_scale=(-3.0, 0.5), lidar_frac=0.05):
    """The 160x120 single-view workload: uniform means in front of an identity camera.

    Means x,y ~ U[-xy, xy], z ~ U[z]; log-scales ~ N(log_scale); random unit
    quaternions; opacity logits ~ N(0,1); SH band 0 chosen so the base colour
    is U[0,1] (coefficient U[-sqrt(pi), sqrt(pi)]), higher bands ~ N(0, 0.1).
    Target RGB ~ U[0,1] per pixel; LiDAR depth U[z] at ``lidar_frac`` of the
    pixels (chosen without replacement), 0 elsewhere.
    """
    rng = _rng(seed)
    kmax = sh_degree if sh_max_degree is None else sh_max_degree
    K = (kmax + 1) ** 2
    means = np.empty((n, 3), np.float32)
    means[:, 0] = rng.uniform(-xy, xy, n)
    means[:, 1] = rng.uniform(-xy, xy, n)
    means[:, 2] = rng.uniform(z[0], z[1], n)
    log_scales = rng.normal(log_scale[0], log_scale[1], (n, 3)).astype(np.float32)
    quats = random_quats(rng, n)
    opacity_logits = rng.normal(0.0, 1.0, n).astype(np.float32)
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, K - 1, 3))
    params = dict(means=means, log_scales=log_scales, quats=quats,
                  opacity_logits=opacity_logits, sh=sh, sh_degree=sh_degree)
    cam = identity_camera(W, H, f)
    gt = rng.uniform(0.0, 1.0, (3, H, W)).astype(np.float32)
    lidar = np.zeros(H * W, np.float32)
    k = int(round(lidar_frac * H * W))
    idx = rng.choice(H * W, size=k, replace=False)
    lidar[idx] = rng.uniform(z[0], z[1], k)
    return params, cam, gt, lidar.reshape(H, W)


# ---------------------------------------------------------------------------
# LiDAR-sweep scenes for the 1280x1024 workloads
# ---------------------------------------------------------------------------

def _boxes(rng, n_boxes=40):
    """Axis-aligned facades beside a trajectory along +x (footprint 5-20 m, height 3-15 m)."""
    lo = np.zeros((n_boxes, 3))
    hi = np.zeros((n_boxes, 3))
    for i in range(n_boxes):
        sx, sy = rng.uniform(5, 20, 2)
        h = rng.uniform(3, 15)
        cxw = rng.uniform(-20, 80)
        side = rng.choice([-1.0, 1.0])
        dist = rng.uniform(8, 50)
        cyw = side * (dist + sy / 2)
        lo[i] = (cxw - sx / 2, cyw - sy / 2, 0.0)
        hi[i] = (cxw + sx / 2, cyw + sy / 2, h)
    return lo, hi


def _texture(p):
    """Procedural colour of a world position (structured, in [0,1])."""
    r = 0.5 + 0.35 * np.sin(0.9 * p[:, 0] + 0.3 * p[:, 2]) * np.cos(0.7 * p[:, 1])
    g = 0.5 + 0.35 * np.sin(0.5 * p[:, 1] + 1.3 * p[:, 2] + 1.0)
    b = 0.5 + 0.35 * np.cos(0.6 * p[:, 0] - 0.8 * p[:, 1] + 0.5 * p[:, 2])
    stripes = 0.12 * np.sign(np.sin(3.0 * p[:, 0]) * np.sin(3.0 * p[:, 1] + 2.0 * p[:, 2]))
    return np.clip(np.stack([r, g, b], 1) + stripes[:, None], 0.0, 1.0)


def _ray_cast(origin, d, lo, hi):
    """Distance along unit directions d from origin to the first hit of the
    ground plane z=0 or a box (inf where a ray hits nothing)."""
    tbest = np.full(d.shape[0], np.inf)
    down = d[:, 2] < 0
    tbest[down] = origin[2] / (-d[down, 2])
    inv = 1.0 / np.where(np.abs(d) < 1e-12, 1e-12, d)
    for c0 in range(0, d.shape[0], 16384):
        sl = slice(c0, c0 + 16384)
        t0 = (lo[None] - origin) * inv[sl, None, :]
        t1 = (hi[None] - origin) * inv[sl, None, :]
        tmin = np.minimum(t0, t1).max(2)
        tmax = np.maximum(t0, t1).min(2)
        tmin = np.where((tmax >= tmin) & (tmin > 0), tmin, np.inf).min(1)
        tbest[sl] = np.minimum(tbest[sl], tmin)
    return tbest


def lidar_sweep(origin, lo, hi, n_beams=64, az_step_deg=0.2, elev=(-25.0, 15.0), rng_lim=(2.0, 60.0)):
    """Ray-cast one 360-degree sweep against the ground plane z=0 and the boxes."""
    el = np.deg2rad(np.linspace(elev[0], elev[1], n_beams))
    az = np.deg2rad(np.arange(0.0, 360.0, az_step_deg))
    E, A = np.meshgrid(el, az, indexing="ij")
    d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    tbest = _ray_cast(origin, d, lo, hi)
    keep = (tbest >= rng_lim[0]) & (tbest <= rng_lim[1])
    return origin + d[keep] * tbest[keep, None]


def world(seed=BASE_SEED + 2):
    """The ground and box facades of the LiDAR scenes drawn with ``seed``
    (the same draw as ``lidar_scene``), and its trajectory phase."""
    rng = _rng(seed)
    lo, hi = _boxes(rng)
    phase = float(rng.uniform(0, 2 * math.pi))
    return lo, hi, phase


def trajectory_pose(s, seed_phase=0.0, length=50.0, height=1.8):
    """Camera/sensor pose at arc position s in [0,1] of a 50 m straight path with a yaw sinusoid."""
    x = s * length
    yaw = 0.25 * math.sin(2 * math.pi * s * 1.5 + seed_phase)
    y = 0.8 * math.sin(2 * math.pi * s + seed_phase)
    return np.array([x, y, height]), yaw


def camera_at(pos, yaw, W=1280, H=1024, f=860.0):
    """World->camera pose of a forward-looking camera (x right, y down, z forward)."""
    fwd = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.array([0.0, 0.0, -1.0])
    R = np.stack([right, down, fwd]).astype(np.float32)
    t = (-R.astype(np.float64) @ pos).astype(np.float32)
    return CameraSpec(R, t, float(f), float(f), W / 2.0, H / 2.0, W, H)


def lidar_scene(n, seed=BASE_SEED + 2, sh_degree=3, log_scale=(-3.0, 0.5)):
    """Gaussians initialised from a seeded LiDAR map: sweeps along the trajectory until n points.

    64 beams over [-25, 15] degrees, 0.2 degree azimuth, hits in [2, 60] m on a
    ground plane plus 40 box facades, kept in acquisition order (the order a
    map grown from keyframe point clouds stores them); colour from a
    procedural texture; SH
    band 0 set from the colour, higher bands ~ N(0, 0.1); opacity logit
    ~ N(0,1); log-scale ~ N(log_scale); random unit quaternions.
    """
    rng = _rng(seed)
    lo, hi = _boxes(rng)
    phase = float(rng.uniform(0, 2 * math.pi))
    pts = []
    total = 0
    k = 0
    n_pos = 16
    while True:
        # sweeps at evenly spaced positions, then at the midpoints between them, ...
        rnd, j = divmod(k, n_pos)
        s = (j + 0.5 + (0.5 * rnd) % 1.0) / n_pos
        origin, _ = trajectory_pose(s, phase)
        p = lidar_sweep(origin, lo, hi)
        pts.append(p)
        total += p.shape[0]
        k += 1
        if k % n_pos == 0 and total >= n:
            break
    P = np.concatenate(pts)
    # subsample, keeping acquisition order (sweep by sweep, beam by beam): a map
    # grown from keyframe point clouds stores each frame's points together
    P = P[np.sort(rng.choice(P.shape[0], size=n, replace=False))]
    col = _texture(P)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = (col - 0.5) * (2.0 * math.sqrt(math.pi))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, K - 1, 3))
    params = dict(means=P.astype(np.float32),
                  log_scales=rng.normal(log_scale[0], log_scale[1], (n, 3)).astype(np.float32),
                  quats=random_quats(rng, n),
                  opacity_logits=rng.normal(0.0, 1.0, n).astype(np.float32),
                  sh=sh, sh_degree=sh_degree)
    return params, phase


def fresh_scan(n, step, seed=BASE_SEED + 2):
    """Colourised points of one new LiDAR sweep of the ``lidar_scene`` world (the
    same ground and facades), taken at a seeded trajectory position for map
    expansion step ``step``: at most n points, in acquisition order, with their
    procedural colours in [0, 1].  Returns float32 (points [k,3], colours [k,3])."""
    lo, hi, phase = world(seed)
    r2 = _rng(seed + 1000 + int(step))
    origin, _ = trajectory_pose(float(r2.uniform(0.05, 0.95)), phase)
    P = lidar_sweep(origin, lo, hi)
    if P.shape[0] > n:
        P = P[np.sort(r2.choice(P.shape[0], size=n, replace=False))]
    return P.astype(np.float32), _texture(P).astype(np.float32)


def trajectory_cameras(n_views, seed=BASE_SEED + 3, phase=0.0, W=1280, H=1024, f=860.0):
    """Keyframe cameras at seeded positions along the trajectory."""
    rng = _rng(seed)
    ss = np.sort(rng.uniform(0.05, 0.95, n_views))
    cams = []
    for s in ss:
        pos, yaw = trajectory_pose(float(s), phase)
        cams.append(camera_at(pos, yaw, W, H, f))
    return cams


def camera_centre(cam: CameraSpec):
    """World position of the camera: -R^T t."""
    return -(np.asarray(cam.R, np.float64).T @ np.asarray(cam.t, np.float64))


def camera_image(cam: CameraSpec, seed, world_seed=BASE_SEED + 2, noise=0.01):
    """What the keyframe camera sees of the LiDAR scenes' world: each pixel's
    ray (through the pixel's integer coordinate) is cast against the ground
    and the facades and takes the procedural colour of the hit point, the
    colour the map's LiDAR points carry; rays that hit nothing within 200 m
    see a sky gradient.  Seeded sensor noise N(0, noise), clipped to [0, 1]."""
    lo, hi, _ = world(world_seed)
    R = np.asarray(cam.R, np.float64)
    C = camera_centre(cam)
    ys, xs = np.mgrid[0:cam.H, 0:cam.W]
    dc = np.stack([(xs - cam.cx) / cam.fx, (ys - cam.cy) / cam.fy, np.ones_like(xs, np.float64)], -1)
    d = dc @ R  # R^T d_cam, per pixel
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    t = np.full((cam.H, cam.W), np.inf)
    down = d[..., 2] < 0
    t[down] = C[2] / (-d[..., 2][down])
    # each facade only where its projected bounding rectangle lies
    for b in range(lo.shape[0]):
        corners = np.array([[x, y, z] for x in (lo[b, 0], hi[b, 0]) for y in (lo[b, 1], hi[b, 1])
                            for z in (lo[b, 2], hi[b, 2])])
        pc = corners @ R.T + np.asarray(cam.t, np.float64)
        if (pc[:, 2] <= 0).all():
            continue
        if (pc[:, 2] <= 1e-3).any():
            x0, x1, y0, y1 = 0, cam.W, 0, cam.H
        else:
            u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
            v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
            x0, x1 = max(0, int(np.floor(u.min()))), min(cam.W, int(np.ceil(u.max())) + 1)
            y0, y1 = max(0, int(np.floor(v.min()))), min(cam.H, int(np.ceil(v.max())) + 1)
            if x0 >= x1 or y0 >= y1:
                continue
        db = d[y0:y1, x0:x1]
        inv = 1.0 / np.where(np.abs(db) < 1e-12, 1e-12, db)
        t0 = (lo[b] - C) * inv
        t1 = (hi[b] - C) * inv
        tmin = np.minimum(t0, t1).max(-1)
        tmax = np.maximum(t0, t1).min(-1)
        tb = np.where((tmax >= tmin) & (tmin > 0), tmin, np.inf)
        t[y0:y1, x0:x1] = np.minimum(t[y0:y1, x0:x1], tb)
    d = d.reshape(-1, 3)
    t = t.reshape(-1)
    hit = np.isfinite(t) & (t < 200.0)
    img = np.empty((d.shape[0], 3))
    img[hit] = _texture(C + d[hit] * t[hit, None])
    up = np.clip(d[~hit, 2], 0.0, 1.0)[:, None]
    img[~hit] = np.array([0.62, 0.74, 0.90]) * (1 - up) + np.array([0.30, 0.45, 0.80]) * up
    img = img.reshape(cam.H, cam.W, 3).transpose(2, 0, 1)
    img = img + _rng(seed).normal(0.0, noise, img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def lidar_depth_image(cam: CameraSpec, world_seed=BASE_SEED + 2, z_near=0.2):
    """Sparse LiDAR depth target of a keyframe: one sweep of the world taken
    from the camera's position, projected into the camera (pinhole, nearest
    pixel), keeping the nearest return per pixel (a z-buffer).  Values are
    view-space depths; pixels without a return hold 0."""
    lo, hi, _ = world(world_seed)
    C = camera_centre(cam)
    P = lidar_sweep(C, lo, hi)
    R = np.asarray(cam.R, np.float64)
    pc = P @ R.T + np.asarray(cam.t, np.float64)
    z = pc[:, 2]
    front = z > z_near
    u = np.rint(cam.fx * pc[front, 0] / z[front] + cam.cx).astype(np.int64)
    v = np.rint(cam.fy * pc[front, 1] / z[front] + cam.cy).astype(np.int64)
    zf = z[front]
    inb = (u >= 0) & (u < cam.W) & (v >= 0) & (v < cam.H)
    depth = np.full(cam.H * cam.W, np.inf)
    np.minimum.at(depth, v[inb] * cam.W + u[inb], zf[inb])
    depth[~np.isfinite(depth)] = 0.0
    return depth.reshape(cam.H, cam.W).astype(np.float32)


def target_images(cam: CameraSpec, seed, world_seed=BASE_SEED + 2):
    """Level-0 targets of one keyframe of the LiDAR scenes: the camera's image
    of the world (``camera_image``, noise seeded by ``seed``) and the sparse
    LiDAR depth of a sweep from the keyframe's position (``lidar_depth_image``)."""
    return camera_image(cam, seed, world_seed), lidar_depth_image(cam, world_seed)


def mixed_level_views(n_views, seed=BASE_SEED + 4, levels=(0, 1, 2)):
    """Pyramid level per keyframe, drawn uniformly from ``levels``."""
    rng = _rng(seed)
    return [int(v) for v in rng.choice(levels, size=n_views)]


def workload(name):
    """Named workloads (all seeded).  Returns a dict of params, cameras, levels, targets."""
    if name == "small_160x120_2k":
        params, cam, gt, lidar = small_scene()
        return dict(params=params, cams=[cam], levels=[0], gts=[gt], lidars=[lidar],
                    lam=0.0, lam_d=1.0)
    if name.startswith("pyramid_"):
        # pyramid_<N> : one keyframe rendered at pyramid levels 0, 1 and 2 from N Gaussians
        n = int(name.split("_")[1])
        params, phase = lidar_scene(n)
        cam = trajectory_cameras(1, phase=phase)[0]
        gt, li = target_images(cam, BASE_SEED + 100)
        return dict(params=params, cams=[cam, cam, cam], levels=[0, 1, 2], gts=[gt, gt, gt],
                    lidars=[li, li, li], lam=0.2, lam_d=0.1)
    if name.startswith("lidar_"):
        # lidar_<N>_<V>v : N Gaussians, V keyframes at mixed levels
        _, n, v = name.split("_")
        n = int(n)
        V = int(v.rstrip("v"))
        params, phase = lidar_scene(n)
        cams = trajectory_cameras(V, phase=phase)
        levels = [0] if V == 1 else mixed_level_views(V)
        tg = [target_images(c, BASE_SEED + 100 + i) for i, c in enumerate(cams)]
        return dict(params=params, cams=cams, levels=levels, gts=[t[0] for t in tg],
                    lidars=[t[1] for t in tg], lam=0.2, lam_d=0.1)
    raise KeyError(name)
