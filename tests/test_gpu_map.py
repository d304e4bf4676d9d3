"""GPU parity of the map-maintenance calls (through the C ABI) against the
oracle of ``oracle/map_ops.py``: the Adam step, map expansion from colourised
LiDAR points (nearest-neighbour scales, initial values, the visibility filter)
and pruning.

Bars: integer and selection results (which points are kept, which Gaussians
survive pruning, row order) bit-exact; copied values (centres, quaternions)
bit-exact; log-scales within 1e-5 absolute; the Adam update within 1e-3 of
its size plus binary32 rounding of the parameter; moments within 1e-6
relative.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from oracle import map_ops as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = M.PARAM_KEYS


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P

    P.load()
    return P


@pytest.fixture(scope="module")
def ctx(pkg):
    return pkg.Context()


def _rand(rng, n, K):
    return {"means": rng.normal(0, 5, (n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
            "quats": rng.normal(0, 1, (n, 4)), "opacity_logits": rng.normal(0, 1, n),
            "sh": rng.normal(0, 0.3, (n, K, 3))}


def _f32(d):
    return {k: np.asarray(v, np.float32) for k, v in d.items()}


def _dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def _host(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _adam_gpu(lib, P, G, Mo, V, n, K, step, zero_grads=0, offset=0):
    from paper_2411_02703_gb300 import _lib as L

    def bufs(d):
        return L.ParamBuffers(*(d[k].data_ptr() + offset * 4 for k in KEYS))

    g = L.Grads(*(G[k].data_ptr() + offset * 4 for k in KEYS), 0)
    code = lib.lvigs_adam_step(ctypes.byref(bufs(P)), ctypes.byref(g), ctypes.byref(bufs(Mo)), ctypes.byref(bufs(V)),
                               n, K, step, None, zero_grads, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0


def _check_adam(before, after_gpu, g, step):
    """Moments: within 1e-6 of the sum of the magnitudes of their two terms (the
    binary32 rounding bound of b m + (1 - b) g, which may cancel).  Parameters:
    the oracle's update computed from the moments the GPU produced, within 1e-3
    of the update plus binary32 rounding of the parameter."""
    (p0, m0, v0), (p1, m1, v1) = before, after_gpu
    cfg = M.ADAM_DEFAULTS
    b1, b2 = cfg["beta1"], cfg["beta2"]
    _, mr, vr = M.adam_step(p0, g, m0, v0, step)
    for k in p0:
        gk = np.asarray(g[k], np.float64)
        mb = 1e-6 * (b1 * np.abs(m0[k]) + (1 - b1) * np.abs(gk)) + 1e-37
        assert np.all(np.abs(m1[k] - mr[k]) <= mb), k
        vb = 1e-6 * (b2 * np.abs(v0[k]) + (1 - b2) * gk * gk) + 1e-40
        assert np.all(np.abs(v1[k] - vr[k]) <= vb), k
    # the update given the GPU's moments
    pr, _, _ = M.adam_step(p0, {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in g.items()},
                           {k: np.asarray(m1[k], np.float64) / b1 for k in p0},
                           {k: np.asarray(v1[k], np.float64) / b2 for k in p0}, step)
    for k in p0:
        d = np.abs(pr[k] - p0[k])
        assert np.all(np.abs(p1[k] - pr[k]) <= 1e-3 * d + 2.5e-7 * np.abs(pr[k]) + 1e-30), k


@pytest.mark.parametrize("n,K", [(10001, 16), (777, 1), (1, 4)])
def test_adam_step_parity(pkg, n, K):
    from paper_2411_02703_gb300 import _lib as L

    lib = L.load()
    rng = np.random.default_rng(10 + n)
    P = _dev(_f32(_rand(rng, n, K)))
    Mo = _dev({k: np.zeros_like(v.cpu().numpy()) for k, v in P.items()})
    V = _dev({k: np.zeros_like(v.cpu().numpy()) for k, v in P.items()})
    for step in range(1, 4):
        g = _f32(_rand(rng, n, K))
        if step == 2:
            g["opacity_logits"][: n // 2] = 0.0
        G = _dev(g)
        before = (_host(P), _host(Mo), _host(V))
        _adam_gpu(lib, P, G, Mo, V, n, K, step)
        torch.cuda.synchronize()
        _check_adam(before, (_host(P), _host(Mo), _host(V)), g, step)


def test_adam_unaligned_buffers_and_zero_grads(pkg):
    """Buffers starting 4 bytes past a 16-byte boundary take the scalar path."""
    from paper_2411_02703_gb300 import _lib as L

    lib = L.load()
    n, K = 513, 16
    rng = np.random.default_rng(3)
    big = _f32(_rand(rng, n + 1, K))
    P = _dev(big)
    Mo = _dev({k: np.abs(v) * 0.1 for k, v in _f32(_rand(rng, n + 1, K)).items()})
    V = _dev({k: np.abs(v) * 0.01 for k, v in _f32(_rand(rng, n + 1, K)).items()})
    g = _f32(_rand(rng, n + 1, K))
    G = _dev(g)
    flat = lambda d: {k: v.reshape(-1) for k, v in _host(d).items()}
    b0 = (flat(P), flat(Mo), flat(V))
    _adam_gpu(lib, P, G, Mo, V, n, K, 5, zero_grads=1, offset=1)
    torch.cuda.synchronize()
    gf = {k: v.reshape(-1) for k, v in g.items()}
    # rows shifted by one float: the call sees elements [1, 1 + n * width).
    # (SH is left out: its learning rate follows the coefficient index, which
    # the one-float shift moves)
    width = {"means": 3, "log_scales": 3, "quats": 4, "opacity_logits": 1}
    sl = {k: slice(1, 1 + n * w) for k, w in width.items()}
    sub = lambda d: {k: d[k][sl[k]] for k in width}
    a1 = (flat(P), flat(Mo), flat(V))
    _check_adam((sub(b0[0]), sub(b0[1]), sub(b0[2])), (sub(a1[0]), sub(a1[1]), sub(a1[2])), sub(gf), 5)
    for k in width:
        assert a1[0][k][0] == b0[0][k][0]  # untouched element before the view
    gz = flat(G)
    sl["sh"] = slice(1, 1 + n * 3 * K)
    for k in KEYS:
        assert np.all(gz[k][sl[k]] == 0.0) and gz[k][0] == gf[k][0]


def test_adam_full_size(pkg):
    """One step over 1,000,000 Gaussians at SH degree 3 (every element)."""
    from paper_2411_02703_gb300 import _lib as L

    lib = L.load()
    n, K = 1_000_000, 16
    rng = np.random.default_rng(4)
    p = _f32(_rand(rng, n, K))
    g = _f32(_rand(rng, n, K))
    m = {k: (0.1 * v).astype(np.float32) for k, v in _f32(_rand(rng, n, K)).items()}
    v = {k: (0.01 * np.abs(x)).astype(np.float32) for k, x in _f32(_rand(rng, n, K)).items()}
    P, G, Mo, V = _dev(p), _dev(g), _dev(m), _dev(v)
    _adam_gpu(lib, P, G, Mo, V, n, K, 12)
    torch.cuda.synchronize()
    _check_adam((p, m, v), (_host(P), _host(Mo), _host(V)), g, 12)


def _append(pkg, ctx, pts, col, n0=0, cam=None, level=0, alpha=None, cfg=None, K=16):
    gm = pkg.GaussianMap(capacity=n0 + pts.shape[0] + 5, sh_stride_k=K)
    if n0:
        gm.n = n0
    added = gm.append(ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(col).cuda(), cam, level,
                      None if alpha is None else torch.from_numpy(alpha).cuda(), cfg)
    torch.cuda.synchronize()
    return gm, added


def _check_init(gm, n0, pts, col, K):
    ref = M.init_gaussians(pts, col, sh_stride_k=K)
    n = pts.shape[0]
    got = {k: v.cpu().numpy()[n0:n0 + n] for k, v in gm.params().items() if k != "sh_degree"}
    np.testing.assert_array_equal(got["means"], pts)
    assert np.abs(got["log_scales"] - ref["log_scales"]).max() <= 1e-5
    np.testing.assert_array_equal(got["quats"], ref["quats"].astype(np.float32))
    np.testing.assert_allclose(got["opacity_logits"], ref["opacity_logits"], rtol=1e-6)
    np.testing.assert_allclose(got["sh"][:, 0], ref["sh"][:, 0], rtol=1e-6, atol=1e-6)
    assert np.all(got["sh"][:, 1:] == 0.0)
    m, v = gm.adam_state()
    for k in KEYS:
        assert np.all(m[k].cpu().numpy()[n0:] == 0.0) and np.all(v[k].cpu().numpy()[n0:] == 0.0)


def test_append_fresh_scan(pkg, ctx):
    """50,000 points of a new sweep (the per-step expansion of the large map)."""
    pts, col = S.fresh_scan(50_000, step=0)
    gm, added = _append(pkg, ctx, pts, col, n0=0)
    assert added == pts.shape[0] and gm.n == pts.shape[0]
    _check_init(gm, 0, pts, col, 16)


def test_append_first_frame_large_cloud(pkg, ctx):
    """A whole 300,000-point map cloud initialised at once (the first frame)."""
    params, _ = S.lidar_scene(300_000)
    pts = params["means"]
    col = np.clip(0.5 + params["sh"][:, 0, :] / (2.0 * np.sqrt(np.pi)), 0, 1).astype(np.float32)
    gm, added = _append(pkg, ctx, pts, col, n0=0, K=4)
    assert added == pts.shape[0]
    _check_init(gm, 0, pts, col, 4)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7])
def test_append_few_points(pkg, ctx, k):
    rng = np.random.default_rng(20 + k)
    pts = rng.normal(0, 1, (k, 3)).astype(np.float32)
    col = rng.uniform(0, 1, (k, 3)).astype(np.float32)
    gm, added = _append(pkg, ctx, pts, col, n0=3, K=1)
    assert added == k and gm.n == 3 + k
    _check_init(gm, 3, pts, col, 1)


def _alpha_field(H, W, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, W), indexing="ij")
    a = 0.5 + 0.45 * np.sin(7 * xx + rng.uniform(0, 6)) * np.cos(5 * yy + rng.uniform(0, 6))
    a = a.astype(np.float32)
    a[::7, ::5] = 0.5  # exactly at the threshold
    return a


@pytest.mark.parametrize("literal", [0, 1])
def test_append_visibility_filter(pkg, ctx, literal):
    pts, col = S.fresh_scan(50_000, step=1)
    spec = S.trajectory_cameras(3, phase=0.3)[1]
    import oracle as O

    cam = O.level_camera(O.Camera(spec.R, spec.t, spec.fx, spec.fy, spec.cx, spec.cy, spec.W, spec.H), 1)
    alpha = _alpha_field(cam.H, cam.W, 5)
    keep = M.visibility_keep(pts, cam, alpha, tau_alpha=0.5, literal=bool(literal))
    assert 0 < keep.sum() < keep.size
    gm, added = _append(pkg, ctx, pts, col, n0=10, cam=spec, level=1, alpha=alpha, cfg={"filter_literal": literal})
    assert added == int(keep.sum())
    _check_init(gm, 10, pts[keep], col[keep], 16)


def test_append_capacity_error(pkg, ctx):
    gm = pkg.GaussianMap(capacity=4, sh_stride_k=1)
    pts = torch.zeros((5, 3), device="cuda")
    from paper_2411_02703_gb300 import _lib as L

    n_out = ctypes.c_int64()
    code = L.load().lvigs_append_gaussians(
        ctx._h, ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(pts.data_ptr()), 5, None, 0, None, None,
        ctypes.byref(L.ParamBuffers(*(gm._p[k].data_ptr() for k in KEYS))), None, None, 0, 4, 1,
        ctypes.byref(n_out), None)
    assert code == 4  # LVIGS_ERR_CAPACITY


def test_prune_parity(pkg, ctx):
    rng = np.random.default_rng(6)
    n, K = 20011, 16
    params = _f32(_rand(rng, n, K))
    params["opacity_logits"] = rng.normal(-4, 2, n).astype(np.float32)
    thr = np.float32(np.log(0.005 / 0.995))
    params["opacity_logits"][::97] = thr  # exactly at the threshold: kept
    params["opacity_logits"][1::97] = np.nextafter(thr, np.float32(-np.inf))
    gm = pkg.GaussianMap.from_params(dict(params, sh_degree=3), capacity=n + 100)
    m, v = gm.adam_state()
    mh = _f32(_rand(rng, n, K))
    vh = {k: np.abs(x) for k, x in _f32(_rand(rng, n, K)).items()}
    for k in KEYS:
        m[k].copy_(torch.from_numpy(mh[k]))
        v[k].copy_(torch.from_numpy(vh[k]))
    removed = gm.prune(ctx, 0.005)
    torch.cuda.synchronize()
    keep = M.prune_keep(params["opacity_logits"], 0.005)
    assert removed == n - keep.sum() and gm.n == keep.sum()
    m2, v2 = gm.adam_state()
    for got, src in ((gm.params(), params), (m2, mh), (v2, vh)):
        ref = M.compact_rows(src, keep)
        for k in KEYS:
            np.testing.assert_array_equal(got[k].cpu().numpy(), ref[k])


def test_appended_map_renders_like_oracle(pkg, ctx):
    """Expand a small map, then render it: the capacity growth and the new rows
    feed the renderer like any parameter set."""
    import oracle as O

    params, cam, _, _ = S.small_scene(n=500, W=64, H=48, f=60.0)
    gm = pkg.GaussianMap.from_params(params, capacity=600)
    rng = np.random.default_rng(7)
    pts = np.stack([rng.uniform(-2, 2, 800), rng.uniform(-1.5, 1.5, 800), rng.uniform(3, 8, 800)], 1).astype(np.float32)
    col = rng.uniform(0, 1, (800, 3)).astype(np.float32)
    gm.append(ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(col).cuda())
    assert gm.n == 1300 and gm.capacity >= 1300
    p = gm.params()
    rgb, depth, alpha, slot = ctx.render(p, cam, 0)
    ctx.release(slot)
    host = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in p.items()}
    ref = O.render_view(host, O.Camera(cam.R, cam.t, cam.fx, cam.fy, cam.cx, cam.cy, cam.W, cam.H), 0)
    ok = ref["margin"] > 1e-4
    assert ok.mean() > 0.95
    assert np.abs(rgb.cpu().numpy() - ref["rgb"])[:, ok].max() <= 1e-4


def test_mapper_reduces_loss(pkg, ctx):
    """A short mapping run (expansion from fresh sweeps, coarse-to-fine
    schedule, Adam) lowers every keyframe's full-resolution loss."""
    cams = S.trajectory_cameras(3, phase=0.7, W=256, H=192, f=172.0)
    tg = [S.target_images(c, 300 + i) for i, c in enumerate(cams)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gm = pkg.GaussianMap(capacity=1000, sh_stride_k=16)
    mapper = pkg.Mapper(ctx, gm, pkg.MappingSchedule(max_iters=30, top_level=2, sh_interval=15, views_per_step=2,
                                                     seed=1), delay=0)
    kfs = []
    for i, c in enumerate(cams):
        pts, col = S.fresh_scan(20_000, step=10 + i)
        kf = pkg.Keyframe(cam=c, gt_rgb=t(tg[i][0]), lidar=t(tg[i][1]), points=t(pts), colours=t(col))
        mapper.add_keyframe(kf)
        kfs.append(kf)
    assert gm.n > 20_000  # the first sweep unfiltered, the later ones filtered

    def full_res_losses():
        out = []
        for kf in kfs:
            rgb, depth, alpha, slot = ctx.render(gm.params(), kf.cam, 0)
            ctx.release(slot)
            terms, _, _ = ctx.loss(rgb, depth, kf.gt_rgb, kf.lidar, 0.2, 0.1, grads=False)
            out.append(float(terms[0]))
        return out

    before = full_res_losses()
    steps = 0
    while mapper.step() is not None:
        steps += 1
    after = full_res_losses()
    print(f"  {steps} steps, n={gm.n}, loss before {before} after {after}")
    assert sum(kf.iters for kf in kfs) == 3 * 30 and steps >= 3 + 87 // 2
    assert all(a < 0.9 * b for a, b in zip(after, before))
    assert gm.sh_degree == 3


def test_map_edge_cases(pkg, ctx):
    """Empty appends, a filter that drops every point, pruning everything, and
    an Adam step on an empty map."""
    rng = np.random.default_rng(8)
    pts = rng.normal(0, 1, (100, 3)).astype(np.float32) + np.array([0, 0, 6], np.float32)
    col = rng.uniform(0, 1, (100, 3)).astype(np.float32)
    gm = pkg.GaussianMap(capacity=8, sh_stride_k=4)
    # nothing to add
    assert gm.append(ctx, torch.zeros((0, 3), device="cuda"), torch.zeros((0, 3), device="cuda")) == 0
    assert gm.n == 0
    gm.adam_step()  # empty map: no work, no error
    # a fully opaque keyframe drops every point in view; the rest (none) is kept
    cam = S.CameraSpec(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 50.0, 50.0, 32.0, 24.0, 64, 48)
    import oracle as O

    _, _, inview = M.point_pixels(pts, O.Camera(cam.R, cam.t, cam.fx, cam.fy, cam.cx, cam.cy, cam.W, cam.H))
    alpha = torch.ones((48, 64), device="cuda")
    added = gm.append(ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(col).cuda(), cam, 0, alpha)
    assert added == int((~inview).sum())
    n_keep = gm.n
    # a transparent keyframe keeps everything (and grows the buffers)
    added = gm.append(ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(col).cuda(), cam, 0,
                      torch.zeros((48, 64), device="cuda"))
    assert added == 100 and gm.n == n_keep + 100 and gm.capacity >= gm.n
    # opacity 0.1 everywhere: pruning at 0.5 removes all, at 0.05 none
    assert gm.prune(ctx, 0.05) == 0
    assert gm.prune(ctx, 0.5) == n_keep + 100 and gm.n == 0
    gm.adam_step()
