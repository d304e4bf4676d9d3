"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: tile keys and sort order bit-exact; rgb / depth / alpha within 1e-4
absolute; gradients within 1e-3 relative (with an absolute floor of 1e-3 of
the tensor's largest entry).  Pixels where the oracle sees a threshold test
(power vs 0, alpha vs 1/255, o*G vs 0.99, T vs 1e-4) within a relative
margin of 1e-4 may take the other branch in binary32; they are excused and
counted, and so are the gradients of Gaussians listed in their tiles.  The
oracle's margin of the alpha, o*G and T tests is net of the deviation that the
binary32 screen position and covariance (bit-exact on both sides) and the
binary32 evaluation of the exponent may cause: a Gaussian one pixel wide at
u = 600 moves its exponent by ~1e-4 from the rounding of u alone.
"""
import functools
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 1e-4
IMG_TOL = 1e-4
GRAD_RTOL = 1e-3


@functools.lru_cache(maxsize=None)
def lidar(n):
    return S.lidar_scene(n)


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P

    P.load()
    return P


_ctx_cache = {}


def ctx_for(pkg, tile=(16, 16)):
    if tile not in _ctx_cache:
        _ctx_cache[tile] = pkg.Context(tile=tile)
    return _ctx_cache[tile]


def dev_params(params):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
            for k, v in params.items()}


def ocam(spec):
    return O.Camera(spec.R, spec.t, spec.fx, spec.fy, spec.cx, spec.cy, spec.W, spec.H)


def excused_tiles_gaussians(ref, tile, W, H, excused_px):
    """Gaussians listed in any tile that holds an excused pixel."""
    tx_n = (W + tile[0] - 1) // tile[0]
    ys, xs = np.nonzero(excused_px)
    tiles = np.unique((ys // tile[1]) * tx_n + xs // tile[0])
    out = set()
    for t in tiles:
        s, e = ref["ranges"][t]
        out.update(ref["vals"][s:e].tolist())
    return np.array(sorted(out), dtype=np.int64)


def compare_images(gpu, ref, excused, tol=IMG_TOL):
    rgb, depth, alpha = (x.cpu().numpy().astype(np.float64) for x in gpu)
    ok = ~excused
    e_rgb = np.abs(rgb - ref["rgb"])[:, ok].max(initial=0.0)
    e_d = np.abs(depth - ref["depth"])[ok].max(initial=0.0)
    e_a = np.abs(alpha - ref["alpha"])[ok].max(initial=0.0)
    return e_rgb, e_d, e_a


def grad_check(name, g, r, excl=None, rtol=GRAD_RTOL):
    g = np.asarray(g, np.float64).reshape(r.shape[0], -1)
    r = np.asarray(r, np.float64).reshape(r.shape[0], -1)
    mask = np.ones(r.shape[0], bool)
    if excl is not None and len(excl):
        mask[excl] = False
    scale = np.abs(r[mask]).max(initial=0.0)
    err = np.abs(g - r)[mask]
    bound = rtol * np.abs(r[mask]) + rtol * scale
    worst = (err / np.maximum(bound, 1e-30)).max(initial=0.0)
    rel_norm = np.linalg.norm(err) / max(np.linalg.norm(r[mask]), 1e-30)
    msg = f"  grad {name}: max err/bound {worst:.3f}  rel-norm err {rel_norm:.2e}  scale {scale:.3e}"
    if not mask.all():
        # the excused rows still count in the whole tensor's relative norm: a
        # branch taken the other way moves a few pixels' terms, not the tensor
        all_norm = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
        msg += f"  (all rows: rel-norm err {all_norm:.2e})"
        assert all_norm <= rtol, f"{name}: relative norm error {all_norm:.2e} over all rows"
    print(msg)
    assert (err <= bound).all(), f"{name}: {int((err > bound).sum())} entries beyond tolerance"


# ---------------------------------------------------------------------------
# a1-a4: keys and order bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_keys_bit_exact_small(pkg, tile):
    params, spec, _, _ = S.small_scene()
    lv = ctx_for(pkg, tile)
    _, _, _, slot = lv.render(dev_params(params), spec, 0)
    keys, vals = lv.debug_keys(slot)
    lv.release(slot)
    pre = O.preprocess(params, ocam(spec), tile)
    rk, rv = O.build_keys(pre)
    assert keys.shape[0] == rk.shape[0]
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), rk)
    np.testing.assert_array_equal(vals.cpu().numpy().view(np.uint32), rv)


def test_keys_bit_exact_full_size_lidar(pkg):
    """1280x1024, 200k Gaussians from the LiDAR generator, SH degree 3."""
    params, phase = lidar(200_000)
    cams = S.trajectory_cameras(2, phase=phase)
    lv = ctx_for(pkg)
    dp = dev_params(params)
    for spec in cams:
        for level in (0, 2):
            _, _, _, slot = lv.render(dp, spec, level)
            keys, vals = lv.debug_keys(slot)
            lv.release(slot)
            pre = O.preprocess(params, O.level_camera(ocam(spec), level))
            rk, rv = O.build_keys(pre)
            assert keys.shape[0] == rk.shape[0] > 10000
            np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), rk)
            np.testing.assert_array_equal(vals.cpu().numpy().view(np.uint32), rv)


def test_key_exp_bit_exact(pkg):
    """The key stage's binary32 exp (table-driven, binary64 only where the
    rounding is not certain) against the oracle's binary64 exp rounded once:
    16.8M values over the log-scale range, the reduction's boundaries, the
    fallback range and special values."""
    import ctypes

    from paper_2411_02703_gb300 import _lib as L

    rng = np.random.default_rng(5)
    step = np.log(2.0) / 32.0
    k = np.arange(-2000, 2000)
    edges = np.concatenate([(k + 0.5) * step, k * step])
    x = np.concatenate([rng.uniform(-12, 8, 12_000_000), rng.normal(-3, 0.5, 4_000_000),
                        edges, np.nextafter(edges.astype(np.float32), np.float32(np.inf)),
                        np.nextafter(edges.astype(np.float32), np.float32(-np.inf)),
                        rng.uniform(-90, 90, 100_000),
                        [0.0, -0.0, 1e-30, -1e-30, 59.999, -59.999, 60.0, -60.0, 88.7, -103.0]]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    code = L.load().lvigs_debug_exp_key(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), x.size,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    ref = O.exp_key(x)
    got = yd.cpu().numpy()
    bad = np.nonzero(got.view(np.uint32) != ref.view(np.uint32))[0]
    assert bad.size == 0, (bad.size, x[bad[:5]], got[bad[:5]], ref[bad[:5]])


def test_ranges_and_contributors(pkg):
    params, spec, _, _ = S.small_scene()
    lv = ctx_for(pkg)
    _, _, _, slot = lv.render(dev_params(params), spec, 0)
    ranges, nc, ft = lv.debug_state(slot, spec.H, spec.W)
    lv.release(slot)
    ref = O.render_view(params, ocam(spec), 0)
    np.testing.assert_array_equal(ranges.cpu().numpy().view(np.uint32), ref["ranges"])
    ok = ref["margin"] > MARGIN
    np.testing.assert_array_equal(nc.cpu().numpy()[ok], ref["n_contrib"][ok])
    np.testing.assert_allclose(ft.cpu().numpy()[ok], ref["final_T"][ok], atol=IMG_TOL)


# ---------------------------------------------------------------------------
# a5: images
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_forward_images_small(pkg, tile):
    params, spec, _, _ = S.small_scene()
    lv = ctx_for(pkg, tile)
    rgb, depth, alpha, slot = lv.render(dev_params(params), spec, 0)
    lv.release(slot)
    ref = O.render_view(params, ocam(spec), 0, tile)
    exc = ref["margin"] <= MARGIN
    e = compare_images((rgb, depth, alpha), ref, exc)
    print(f"  tile {tile}: excused {exc.mean():.4%}  max err rgb {e[0]:.2e} depth {e[1]:.2e} alpha {e[2]:.2e}")
    assert exc.mean() < 0.01
    assert max(e) < IMG_TOL


def test_forward_sampled_full_size(pkg):
    """1280x1024, 200k Gaussians: oracle on 48 sampled tiles of each view."""
    params, phase = lidar(200_000)
    cams = S.trajectory_cameras(3, phase=phase)
    lv = ctx_for(pkg)
    dp = dev_params(params)
    rng = np.random.default_rng(0)
    for spec in cams:
        rgb, depth, alpha, slot = lv.render(dp, spec, 0)
        lv.release(slot)
        cam = ocam(spec)
        n_tiles = 80 * 64
        sel = rng.choice(n_tiles, 48, replace=False).astype(np.int32)
        ref = O.render_view(params, cam, 0, sel_tiles=sel)
        mask = np.zeros((spec.H, spec.W), bool)
        for t in sel:
            ty, tx = divmod(int(t), 80)
            mask[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
        exc = (ref["margin"] <= MARGIN) | ~mask
        e = compare_images((rgb, depth, alpha), ref, exc)
        frac = ((ref["margin"] <= MARGIN) & mask).sum() / mask.sum()
        print(f"  excused {frac:.4%}  max err rgb {e[0]:.2e} depth {e[1]:.2e} alpha {e[2]:.2e}")
        assert frac < 0.02
        assert e[0] < IMG_TOL and e[2] < IMG_TOL
        # depth is an opacity-weighted sum of metres: the same relative bar
        assert e[1] < IMG_TOL * max(1.0, float(np.abs(ref["depth"][mask]).max()))


def test_edge_cases(pkg):
    lv = ctx_for(pkg)
    # ragged image (tiles cut by the border) and few Gaussians
    params, spec, _, _ = S.small_scene(n=40, W=37, H=23, f=30.0)
    rgb, depth, alpha, slot = lv.render(dev_params(params), spec, 0)
    lv.release(slot)
    ref = O.render_view(params, ocam(spec), 0)
    e = compare_images((rgb, depth, alpha), ref, ref["margin"] <= MARGIN)
    assert max(e[0], e[2]) < IMG_TOL
    # empty map
    empty = {k: (v[:0].copy() if isinstance(v, np.ndarray) else v) for k, v in params.items()}
    rgb, depth, alpha, slot = lv.render(dev_params(empty), spec, 0)
    g = lv.backward(slot, dev_params(empty), torch.ones_like(rgb), torch.ones_like(depth))
    lv.release(slot)
    assert float(rgb.abs().max()) == 0.0 and float(alpha.abs().max()) == 0.0
    assert g["means"].numel() == 0
    # everything behind the camera
    behind = dict(params)
    behind["means"] = params["means"] * np.array([1, 1, -1], np.float32)
    rgb, depth, alpha, slot = lv.render(dev_params(behind), spec, 0)
    keys, _ = lv.debug_keys(slot)
    lv.release(slot)
    assert keys.numel() == 0 and float(alpha.abs().max()) == 0.0
    # deepest pyramid level
    params, spec, _, _ = S.small_scene(n=300)
    rgb, depth, alpha, slot = lv.render(dev_params(params), spec, 4)
    lv.release(slot)
    assert rgb.shape == (3, 120 >> 4, 160 >> 4)
    ref = O.render_view(params, ocam(spec), 4)
    e = compare_images((rgb, depth, alpha), ref, ref["margin"] <= MARGIN)
    assert max(e[0], e[2]) < IMG_TOL
    # invalid arguments come back as errors, not faults
    with pytest.raises(pkg.LvigsError):
        lv.render(dev_params(params), spec, 9)
    with pytest.raises(pkg.LvigsError):
        lv.backward(123456, dev_params(params), torch.ones(3, 4, 4, device="cuda"))


# ---------------------------------------------------------------------------
# a8 + a9: loss and pyramid
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,lam,lamd", [((120, 160), 0.0, 1.0), ((120, 160), 0.2, 0.1), ((250, 331), 0.2, 0.1)])
def test_loss_parity(pkg, shape, lam, lamd):
    H, W = shape
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1).astype(np.float32)
    d = rng.uniform(2, 10, (H, W)).astype(np.float32)
    li = np.where(rng.uniform(size=(H, W)) < 0.05, rng.uniform(2, 10, (H, W)), 0).astype(np.float32)
    lv = ctx_for(pkg)
    t = lambda a: torch.from_numpy(a).cuda()
    terms, d_img, d_dep = lv.loss(t(x), t(d), t(y), t(li), lam, lamd)
    rterms, r_img, r_dep = O.loss(x, y, d, li, lam, lamd)
    np.testing.assert_allclose(terms.cpu().numpy(), rterms, rtol=1e-5, atol=1e-7)
    gi = d_img.cpu().numpy()
    scale = np.abs(r_img).max()
    assert np.abs(gi - r_img).max() <= 1e-3 * scale
    np.testing.assert_allclose(d_dep.cpu().numpy(), r_dep, rtol=1e-5, atol=1e-12)


def test_loss_full_size(pkg):
    H, W = 1024, 1280
    spec = S.camera_at(np.array([5.0, 0.0, 1.8]), 0.1)
    gt, li = S.target_images(spec, 7)
    rng = np.random.default_rng(2)
    x = np.clip(gt + rng.normal(0, 0.1, gt.shape), 0, 1).astype(np.float32)
    d = rng.uniform(2, 60, (H, W)).astype(np.float32)
    lv = ctx_for(pkg)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    terms, d_img, d_dep = lv.loss(t(x), t(d), t(gt), t(li), 0.2, 0.1)
    rterms, r_img, r_dep = O.loss(x, gt, d, li, 0.2, 0.1)
    np.testing.assert_allclose(terms.cpu().numpy(), rterms, rtol=1e-5)
    assert np.abs(d_img.cpu().numpy() - r_img).max() <= 1e-3 * np.abs(r_img).max()


def test_pyramid_parity(pkg):
    rng = np.random.default_rng(3)
    rgb = rng.uniform(size=(3, 64, 90)).astype(np.float32)
    dep = np.where(rng.uniform(size=(64, 90)) < 0.3, rng.uniform(1, 9, (64, 90)), 0).astype(np.float32)
    lv = ctx_for(pkg)
    r1, d1 = lv.pyramid_down(torch.from_numpy(rgb).cuda(), torch.from_numpy(dep).cuda())
    rr, rd = O.pyramid_down(rgb, dep)
    np.testing.assert_allclose(r1.cpu().numpy(), rr, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(d1.cpu().numpy(), rd, rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------------------
# a6 + a7: gradients
# ---------------------------------------------------------------------------
def _backward_case(pkg, params, spec, level, tile=(16, 16), seed=4):
    lv = ctx_for(pkg, tile)
    dp = dev_params(params)
    rgb, depth, alpha, slot = lv.render(dp, spec, level)
    H, W = depth.shape
    rng = np.random.default_rng(seed)
    g_rgb = (rng.normal(size=(3, H, W)) * 1e-3).astype(np.float32)
    g_dep = (rng.normal(size=(H, W)) * 1e-4).astype(np.float32)
    g_alp = (rng.normal(size=(H, W)) * 1e-3).astype(np.float32)
    grads = lv.backward(slot, dp, torch.from_numpy(g_rgb).cuda(), torch.from_numpy(g_dep).cuda(),
                        torch.from_numpy(g_alp).cuda())
    lv.release(slot)
    cam = O.level_camera(ocam(spec), level)
    ref = O.render_view(params, ocam(spec), level, tile)
    g2 = O.backward_render(ref["pre"], ref["vals"], ref["ranges"], cam.W, cam.H, g_rgb, g_dep, g_alp, tile)
    rg = O.backward_preprocess(params, cam, ref["pre"], g2)
    exc_px = ref["margin"] <= MARGIN
    excl = excused_tiles_gaussians(ref, tile, cam.W, cam.H, exc_px)
    print(f"  excused pixels {exc_px.mean():.4%}, excused Gaussians {len(excl)}")
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_check(k, grads[k].cpu().numpy(), rg[k], excl)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_backward_small(pkg, tile):
    params, spec, _, _ = S.small_scene()
    _backward_case(pkg, params, spec, 0, tile)


def test_backward_lidar_sh3(pkg):
    params, phase = lidar(30_000)
    spec = S.trajectory_cameras(1, phase=phase, W=320, H=256, f=215.0)[0]
    _backward_case(pkg, params, spec, 0)
    _backward_case(pkg, params, spec, 1)


def test_dense_coarse_level_multi_chunk(pkg):
    """Level 2 of a 200k-Gaussian LiDAR map: tile lists of several thousand
    entries, composited list-parallel in chunks (forward and backward)."""
    params, phase = lidar(200_000)
    spec = S.trajectory_cameras(8, phase=phase)[0]  # the first keyframe of the 8-view workload
    lv = ctx_for(pkg)
    rgb, depth, alpha, slot = lv.render(dev_params(params), spec, 2)
    lv.release(slot)
    ref = O.render_view(params, ocam(spec), 2)
    lens = ref["ranges"][:, 1].astype(np.int64) - ref["ranges"][:, 0]
    assert lens.max() > 4 * 1024
    exc = ref["margin"] <= MARGIN
    e = compare_images((rgb, depth, alpha), ref, exc)
    print(f"  longest list {lens.max()}, excused {exc.mean():.4%}, max err rgb {e[0]:.2e} alpha {e[2]:.2e}")
    assert e[0] < IMG_TOL and e[2] < IMG_TOL
    assert e[1] < IMG_TOL * max(1.0, float(np.abs(ref["depth"]).max()))
    _backward_case(pkg, params, spec, 2)


def test_autograd_function(pkg):
    params, spec, _, _ = S.small_scene(n=300, sh_degree=1)
    lv = ctx_for(pkg)
    dp = {k: (v.clone().requires_grad_(True) if isinstance(v, torch.Tensor) else v)
          for k, v in dev_params(params).items()}
    rgb, depth, alpha = pkg.render(lv, dp, spec, 0)
    w = torch.linspace(0, 1, rgb.numel(), device="cuda").reshape(rgb.shape)
    loss = (rgb * w).sum() + 0.01 * depth.sum() + 0.5 * alpha.sum()
    loss.backward()
    ref = O.render_view(params, ocam(spec), 0)
    g2 = O.backward_render(ref["pre"], ref["vals"], ref["ranges"], spec.W, spec.H,
                           w.cpu().numpy().astype(np.float64), np.full((spec.H, spec.W), 0.01),
                           np.full((spec.H, spec.W), 0.5))
    rg = O.backward_preprocess(params, ocam(spec), ref["pre"], g2)
    excl = excused_tiles_gaussians(ref, (16, 16), spec.W, spec.H, ref["margin"] <= MARGIN)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_check(k, dp[k].grad.cpu().numpy(), rg[k], excl)


# ---------------------------------------------------------------------------
# a10: batched step == plain calls
# ---------------------------------------------------------------------------
def test_batched_matches_plain_and_oracle(pkg):
    params, phase = lidar(30_000)
    cams = S.trajectory_cameras(4, phase=phase, W=320, H=256, f=215.0)
    levels = [0, 1, 2, 0]
    tg = [S.target_images(c, 100 + i) for i, c in enumerate(cams)]
    lv_b = pkg.Context()
    lv_p = ctx_for(pkg)
    dp = dev_params(params)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gts = [t(x[0]) for x in tg]
    lis = [t(x[1]) for x in tg]
    outs = []
    for c, l in zip(cams, levels):
        W, H = c.W >> l, c.H >> l
        outs.append((torch.empty(3, H, W, device="cuda"), torch.empty(H, W, device="cuda"),
                     torch.empty(H, W, device="cuda")))
    for graph in (False, True, True):
        losses, grads = lv_b.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, graph=graph, outputs=outs)
        torch.cuda.synchronize()
        lv_b.sync_status()
    # plain: per view pyramid -> render -> loss -> backward (accumulate)
    pgrads = {k: torch.zeros_like(dp[k]) for k in pkg.PARAM_NAMES}
    for i, (c, l) in enumerate(zip(cams, levels)):
        g_l, d_l = gts[i], lis[i]
        for _ in range(l):
            g_l, d_l = lv_p.pyramid_down(g_l, d_l)
        rgb, depth, alpha, slot = lv_p.render(dp, c, l)
        assert torch.equal(rgb, outs[i][0]) and torch.equal(depth, outs[i][1]) and torch.equal(alpha, outs[i][2])
        terms, d_rgb, d_dep = lv_p.loss(rgb, depth, g_l, d_l, 0.2, 0.1)
        np.testing.assert_allclose(terms.cpu().numpy(), losses[i].cpu().numpy(), rtol=1e-12)
        lv_p.backward(slot, dp, d_rgb, d_dep, grads=pgrads, accumulate=True)
        lv_p.release(slot)
    for k in pkg.PARAM_NAMES:
        a, b = grads[k].cpu().numpy(), pgrads[k].cpu().numpy()
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-4 * scale + 1e-12, k
    # and the whole step against the oracle
    ocams = [ocam(c) for c in cams]
    out, rgrads = O.train_step(params, ocams, levels, [x[0] for x in tg], [x[1] for x in tg], 0.2, 0.1)
    for i in range(len(cams)):
        np.testing.assert_allclose(losses[i].cpu().numpy()[0], out[i]["terms"][0], rtol=2e-4)
    excl = set()
    for i, (c, l) in enumerate(zip(cams, levels)):
        r = out[i]["render"]
        # the loss window spreads a flipped pixel over 11x11 neighbours: dilate
        exc = r["margin"] <= MARGIN
        if exc.any():
            from scipy.ndimage import binary_dilation
            exc = binary_dilation(exc, iterations=5)
        excl.update(excused_tiles_gaussians(r, (16, 16), r["cam"].W, r["cam"].H, exc).tolist())
    excl = np.array(sorted(excl), dtype=np.int64)
    for k in pkg.PARAM_NAMES:
        grad_check(k, grads[k].cpu().numpy(), rgrads[k], excl, rtol=2e-3)


def test_autotune_then_batched_matches_plain(pkg):
    """The autotuner leaves a valid configuration; a batched step with it equals
    plain renders at the chosen tile size."""
    params, phase = lidar(30_000)
    cams = S.trajectory_cameras(3, phase=phase, W=320, H=256, f=215.0)
    levels = [0, 1, 2]
    tg = [S.target_images(c, 200 + i) for i, c in enumerate(cams)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dp = dev_params(params)
    gts, lis = [t(x[0]) for x in tg], [t(x[1]) for x in tg]
    lv = pkg.Context()
    tile, bd, times = lv.autotune(dp, cams, levels, gts, lis, 0.2, 0.1, trials=2)
    print(f"  autotune chose {tile}/{bd}: {times}")
    assert tile in [(16, 16), (8, 8), (32, 16)] and bd in (32, 64)
    assert all(v > 0 for v in times.values())
    outs = [(torch.empty(3, c.H >> l, c.W >> l, device="cuda"), torch.empty(c.H >> l, c.W >> l, device="cuda"),
             torch.empty(c.H >> l, c.W >> l, device="cuda")) for c, l in zip(cams, levels)]
    lv.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, outputs=outs)
    torch.cuda.synchronize()
    plain = pkg.Context(tile=tile, batch_depth=bd)
    for i, (c, l) in enumerate(zip(cams, levels)):
        rgb, depth, alpha, slot = plain.render(dp, c, l)
        plain.release(slot)
        assert torch.equal(rgb, outs[i][0]) and torch.equal(alpha, outs[i][2])


@pytest.mark.parametrize("workload", ["lidar_200000_1v", "pyramid_500000", "lidar_1000000_8v"])
def test_full_step_vs_oracle(pkg, workload):
    """Whole steps of the measured configurations against the oracle's full step:
    one 1280x1024 keyframe on 200k Gaussians; one keyframe at pyramid levels 0, 1
    and 2 on 500k; and the benchmarked step, 1M Gaussians (SH 3) and 8 keyframes
    at levels [2,2,2,2,1,0,2,1].  One graph-replayed batched call (16x16 tiles).
    Every pixel of every view, the four loss terms of every view and every
    parameter gradient, with the threshold excusals of the other chained-step
    tests (pixels within the 1e-4 margin, dilated by the SSIM half-window, and
    the Gaussians listed in their tiles), to which the loss's own branches are
    added: pixels whose L1 residual (colour, or depth where LiDAR returns) lies
    within the image tolerance of zero, and Gaussians whose SH colour lies
    within 1e-5 (relative to its terms) of the clamp at 0."""
    from scipy.ndimage import binary_dilation

    margin = MARGIN

    wl = S.workload(workload)
    params, cams, levels = wl["params"], wl["cams"], wl["levels"]
    lv = pkg.Context(tile=(16, 16))
    dp = dev_params(params)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gts, lis = [t(x) for x in wl["gts"]], [t(x) for x in wl["lidars"]]
    outs = [(torch.empty(3, c.H >> l, c.W >> l, device="cuda"), torch.empty(c.H >> l, c.W >> l, device="cuda"),
             torch.empty(c.H >> l, c.W >> l, device="cuda")) for c, l in zip(cams, levels)]
    for _ in range(3):  # eager sizing, capture, replay
        losses, grads = lv.train_step_batched(dp, cams, levels, gts, lis, wl["lam"], wl["lam_d"], outputs=outs)
    torch.cuda.synchronize()
    lv.sync_status()
    ocams = [ocam(c) for c in cams]
    out, rgrads = O.train_step(params, ocams, levels, wl["gts"], wl["lidars"], wl["lam"], wl["lam_d"])
    excl = set()
    for i, (c, l) in enumerate(zip(cams, levels)):
        r = out[i]["render"]
        exc = r["margin"] <= margin
        e = compare_images(outs[i], r, exc)
        print(f"  view {i} level {l}: excused {exc.mean():.4%}, max err rgb {e[0]:.2e} depth {e[1]:.2e} "
              f"alpha {e[2]:.2e}")
        assert exc.mean() < 0.02
        assert e[0] < IMG_TOL and e[2] < IMG_TOL
        assert e[1] < IMG_TOL * max(1.0, float(np.abs(r["depth"]).max()))
        np.testing.assert_allclose(losses[i].cpu().numpy(), out[i]["terms"], rtol=2e-4, atol=1e-7)
        # the gradients also take the loss's own branches: the sign of an L1
        # residual within the image tolerance of zero, and the SH colour's clamp
        # at 0 within binary32 rounding, may go either way
        gt_l, li_l = out[i]["gt"], out[i]["lidar"]
        kink = (np.abs(r["rgb"] - gt_l) <= IMG_TOL).any(axis=0)
        kink |= (li_l > 0) & (np.abs(r["depth"] - li_l) <= IMG_TOL * np.maximum(1.0, np.abs(r["depth"])))
        exc = exc | kink
        if exc.any():
            exc = binary_dilation(exc, iterations=5)
        excl.update(excused_tiles_gaussians(r, (16, 16), r["cam"].W, r["cam"].H, exc).tolist())
        excl.update(np.nonzero(r["pre"]["rgb_margin"] <= 1e-5)[0].tolist())
    excl = np.array(sorted(excl), dtype=np.int64)
    print(f"  Gaussians excused from the gradient bar: {len(excl)} of {params['means'].shape[0]}")
    for k in pkg.PARAM_NAMES:
        grad_check(k, grads[k].cpu().numpy(), rgrads[k], excl, rtol=2e-3)
    lv.close()
