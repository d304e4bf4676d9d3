"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(one or two isotropic Gaussians, constant images), invariants (weights plus
final transmittance sum to one), library routines (numpy sort / eigvalsh /
scipy's complex spherical harmonics and correlate), finite differences of the
projection and of the whole loss, and brute-force enumeration.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S


def cam_of(spec):
    return O.Camera(spec.R, spec.t, spec.fx, spec.fy, spec.cx, spec.cy, spec.W, spec.H)


def one_gaussian_params(means, log_s, logits, colours, quats=None):
    n = len(means)
    sh = np.zeros((n, 1, 3), np.float32)
    sh[:, 0, :] = (np.asarray(colours) - 0.5) * math.sqrt(4 * math.pi)  # Y_00 = 1/sqrt(4 pi)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else quats
    return dict(means=np.asarray(means, np.float32),
                log_scales=np.full((n, 3), 0, np.float32) + np.asarray(log_s, np.float32)[:, None],
                quats=np.asarray(q, np.float32), opacity_logits=np.asarray(logits, np.float32),
                sh=sh, sh_degree=0)


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


# --------------------------------------------------------------------------
# a5 closed forms (Eq. 3-6): one and two isotropic Gaussians on the optical axis
# --------------------------------------------------------------------------
@pytest.mark.parametrize("screen", ["f64", "key"])
def test_single_isotropic_gaussian_closed_form(screen):
    """With the binary64 projection the image is the closed form to rounding;
    with the key stage's (binary32 covariance, centre exact here) alpha moves by
    at most the covariance's binary32 rounding (a few 2^-24 relative) times
    the exponent, and a pixel that close to the 1/255 cut may go either way."""
    W, H, f = 64, 48, 50.0
    cam = O.Camera(np.eye(3), np.zeros(3), f, f, 32.0, 24.0, W, H)
    z, s, logit, col = 4.0, 0.2, 1.0, np.array([0.9, 0.5, 0.2])
    p = one_gaussian_params([[0, 0, z]], [math.log(s)], [logit], [col])
    r = O.render_view(p, cam, 0, screen=screen)
    s_eff = math.exp(float(np.float32(math.log(s))))  # the parameter is a binary32 log-scale
    sig2 = (f * s_eff / z) ** 2 + 0.3
    # radius from the eigenvalues of sig2*I (both equal; discriminant floored at 0.1)
    rad = math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    assert r["pre"]["radius"][0] == rad
    o = sigmoid(logit)
    yy, xx = np.mgrid[0:H, 0:W]
    power = -((xx - 32.0) ** 2 + (yy - 24.0) ** 2) / (2 * sig2)
    a = o * np.exp(power)
    a = np.minimum(a, 0.99)
    near_cut = np.abs(a * 255 - 1) < 1e-5
    a[a < 1 / 255] = 0
    # only the tiles of the covered rectangle are composited
    x0, x1 = int((32 - rad) / 16), int((32 + rad + 15) / 16)
    y0, y1 = int((24 - rad) / 16), int((24 + rad + 15) / 16)
    cover = np.zeros((H, W), bool)
    cover[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
    a[~cover] = 0
    if screen == "f64":
        tol, ok = 1e-12, np.ones((H, W), bool)
    else:
        tol, ok = 1e-6 * a * (np.abs(power) + 1) + 1e-15, ~near_cut
    assert ok.mean() > 0.95
    assert np.all(np.abs(r["alpha"] - a)[ok] <= tol if np.isscalar(tol) else np.abs(r["alpha"] - a)[ok] <= tol[ok])
    assert np.all(np.abs(r["depth"] - z * a)[ok] <= 10 * (tol if np.isscalar(tol) else tol[ok]))
    for ch in range(3):
        np.testing.assert_allclose(r["rgb"][ch][ok], (col[ch] * a)[ok],
                                   atol=1e-12 if screen == "f64" else 1e-6 * 6.5)
    np.testing.assert_allclose(r["final_T"][ok], (1 - a)[ok], atol=1e-12 if screen == "f64" else 1e-6 * 6.5)


def test_two_gaussians_closed_form():
    W, H, f = 32, 32, 40.0
    cam = O.Camera(np.eye(3), np.zeros(3), f, f, 16.0, 16.0, W, H)
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.8, 0.6])
    # the nearer Gaussian is listed second to check the depth ordering
    # both on the optical axis, where the projected covariance is isotropic
    p = one_gaussian_params([[0, 0, 6.0], [0, 0, 3.0]], [math.log(0.3), math.log(0.15)],
                            [0.5, -0.2], [c2, c1])
    r = O.render_view(p, cam, 0, tile=(32, 32))
    o1, o2 = sigmoid(-0.2), sigmoid(0.5)
    s1 = (f * math.exp(float(np.float32(math.log(0.15)))) / 3.0) ** 2 + 0.3
    s2 = (f * math.exp(float(np.float32(math.log(0.3)))) / 6.0) ** 2 + 0.3
    u2 = 16.0
    for (px, py) in [(16, 16), (18, 15), (20, 20), (13, 17)]:
        a1 = min(0.99, o1 * math.exp(-((px - 16) ** 2 + (py - 16) ** 2) / (2 * s1)))
        a2 = min(0.99, o2 * math.exp(-((px - u2) ** 2 + (py - 16) ** 2) / (2 * s2)))
        a1 = a1 if a1 >= 1 / 255 else 0.0
        a2 = a2 if a2 >= 1 / 255 else 0.0
        C = c1 * a1 + c2 * a2 * (1 - a1)
        D = 3.0 * a1 + 6.0 * a2 * (1 - a1)
        np.testing.assert_allclose(r["rgb"][:, py, px], C, atol=1e-6)
        np.testing.assert_allclose(r["depth"][py, px], D, atol=1e-5)
        np.testing.assert_allclose(r["alpha"][py, px], 1 - (1 - a1) * (1 - a2), atol=1e-6)


# --------------------------------------------------------------------------
# a5 invariants: sum_i alpha_i T_i + T_final = 1, T bounded by the stop rule
# --------------------------------------------------------------------------
def test_weights_plus_transmittance_is_one():
    params, spec, _, _ = S.small_scene()
    params = dict(params)
    sh = params["sh"].copy()
    sh[:, 0, :] = 0.5 * math.sqrt(4 * math.pi)  # every colour = 1
    params["sh"] = sh
    r = O.render_view(params, cam_of(spec), 0)
    for ch in range(3):
        np.testing.assert_allclose(r["rgb"][ch] + r["final_T"], 1.0, atol=1e-12)
    assert (r["final_T"] >= 1e-4).all() and (r["final_T"] <= 1).all()
    assert (r["alpha"] >= 0).all() and (r["alpha"] <= 1).all()
    assert r["n_contrib"].max() > 5


def test_early_stop_closed_form():
    # 20 identical on-axis Gaussians with opacity 1/2: alpha = 1/2 exactly at the centre pixel,
    # T after k of them is 2^-k; 2^-13 >= 1e-4 > 2^-14, so the 14th is excluded and the pixel stops.
    W = H = 16
    cam = O.Camera(np.eye(3), np.zeros(3), 20.0, 20.0, 8.0, 8.0, W, H)
    n = 20
    cols = np.random.default_rng(9).uniform(0.1, 0.9, (n, 3))
    p = one_gaussian_params([[0, 0, 2.0 + 0.25 * i] for i in range(n)], [math.log(0.05)] * n,
                            [0.0] * n, cols)
    r = O.render_view(p, cam, 0)
    w = 0.5 * 0.5 ** np.arange(13)
    assert r["n_contrib"][8, 8] == 13
    assert r["final_T"][8, 8] == pytest.approx(2.0 ** -13, rel=1e-14)
    # colours pass through a binary32 SH coefficient, hence the looser tolerance
    np.testing.assert_allclose(r["rgb"][:, 8, 8], (cols[:13] * w[:, None]).sum(0), rtol=1e-6)
    np.testing.assert_allclose(r["depth"][8, 8], ((2.0 + 0.25 * np.arange(13)) * w).sum(), rtol=1e-13)


# --------------------------------------------------------------------------
# a5: the other branch of close calls (flip), on closed forms
# --------------------------------------------------------------------------
def test_flip_takes_the_other_branch_closed_forms():
    """A test within ``close_margin`` of its threshold takes the other branch
    under ``flip``; the result is again the closed form, for that branch."""
    W = H = 16
    cam = O.Camera(np.eye(3), np.zeros(3), 20.0, 20.0, 8.0, 8.0, W, H)
    # (a) the stop: 20 on-axis Gaussians, alpha = 1/2 at the centre pixel; T after
    # 13 of them, 2^-13, is 22 % above 1e-4: with close_margin 0.3 that test is
    # close, so the flipped walk stops before the 13th (T = 2^-12)
    n = 20
    cols = np.random.default_rng(9).uniform(0.1, 0.9, (n, 3))
    zs = [2.0 + 0.25 * i for i in range(n)]
    p = one_gaussian_params([[0, 0, z] for z in zs], [math.log(0.05)] * n, [0.0] * n, cols)
    r0 = O.render_view(p, cam, 0, screen="f64", close_margin=0.3)
    r1 = O.render_view(p, cam, 0, screen="f64", close_margin=0.3, flip=True)
    assert r0["n_contrib"][8, 8] == 13 and r0["n_close"][8, 8] >= 1
    assert r1["n_contrib"][8, 8] == 12
    assert r1["final_T"][8, 8] == pytest.approx(2.0 ** -12, rel=1e-14)
    w = 0.5 * 0.5 ** np.arange(12)
    np.testing.assert_allclose(r1["rgb"][:, 8, 8], (cols[:12] * w[:, None]).sum(0), rtol=1e-6)
    np.testing.assert_allclose(r1["depth"][8, 8], (np.array(zs[:12]) * w).sum(), rtol=1e-13)
    # without flip, close_margin only counts
    r2 = O.render_view(p, cam, 0, screen="f64")
    for k in ("rgb", "depth", "alpha", "n_contrib"):
        assert np.array_equal(r0[k], r2[k])
    # ... and no close test, no flip
    r3 = O.render_view(p, cam, 0, screen="f64", flip=True)
    for k in ("rgb", "depth", "alpha", "n_contrib"):
        assert np.array_equal(r3[k], r2[k])
    # the backward over the flipped walk is the backward of the first 12 alone
    rng = np.random.default_rng(4)
    d_rgb = np.zeros((3, H, W)); d_rgb[:, 8, 8] = rng.normal(size=3)
    d_dep = np.zeros((H, W)); d_dep[8, 8] = 0.3
    d_alp = np.zeros((H, W)); d_alp[8, 8] = -0.7
    g_flip = O.backward_render(r1["pre"], r1["vals"], r1["ranges"], W, H, d_rgb, d_dep, d_alp,
                               close_margin=0.3, flip=True)
    p12 = {k: (v[:12] if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    r12 = O.render_view(p12, cam, 0, screen="f64")
    assert r12["n_contrib"][8, 8] == 12
    g12 = O.backward_render(r12["pre"], r12["vals"], r12["ranges"], W, H, d_rgb, d_dep, d_alp)
    np.testing.assert_allclose(g_flip[:12], g12, rtol=1e-12, atol=1e-15)
    assert np.all(g_flip[12:] == 0)

    # (b) the clamp: o = 0.995 at the centre of one Gaussian, 0.5 % above 0.99
    p = one_gaussian_params([[0, 0, 3.0]], [math.log(0.05)], [math.log(0.995 / 0.005)], [[0.3, 0.6, 0.9]])
    o = sigmoid(float(p["opacity_logits"][0]))
    r0 = O.render_view(p, cam, 0, screen="f64", close_margin=0.01)
    r1 = O.render_view(p, cam, 0, screen="f64", close_margin=0.01, flip=True)
    assert r0["alpha"][8, 8] == pytest.approx(0.99, rel=1e-14)
    assert r1["alpha"][8, 8] == pytest.approx(o, rel=1e-14)

    # (c) the 1/255 cut: a wide Gaussian (sigma ~ 6 px); every pixel whose only
    # close test is its cut shows the closed form alpha when taken, 0 when not
    W2 = H2 = 48
    cam2 = O.Camera(np.eye(3), np.zeros(3), 60.0, 60.0, 24.0, 24.0, W2, H2)
    z, sc, logit = 2.0, 0.2, -1.0
    p = one_gaussian_params([[0, 0, z]], [math.log(sc)], [logit], [[1.0, 1.0, 1.0]])
    o = sigmoid(float(p["opacity_logits"][0]))
    s_eff = math.exp(float(np.float32(math.log(sc))))
    sig2 = (60.0 * s_eff / z) ** 2 + 0.3
    yy, xx = np.mgrid[0:H2, 0:W2]
    a = o * np.exp(-((xx - 24.0) ** 2 + (yy - 24.0) ** 2) / (2 * sig2))
    r0 = O.render_view(p, cam2, 0, tile=(48, 48), screen="f64", close_margin=0.05)
    r1 = O.render_view(p, cam2, 0, tile=(48, 48), screen="f64", close_margin=0.05, flip=True)
    close = r0["n_close"] > 0
    assert close.sum() >= 8 and np.all(np.abs(a[close] * 255 - 1) <= 0.05)
    want = np.where(a >= 1 / 255, 0.0, a)  # the other branch of the cut
    np.testing.assert_allclose(r1["alpha"][close], want[close], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(r1["alpha"][~close], r0["alpha"][~close])


# --------------------------------------------------------------------------
# a1: EWA covariance against a finite-difference Jacobian of the projection
# --------------------------------------------------------------------------
def _quat_R(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_projection_covariance_matches_fd_jacobian():
    rng = np.random.default_rng(5)
    n = 40
    ang = rng.normal(size=3)
    Rw = _quat_R(np.array([1.0, *(0.1 * ang)]))
    t = np.array([0.2, -0.1, 0.5])
    cam = O.Camera(Rw.astype(np.float32), t.astype(np.float32), 300.0, 280.0, 160.0, 120.0, 320, 240)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(3, 8, n)], 1)
    params = dict(means=means.astype(np.float32),
                  log_scales=rng.normal(-2.5, 0.4, (n, 3)).astype(np.float32),
                  quats=rng.normal(size=(n, 4)).astype(np.float32),
                  opacity_logits=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32),
                  sh_degree=0)
    pre = O.preprocess(params, cam, screen="f64")
    # the key stage's screen-space Gaussian is the same projection in binary32
    prek = O.preprocess(params, cam, screen="key")
    Rd, td = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)

    def proj(p):
        return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

    for i in range(n):
        pc = Rd @ means[i].astype(np.float32).astype(np.float64) + td
        Jfd = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-6
            Jfd[:, k] = (proj(pc + e) - proj(pc - e)) / 2e-6
        Rq = _quat_R(params["quats"][i].astype(np.float64))
        s = np.exp(params["log_scales"][i].astype(np.float64))
        Sig = Rq @ np.diag(s * s) @ Rq.T
        cov = Jfd @ Rd @ Sig @ Rd.T @ Jfd.T + 0.3 * np.eye(2)
        inv = np.linalg.inv(cov)
        np.testing.assert_allclose(pre["conic"][i], [inv[0, 0], inv[0, 1], inv[1, 1]],
                                   rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(pre["uv"][i], proj(pc), rtol=1e-12)
        assert pre["depth"][i] == pytest.approx(pc[2], rel=1e-12)
        ref = np.array([inv[0, 0], inv[0, 1], inv[1, 1]])
        assert np.abs(prek["conic"][i] - ref).max() <= 1e-5 * np.abs(ref).max()
        np.testing.assert_allclose(prek["uv"][i], proj(pc), rtol=1e-6)
        assert prek["depth"][i] == pytest.approx(pc[2], rel=1e-6)
        assert prek["uv"][i, 0] == float(prek["uv_f"][i, 0]) and prek["depth"][i] == float(prek["z_f"][i])


def test_quaternion_sign_invariance_and_radius_eigen():
    params, spec, _, _ = S.small_scene(n=500)
    cam = cam_of(spec)
    pre = O.preprocess(params, cam)
    neg = dict(params); neg["quats"] = -params["quats"]
    pre2 = O.preprocess(neg, cam)
    np.testing.assert_array_equal(pre["rect"], pre2["rect"])
    np.testing.assert_array_equal(pre["radius"], pre2["radius"])
    np.testing.assert_allclose(pre["conic"], pre2["conic"], rtol=1e-12)
    vis = pre["tiles"] > 0
    checked = 0
    for i in np.nonzero(vis)[0]:
        A, B, C = pre["conic"][i]
        cov = np.linalg.inv(np.array([[A, B], [B, C]]))
        lam = np.linalg.eigvalsh(cov)
        mid = 0.5 * (lam[0] + lam[1])
        r_expect = 3 * math.sqrt(mid + math.sqrt(max(0.1, (0.5 * (lam[1] - lam[0])) ** 2)))
        if abs(r_expect - round(r_expect)) < 1e-3:
            continue  # too close to an integer for a binary32 / binary64 comparison
        assert pre["radius"][i] == math.ceil(r_expect)
        checked += 1
    assert checked > 100


def test_tile_rect_covers_three_sigma_ellipse():
    params, spec, _, _ = S.small_scene(n=400)
    cam = cam_of(spec)
    pre = O.preprocess(params, cam)
    T = 16
    for i in np.nonzero(pre["tiles"] > 0)[0]:
        A, B, C = pre["conic"][i]
        cov = np.linalg.inv(np.array([[A, B], [B, C]]))
        hx, hy = 3 * math.sqrt(cov[0, 0]), 3 * math.sqrt(cov[1, 1])  # ellipse bounding box
        u, v = pre["uv"][i]
        x0, y0, x1, y1 = pre["rect"][i]
        lo_x, hi_x = max(0.0, u - hx), min(cam.W - 1.0, u + hx)
        lo_y, hi_y = max(0.0, v - hy), min(cam.H - 1.0, v + hy)
        # the rectangle (x0 = trunc((u-r)/T), x1 = trunc((u+r+T-1)/T)) covers every pixel
        # column in [u - r, u + r - 1], and r >= 3 sigma along each axis
        if lo_x <= hi_x - 1 and lo_y <= hi_y - 1:
            assert x0 * T <= math.ceil(lo_x) and math.floor(hi_x - 1) <= x1 * T - 1
            assert y0 * T <= math.ceil(lo_y) and math.floor(hi_y - 1) <= y1 * T - 1


# --------------------------------------------------------------------------
# a2-a4: keys, sort order and ranges by brute-force enumeration + numpy sort
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_keys_sort_ranges_brute_force(tile):
    params, spec, _, _ = S.small_scene()
    cam = cam_of(spec)
    pre = O.preprocess(params, cam, tile)
    tx_n = pre["tiles_x"]
    keys, vals = [], []
    for i in range(pre["tiles"].shape[0]):
        x0, y0, x1, y1 = pre["rect"][i]
        if pre["tiles"][i] == 0:
            continue
        zb = int(pre["z_f"][i:i + 1].view(np.uint32)[0])
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                keys.append(((ty * tx_n + tx) << 32) | zb)
                vals.append(i)
    keys = np.array(keys, np.uint64)
    vals = np.array(vals, np.uint32)
    order = np.lexsort((vals, keys))
    ok, ov = O.build_keys(pre)
    np.testing.assert_array_equal(ok, keys[order])
    np.testing.assert_array_equal(ov, vals[order])
    n_tiles = tx_n * pre["tiles_y"]
    rg = O.tile_ranges(ok, n_tiles)
    tid = (ok >> np.uint64(32)).astype(np.int64)
    for t in range(n_tiles):
        idx = np.nonzero(tid == t)[0]
        if idx.size == 0:
            assert rg[t, 0] == rg[t, 1] == 0
        else:
            assert rg[t, 0] == idx[0] and rg[t, 1] == idx[-1] + 1
            assert (np.diff(idx) == 1).all()


def test_depth_key_is_float_order():
    # positive binary32 values order like their bit patterns (what the key relies on)
    z = np.sort(np.random.default_rng(0).uniform(0.2, 1000, 10000).astype(np.float32))
    assert (np.diff(z.view(np.uint32).astype(np.int64)) >= 0).all()


# --------------------------------------------------------------------------
# SH basis: orthonormal (quadrature), equal to scipy's complex SH made real
# --------------------------------------------------------------------------
def _sphere_quadrature(n_t=40, n_p=80):
    xg, wg = np.polynomial.legendre.leggauss(n_t)
    phi = (np.arange(n_p) + 0.5) * 2 * math.pi / n_p
    pts, wts = [], []
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for p in phi:
            pts.append((st * math.cos(p), st * math.sin(p), ct))
            wts.append(w * 2 * math.pi / n_p)
    return np.array(pts), np.array(wts)


def test_sh_orthonormal():
    pts, wts = _sphere_quadrature()
    Y = np.array([O.sh_basis(p)[0] for p in pts])
    G = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_scipy_real_form():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        theta = math.acos(d[2]); phi = math.atan2(d[1], d[0])
        Y = O.sh_basis(d)[0]
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(sp.sph_harm_y(l, abs(m), theta, phi))
                if m > 0:
                    ref = math.sqrt(2) * c.real
                elif m < 0:
                    ref = math.sqrt(2) * c.imag
                else:
                    ref = c.real
                assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-12)


def test_sh_gradient_fd():
    rng = np.random.default_rng(2)
    d = rng.normal(size=3)
    _, dY = O.sh_basis(d)
    for k in range(3):
        e = np.zeros(3); e[k] = 1e-6
        fd = (O.sh_basis(d + e)[0] - O.sh_basis(d - e)[0]) / 2e-6
        np.testing.assert_allclose(dY[:, k], fd, atol=1e-7)


# --------------------------------------------------------------------------
# a8: loss pins (Eq. 10-12)
# --------------------------------------------------------------------------
def _ssim_scipy(x, y):
    nd = pytest.importorskip("scipy.ndimage")
    g = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2)); g /= g.sum()
    w = np.outer(g, g)
    f = lambda a: nd.correlate(a, w, mode="constant", cval=0.0)
    out = []
    for ch in range(x.shape[0]):
        a, b = x[ch], y[ch]
        mx, my = f(a), f(b)
        sx, sy, sxy = f(a * a) - mx * mx, f(b * b) - my * my, f(a * b) - mx * my
        C1, C2 = 0.01 ** 2, 0.03 ** 2
        out.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2)))
    return np.array(out)


def test_ssim_matches_library_correlate():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (3, 23, 31)); y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    lidar = np.zeros((23, 31))
    terms, _, _ = O.loss(x, y, np.zeros((23, 31)), lidar, 1.0, 0.0, grads=False)
    assert terms[2] == pytest.approx(_ssim_scipy(x, y).mean(), abs=1e-13)


def test_ssim_identity_and_constant_closed_form():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (3, 20, 20))
    terms, d_img, _ = O.loss(x, x, np.zeros((20, 20)), np.zeros((20, 20)), 1.0, 0.0)
    assert terms[0] == pytest.approx(0.0, abs=1e-14)
    assert np.abs(d_img).max() < 1e-14
    # constant images a, b: interior pixels have SSIM (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.3, 0.7
    xs, ys = np.full((3, 30, 30), a), np.full((3, 30, 30), b)
    smap = _ssim_scipy(xs, ys)
    expect = (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)
    np.testing.assert_allclose(smap[:, 5:-5, 5:-5], expect, rtol=1e-12)


def test_l1_and_depth_terms_closed_form():
    x = np.zeros((3, 2, 2)); y = np.zeros((3, 2, 2)); y[0, 0, 0] = 0.6; y[2, 1, 1] = -0.3
    depth = np.array([[1.0, 2.0], [3.0, 4.0]]); lidar = np.array([[0.0, 2.5], [1.0, 0.0]])
    terms, d_img, d_depth = O.loss(x, y, depth, lidar, 0.0, 0.5)
    assert terms[1] == pytest.approx(0.9 / 12)
    assert terms[3] == pytest.approx((0.5 + 2.0) / 2)
    assert terms[0] == pytest.approx(0.9 / 12 + 0.5 * 1.25)
    assert d_img[0, 0, 0] == pytest.approx(-1 / 12) and d_img[2, 1, 1] == pytest.approx(1 / 12)
    assert d_img[1, 0, 0] == 0.0  # sign(0) = 0
    np.testing.assert_allclose(d_depth, [[0, -0.25], [0.25, 0]])
    # residuals within the kink margins take the other sign under flip; the
    # values do not change
    x2 = x.copy(); x2[0, 0, 0] = 0.6 + 1e-5
    d2 = depth.copy(); d2[0, 1] = 2.5 - 2e-4
    t_a, g_a, gd_a = O.loss(x2, y, d2, lidar, 0.0, 0.5)
    t_b, g_b, gd_b = O.loss(x2, y, d2, lidar, 0.0, 0.5, kink_margin=1e-4, depth_kink_margin=1e-3, flip=True)
    np.testing.assert_array_equal(t_a, t_b)
    assert g_a[0, 0, 0] == pytest.approx(1 / 12) and g_b[0, 0, 0] == pytest.approx(-1 / 12)
    assert gd_a[0, 1] == pytest.approx(-0.25) and gd_b[0, 1] == pytest.approx(0.25)
    g_b[0, 0, 0] = g_a[0, 0, 0]; gd_b[0, 1] = gd_a[0, 1]
    np.testing.assert_array_equal(g_a, g_b); np.testing.assert_array_equal(gd_a, gd_b)


def test_loss_gradient_fd():
    rng = np.random.default_rng(6)
    H, W = 14, 17
    x = rng.uniform(0, 1, (3, H, W)); y = rng.uniform(0, 1, (3, H, W))
    depth = rng.uniform(2, 6, (H, W)); lidar = np.where(rng.uniform(size=(H, W)) < 0.3, rng.uniform(2, 6, (H, W)), 0)
    _, d_img, d_depth = O.loss(x, y, depth, lidar, 0.2, 0.1)
    eps = 1e-6
    for (ch, i, j) in [(0, 0, 0), (1, 5, 7), (2, 13, 16), (0, 7, 3), (2, 2, 11)]:
        xp, xm = x.copy(), x.copy(); xp[ch, i, j] += eps; xm[ch, i, j] -= eps
        fd = (O.loss(xp, y, depth, lidar, 0.2, 0.1, False)[0][0] - O.loss(xm, y, depth, lidar, 0.2, 0.1, False)[0][0]) / (2 * eps)
        assert d_img[ch, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-11)
    for (i, j) in zip(*np.nonzero(lidar)):
        dp, dm = depth.copy(), depth.copy(); dp[i, j] += eps; dm[i, j] -= eps
        fd = (O.loss(x, y, dp, lidar, 0.2, 0.1, False)[0][0] - O.loss(x, y, dm, lidar, 0.2, 0.1, False)[0][0]) / (2 * eps)
        assert d_depth[i, j] == pytest.approx(fd, rel=1e-6)
        break


# --------------------------------------------------------------------------
# a9: pyramid
# --------------------------------------------------------------------------
def test_pyramid_box_and_valid_mean():
    rng = np.random.default_rng(7)
    rgb = rng.uniform(size=(3, 8, 12))
    depth = np.where(rng.uniform(size=(8, 12)) < 0.4, rng.uniform(1, 9, (8, 12)), 0.0)
    r1, d1 = O.pyramid_down(rgb, depth)
    np.testing.assert_allclose(r1, rgb.reshape(3, 4, 2, 6, 2).mean((2, 4)), rtol=1e-15)
    blk = depth.reshape(4, 2, 6, 2).transpose(0, 2, 1, 3).reshape(4, 6, 4)
    cnt = (blk > 0).sum(-1)
    expect = np.where(cnt > 0, blk.sum(-1) / np.maximum(cnt, 1), 0.0)
    np.testing.assert_allclose(d1, expect, rtol=1e-15)
    rc, dc = O.pyramid(np.full((3, 16, 16), 0.37), np.full((16, 16), 5.0), 2)
    np.testing.assert_allclose(rc, 0.37, rtol=1e-15); np.testing.assert_allclose(dc, 5.0)


def test_level_camera_aligns_block_centres():
    spec = S.identity_camera(1280, 1024, 860.0)
    cam0 = cam_of(spec)
    params, _, _, _ = S.small_scene(n=50)
    pre0 = O.preprocess(params, cam0)
    for lvl in (1, 2):
        cam = O.level_camera(cam0, lvl)
        assert (cam.W, cam.H) == (1280 >> lvl, 1024 >> lvl)
        pre = O.preprocess(params, cam)
        k = 2 ** lvl
        # a level-l pixel p covers level-0 pixels k p .. k p + k - 1 (centre k p + (k-1)/2)
        np.testing.assert_allclose(pre["uv"], (pre0["uv"] - (k - 1) / 2) / k, rtol=1e-6, atol=1e-5)


# --------------------------------------------------------------------------
# a6 + a7: hand-derived gradients against central finite differences
# --------------------------------------------------------------------------
def _fd_scene():
    rng = np.random.default_rng(11)
    n = 64
    means = np.stack([rng.uniform(-0.9, 0.9, n), rng.uniform(-0.9, 0.9, n), rng.uniform(3, 6, n)], 1)
    K = 16
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = (rng.uniform(0.25, 0.75, (n, 3)) - 0.5) * math.sqrt(4 * math.pi)
    sh[:, 1:, :] = rng.normal(0, 0.1, (n, K - 1, 3))
    params = dict(means=means.astype(np.float32),
                  log_scales=rng.normal(-2.2, 0.3, (n, 3)).astype(np.float32),
                  quats=S.random_quats(rng, n), opacity_logits=rng.normal(0, 1, n).astype(np.float32),
                  sh=sh, sh_degree=3)
    R = _quat_R(np.array([1.0, 0.05, -0.03, 0.02])).astype(np.float32)
    cam = O.Camera(R, np.array([0.05, -0.02, 0.1], np.float32), 40.0, 40.0, 16.0, 16.0, 32, 32)
    gt = rng.uniform(0, 1, (3, 32, 32))
    lidar = np.where(rng.uniform(size=(32, 32)) < 0.2, rng.uniform(3, 6, (32, 32)), 0.0)
    return params, cam, gt, lidar


def _vis_weights(cam):
    """Seeded weights of a visibility term sum_p w_p V_p (Eq. 5), of the size
    of the loss's per-pixel image gradients, so that the dL/dV path of the
    backward carries a share of every gradient comparable to colour and depth."""
    return np.random.default_rng(13).normal(0, 3e-4, (cam.H, cam.W))


def _loss_of(params, cam, gt, lidar, wv):
    r = O.render_view(params, cam, 0, screen="f64")
    terms, _, _ = O.loss(r["rgb"], gt, r["depth"], lidar, 0.2, 0.1, grads=False)
    return terms[0] + float((wv * r["alpha"]).sum()), r


def _analytic_grads(params, cam, gt, lidar, wv):
    """render -> loss + sum w V -> backward, all binary64 (smooth projection)."""
    r = O.render_view(params, cam, 0, screen="f64")
    _, d_img, d_dep = O.loss(r["rgb"], gt, r["depth"], lidar, 0.2, 0.1)
    g2 = O.backward_render(r["pre"], r["vals"], r["ranges"], cam.W, cam.H, d_img, d_dep, wv)
    return O.backward_preprocess(params, cam, r["pre"], g2), r


def test_backward_matches_central_fd():
    """Central differences (eps 1e-4, binary64) of L + sum_p w_p V_p through the
    whole render -> loss pipeline against the hand-derived backward, on every
    parameter of the visible Gaussians (SH rows on 8 of them).  The V term
    pins the visibility gradient dV/dalpha_i = T_i - (sum of the weights behind
    i) / (1 - alpha_i) of Eq. (5); without it the check would not see a
    mistake there."""
    params, cam, gt, lidar = _fd_scene()
    wv = _vis_weights(cam)
    grads, base = _analytic_grads(params, cam, gt, lidar, wv)
    grads_nov, _ = _analytic_grads(params, cam, gt, lidar, np.zeros_like(wv))
    # the visibility term moves every parameter's gradient materially
    for name in ("means", "log_scales", "quats", "opacity_logits"):
        d = np.linalg.norm(grads[name] - grads_nov[name]) / np.linalg.norm(grads[name])
        assert d > 0.05, (name, d)
    assert (base["pre"]["tiles"] > 0).sum() > 40
    eps = 1e-4
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    rng = np.random.default_rng(12)
    visible = np.nonzero(base["pre"]["tiles"] > 0)[0]
    sh_gids = rng.choice(visible, 8, replace=False)
    n_checked = n_skipped = 0
    worst = 0.0
    for name in names:
        g_all = grads[name]
        scale = np.abs(g_all).max()
        for gi in (sh_gids if name == "sh" else visible):
            flat_idx = range(int(np.prod(params[name].shape[1:])))
            for k in flat_idx:
                pp, pm = {k2: (v.copy() if isinstance(v, np.ndarray) else v) for k2, v in params.items()}, \
                         {k2: (v.copy() if isinstance(v, np.ndarray) else v) for k2, v in params.items()}
                ap = pp[name].reshape(params[name].shape[0], -1)
                am = pm[name].reshape(params[name].shape[0], -1)
                ap[gi, k] += np.float32(eps)
                am[gi, k] -= np.float32(eps)
                h = float(ap[gi, k]) - float(am[gi, k])
                lp, rp = _loss_of(pp, cam, gt, lidar, wv)
                lm, rm = _loss_of(pm, cam, gt, lidar, wv)
                # same tile lists in the same order (the depth bits of the keys may move)
                same = (np.array_equal(rp["keys"] >> np.uint64(32), rm["keys"] >> np.uint64(32))
                        and np.array_equal(rp["vals"], rm["vals"])
                        and np.array_equal(rp["signature"], rm["signature"])
                        and np.array_equal(rp["signature"], base["signature"])
                        # nor may an L1 term change sign (its kink)
                        and np.array_equal(np.sign(rp["rgb"] - gt), np.sign(rm["rgb"] - gt))
                        and np.array_equal(np.sign(rp["depth"] - lidar), np.sign(rm["depth"] - lidar)))
                if not same:
                    n_skipped += 1
                    continue
                fd = (lp - lm) / h
                an = g_all.reshape(params[name].shape[0], -1)[gi, k]
                err = abs(fd - an) / (abs(an) + 1e-3 * scale + 1e-12)
                worst = max(worst, err)
                assert err < 2e-5, (name, gi, k, fd, an)
                n_checked += 1
    print(f"  checked {n_checked}, skipped {n_skipped}, worst {worst:.2e}")
    # a perturbation that flips any threshold test anywhere in the image is skipped
    assert n_checked > 900 and n_skipped < 0.1 * (n_checked + n_skipped)


def test_exp_key_is_binary64_exp_rounded_once():
    """The key stage's scale: numpy's binary64 exp rounded to binary32 is an
    independent evaluation of the same definition."""
    rng = np.random.default_rng(21)
    x = np.concatenate([rng.uniform(-12, 8, 1_000_000), rng.normal(-3, 0.5, 200_000),
                        [0.0, -0.0, 1e-30, -1e-30, 59.9, -59.9, 88.0, -100.0]]).astype(np.float32)
    ref = np.exp(x.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(O.exp_key(x), ref)


def test_render_margin_allowance_covers_binary32_evaluation():
    """The render margin's binary32 allowance: (1) the conic of the binary32
    covariance is the float64 conic up to binary32 rounding (amplified where
    the projection cancels a 3D covariance elongated along the ray); (2) with
    the binary64 projection the deviation of the binary32 inputs is charged
    too, which only lowers margins; (3) an independent binary32 evaluation of
    every examined alpha (numpy float32: the key stage's centre, that conic
    rounded to binary32, float32 exp) takes the 1/255 and 0.99 decisions the
    other way only at pixels whose margin is at most 0."""
    params, phase = S.lidar_scene(300_000)
    cam = O.level_camera(cam_of(S.trajectory_cameras(1, phase=phase)[0]), 1)
    pre = O.preprocess(params, cam)
    pre64 = O.preprocess(params, cam, screen="f64")
    vis = pre["radius"] > 0
    cf, c64 = pre["conic_f"][vis], pre64["conic"][vis]
    dev = np.abs(cf - c64).max(axis=1) / np.abs(c64).max(axis=1)
    assert np.median(dev) < 1e-6 and dev.max() < 1e-4
    # the values composited are the key stage's
    assert np.array_equal(pre["conic"], pre["conic_f"]) and np.array_equal(pre["uv"], pre["uv_f"].astype(np.float64))

    keys, vals = O.build_keys(pre)
    ranges = O.tile_ranges(keys, pre["tiles_x"] * pre["tiles_y"])
    sel = np.random.default_rng(5).choice(ranges.shape[0], 160, replace=False).astype(np.int32)
    img = O.render(pre, vals, ranges, cam.W, cam.H, sel_tiles=sel)
    plain = dict(pre)
    del plain["conic_f"]
    img0 = O.render(plain, vals, ranges, cam.W, cam.H, sel_tiles=sel)
    # in the key stage's values the binary32 inputs deviate by nothing
    assert np.array_equal(img["margin"], img0["margin"])
    assert np.array_equal(img["rgb"], img0["rgb"]) and np.array_equal(img["n_contrib"], img0["n_contrib"])
    img64 = O.render(pre64, vals, ranges, cam.W, cam.H, sel_tiles=sel)
    plain64 = dict(pre64)
    del plain64["conic_f"]
    img64p = O.render(plain64, vals, ranges, cam.W, cam.H, sel_tiles=sel)
    fin = np.isfinite(img64p["margin"])
    assert np.all(img64["margin"] <= img64p["margin"]) and (img64["margin"] < img64p["margin"])[fin].mean() > 0.5

    f = np.float32
    uvf = pre["uv_f"]
    cf32 = pre["conic_f"].astype(f)
    op32 = pre["opacity"].astype(f)
    flips = plain_beyond = 0
    tx_n = pre["tiles_x"]
    for t in sel:
        s, e = (int(x) for x in ranges[t])
        if e <= s:
            continue
        g = vals[s:e]
        ty, tx = divmod(t, tx_n)
        ys, xs = np.mgrid[ty * 16:min(ty * 16 + 16, cam.H), tx * 16:min(tx * 16 + 16, cam.W)]
        ys, xs = ys.ravel(), xs.ravel()
        dx64 = pre["uv"][g, 0][None] - xs[:, None]
        dy64 = pre["uv"][g, 1][None] - ys[:, None]
        A, B, C = (pre["conic"][g, k][None] for k in range(3))
        p64 = -0.5 * (A * dx64 * dx64 + C * dy64 * dy64) - B * dx64 * dy64
        a64 = pre["opacity"][g][None] * np.exp(p64)
        dx = uvf[g, 0][None] - xs[:, None].astype(f)
        dy = uvf[g, 1][None] - ys[:, None].astype(f)
        A32, B32, C32 = (cf32[g, k][None] for k in range(3))
        p32 = f(-0.5) * (A32 * dx * dx + C32 * dy * dy) - B32 * dx * dy
        a32 = op32[g][None] * np.exp(p32)
        examined = np.arange(e - s)[None] < img["n_contrib"][ys, xs][:, None]
        flip = examined & (p64 <= 0) & (((a64 >= 1 / 255) != (a32 >= f(1 / 255))) | ((a64 >= 0.99) != (a32 >= f(0.99))))
        rows = np.nonzero(flip.any(axis=1))[0]
        flips += rows.size
        plain_beyond += int((img0["margin"][ys[rows], xs[rows]] > 0.0).sum())
        assert np.all(img["margin"][ys[rows], xs[rows]] <= 0.0)
    print(f"  binary32 decision flips at {flips} pixels, all within the allowance "
          f"({plain_beyond} beyond the plain margin)")
    assert flips > 0


def test_colour_clamp_margin_closed_form():
    """The SH colour's clamp margin: |0.5 + sum sh Y| over 0.5 + sum |sh Y|,
    the smallest over channels.  Degree 0 (Y_00 = 1/(2 sqrt(pi))): a colour c in
    [0, 1] has raw = c, terms 0.5 + |c - 0.5|."""
    W, H, f = 32, 32, 40.0
    cam = O.Camera(np.eye(3), np.zeros(3), f, f, 16.0, 16.0, W, H)
    cols = [[0.0, 0.5, 1.0], [0.25, 0.9, 0.6]]
    p = one_gaussian_params([[0, 0, 4.0], [0.5, 0, 5.0]], [math.log(0.2)] * 2, [1.0, 1.0], cols)
    pre = O.preprocess(p, cam)
    for i in range(len(cols)):
        c = p["sh"][i, 0, :].astype(np.float64)  # the binary32 band-0 coefficients
        raw = 0.5 + c / math.sqrt(4 * math.pi)
        want = (np.abs(raw) / (0.5 + np.abs(c / math.sqrt(4 * math.pi)))).min()
        assert abs(pre["rgb_margin"][i] - want) <= 1e-12
    assert pre["rgb_margin"][0] < 1e-7  # a black channel sits on the clamp
    # a culled Gaussian has no clamp
    p2 = one_gaussian_params([[0, 0, -4.0]], [math.log(0.2)], [1.0], [[0.5, 0.5, 0.5]])
    assert np.isinf(O.preprocess(p2, cam)["rgb_margin"][0])
