"""Planted mistakes in the oracle must fail its pins.

Each case copies ``oracle/`` to a temporary directory, replaces one statement
of ``lvigs_oracle.c`` with a plausible mistake (a wrong constant, a dropped
term or factor, a flipped sign, an off-by-one in the stop rule, a reversed tie
order), builds that copy, and runs the checks below against it; at least one
must fail, and all of them must pass on the unmodified oracle.  The checks
restate the pins of ``tests/test_oracle_pins.py`` in small form (closed forms,
invariants, library routines, brute force, central differences), so this shows
that the pins see a mistake anywhere in the oracle, not only that the oracle
passes them.
"""
import importlib.util
import math
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle")


def load_oracle(tmp_path, name, replace=None):
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(SRC, "__init__.py"), d / "__init__.py")
    src = open(os.path.join(SRC, "lvigs_oracle.c")).read()
    if replace is not None:
        old, new = replace
        assert src.count(old) == 1, f"mutation target not unique: {old!r}"
        src = src.replace(old, new)
    (d / "lvigs_oracle.c").write_text(src)
    name = f"{name}_{abs(hash(str(d)))}"
    spec = importlib.util.spec_from_file_location(name, d / "__init__.py", submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod  # the module's dataclasses look themselves up there
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def gaussians(means, log_s, logits, colours, quats=None, extra_sh=None):
    n = len(means)
    K = 1 if extra_sh is None else extra_sh.shape[1] + 1
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = (np.asarray(colours) - 0.5) * math.sqrt(4 * math.pi)
    if extra_sh is not None:
        sh[:, 1:, :] = extra_sh
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else quats
    ls = np.asarray(log_s, np.float32)
    ls = np.repeat(ls[:, None], 3, 1) if ls.ndim == 1 else ls
    return dict(means=np.asarray(means, np.float32), log_scales=ls.astype(np.float32),
                quats=np.asarray(q, np.float32), opacity_logits=np.asarray(logits, np.float32), sh=sh,
                sh_degree=int(round(math.sqrt(K))) - 1)


# --------------------------------------------------------------------------
# checks (each raises on a mismatch)
# --------------------------------------------------------------------------
def check_closed_forms(O):
    # one wide isotropic Gaussian: alpha = min(0.99, o exp(-r^2 / 2 s^2)) where >= 1/255
    W, H, f = 48, 48, 60.0
    cam = O.Camera(np.eye(3), np.zeros(3), f, f, 24.0, 24.0, W, H)
    z, s, logit = 2.0, 0.2, -1.0
    p = gaussians([[0, 0, z]], [math.log(s)], [logit], [[1.0, 1.0, 1.0]])
    r = O.render_view(p, cam, 0, tile=(48, 48), screen="f64")
    s_eff = math.exp(float(np.float32(math.log(s))))
    sig2 = (f * s_eff / z) ** 2 + 0.3
    assert r["pre"]["radius"][0] == math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    yy, xx = np.mgrid[0:H, 0:W]
    a = min(1.0, sigmoid(logit)) * np.exp(-((xx - 24.0) ** 2 + (yy - 24.0) ** 2) / (2 * sig2))
    a = np.minimum(a, 0.99)
    a[a < 1 / 255] = 0
    np.testing.assert_allclose(r["alpha"], a, atol=1e-12)
    np.testing.assert_allclose(r["depth"], z * a, atol=1e-11)
    # the key stage's projection: the same image to its binary32 covariance rounding
    rk = O.render_view(p, cam, 0, tile=(48, 48))
    power = -((xx - 24.0) ** 2 + (yy - 24.0) ** 2) / (2 * sig2)
    ok = np.abs(min(1.0, sigmoid(logit)) * np.exp(power) * 255 - 1) > 1e-5
    assert np.all(np.abs(rk["alpha"] - a)[ok] <= (1e-6 * a * (np.abs(power) + 1) + 1e-15)[ok])
    # the 1/255 cut: an opacity that puts the pixel at offset (6, 8) between 1/256 and 1/255
    lo = np.float32(math.log((1 / 255.5) * math.exp(100 / (2 * sig2)) / (1 - (1 / 255.5) * math.exp(100 / (2 * sig2)))))
    a68 = sigmoid(float(lo)) * math.exp(-100 / (2 * sig2))
    assert 1 / 256 < a68 < 1 / 255
    p2 = gaussians([[0, 0, z]], [math.log(s)], [float(lo)], [[1.0, 1.0, 1.0]])
    r2 = O.render_view(p2, cam, 0, tile=(48, 48), screen="f64")
    assert r2["alpha"][24 + 8, 24 + 6] == 0.0 and r2["alpha"][24, 24] > 0
    # the clamp: o = 0.995 at the centre gives alpha 0.99
    p = gaussians([[0, 0, 3.0]], [math.log(0.05)], [math.log(0.995 / 0.005)], [[0.3, 0.6, 0.9]])
    cam2 = O.Camera(np.eye(3), np.zeros(3), 20.0, 20.0, 8.0, 8.0, 16, 16)
    r = O.render_view(p, cam2, 0, screen="f64")
    assert abs(r["alpha"][8, 8] - 0.99) < 1e-14
    # the stop: 20 stacked alpha = 1/2 Gaussians; 2^-13 >= 1e-4 > 2^-14 so 13 contribute
    n = 20
    cols = np.random.default_rng(9).uniform(0.1, 0.9, (n, 3))
    p = gaussians([[0, 0, 2.0 + 0.25 * i] for i in range(n)], [math.log(0.05)] * n, [0.0] * n, cols)
    r = O.render_view(p, cam2, 0, screen="f64")
    assert r["n_contrib"][8, 8] == 13
    assert abs(r["final_T"][8, 8] - 2.0 ** -13) < 1e-18
    w = 0.5 * 0.5 ** np.arange(13)
    np.testing.assert_allclose(r["rgb"][:, 8, 8], (cols[:13] * w[:, None]).sum(0), rtol=1e-6)


def check_weights_sum_to_one(O):
    rng = np.random.default_rng(3)
    n = 300
    means = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(3, 8, n)], 1)
    p = gaussians(means, rng.normal(-2.5, 0.4, n), rng.normal(0, 1, n), np.ones((n, 3)))
    cam = O.Camera(np.eye(3), np.zeros(3), 40.0, 40.0, 20.0, 16.0, 40, 32)
    r = O.render_view(p, cam, 0)
    for ch in range(3):
        np.testing.assert_allclose(r["rgb"][ch] + r["final_T"], 1.0, atol=1e-12)
    assert r["n_contrib"].max() > 3


def check_keys_brute_force(O):
    rng = np.random.default_rng(4)
    n = 200
    means = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(3, 8, n)], 1)
    means[100:150] = means[50:100]  # duplicates: equal keys, ordered by index
    p = gaussians(means, rng.normal(-2.5, 0.4, n), rng.normal(0, 1, n), rng.uniform(0, 1, (n, 3)))
    cam = O.Camera(np.eye(3), np.zeros(3), 40.0, 40.0, 20.0, 16.0, 40, 32)
    pre = O.preprocess(p, cam, (8, 8))
    keys, vals = O.build_keys(pre)
    kk, vv = [], []
    tx_n = pre["tiles_x"]
    for i in range(n):
        x0, y0, x1, y1 = pre["rect"][i]
        zb = int(np.float32(pre["z_f"][i]).view(np.uint32))
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                kk.append(((ty * tx_n + tx) << 32) | zb)
                vv.append(i)
    order = np.lexsort((np.array(vv), np.array(kk, dtype=np.uint64)))
    np.testing.assert_array_equal(keys, np.array(kk, dtype=np.uint64)[order])
    np.testing.assert_array_equal(vals, np.array(vv, dtype=np.uint32)[order])


def ssim_reference(x, y):
    from scipy.ndimage import correlate

    g = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2))
    g /= g.sum()
    w2 = np.outer(g, g)
    f = lambda a: correlate(a, w2, mode="constant", cval=0.0)
    mx, my = f(x), f(y)
    sx, sy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2))


def check_loss(O):
    rng = np.random.default_rng(6)
    H, W = 14, 17
    x = rng.uniform(0, 1, (3, H, W))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)
    depth = rng.uniform(2, 9, (H, W))
    lidar = np.where(rng.uniform(size=(H, W)) < 0.3, rng.uniform(2, 9, (H, W)), 0.0)
    terms, d_img, d_depth = O.loss(x, y, depth, lidar, 0.2, 0.1)
    ssim = np.mean([ssim_reference(x[c], y[c]).mean() for c in range(3)])
    l1 = np.abs(x - y).mean()
    ld = np.abs(depth - lidar)[lidar > 0].mean()
    np.testing.assert_allclose(terms, [0.8 * l1 + 0.2 * (1 - ssim) + 0.1 * ld, l1, ssim, ld], rtol=1e-12)
    eps = 1e-6
    for (c, i, j) in [(0, 3, 4), (1, 7, 9), (2, 12, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += eps
        xm[c, i, j] -= eps
        fd = (O.loss(xp, y, depth, lidar, 0.2, 0.1, False)[0][0] - O.loss(xm, y, depth, lidar, 0.2, 0.1, False)[0][0]) / (2 * eps)
        assert abs(fd - d_img[c, i, j]) <= 1e-6 * abs(d_img[c, i, j]) + 1e-12
    i, j = np.argwhere(lidar > 0)[0]
    dp, dm = depth.copy(), depth.copy()
    dp[i, j] += eps
    dm[i, j] -= eps
    fd = (O.loss(x, y, dp, lidar, 0.2, 0.1, False)[0][0] - O.loss(x, y, dm, lidar, 0.2, 0.1, False)[0][0]) / (2 * eps)
    assert abs(fd - d_depth[i, j]) <= 1e-6 * abs(d_depth[i, j]) + 1e-12


def check_pyramid_and_levels(O):
    rng = np.random.default_rng(7)
    rgb = rng.uniform(size=(3, 8, 10))
    dep = np.where(rng.uniform(size=(8, 10)) < 0.5, rng.uniform(1, 5, (8, 10)), 0.0)
    r1, d1 = O.pyramid_down(rgb, dep)
    np.testing.assert_allclose(r1, rgb.reshape(3, 4, 2, 5, 2).mean(axis=(2, 4)), rtol=1e-15)
    blocks = dep.reshape(4, 2, 5, 2).transpose(0, 2, 1, 3).reshape(4, 5, 4)
    cnt = (blocks > 0).sum(-1)
    np.testing.assert_allclose(d1, np.where(cnt > 0, blocks.sum(-1) / np.maximum(cnt, 1), 0.0), rtol=1e-15)
    cam0 = O.Camera(np.eye(3), np.zeros(3), 860.0, 860.0, 640.0, 512.0, 1280, 1024)
    p = gaussians([[0.3, -0.2, 5.0], [-1.0, 0.5, 7.0]], [math.log(0.05)] * 2, [0.0] * 2, [[0.5] * 3] * 2)
    u0 = O.preprocess(p, cam0, screen="f64")["uv"]
    for lvl in (1, 2):
        k = 2 ** lvl
        u = O.preprocess(p, O.level_camera(cam0, lvl), screen="f64")["uv"]
        np.testing.assert_allclose(u, (u0 - (k - 1) / 2) / k, rtol=1e-6, atol=1e-5)


def check_sh(O):
    from scipy.special import sph_harm_y

    rng = np.random.default_rng(8)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = O.sh_basis(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(sph_harm_y(l, abs(m), theta, phi))
                ref = c.real if m == 0 else (math.sqrt(2) * (c.real if m > 0 else c.imag))
                assert abs(Y[l * l + l + m] - ref) < 1e-12, (l, m)


def _fd_case():
    rng = np.random.default_rng(11)
    n = 24
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), rng.uniform(3, 5, n)], 1)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    p = gaussians(means, rng.normal(-2.0, 0.3, (n, 3)), rng.normal(0, 1, n), rng.uniform(0.25, 0.75, (n, 3)),
                  quats=q, extra_sh=rng.normal(0, 0.1, (n, 3, 3)).astype(np.float32))
    gt = rng.uniform(0, 1, (3, 24, 24))
    lidar = np.where(rng.uniform(size=(24, 24)) < 0.3, rng.uniform(3, 5, (24, 24)), 0.0)
    wv = rng.normal(0, 3e-4, (24, 24))
    return p, gt, lidar, wv


def check_gradients_fd(O):
    p, gt, lidar, wv = _fd_case()
    th = 0.03
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]], np.float32)
    cam = O.Camera(R, np.array([0.05, -0.02, 0.1], np.float32), 30.0, 30.0, 12.0, 12.0, 24, 24)

    def total(pp):
        r = O.render_view(pp, cam, 0, screen="f64")
        t, _, _ = O.loss(r["rgb"], gt, r["depth"], lidar, 0.2, 0.1, False)
        return t[0] + float((wv * r["alpha"]).sum()), r

    r = O.render_view(p, cam, 0, screen="f64")
    _, d_img, d_dep = O.loss(r["rgb"], gt, r["depth"], lidar, 0.2, 0.1)
    g2 = O.backward_render(r["pre"], r["vals"], r["ranges"], 24, 24, d_img, d_dep, wv)
    g = O.backward_preprocess(p, cam, r["pre"], g2)
    vis = np.nonzero(r["pre"]["tiles"] > 0)[0][:8]
    eps = 1e-4
    checked = 0
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        flat = p[name].reshape(p[name].shape[0], -1)
        scale = np.abs(g[name]).max()
        for gi in vis:
            for k in range(flat.shape[1]):
                pp = {a: (b.copy() if isinstance(b, np.ndarray) else b) for a, b in p.items()}
                pm = {a: (b.copy() if isinstance(b, np.ndarray) else b) for a, b in p.items()}
                pp[name].reshape(flat.shape)[gi, k] += np.float32(eps)
                pm[name].reshape(flat.shape)[gi, k] -= np.float32(eps)
                h = float(pp[name].reshape(flat.shape)[gi, k]) - float(pm[name].reshape(flat.shape)[gi, k])
                lp, rp = total(pp)
                lm, rm = total(pm)
                if not (np.array_equal(rp["signature"], r["signature"]) and np.array_equal(rm["signature"], r["signature"])
                        and np.array_equal(rp["vals"], r["vals"]) and np.array_equal(rm["vals"], r["vals"])
                        and np.array_equal(np.sign(rp["rgb"] - gt), np.sign(rm["rgb"] - gt))):
                    continue
                an = g[name].reshape(flat.shape)[gi, k]
                assert abs((lp - lm) / h - an) <= 1e-4 * (abs(an) + 1e-3 * scale) + 1e-15, (name, gi, k)
                checked += 1
    assert checked > 150


CHECKS = [check_closed_forms, check_weights_sum_to_one, check_keys_brute_force, check_loss,
          check_pyramid_and_levels, check_sh, check_gradients_fd]

# (what the mistake is, statement in lvigs_oracle.c, its mistaken form)
MUTATIONS = [
    ("dilation of the composited covariance", "g->a = a + 0.3;", "g->a = a + 0.35;"),
    ("dilation in the key stage", "    a = a + 0.3f;\n", "    a = a + 0.25f;\n"),
    ("alpha clamp", "#define ALPHA_MAX 0.99", "#define ALPHA_MAX 0.995"),
    ("1/255 cut", "#define ALPHA_MIN (1.0 / 255.0)", "#define ALPHA_MIN (1.0 / 256.0)"),
    ("stop threshold", "#define T_MIN 1e-4", "#define T_MIN 1e-3"),
    ("stop tested before the Gaussian's alpha", "int stop = Tn < T_MIN;", "int stop = T < T_MIN;"),
    ("sign of dL/du", "o[0] += dLdpow * (-(A * c->dx + B * c->dy));", "o[0] += dLdpow * (A * c->dx + B * c->dy);"),
    ("depth behind a Gaussian added, not subtracted",
     "dLda += gd * (depth[g] * c->T - suf[5 * (i + 1) + 3] * inv);",
     "dLda += gd * (depth[g] * c->T + suf[5 * (i + 1) + 3] * inv);"),
    ("visibility term without T", "dLda += ga * (c->T - suf[5 * (i + 1) + 4] * inv);",
     "dLda += ga * (1.0 - suf[5 * (i + 1) + 4] * inv);"),
    ("sigmoid derivative dropped", "d_opacity_logits[i] += dop * g.opacity * (1.0 - g.opacity);",
     "d_opacity_logits[i] += dop * g.opacity;"),
    ("quaternion gradient not projected",
     "for (int k = 0; k < 4; ++k) d_quats[4 * i + k] += (dqn[k] - g.qn[k] * dot) / g.qnorm;",
     "for (int k = 0; k < 4; ++k) d_quats[4 * i + k] += dqn[k] / g.qnorm;"),
    ("factor 2 dropped in the conic derivative",
     "double db = dA * (2.0 * b * c / det2)", "double db = dA * (1.0 * b * c / det2)"),
    ("transposed covariance chain", "dT[r] = 2.0 * da * s0 + db * s1;", "dT[r] = 2.0 * da * s1 + db * s0;"),
    ("SH band-1 constant", "const double k1 = sqrt(3.0 / (4.0 * PI));", "const double k1 = sqrt(3.0 / (2.0 * PI));"),
    ("SSIM constant C2", "const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;",
     "const double C1 = 0.01 * 0.01, C2 = 0.02 * 0.02;"),
    ("L1 gradient sign", "d_img[i] = (1.0 - lambda) * sgn_flip(img[i] - gt[i], kink_margin, flip) / (3.0 * P);",
     "d_img[i] = (1.0 - lambda) * sgn_flip(gt[i] - img[i], kink_margin, flip) / (3.0 * P);"),
    ("depth loss normalised by all pixels", "if (nvalid) ld /= (double)nvalid;", "if (nvalid) ld /= (double)P;"),
    ("pyramid depth averaged over four", "depth_out[(size_t)y * W2 + x] = cnt ? sum / cnt : 0.0;",
     "depth_out[(size_t)y * W2 + x] = sum / 4.0;"),
    ("level principal point not centred", "out->cx = (c0->cx + 0.5f) * scale - 0.5f;", "out->cx = c0->cx * scale;"),
    ("equal keys in reverse index order", "if (a->val != b->val) return a->val < b->val ? -1 : 1;",
     "if (a->val != b->val) return a->val < b->val ? 1 : -1;"),
]


def test_checks_pass_on_the_oracle(tmp_path):
    O = load_oracle(tmp_path, "oracle_plain")
    for check in CHECKS:
        check(O)


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    O = load_oracle(tmp_path, "oracle_mut", (old, new))
    failed = []
    for check in CHECKS:
        try:
            check(O)
        except Exception as e:  # an assertion, or an error the mistake causes
            failed.append(f"{check.__name__}: {type(e).__name__}")
            break
    assert failed, f"no check fails with the mistake: {what}"
    print(f"  {what}: {failed[0]}")
