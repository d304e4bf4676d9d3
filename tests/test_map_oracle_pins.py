"""Pins of the map-maintenance oracle (``oracle/map_ops.py``) against what the
mathematics and independent routines fix: the Adam update's closed forms and
PyTorch's own Adam (an independent implementation of the same textbook
definition), nearest-neighbour scales on a lattice and by brute force, the SH
band-0 colour against the renderer's basis, the visibility filter's pixel
rounding and inequality, and the pruning threshold."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import map_ops as M


def _rand_params(rng, n, K=16):
    return {
        "means": rng.normal(0, 5, (n, 3)),
        "log_scales": rng.normal(-3, 0.5, (n, 3)),
        "quats": rng.normal(0, 1, (n, 4)),
        "opacity_logits": rng.normal(0, 1, n),
        "sh": rng.normal(0, 0.3, (n, K, 3)),
    }


def _zeros_like(d):
    return {k: np.zeros_like(v) for k, v in d.items()}


def test_adam_first_step_is_signed_learning_rate():
    """With zero moments, m_hat = g and v_hat = g^2: p -= lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p = _rand_params(rng, 50)
    g = _rand_params(rng, 50)
    P, Mo, V = M.adam_step(p, g, _zeros_like(p), _zeros_like(p), 1)
    cfg = M.ADAM_DEFAULTS
    lr = {"means": cfg["lr_means"], "log_scales": cfg["lr_log_scales"], "quats": cfg["lr_quats"],
          "opacity_logits": cfg["lr_opacity"]}
    for k, l in lr.items():
        np.testing.assert_allclose(P[k], p[k] - l * g[k] / (np.abs(g[k]) + cfg["eps"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(P["sh"][:, 0], p["sh"][:, 0] - cfg["lr_sh_dc"] * np.sign(g["sh"][:, 0]), atol=1e-15)
    np.testing.assert_allclose(P["sh"][:, 1:], p["sh"][:, 1:] - cfg["lr_sh_rest"] * np.sign(g["sh"][:, 1:]),
                               atol=1e-15)
    np.testing.assert_allclose(Mo["means"], (1 - cfg["beta1"]) * g["means"], rtol=1e-15)
    np.testing.assert_allclose(V["means"], (1 - cfg["beta2"]) * g["means"] ** 2, rtol=1e-15)


def test_adam_zero_gradient_decays_moments():
    rng = np.random.default_rng(1)
    p = _rand_params(rng, 20)
    m = _rand_params(rng, 20)
    v = {k: np.abs(x) for k, x in _rand_params(rng, 20).items()}
    P, Mo, V = M.adam_step(p, _zeros_like(p), m, v, 7)
    for k in M.PARAM_KEYS:
        np.testing.assert_allclose(Mo[k], 0.9 * m[k], rtol=1e-15)
        np.testing.assert_allclose(V[k], 0.999 * v[k], rtol=1e-15)
    bc1, bc2 = 1 - 0.9 ** 7, 1 - 0.999 ** 7
    exp = p["quats"] - 1e-3 * (0.9 * m["quats"] / bc1) / (np.sqrt(0.999 * v["quats"] / bc2) + 1e-15)
    np.testing.assert_allclose(P["quats"], exp, rtol=1e-14)


def test_adam_matches_torch_adam_over_steps():
    """torch.optim.Adam (float64, CPU) is an independent implementation."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    n, K = 40, 16
    p = _rand_params(rng, n, K)
    cfg = M.ADAM_DEFAULTS
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items() if k != "sh"}
    sh0 = torch.tensor(p["sh"][:, :1], dtype=torch.float64, requires_grad=True)
    shr = torch.tensor(p["sh"][:, 1:], dtype=torch.float64, requires_grad=True)
    groups = [{"params": [tp["means"]], "lr": cfg["lr_means"]},
              {"params": [tp["log_scales"]], "lr": cfg["lr_log_scales"]},
              {"params": [tp["quats"]], "lr": cfg["lr_quats"]},
              {"params": [tp["opacity_logits"]], "lr": cfg["lr_opacity"]},
              {"params": [sh0], "lr": cfg["lr_sh_dc"]}, {"params": [shr], "lr": cfg["lr_sh_rest"]}]
    opt = torch.optim.Adam(groups, betas=(cfg["beta1"], cfg["beta2"]), eps=cfg["eps"])
    P, Mo, V = p, _zeros_like(p), _zeros_like(p)
    for step in range(1, 6):
        g = _rand_params(rng, n, K)
        if step == 3:
            g["opacity_logits"][:] = 0.0  # a step without gradient for one group
        for k, t in tp.items():
            t.grad = torch.tensor(g[k], dtype=torch.float64)
        sh0.grad = torch.tensor(g["sh"][:, :1], dtype=torch.float64)
        shr.grad = torch.tensor(g["sh"][:, 1:], dtype=torch.float64)
        opt.step()
        P, Mo, V = M.adam_step(P, g, Mo, V, step)
        for k, t in tp.items():
            np.testing.assert_allclose(P[k], t.detach().numpy(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(P["sh"], np.concatenate([sh0.detach().numpy(), shr.detach().numpy()], 1),
                                   rtol=1e-12, atol=1e-14)


def test_knn_scale_on_cubic_lattice():
    """On a lattice of spacing a every point has at least three neighbours at
    distance a and none closer: log-scale = ln a."""
    a = 0.37
    g = np.arange(5) * a
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + np.array([3.0, -2.0, 1.0])
    init = M.init_gaussians(pts, np.full_like(pts, 0.5), sh_stride_k=1)
    np.testing.assert_allclose(init["log_scales"], math.log(a), atol=1e-12)


def test_knn_matches_brute_force():
    rng = np.random.default_rng(3)
    pts = rng.normal(0, 1, (300, 3))
    pts[10] = pts[11]  # a duplicate pair
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    ref = np.sort(d2, axis=1)[:, :3].mean(1)
    np.testing.assert_allclose(M.knn_mean_dist2(pts), ref, rtol=1e-12, atol=1e-15)
    # few points: the mean over the others; a lone point gets 0 (then the floor)
    np.testing.assert_allclose(M.knn_mean_dist2(pts[:3]), np.sort(d2[:3, :3], 1)[:, :2].mean(1), rtol=1e-12)
    assert M.knn_mean_dist2(pts[:1])[0] == 0.0


def test_init_floor_identity_opacity_and_colour():
    pts = np.array([[1.0, 2.0, 3.0]] * 4 + [[5.0, 5.0, 5.0]])
    col = np.array([[0.2, 0.5, 0.9]] * 4 + [[0.0, 1.0, 0.3]])
    init = M.init_gaussians(pts, col, sh_stride_k=16)
    # four coincident points: distance 0, floored at 1e-7
    np.testing.assert_allclose(init["log_scales"][:4], 0.5 * math.log(1e-7), rtol=1e-12)
    np.testing.assert_array_equal(init["quats"], np.tile([1.0, 0, 0, 0], (5, 1)))
    np.testing.assert_allclose(1.0 / (1.0 + np.exp(-init["opacity_logits"])), 0.1, rtol=1e-12)
    # the renderer's degree-0 colour (basis value Y_00, offset 0.5) gives back the point colour
    Y, _ = O.sh_basis(np.array([0.0, 0.0, 1.0]))
    np.testing.assert_allclose(Y[0] * init["sh"][:, 0, :] + 0.5, col, atol=1e-12)
    assert np.all(init["sh"][:, 1:, :] == 0.0)


def _cam(W=64, H=48):
    return O.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 50.0, 50.0, 32.0, 24.0, W, H)


def test_point_pixels_round_to_nearest_centre():
    cam = _cam()
    # at depth 2, u = 25 x + 32: x = 0.0396 -> u = 32.99 -> 33; x = -0.0204 -> u = 31.49 -> 31
    pts = np.array([[0.0396, 0.0, 2.0], [-0.0204, 0.0, 2.0], [0.0, 0.0196, 2.0], [0.0, 0.0, 0.1],
                    [10.0, 0.0, 2.0]], np.float32)
    px, py, inside = M.point_pixels(pts, cam)
    assert px[:3].tolist() == [33, 31, 32]
    assert py[:3].tolist() == [24, 24, 24]
    assert inside.tolist() == [True, True, True, False, False]


def test_visibility_filter_inequality_and_outside_points():
    cam = _cam()
    alpha = np.zeros((48, 64), np.float32)
    alpha[24, 33] = 0.9   # opaque: transparency 0.1
    alpha[24, 31] = 0.2   # transparent: 0.8
    alpha[24, 32] = 0.5   # transparency exactly tau
    pts = np.array([[0.0396, 0.0, 2.0], [-0.0204, 0.0, 2.0], [0.0, 0.0, 2.0], [0.0, 0.0, -3.0],
                    [10.0, 0.0, 2.0]], np.float32)
    keep = M.visibility_keep(pts, cam, alpha, tau_alpha=0.5)
    assert keep.tolist() == [False, True, False, True, True]
    lit = M.visibility_keep(pts, cam, alpha, tau_alpha=0.5, literal=True)
    assert lit.tolist() == [True, False, False, True, True]


def test_prune_threshold_on_logits():
    rng = np.random.default_rng(4)
    logits = rng.normal(-3, 3, 5000).astype(np.float32)
    op = 1.0 / (1.0 + np.exp(-logits.astype(np.float64)))
    keep = M.prune_keep(logits, 0.005)
    far = np.abs(op - 0.005) > 1e-9
    np.testing.assert_array_equal(keep[far], (op >= 0.005)[far])
    arrs = {"a": np.arange(5000), "b": np.arange(5000 * 3).reshape(5000, 3)}
    c = M.compact_rows(arrs, keep)
    assert np.all(np.diff(c["a"]) > 0) and c["a"].shape[0] == keep.sum()
    np.testing.assert_array_equal(c["b"][:, 0], c["a"] * 3)
