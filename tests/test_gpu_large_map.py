"""The large outdoor map-expansion step at full size: 3,000,000 Gaussians (SH
degree 3), one 50,000-point sweep appended, 16 keyframes at 1280x1024 in one
batched forward + backward with the full loss, then an Adam update of every
parameter.

What is compared (the oracle cannot run the whole step in seconds):
  * the appended rows against the oracle's initialisation of the sweep
    (nearest-neighbour scales over the 50,000 points), all of them;
  * 24 sampled 16x16 tiles of three of the views against the oracle renderer
    run on the whole 3,050,000-Gaussian map (bars of the forward parity tests);
  * the batched step's gradients against the plain single-view path (render,
    loss, backward accumulated over the 16 views), within 1e-4 of the largest
    entry (atomic summation order differs);
  * the Adam step on 20,000 sampled rows against the oracle's update, given
    the moments the GPU produced (which are checked against their binary32
    rounding bound).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import map_ops as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = M.PARAM_KEYS
MARGIN = 1e-4
IMG_TOL = 1e-4


def test_large_map_expansion_step():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P

    ctx = P.Context()
    params, phase = S.lidar_scene(3_000_000)
    n0 = params["means"].shape[0]
    gm = P.GaussianMap.from_params(params, capacity=n0 + 50_000)
    pts, col = S.fresh_scan(50_000, step=3)
    added = gm.append(ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(col).cuda())
    assert added == pts.shape[0]

    # appended rows
    ref = M.init_gaussians(pts, col, sh_stride_k=16)
    got = {k: v[n0:].cpu().numpy() for k, v in gm.params().items() if k != "sh_degree"}
    np.testing.assert_array_equal(got["means"], pts)
    assert np.abs(got["log_scales"] - ref["log_scales"]).max() <= 1e-5
    np.testing.assert_allclose(got["sh"][:, 0], ref["sh"][:, 0], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(got["opacity_logits"], ref["opacity_logits"], rtol=1e-6)

    # the 16-view batched step on the expanded map
    cams = S.trajectory_cameras(16, phase=phase)
    levels = [0] * 16
    tg = [S.target_images(c, 500 + i) for i, c in enumerate(cams)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gts, lis = [t(x[0]) for x in tg], [t(x[1]) for x in tg]
    outs = [(torch.empty(3, c.H, c.W, device="cuda"), torch.empty(c.H, c.W, device="cuda"),
             torch.empty(c.H, c.W, device="cuda")) for c in cams]
    gm.sh_degree = 3
    dp = gm.params()
    losses, grads = ctx.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, grads=gm.grads(), outputs=outs)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert torch.isfinite(losses).all()

    host = {k: v.cpu().numpy() for k, v in dp.items() if k != "sh_degree"}
    host["sh_degree"] = 3
    rng = np.random.default_rng(9)
    for vi in (0, 7, 15):
        spec = cams[vi]
        sel = rng.choice(80 * 64, 8, replace=False).astype(np.int32)
        r = O.render_view(host, O.Camera(spec.R, spec.t, spec.fx, spec.fy, spec.cx, spec.cy, spec.W, spec.H), 0,
                          sel_tiles=sel)
        mask = np.zeros((spec.H, spec.W), bool)
        for tt in sel:
            ty, tx = divmod(int(tt), 80)
            mask[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
        ok = mask & (r["margin"] > MARGIN)
        assert ok.sum() > 0.95 * mask.sum()
        rgb, depth, alpha = (o.cpu().numpy() for o in outs[vi])
        assert np.abs(rgb - r["rgb"])[:, ok].max() < IMG_TOL
        assert np.abs(alpha - r["alpha"])[ok].max() < IMG_TOL
        assert np.abs(depth - r["depth"])[ok].max() < IMG_TOL * max(1.0, float(np.abs(r["depth"][ok]).max()))

    # batched gradients against the plain single-view path
    pgrads = {k: torch.zeros_like(dp[k]) for k in P.PARAM_NAMES}
    for i, c in enumerate(cams):
        rgb, depth, alpha, slot = ctx.render(dp, c, 0)
        # bit-identical, or within float rounding where a list of a few chunks
        # was walked whole in the batched step and chunk by chunk here
        if not torch.equal(rgb, outs[i][0]):
            assert float((rgb - outs[i][0]).abs().max()) <= 1e-5
        _, d_rgb, d_dep = ctx.loss(rgb, depth, gts[i], lis[i], 0.2, 0.1)
        ctx.backward(slot, dp, d_rgb, d_dep, grads=pgrads, accumulate=i > 0)
        ctx.release(slot)
    torch.cuda.synchronize()
    for k in P.PARAM_NAMES:
        a, b = grads[k].cpu().numpy(), pgrads[k].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, k

    # Adam on sampled rows
    rows = np.sort(rng.choice(gm.n, 20_000, replace=False))
    ri = torch.from_numpy(rows).cuda()
    m_, v_ = gm.adam_state()
    take = lambda d: {k: d[k][ri].cpu().numpy().astype(np.float64) for k in KEYS}
    p0, g0, m0, v0 = take(gm.params()), take(gm.grads()), take(m_), take(v_)
    gm.adam_step()
    torch.cuda.synchronize()
    m_, v_ = gm.adam_state()
    p1, m1, v1 = take(gm.params()), take(m_), take(v_)
    _, mr, vr = M.adam_step(p0, g0, m0, v0, 1)
    b1, b2 = M.ADAM_DEFAULTS["beta1"], M.ADAM_DEFAULTS["beta2"]
    for k in KEYS:
        assert np.all(np.abs(m1[k] - mr[k]) <= 1e-6 * (b1 * np.abs(m0[k]) + (1 - b1) * np.abs(g0[k])) + 1e-37), k
        assert np.all(np.abs(v1[k] - vr[k]) <= 1e-6 * (b2 * v0[k] + (1 - b2) * g0[k] ** 2) + 1e-40), k
    pr, _, _ = M.adam_step(p0, {k: np.zeros_like(g0[k]) for k in KEYS}, {k: m1[k] / b1 for k in KEYS},
                           {k: v1[k] / b2 for k in KEYS}, 1)
    for k in KEYS:
        d = np.abs(pr[k] - p0[k])
        assert np.all(np.abs(p1[k] - pr[k]) <= 1e-3 * d + 2.5e-7 * np.abs(pr[k]) + 1e-30), k
    # the gradients were cleared by the step
    assert all(float(gm.grads()[k].abs().max()) == 0.0 for k in KEYS)
    ctx.close()
