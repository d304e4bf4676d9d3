"""Host logic of the mapping loop (paper_2411_02703_gb300.driver) on CPU, with
fakes standing in for the context and the map: the order keyframes are
optimised in, the per-keyframe iteration cap, the coarse-to-fine level
schedule, the SH degree schedule and the delay buffer of map expansion."""
import pytest

torch = pytest.importorskip("torch")

from paper_2411_02703_gb300.driver import Keyframe, Mapper, MappingSchedule  # noqa: E402


class FakeMap:
    def __init__(self, n=10, K=16):
        self.n, self.K, self.sh_degree = n, K, 0
        self.appended, self.adam_steps = [], 0

    def params(self):
        return {"sh_degree": self.sh_degree}

    def grads(self):
        return {}

    def append(self, ctx, points, colours, cam, level, alpha, cfg):
        self.appended.append((int(points[0, 0]), alpha is not None, cfg["tau_alpha"]))
        self.n += points.shape[0]

    def adam_step(self, cfg=None, zero_grads=True):
        self.adam_steps += 1


class FakeCtx:
    def __init__(self):
        self.steps = []

    def render(self, params, cam, level):
        return None, None, torch.zeros(2, 2), 7

    def release(self, slot):
        assert slot == 7

    def train_step_batched(self, params, cams, levels, gts, lidars, lam, lamd, grads=None):
        self.steps.append((list(cams), list(levels), params["sh_degree"]))
        return torch.zeros(len(cams), 4, dtype=torch.float64), grads


def _kf(i, with_points=False):
    pts = torch.full((5, 3), float(i)) if with_points else None
    return Keyframe(cam=f"cam{i}", gt_rgb=None, lidar=None, points=pts, colours=pts)


def test_level_and_sh_schedules():
    s = MappingSchedule(max_iters=90, top_level=2, sh_interval=100)
    kf = _kf(0)
    levels = []
    for it in range(90):
        kf.iters = it
        levels.append(s.level_for(kf))
    assert levels == [2] * 30 + [1] * 30 + [0] * 30
    assert [s.sh_degree(k) for k in (0, 99, 100, 250, 300, 10_000)] == [0, 0, 1, 2, 3, 3]


def test_fresh_keyframes_first_then_random_pool_with_cap():
    ctx, gm = FakeCtx(), FakeMap()
    m = Mapper(ctx, gm, MappingSchedule(max_iters=4, top_level=1, views_per_step=2, seed=3))
    for i in range(3):
        m.add_keyframe(_kf(i))
    # each new keyframe is optimised alone, in arrival order
    for i in range(3):
        m.step()
        assert ctx.steps[-1][0] == [f"cam{i}"]
    # then pairs drawn from the pool until every keyframe has 4 iterations
    while m.step() is not None:
        cams = ctx.steps[-1][0]
        assert len(cams) == len(set(cams)) and len(cams) <= 2
    counts = {}
    for cams, _, _ in ctx.steps:
        for c in cams:
            counts[c] = counts.get(c, 0) + 1
    assert counts == {"cam0": 4, "cam1": 4, "cam2": 4}
    assert gm.adam_steps == len(ctx.steps)
    # coarse to fine: the first two iterations of a keyframe at level 1, then 0
    seen = {}
    for cams, levels, _ in ctx.steps:
        for c, l in zip(cams, levels):
            seen.setdefault(c, []).append(l)
    assert all(v == [1, 1, 0, 0] for v in seen.values())


def test_sh_degree_capped_by_buffer():
    ctx, gm = FakeCtx(), FakeMap(K=4)
    m = Mapper(ctx, gm, MappingSchedule(max_iters=50, sh_interval=1))
    m.add_keyframe(_kf(0))
    for _ in range(6):
        m.step()
    assert [d for _, _, d in ctx.steps] == [0, 1, 1, 1, 1, 1]


def test_delay_buffer_integrates_points_late_and_filtered():
    ctx, gm = FakeCtx(), FakeMap(n=0)
    m = Mapper(ctx, gm, MappingSchedule(), delay=2, tau_alpha=0.25)
    m.add_keyframe(_kf(0, True))
    m.add_keyframe(_kf(1, True))
    assert gm.appended == []
    m.add_keyframe(_kf(2, True))
    # keyframe 0's points join when keyframe 2 arrives; the map was empty: no filter image
    assert gm.appended == [(0, False, 0.25)]
    m.add_keyframe(_kf(3, True))
    assert gm.appended[-1] == (1, True, 0.25)
    m.flush()
    assert [a[0] for a in gm.appended] == [0, 1, 2, 3]
    assert gm.n == 20


def test_no_step_without_map_or_keyframes():
    ctx, gm = FakeCtx(), FakeMap(n=0)
    m = Mapper(ctx, gm, MappingSchedule())
    assert m.step() is None
    m.add_keyframe(_kf(0))
    assert m.step() is None and ctx.steps == []
    gm.n = 5  # once the map has Gaussians the waiting keyframe is optimised
    assert m.step() is not None and ctx.steps[-1][0] == ["cam0"]
