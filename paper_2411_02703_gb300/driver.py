"""The mapping loop around the differentiable path (Sec. III-C, III-D, III-E):
keyframes arrive with their colourised LiDAR points, the map expands, and
every step renders and differentiates a random choice of keyframes at the
pyramid level their progress calls for, then takes an Adam step.

Schedule (readings of the paper, which describes the policies but gives no
numbers; every value is a constructor argument):
  * a new keyframe is optimised once on its own before it joins the random
    pool (each received keyframe is first optimised as a submap);
  * each step draws ``views_per_step`` keyframes at random, without
    replacement, from the keyframes still below the per-keyframe iteration
    cap; a keyframe that reaches the cap leaves the pool;
  * coarse to fine per keyframe: with pyramid levels 0..L, a keyframe is
    rendered at level L for its first cap/(L+1) iterations, then L-1, ..., and
    at full resolution for the last share;
  * SH degree: 0 at the start, one more every ``sh_interval`` steps, at most 3;
  * expansion: a keyframe's points join the map ``delay`` keyframes after it
    arrives (the delay buffer), filtered against the V_p image of the current
    map at that keyframe.

Host logic only; every render, loss, gradient, optimiser and expansion step
runs in liblvigs.so through ``Context`` and ``GaussianMap``.
"""
from __future__ import annotations

import random
from collections import deque
from dataclasses import dataclass, field

import torch


@dataclass(eq=False)
class Keyframe:
    cam: object                  # level-0 camera (R, t, fx, fy, cx, cy, W, H)
    gt_rgb: torch.Tensor         # [3,H,W] level-0 target, device
    lidar: torch.Tensor          # [H,W] projected LiDAR depth (0 = no return), device
    points: torch.Tensor = None  # [k,3] colourised points that arrived with it (device), optional
    colours: torch.Tensor = None
    iters: int = 0
    kid: int = field(default=-1)


class MappingSchedule:
    def __init__(self, max_iters=100, top_level=2, sh_interval=1000, views_per_step=1, seed=0):
        if max_iters < 1 or top_level < 0 or views_per_step < 1:
            raise ValueError("bad schedule")
        self.max_iters = int(max_iters)
        self.top_level = int(top_level)
        self.sh_interval = int(sh_interval)
        self.views_per_step = int(views_per_step)
        self.rng = random.Random(seed)

    def level_for(self, kf: Keyframe) -> int:
        share = self.max_iters / (self.top_level + 1)
        return max(0, self.top_level - int(kf.iters // share))

    def sh_degree(self, steps_done: int) -> int:
        return min(3, steps_done // self.sh_interval) if self.sh_interval > 0 else 3

    def select(self, fresh: deque, pool: list) -> list:
        """Keyframes for the next step: a fresh keyframe alone if one waits,
        else a random draw from the pool."""
        if fresh:
            return [fresh.popleft()]
        if not pool:
            return []
        k = min(self.views_per_step, len(pool))
        return self.rng.sample(pool, k)


class Mapper:
    def __init__(self, ctx, gmap, schedule: MappingSchedule, lambda_ssim=0.2, lambda_depth=0.1, delay=1,
                 tau_alpha=0.5, adam=None):
        self.ctx, self.gmap, self.sched = ctx, gmap, schedule
        self.lambda_ssim, self.lambda_depth = float(lambda_ssim), float(lambda_depth)
        self.delay = int(delay)
        self.tau_alpha = float(tau_alpha)
        self.adam = adam
        self.fresh = deque()
        self.pool = []
        self.pending = deque()  # keyframes whose points wait in the delay buffer
        self.steps = 0
        self.n_keyframes = 0
        self.history = []       # (step, [kid], [level], [loss]) per step

    def add_keyframe(self, kf: Keyframe):
        kf.kid = self.n_keyframes
        self.n_keyframes += 1
        if kf.points is not None:
            self.pending.append(kf)
        while len(self.pending) > self.delay:
            self._expand(self.pending.popleft())
        self.fresh.append(kf)

    def flush(self):
        """Integrate every buffered keyframe's points now."""
        while self.pending:
            self._expand(self.pending.popleft())

    def _expand(self, kf: Keyframe):
        alpha = None
        if self.gmap.n > 0:
            _, _, alpha, slot = self.ctx.render(self.gmap.params(), kf.cam, 0)
            self.ctx.release(slot)
        self.gmap.append(self.ctx, kf.points, kf.colours, kf.cam if alpha is not None else None, 0, alpha,
                         {"tau_alpha": self.tau_alpha})

    def step(self):
        """One mapping iteration; returns the per-view losses ([V,4] float64)
        or None when no keyframe is left to optimise."""
        if self.gmap.n == 0:
            return None
        views = self.sched.select(self.fresh, self.pool)
        if not views:
            return None
        levels = [self.sched.level_for(kf) for kf in views]
        kmax = int(self.gmap.K ** 0.5) - 1  # highest degree the SH buffer holds
        self.gmap.sh_degree = min(self.sched.sh_degree(self.steps), kmax)
        losses, _ = self.ctx.train_step_batched(self.gmap.params(), [kf.cam for kf in views], levels,
                                                [kf.gt_rgb for kf in views], [kf.lidar for kf in views],
                                                self.lambda_ssim, self.lambda_depth, grads=self.gmap.grads())
        self.gmap.adam_step(self.adam, zero_grads=False)
        self.steps += 1
        for kf in views:
            kf.iters += 1
            if kf.iters < self.sched.max_iters:
                if kf not in self.pool:
                    self.pool.append(kf)
            elif kf in self.pool:
                self.pool.remove(kf)
        self.history.append((self.steps, [kf.kid for kf in views], levels, losses[:, 0].tolist()))
        return losses
