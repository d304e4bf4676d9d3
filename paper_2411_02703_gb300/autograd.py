"""torch.autograd.Function around the CUDA render / backward pair.

forward  -> lvigs_render   (a1-a5, the compositing state stays in a view slot)
backward -> lvigs_backward (a6-a7, transmittance recovered by division)
"""
from __future__ import annotations

import torch

from .context import PARAM_NAMES, Context


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, lv: Context, cam, level: int, sh_degree: int):
        params = dict(means=means.detach().contiguous(), log_scales=log_scales.detach().contiguous(),
                      quats=quats.detach().contiguous(), opacity_logits=opacity_logits.detach().contiguous(),
                      sh=sh.detach().contiguous(), sh_degree=sh_degree)
        rgb, depth, alpha, slot = lv.render(params, cam, level)
        ctx.lv = lv
        ctx.slot = slot
        ctx.params = params  # the library reads these buffers again in backward
        ctx.rgb_shape = tuple(rgb.shape)
        return rgb, depth, alpha

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_alpha):
        params = ctx.params
        if d_rgb is None:
            d_rgb = torch.zeros(ctx.rgb_shape, device=params["means"].device)
        grads = ctx.lv.backward(ctx.slot, params, d_rgb.contiguous().float(),
                                None if d_depth is None else d_depth.contiguous().float(),
                                None if d_alpha is None else d_alpha.contiguous().float())
        ctx.lv.release(ctx.slot)
        return tuple(grads[k] for k in PARAM_NAMES) + (None, None, None, None)


def render(lv: Context, params, cam, level=0):
    """Differentiable render: returns (rgb, depth, alpha) with autograd to the parameters."""
    return RenderFunction.apply(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                                params["sh"], lv, cam, int(level), int(params.get("sh_degree", 0)))
