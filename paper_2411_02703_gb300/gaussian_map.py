"""The Gaussian map as a training system holds it: parameter tensors with spare
capacity, their Adam moments and gradient buffers (PyTorch device memory),
and the map-maintenance calls of the C ABI on them -- the optimiser step,
expansion from colourised LiDAR points, pruning (argument marshalling only;
the arithmetic runs in liblvigs.so).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .context import PARAM_NAMES, Context, _ptr, _stream, camera_struct

_WIDTH = {"means": (3,), "log_scales": (3,), "quats": (4,), "opacity_logits": ()}


def _shape(name, rows, K):
    return (rows, K, 3) if name == "sh" else (rows, *_WIDTH[name])


def _bufs(d):
    return L.ParamBuffers(*(d[k].data_ptr() for k in PARAM_NAMES))


class GaussianMap:
    """Live rows [0, n) of capacity-sized buffers.  ``params()`` and ``grads()``
    return views of the live rows for the render / batched-step calls."""

    def __init__(self, capacity=1024, sh_stride_k=16, sh_degree=0, device="cuda"):
        self.K = int(sh_stride_k)
        self.sh_degree = int(sh_degree)
        self.device = torch.device(device)
        self.n = 0
        self.step = 0
        self.capacity = 0
        self._p = self._m = self._v = self._g = None
        self.reserve(max(int(capacity), 1))

    @classmethod
    def from_params(cls, params, capacity=None, device="cuda"):
        n = int(params["means"].shape[0])
        K = int(params["sh"].shape[1])
        gm = cls(capacity or max(n, 1), K, int(params.get("sh_degree", 0)), device)
        for k in PARAM_NAMES:
            src = torch.as_tensor(params[k], dtype=torch.float32)
            gm._p[k][:n].copy_(src.to(gm.device))
        gm.n = n
        return gm

    def _alloc(self, rows):
        return {k: torch.zeros(_shape(k, rows, self.K), device=self.device, dtype=torch.float32)
                for k in PARAM_NAMES}

    def reserve(self, capacity):
        """Grow every buffer to at least ``capacity`` rows (x1.5 steps), keeping
        the live rows."""
        if capacity <= self.capacity:
            return
        cap = max(int(capacity), int(self.capacity * 1.5))
        new = [self._alloc(cap) for _ in range(4)]
        for old, nw in zip((self._p, self._m, self._v, self._g), new):
            if old is not None and self.n > 0:
                for k in PARAM_NAMES:
                    nw[k][:self.n].copy_(old[k][:self.n])
        self._p, self._m, self._v, self._g = new
        self.capacity = cap

    def params(self):
        d = {k: self._p[k][:self.n] for k in PARAM_NAMES}
        d["sh_degree"] = self.sh_degree
        return d

    def grads(self):
        return {k: self._g[k][:self.n] for k in PARAM_NAMES}

    def adam_state(self):
        return ({k: self._m[k][:self.n] for k in PARAM_NAMES}, {k: self._v[k][:self.n] for k in PARAM_NAMES})

    def adam_step(self, cfg=None, zero_grads=True):
        """One Adam step on the live rows with the gradients in ``grads()``."""
        self.step += 1
        c = L.AdamConfig()
        L.load().lvigs_adam_config_default(ctypes.byref(c))
        for key, val in (cfg or {}).items():
            setattr(c, key, float(val))
        g = L.Grads(*(self._g[k].data_ptr() for k in PARAM_NAMES), 0)
        L.check(L.load().lvigs_adam_step(ctypes.byref(_bufs(self._p)), ctypes.byref(g), ctypes.byref(_bufs(self._m)),
                                         ctypes.byref(_bufs(self._v)), self.n, self.K, self.step, ctypes.byref(c),
                                         int(bool(zero_grads)), _stream()), "lvigs_adam_step")

    def append(self, ctx: Context, points, colours, cam=None, level=0, alpha=None, cfg=None):
        """New Gaussians for colourised points (device float32 [k,3] each),
        optionally filtered against the V_p image ``alpha`` of ``cam`` at
        ``level``.  Returns the number added."""
        k = int(points.shape[0])
        for t, name in ((points, "points"), (colours, "colours")):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == (k, 3)):
                raise ValueError(f"{name} must be a contiguous CUDA float32 tensor [k,3]")
        if alpha is not None and not (alpha.is_cuda and alpha.dtype == torch.float32 and alpha.is_contiguous()):
            raise ValueError("alpha must be a contiguous CUDA float32 tensor")
        self.reserve(self.n + k)
        c = L.InitConfig()
        L.load().lvigs_init_config_default(ctypes.byref(c))
        for key, val in (cfg or {}).items():
            setattr(c, key, type(getattr(c, key))(val))
        cs = camera_struct(cam) if cam is not None else None
        n_out = ctypes.c_int64()
        ctx._chk(L.load().lvigs_append_gaussians(
            ctx._h, _ptr(points), _ptr(colours), k, ctypes.byref(cs) if cs is not None else None, int(level),
            _ptr(alpha), ctypes.byref(c), ctypes.byref(_bufs(self._p)), ctypes.byref(_bufs(self._m)),
            ctypes.byref(_bufs(self._v)), self.n, self.capacity, self.K, ctypes.byref(n_out), _stream()),
            "lvigs_append_gaussians")
        added = int(n_out.value) - self.n
        self.n = int(n_out.value)
        return added

    def prune(self, ctx: Context, min_opacity=0.005):
        """Remove Gaussians below ``min_opacity``; returns the number removed.
        The gradient rows are cleared (they no longer match)."""
        n_out = ctypes.c_int64()
        ctx._chk(L.load().lvigs_prune_gaussians(ctx._h, float(min_opacity), ctypes.byref(_bufs(self._p)),
                                                ctypes.byref(_bufs(self._m)), ctypes.byref(_bufs(self._v)), self.n,
                                                self.K, ctypes.byref(n_out), _stream()), "lvigs_prune_gaussians")
        removed = self.n - int(n_out.value)
        self.n = int(n_out.value)
        if removed:
            for k in PARAM_NAMES:
                self._g[k].zero_()
        return removed
