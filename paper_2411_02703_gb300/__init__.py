"""GB300 (sm_103a) differentiable Gaussian-splatting hot path of LVI-GS
(arxiv 2411.02703): CUDA kernels behind the C ABI of include/lvigs.h and a
thin PyTorch binding (PyTorch supplies device memory and streams only).
"""
from ._lib import LvigsError, load, library_path  # noqa: F401
from .context import Context, PARAM_NAMES, loss_noalloc  # noqa: F401
from .autograd import RenderFunction, render  # noqa: F401
from .gaussian_map import GaussianMap  # noqa: F401
from .driver import Keyframe, Mapper, MappingSchedule  # noqa: F401

__all__ = ["Context", "GaussianMap", "Keyframe", "Mapper", "MappingSchedule", "loss_noalloc", "RenderFunction", "render", "LvigsError", "load", "library_path", "PARAM_NAMES"]
