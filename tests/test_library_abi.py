"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/lvigs.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lvigs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lvigs_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["lvigs_create", "lvigs_destroy", "lvigs_render", "lvigs_backward", "lvigs_loss",
                     "lvigs_pyramid_down", "lvigs_train_step_batched", "lvigs_debug_keys", "lvigs_sync_status",
                     "lvigs_release_view", "lvigs_last_error", "lvigs_stage_targets", "lvigs_adam_step",
                     "lvigs_append_gaussians", "lvigs_prune_gaussians", "lvigs_loss_noalloc"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2411_02703_gb300 import _lib

    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in lvigs.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature in the binding"
    assert lib.lvigs_version().startswith(b"lvigs-gb300")


def test_library_is_built_for_sm_103a():
    from paper_2411_02703_gb300 import build as b

    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)
    assert os.path.exists(b.LIB)


def test_host_side_argument_checks_without_gpu():
    from paper_2411_02703_gb300 import _lib

    lib = _lib.load()
    cam = _lib.Camera()
    cam.width, cam.height = 1280, 1024
    w, h = ctypes.c_int(), ctypes.c_int()
    assert lib.lvigs_level_size(ctypes.byref(cam), 2, ctypes.byref(w), ctypes.byref(h)) == 0
    assert (w.value, h.value) == (320, 256)
    assert lib.lvigs_level_size(ctypes.byref(cam), 9, ctypes.byref(w), ctypes.byref(h)) == 1
    assert lib.lvigs_level_size(None, 0, ctypes.byref(w), ctypes.byref(h)) == 1
    # NULL context / arguments are rejected before any CUDA call
    assert lib.lvigs_render(None, None, None, 0, None, None, None) == 1
    assert lib.lvigs_backward(None, 0, None, None, None, None, None) == 1
    assert lib.lvigs_sync_status(None, None) == 1
    assert lib.lvigs_release_view(None, 0) == 1
    assert lib.lvigs_pyramid_down(1, 1, None, None, None, None, None) == 1
    assert lib.lvigs_stage_targets(None, 0, 1, None, None, None, None) == 1
    bad = _lib.Config(12, 12, 0, 0)
    h_ = ctypes.c_void_p()
    assert lib.lvigs_create(ctypes.byref(h_), ctypes.byref(bad)) == 1
    assert lib.lvigs_last_error(None) == b"no context"


def test_oracle_and_library_share_no_code():
    # the oracle never imports the package and the package never imports the oracle
    pkg = os.path.join(ROOT, "paper_2411_02703_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "lvigs_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2411_02703_gb300" not in txt and "lvigs.h" not in txt and "synthetic" not in txt, f
