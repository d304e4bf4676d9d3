"""lvigs_loss_noalloc: the mapping loss for callers that cannot allocate
device memory (a host whose allocator owns the memory budget, or a real-time
loop where cudaFree would synchronise the device).  Its scratch is a fixed
array in the library's device code instead of a context's workspace.

The GPU test calls it through the C ABI twice in a row, on images of
different sizes and weights, and checks each result against lvigs_loss on the
same inputs with the loss-parity bars (loss terms 1e-5 relative, dL/drgb 1e-3
of its largest entry, dL/ddepth 1e-5 relative).  The second call sees the
scratch as the first one left it, which must not matter.  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

CAPACITY = 4  # LVIGS_ERR_CAPACITY


def _inputs(H, W, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1).astype(np.float32)
    d = rng.uniform(2, 10, (H, W)).astype(np.float32)
    li = np.where(rng.uniform(size=(H, W)) < 0.05, rng.uniform(2, 10, (H, W)), 0).astype(np.float32)
    return x, y, d, li


def test_noalloc_rejects_oversize_images():
    """Size checks come before any CUDA call, so this runs without a GPU."""
    from paper_2411_02703_gb300 import _lib

    lib = _lib.load()
    fake = ctypes.c_void_p(256)  # never dereferenced: the call returns first
    for W, H in ((641, 512), (2049, 100), (100, 2049), (573, 573)):
        code = lib.lvigs_loss_noalloc(W, H, fake, fake, fake, fake, 0.2, 0.1, fake, fake, fake, None)
        assert code == CAPACITY, (W, H, code)


@pytest.mark.gpu
def test_noalloc_loss_matches_lvigs_loss_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P
    from paper_2411_02703_gb300 import _lib

    lib = _lib.load()
    ctx = P.Context()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    # first call at the largest size allowed, the second smaller, ragged and
    # with other weights, so it runs over what the first left in the scratch
    for (H, W, lam, lamd, seed) in ((512, 640, 0.2, 0.1, 11), (197, 333, 0.35, 1.0, 12)):
        x, y, d, li = (torch.from_numpy(a).cuda() for a in _inputs(H, W, seed))
        ref_terms, ref_img, ref_dep = ctx.loss(x, d, y, li, lam, lamd)
        terms = torch.full((4,), float("nan"), device="cuda", dtype=torch.float64)
        d_img = torch.full((3, H, W), float("nan"), device="cuda")
        d_dep = torch.full((H, W), float("nan"), device="cuda")
        code = lib.lvigs_loss_noalloc(W, H, ptr(x), ptr(d), ptr(y), ptr(li), lam, lamd, ptr(terms), ptr(d_img),
                                      ptr(d_dep), stream)
        assert code == 0, code
        torch.cuda.synchronize()
        np.testing.assert_allclose(terms.cpu().numpy(), ref_terms.cpu().numpy(), rtol=1e-5, atol=1e-7)
        r_img = ref_img.cpu().numpy()
        assert np.abs(d_img.cpu().numpy() - r_img).max() <= 1e-3 * np.abs(r_img).max()
        np.testing.assert_allclose(d_dep.cpu().numpy(), ref_dep.cpu().numpy(), rtol=1e-5, atol=1e-12)
