"""lvigs_loss_noalloc: the mapping loss for callers that cannot allocate
device memory (a host whose allocator owns the memory budget, or a real-time
loop where cudaFree would synchronise the device).  Its scratch is a fixed
array in the library's device code instead of a context's workspace.

The GPU tests call it through the C ABI, several times in a row, on images of
different sizes and weights.  It runs the kernels of lvigs_loss in the same
order, so each result must equal lvigs_loss on the same inputs bit for bit;
each is also held to the oracle's loss with the loss-parity bars (loss terms
1e-5 relative, dL/drgb 1e-3 of its largest entry, dL/ddepth 1e-5 relative).
Later calls see the scratch as earlier ones left it, which must not matter.
The optional arguments are covered too: no LiDAR target, no gradients, the
loss terms written into page-locked host memory, and the Python wrapper.
The file is named to be collected last.
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


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_vs_oracle(terms, d_img, d_dep, x, y, d, li, lam, lamd):
    import oracle as O

    rterms, r_img, r_dep = O.loss(x, y, d, np.zeros_like(d) if li is None else li, lam, lamd)
    np.testing.assert_allclose(terms, rterms, rtol=1e-5, atol=1e-7)
    if d_img is not None:
        assert np.abs(d_img - r_img).max() <= 1e-3 * np.abs(r_img).max()
    if d_dep is not None:
        np.testing.assert_allclose(d_dep, r_dep, rtol=1e-5, atol=1e-12)


# (H, W, lambda_ssim, lambda_depth, seed, with LiDAR, with gradients, loss terms in pinned host memory)
CALLS = [
    (512, 640, 0.2, 0.1, 11, True, True, False),   # the largest size allowed
    (197, 333, 0.35, 1.0, 12, True, True, False),  # smaller and ragged, over what the first left
    (240, 320, 0.2, 0.1, 13, False, True, False),  # no LiDAR target
    (120, 160, 0.2, 0.1, 14, True, False, False),  # loss terms only
    (100, 90, 0.0, 1.0, 15, True, True, True),     # terms written into page-locked host memory
]


@pytest.mark.gpu
def test_noalloc_loss_matches_lvigs_loss_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P
    from paper_2411_02703_gb300 import _lib

    lib = _lib.load()
    ctx = P.Context()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (H, W, lam, lamd, seed, with_lidar, with_grads, host_terms) in CALLS:
        x, y, d, li = _inputs(H, W, seed)
        if not with_lidar:
            li = None
        X, Y, D = (torch.from_numpy(a).cuda() for a in (x, y, d))
        LI = None if li is None else torch.from_numpy(li).cuda()
        ref_terms, ref_img, ref_dep = ctx.loss(X, D, Y, LI, lam, lamd, grads=with_grads)
        if host_terms:
            terms = torch.full((4,), float("nan"), dtype=torch.float64).pin_memory()
        else:
            terms = torch.full((4,), float("nan"), device="cuda", dtype=torch.float64)
        d_img = torch.full((3, H, W), float("nan"), device="cuda") if with_grads else None
        d_dep = torch.full((H, W), float("nan"), device="cuda") if with_grads else None
        code = lib.lvigs_loss_noalloc(W, H, _ptr(X), _ptr(D), _ptr(Y), _ptr(LI), lam, lamd, _ptr(terms),
                                      _ptr(d_img), _ptr(d_dep), stream)
        assert code == 0, code
        torch.cuda.synchronize()
        t = terms.cpu().numpy()
        assert np.array_equal(t, ref_terms.cpu().numpy()), (t, ref_terms)
        if with_grads:
            assert torch.equal(d_img, ref_img) and torch.equal(d_dep, ref_dep)
        _check_vs_oracle(t, None if d_img is None else d_img.cpu().numpy(),
                         None if d_dep is None else d_dep.cpu().numpy(), x, y, d, li, lam, lamd)


@pytest.mark.gpu
def test_noalloc_python_wrapper():
    """paper_2411_02703_gb300.loss_noalloc: caller-owned outputs, twice."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P

    ctx = P.Context()
    for (H, W, seed) in ((256, 320, 21), (64, 48, 22)):
        x, y, d, li = _inputs(H, W, seed)
        X, Y, D, LI = (torch.from_numpy(a).cuda() for a in (x, y, d, li))
        terms = torch.empty(4, device="cuda", dtype=torch.float64)
        d_img = torch.empty(3, H, W, device="cuda")
        d_dep = torch.empty(H, W, device="cuda")
        out = P.loss_noalloc(X, D, Y, LI, 0.2, 0.1, terms, d_img, d_dep)
        assert out[0] is terms and out[1] is d_img and out[2] is d_dep
        ref_terms, ref_img, ref_dep = ctx.loss(X, D, Y, LI, 0.2, 0.1)
        torch.cuda.synchronize()
        assert torch.equal(terms, ref_terms) and torch.equal(d_img, ref_img) and torch.equal(d_dep, ref_dep)
        _check_vs_oracle(terms.cpu().numpy(), d_img.cpu().numpy(), d_dep.cpu().numpy(), x, y, d, li, 0.2, 0.1)
    with pytest.raises(P.LvigsError):
        big = torch.zeros(3, 600, 700, device="cuda")
        P.loss_noalloc(big, big[0], big, big[0], 0.2, 0.1, terms)
