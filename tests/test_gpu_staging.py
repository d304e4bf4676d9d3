"""Targets staged from pinned host memory on a second stream (double-buffered
slots) give the same step as targets copied inside the step: images and losses
bit-identical, gradients equal up to the atomics' summation order, including
when the two slots alternate between different target sets."""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_02703_gb300 as P

    params, phase = S.lidar_scene(40_000)
    cams = S.trajectory_cameras(3, phase=phase, W=320, H=256, f=215.0)
    levels = [0, 1, 2]
    dp = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
          for k, v in params.items()}
    sets = []
    for seed in (300, 400):
        tg = [S.target_images(c, seed + i) for i, c in enumerate(cams)]
        sets.append(([torch.from_numpy(np.ascontiguousarray(x[0], np.float32)).pin_memory() for x in tg],
                     [torch.from_numpy(np.ascontiguousarray(x[1], np.float32)).pin_memory() for x in tg]))
    return P, dp, cams, levels, sets


def outs_for(cams, levels):
    return [(torch.empty(3, c.H >> l, c.W >> l, device="cuda"), torch.empty(c.H >> l, c.W >> l, device="cuda"),
             torch.empty(c.H >> l, c.W >> l, device="cuda")) for c, l in zip(cams, levels)]


def grads_close(a, b):
    for k in a:
        x, y = a[k].cpu().numpy(), b[k].cpu().numpy()
        assert np.abs(x - y).max() <= 1e-4 * np.abs(y).max() + 1e-12, k


def test_staged_equals_copied_in_step(setup):
    P, dp, cams, levels, sets = setup
    lv = P.Context(tile=(16, 16))
    # reference per target set: copies inside the step
    ref = []
    for gts, lis in sets:
        o = outs_for(cams, levels)
        for _ in range(2):
            losses, grads = lv.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, host_targets=True,
                                                  host_loss=True, outputs=o)
        ref.append((losses.clone(), {k: v.clone() for k, v in grads.items()}, [tuple(t.clone() for t in x) for x in o]))
    # pipelined: step i uses slot i % 2 and target set i % 2; the next step's copy is in flight
    n = 6
    lv.stage_targets(cams, *sets[0], 0)
    for i in range(n):
        if i + 1 < n:
            lv.stage_targets(cams, *sets[(i + 1) % 2], (i + 1) % 2)
        o = outs_for(cams, levels)
        losses, grads = lv.train_step_batched(dp, cams, levels, None, None, 0.2, 0.1, host_loss=True,
                                              staged_slot=i % 2, outputs=o)
        rl, rg, ro = ref[i % 2]
        assert torch.equal(losses, rl), i
        for a, b in zip(o, ro):
            for x, y in zip(a, b):
                assert torch.equal(x, y), i
        grads_close(grads, rg)
    lv.close()


def test_staging_errors(setup):
    P, dp, cams, levels, sets = setup
    lv = P.Context(tile=(16, 16))
    gts, lis = sets[0]
    # a slot that holds nothing, and a slot that holds other sizes
    with pytest.raises(P.LvigsError):
        lv.train_step_batched(dp, cams, levels, None, None, 0.2, 0.1, host_loss=True, staged_slot=1)
    lv.stage_targets(cams[:2], gts[:2], lis[:2], 0)
    with pytest.raises(P.LvigsError):
        lv.train_step_batched(dp, cams, levels, None, None, 0.2, 0.1, host_loss=True, staged_slot=0)
    with pytest.raises(ValueError):  # device tensors are not host staging sources
        lv.stage_targets(cams, [g.cuda() for g in gts], None, 0)
    with pytest.raises(P.LvigsError):
        lv.stage_targets(cams, gts, lis, 2)
    torch.cuda.synchronize()
    lv.close()


def test_async_host_losses(setup):
    """Losses written by the step's kernels into pinned host memory (no wait in
    the call) equal the synchronous host read-back."""
    P, dp, cams, levels, sets = setup
    lv = P.Context(tile=(16, 16))
    gts, lis = sets[0]
    for _ in range(2):
        ref, _ = lv.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, host_targets=True, host_loss=True)
    host = torch.zeros((len(cams), 4), dtype=torch.float64).pin_memory()
    ev = torch.cuda.Event()
    for _ in range(2):
        lv.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, host_targets=True, losses=host)
        ev.record(torch.cuda.current_stream())
        ev.synchronize()
        assert torch.equal(host, ref)
    with pytest.raises(ValueError):  # pageable host memory cannot be written by a kernel
        lv.train_step_batched(dp, cams, levels, gts, lis, 0.2, 0.1, host_targets=True,
                              losses=torch.zeros((len(cams), 4), dtype=torch.float64))
    torch.cuda.synchronize()
    lv.close()
