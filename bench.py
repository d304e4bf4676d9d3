#!/usr/bin/env python
"""Benchmark of the LVI-GS differentiable splatting hot path on GB300.

One step = every row of the hot path over one batch of keyframes: target
pyramid (a9), preprocess (a1), key expansion and sorts (a2-a4), forward
compositing (a5), fused L1 + SSIM + LiDAR-depth loss (a8), backward
compositing (a6) and the chain rule to all parameters (a7), for 8 keyframes
at mixed pyramid levels sharing 1M Gaussians (SH degree 3), replayed as one
CUDA graph.  The same work is also timed as 8 sequential plain single-view
calls, end to end through the public API with host targets, and (on the CPU)
with the FP64 oracle on a bounded sample.

Prints one JSON line (rank 0).  Under torchrun every rank runs an
independent replica of the step on its own GPU (no collective on the data
path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd train steps/s & Mpix/s (1M Gaussians, 1280x1024), batched vs plain"
BASE_TARGET_SEED = 20241105 + 100
WORKLOAD = "lidar_1000000_8v"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tile", default="auto", help="WxH, or auto (autotuned)")
    ap.add_argument("--batch-depth", type=int, default=0)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-map", action="store_true", help="skip the map-maintenance timings")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def reduce_max(x, dist=None):
    """Maximum of x over the ranks of the default process group (x itself
    without one); the tensor lives on the GPU for NCCL and on the host
    otherwise."""
    if dist is None:
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, ms_per_step_max):
    """Whole-job steps/s of `world` replicas, each timing its own steps: every
    rank completes one step per max-over-ranks step time."""
    return world * 1000.0 / ms_per_step_max


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(gpu_id)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 2070.0, "fallback"


def algorithmic_bytes(N, V, K, n_vis, M, P, loaded, pyr_px=0):
    """Bytes each phase must move (float32 = 4 B), from the step's counts."""
    prm = N * 4 * (11 + 3 * K)
    return {
        "pyramid": pyr_px * 20,
        "preprocess": prm + V * N * 16 + n_vis * 48,
        "compact": V * N * 8 + n_vis * 8,
        "depth_sort": 4 * 20 * n_vis,
        "offsets": n_vis * 12,
        "emit": n_vis * 16 + M * 8,
        "tile_sort": 2 * 20 * M,
        "ranges": M * 4,
        "composite_fwd": loaded * 52 + P * 28,
        "combine": 0,
        "loss": P * (32 + 36 + 36 + 32 + 16),
        "composite_bwd": loaded * 52 + P * 40,
        "preprocess_bwd": 2 * prm + n_vis * 52,
    }


# Kernel source file of each profiled phase: the DRAM traffic recorded from an
# ncu capture is reported only while that file is unchanged since the capture.
PHASE_SOURCE = {"composite_fwd": "composite.cu", "composite_bwd": "composite.cu", "combine": "composite.cu",
                "preprocess": "preprocess.cu", "preprocess_bwd": "preprocess.cu", "loss": "loss.cu", "adam": "map.cu"}


def recorded_traffic(phase, workload):
    """DRAM bytes per launch of the phase's kernel from profiles/dram_traffic.md
    (lines `phase kernel source_sha256 bytes_per_launch workload`), or None
    when no capture matches the current source and the workload."""
    import hashlib

    src = PHASE_SOURCE.get(phase)
    if src is None:
        return None
    try:
        with open(os.path.join(ROOT, "paper_2411_02703_gb300", "csrc", src), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        with open(os.path.join(ROOT, "profiles", "dram_traffic.md")) as f:
            for line in f:
                parts = line.strip().strip("|").split("|")
                parts = [x.strip() for x in parts]
                if len(parts) >= 5 and parts[0] == phase and parts[2] == sha and parts[4] == workload:
                    return float(parts[3])
    except OSError:
        return None
    return None


# FP32 operations charged per visited (pixel, Gaussian) pair: 20 for the
# forward compositing and 60 for the backward (each plus one exponential), the
# per-pair work of Eq. (3)-(6) and of its reverse traversal.  Visited pairs
# are counted as the sum over pixels of the last contributor's list position:
# every pair is charged in full, although most pairs of the coarse levels fail
# the 1/255 test after a few operations, so the achieved rate is an upper bound.
FLOP_PER_PAIR = {"composite_fwd": 20.0, "composite_bwd": 60.0}


def alu_flops(n_contrib_sum):
    return {k: v * n_contrib_sum for k, v in FLOP_PER_PAIR.items()}


def roofline_table(phase_ms, ab, flops, ms_step, hbm_peak, alu_peak):
    """Per phase: device ms (eager step with events per phase), algorithmic
    bytes and the fraction of the HBM peak they reach; for the compositing
    phases also the FP32 rate against the ALU peak.  Plus the whole step:
    every phase's algorithmic bytes over the graph-replayed step time."""
    phases = {}
    for k, ms in phase_ms.items():
        row = {"ms": round(ms, 4)}
        if ab.get(k):
            gbs = ab[k] / (ms / 1e3) / 1e9
            row.update(bytes=int(ab[k]), gbs=round(gbs, 1), hbm_frac=round(gbs / hbm_peak, 3))
        if k in flops:
            tf = flops[k] / (ms / 1e3) / 1e12
            row.update(tflops=round(tf, 2), alu_frac=round(tf / alu_peak, 3))
        phases[k] = row
    total = float(sum(v for k, v in ab.items() if k in phase_ms))
    gbs = total / (ms_step / 1e3) / 1e9
    step = {"bytes": int(total), "ms": round(ms_step, 4), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)}
    return step, phases


def run_ours(args):
    import torch

    import synthetic as S
    import paper_2411_02703_gb300 as P

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tile = (16, 16) if args.tile == "auto" else tuple(int(x) for x in args.tile.split("x"))
    wl = S.workload(args.workload)
    params = wl["params"]
    cams, levels = wl["cams"], wl["levels"]
    lam, lamd = wl["lam"], wl["lam_d"]
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in params.items()}
    gts = [torch.from_numpy(g).cuda() for g in wl["gts"]]
    lis = [torch.from_numpy(g).cuda() for g in wl["lidars"]]
    gts_h = [torch.from_numpy(g).pin_memory() for g in wl["gts"]]
    lis_h = [torch.from_numpy(g).pin_memory() for g in wl["lidars"]]
    lv = P.Context(tile=tile, batch_depth=args.batch_depth)
    grads = {k: torch.zeros_like(dev[k]) for k in P.PARAM_NAMES}
    N = params["means"].shape[0]
    V = len(cams)
    K = params["sh"].shape[1]
    pix = sum((c.W >> l) * (c.H >> l) for c, l in zip(cams, levels))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, dist)

    def step():
        lv.train_step_batched(dev, cams, levels, gts, lis, lam, lamd, grads=grads)

    autotune = None
    if args.tile == "auto":
        t_best, bd_best, times = lv.autotune(dev, cams, levels, gts, lis, lam, lamd, trials=3, grads=grads)
        autotune = {"chosen": f"{t_best[0]}x{t_best[1]}/{bd_best}", "ms_per_step": times}
        tile = t_best

    # warm-up (first call sizes the workspace eagerly, the second captures the graph)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    lv.sync_status()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_uuid = str(local)
    sampler = ClockSampler(gpu_uuid)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    lv.sync_status()
    ms_batched = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    stats = lv.step_stats()
    _, kernels_per_step = lv.profile_read()

    # the same keyframes all at full resolution (level 0): the heaviest mix of
    # the configuration's levels, timed the same way after its own warm-up
    full_res = None
    if any(l != 0 for l in levels):
        lv0 = [0] * V
        ctx0 = P.Context(tile=tile, batch_depth=bd_best if autotune else args.batch_depth)  # own graph, lists

        def step0():
            ctx0.train_step_batched(dev, cams, lv0, gts, lis, lam, lamd, grads=grads)
        for _ in range(3):
            step0()
        torch.cuda.synchronize()
        k0 = max(5, args.steps // 4)
        barrier()
        e0.record(stream)
        for _ in range(k0):
            step0()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms0 = max_over_ranks(e0.elapsed_time(e1) / k0)
        pix0 = sum(c.W * c.H for c in cams)
        ctx0.sync_status()
        ctx0.close()
        full_res = {"levels": lv0, "ms_per_step": round(ms0, 4), "steps_per_s": round(world * 1000.0 / ms0, 3),
                    "mpix_per_s": round(world * pix0 * 1000.0 / ms0 / 1e6, 1), "steps": k0}

    # plain path: 8 sequential single-view calls (render, loss, backward) per step,
    # with renders that do not wait on the stream (lists sized from the earlier
    # renders of the context), and with renders that wait once each to size them
    ms_plain = ms_plain_sync = None
    if not args.skip_plain:
        pgrads = {k: torch.zeros_like(dev[k]) for k in P.PARAM_NAMES}

        def plain_step(wait):
            for i, (c, l) in enumerate(zip(cams, levels)):
                g_l, d_l = gts[i], lis[i]
                for _ in range(l):
                    g_l, d_l = lv.pyramid_down(g_l, d_l)
                rgb, depth, alpha, slot = lv.render(dev, c, l, wait=wait)
                _, d_rgb, d_dep = lv.loss(rgb, depth, g_l, d_l, lam, lamd)
                lv.backward(slot, dev, d_rgb, d_dep, grads=pgrads, accumulate=i > 0)
                lv.release(slot)

        def time_plain(wait):
            for _ in range(2):
                plain_step(True)
            torch.cuda.synchronize()
            kp = max(3, args.steps // 4)
            barrier()
            e0.record(stream)
            for _ in range(kp):
                plain_step(wait)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            lv.sync_status()
            return max_over_ranks(e0.elapsed_time(e1) / kp)

        ms_plain = time_plain(False)
        ms_plain_sync = time_plain(True)

    # per-phase device time of the same step enqueued eagerly (events per phase)
    lv.profile(True)
    kprof = 5
    for _ in range(kprof):
        lv.train_step_batched(dev, cams, levels, gts, lis, lam, lamd, grads=grads, graph=False)
    torch.cuda.synchronize()
    phases, _ = lv.profile_read()
    lv.profile(False)
    phase_ms = {k: v[0] / kprof for k, v in phases.items()}  # ms per step

    # end to end through the public API: every step copies its targets in from pinned host memory
    # and reads its losses back.  Pipelined: the next step's targets are copied on a second stream
    # (stage_targets, two slots) while the current step computes, and each step's losses are copied
    # to pinned host memory behind it and read on the host while the next step runs.  Serial: the
    # copies are part of the step on its own stream and the call waits for its losses.
    loss_host = [torch.zeros((V, 4), dtype=torch.float64).pin_memory() for _ in range(2)]
    loss_ev = [torch.cuda.Event() for _ in range(2)]
    loss_seen = []

    def e2e_pipelined(k):
        lv.stage_targets(cams, gts_h, lis_h, 0)
        prev = None
        for i in range(k):
            j = i % 2
            if i + 1 < k:
                lv.stage_targets(cams, gts_h, lis_h, (i + 1) % 2)
            # the step's loss kernel writes its terms straight into pinned host memory
            lv.train_step_batched(dev, cams, levels, None, None, lam, lamd, grads=grads, staged_slot=j,
                                  losses=loss_host[j])
            loss_ev[j].record(stream)
            if prev is not None:
                loss_ev[prev].synchronize()
                loss_seen.append(float(loss_host[prev][:, 0].sum()))
            prev = j
        loss_ev[prev].synchronize()
        loss_seen.append(float(loss_host[prev][:, 0].sum()))

    def e2e_serial(k):
        for _ in range(k):
            lv.train_step_batched(dev, cams, levels, gts_h, lis_h, lam, lamd, grads=grads, host_targets=True,
                                  host_loss=True)

    ke = max(5, args.steps // 2)
    t_e2e = {}
    for name, fn in (("pipelined", e2e_pipelined), ("serial", e2e_serial)):
        fn(3)  # warm-up: sizes the staging buffers and captures the graphs
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn(ke)
        torch.cuda.synchronize()
        t_e2e[name] = max_over_ranks((time.perf_counter() - t0) / ke)
    h2d = sum(g.numel() * 4 for g in gts_h) + sum(x.numel() * 4 for x in lis_h)
    d2h = V * 4 * 8

    map_ops = None if args.skip_map else time_map_ops(P, S, lv, params, grads, cams[0], stream, peaks()[0],
                                                       peaks()[2], args.workload)

    n_vis, M, nc_sum, P_px = stats
    # instances the compositing kernels gather: bounded by M; use M (upper bound)
    # pyramid: each level-down reads rgb + depth (16 B) and writes a quarter of it
    pyr_px = sum(sum((c.W >> i) * (c.H >> i) for i in range(l)) for c, l in zip(cams, levels))
    ab = algorithmic_bytes(N, V, K, n_vis, M, P_px, M, pyr_px)
    flops = alu_flops(nc_sum)
    hbm_peak, sm_max, peak_kind = peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # FP32 FMA pipe: SMs x 128 lanes x 2 FLOP x max SM clock
    alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    dominant = max(phase_ms, key=lambda k: phase_ms[k])
    t_dom = phase_ms[dominant] / 1e3
    if dominant in flops:
        roof = {"bound": "alu", "kernel": dominant, "achieved": flops[dominant] / t_dom / 1e12,
                "peak": alu_peak, "unit": "TFLOP/s",
                "frac": flops[dominant] / t_dom / 1e12 / alu_peak, "traffic": recorded_traffic(dominant, args.workload),
                "peak_source": f"{n_sm} SM x 128 FP32 lanes x 2 x sm_max_mhz",
                "flop_per_pair": FLOP_PER_PAIR[dominant],
                "hbm_achieved_gbs": ab[dominant] / t_dom / 1e9}
    else:
        ach = ab[dominant] / t_dom / 1e9
        roof = {"bound": "hbm", "kernel": dominant, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": recorded_traffic(dominant, args.workload), "peak_source": peak_kind}
    roof["step"], roof["phases"] = roofline_table(phase_ms, ab, flops, ms_batched, hbm_peak, alu_peak)
    roof["step"]["peak_source"] = peak_kind

    steps_per_s = 1000.0 / ms_batched
    value = job_throughput(world, ms_batched)
    param_mb = N * (3 + 3 + 4 + 1 + 3 * K) * 4 / 1e6
    l2_note = (f"inputs larger than L2 ({param_mb:.0f} MB of parameters per step)" if param_mb > 129 else
               f"inputs smaller than L2 ({param_mb:.1f} MB of parameters), L2 not flushed between steps")
    metric = METRIC if args.workload == WORKLOAD else (
        f"fwd+bwd train steps/s & Mpix/s ({N} Gaussians, {cams[0].W}x{cams[0].H}, {V} views)")
    out = {
        "metric": metric,
        "value": round(value, 4),
        "unit": "train steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_batched, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded LiDAR-sweep scene; targets: the camera image of the world and a z-buffered LiDAR sweep)",
        "config": {"workload": args.workload, "gaussians": N, "views": V, "levels": levels,
                   "base_resolution": f"{cams[0].W}x{cams[0].H}", "sh_degree": int(params["sh_degree"]),
                   "tile": f"{tile[0]}x{tile[1]}", "autotune": autotune,
                   "loss": f"{1 - lam:g} L1 + {lam:g} (1-SSIM) + {lamd:g} depth L1",
                   "parallelism": f"replicas x{world}", "l2": l2_note},
        "mpix_per_s": round(world * pix * steps_per_s / 1e6, 3),
        "plain_ms_per_step": None if ms_plain is None else round(ms_plain, 4),
        "batched_vs_plain": None if ms_plain is None else round(ms_plain / ms_batched, 3),
        "plain_sync_ms_per_step": None if ms_plain_sync is None else round(ms_plain_sync, 4),
        "all_views_full_resolution": full_res,
        "batched_vs_plain_sync": None if ms_plain_sync is None else round(ms_plain_sync / ms_batched, 3),
        "e2e": {"value": round(world / t_e2e["pipelined"], 4), "unit": "train steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "copies": "each step's targets copied from pinned host memory on a second stream while the "
                          "previous step computes; each step's losses written by its loss kernel into pinned "
                          "host memory and read on the host while the next step runs",
                "losses_finite": bool(np.isfinite(loss_seen).all()) if loss_seen else None,
                "serial_value": round(world / t_e2e["serial"], 4)},
        "gpu_launches": int(kernels_per_step) * args.steps,
        "roofline": roof,
        "phases_ms": {k: round(v, 4) for k, v in phase_ms.items()},
        "counts": {"visible_pairs": n_vis, "instances": M, "contrib_sum": nc_sum, "pixels": P_px},
        "clocks": clocks,
        "map_ops": map_ops,
    }
    if rank == 0 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(wl, pix)
    lv.close()
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_expand(args):
    """The large map-expansion training step (`expand_<N>_<V>v`): every step
    appends the Gaussians of a fresh 50,000-point sweep, renders and
    differentiates V keyframes at full resolution in one batched call, and
    takes an Adam step over every parameter.  The Gaussian count grows every
    step, so the batched call runs without graph replay (it waits once to size
    its lists).  Device-resident inputs; CUDA events over the timed steps."""
    import torch

    import synthetic as S
    import paper_2411_02703_gb300 as P

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    _, n_s, v_s = args.workload.split("_")
    N, V = int(n_s), int(v_s.rstrip("v"))
    steps, warm = args.steps, max(3, args.warmup)
    params, phase = S.lidar_scene(N)
    gm = P.GaussianMap.from_params(params, capacity=N + (steps + warm + 1) * 50_000)
    gm.sh_degree = 3
    cams = S.trajectory_cameras(V, phase=phase)
    levels = [0] * V
    tg = [S.target_images(c, 500 + i) for i, c in enumerate(cams)]
    gts = [torch.from_numpy(np.ascontiguousarray(t[0])).cuda() for t in tg]
    lis = [torch.from_numpy(np.ascontiguousarray(t[1])).cuda() for t in tg]
    scans = [S.fresh_scan(50_000, step=i) for i in range(steps + warm)]
    scans = [(torch.from_numpy(p).cuda(), torch.from_numpy(c).cuda()) for p, c in scans]
    tile = (16, 16) if args.tile == "auto" else tuple(int(x) for x in args.tile.split("x"))
    lv = P.Context(tile=tile, batch_depth=args.batch_depth)

    def step(i):
        gm.append(lv, scans[i][0], scans[i][1])
        lv.train_step_batched(gm.params(), cams, levels, gts, lis, 0.2, 0.1, grads=gm.grads(), graph=False)
        gm.adam_step()

    for i in range(warm):
        step(i)
    torch.cuda.synchronize()
    lv.sync_status()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = gm.n
    e0.record(stream)
    for i in range(warm, warm + steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    lv.sync_status()
    ms = e0.elapsed_time(e1) / steps
    pix = V * cams[0].W * cams[0].H
    out = {"metric": "map-expansion train steps/s (3M + 50k Gaussians per step, 16 views 1280x1024, + Adam)",
           "value": round(world * 1000.0 / ms, 4), "unit": "train steps/s", "n_gpus": world, "steps": steps,
           "warmup": warm, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded LiDAR-sweep scene, fresh sweeps, "
                                                        "targets from the world)",
           "config": {"workload": args.workload, "gaussians_start": N, "gaussians_end": gm.n,
                      "appended_per_step": (gm.n - n0) // steps, "views": V, "levels": levels,
                      "tile": f"{tile[0]}x{tile[1]}", "loss": "0.8 L1 + 0.2 (1-SSIM) + 0.1 depth L1",
                      "optimiser": "Adam", "parallelism": f"replicas x{world}"},
           "mpix_per_s": round(world * pix * 1000.0 / ms / 1e6, 3)}
    lv.close()
    if rank == 0:
        print(json.dumps(out))


def run_mapping(args):
    """One keyframe of the mapping thread (`mapping_<W>x<H>`): the map starts
    empty, the keyframe's colourised LiDAR sweep is integrated, and the mapping
    driver optimises it for 105 iterations (coarse to fine over levels 2, 1, 0,
    SH degree raised every 35 iterations), the iteration count the paper
    reports for one keyframe to reach photo-realistic quality.  Reports the
    driver's iterations per second (wall clock, every step synchronised by the
    driver's loss read-back) and the loss and full-resolution PSNR along the
    way."""
    import torch

    import synthetic as S
    import paper_2411_02703_gb300 as P

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    W, H = (int(x) for x in args.workload.split("_")[1].split("x"))
    lo, hi, phase = S.world()
    cam = S.trajectory_cameras(1, phase=phase, W=W, H=H, f=860.0 * W / 1280.0)[0]
    gt, lidar = S.target_images(cam, BASE_TARGET_SEED)
    pts = S.lidar_sweep(S.camera_centre(cam), lo, hi)
    col = S._texture(pts)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    gt_d, li_d = t(gt), t(lidar)
    iters = 105

    marks = (0, 15, 35, 70, 105)

    def run(measure_psnr):
        lv = P.Context(tile=(16, 16))
        gm = P.GaussianMap(capacity=pts.shape[0] + 1024, sh_stride_k=16)
        mp = P.Mapper(lv, gm, P.MappingSchedule(max_iters=iters, top_level=2, sh_interval=35, views_per_step=1),
                      delay=0)
        kf = P.Keyframe(cam=cam, gt_rgb=gt_d, lidar=li_d, points=t(pts), colours=t(col))
        psnr = {}

        def measure(k):
            # PSNR at full resolution over the whole image and over the pixels the
            # map covers (alpha >= 0.5; the sky is never covered by LiDAR points)
            rgb, _, alpha, slot = lv.render(gm.params(), cam, 0)
            lv.release(slot)
            err = ((rgb - gt_d) ** 2).mean(0)
            cov = alpha >= 0.5
            db = lambda m: round(10.0 * math.log10(1.0 / max(m, 1e-12)), 3)
            psnr[str(k)] = {"all": db(float(err.mean())), "covered": db(float(err[cov].mean())) if bool(cov.any())
                            else None, "covered_frac": round(float(cov.float().mean()), 4)}

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mp.add_keyframe(kf)
        if measure_psnr:
            mp.flush()
            measure(0)
        n = 0
        while mp.step() is not None:
            n += 1
            if measure_psnr and n in marks:
                measure(n)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        losses = [h[3][0] for h in mp.history]
        curve = {str(k): round(losses[k - 1], 5) for k in marks if 0 < k <= len(losses)}
        out = dict(wall_s=wall, n=n, gaussians=gm.n, losses=curve, psnr=psnr, levels=[h[2][0] for h in mp.history])
        lv.close()
        return out

    run(False)  # warm-up: builds and captures
    res = run(False)
    res["psnr"] = run(True)["psnr"]
    value = res["n"] / res["wall_s"]
    lv_first = res["levels"].index(0) if 0 in res["levels"] else None
    out = {"metric": f"mapping iterations/s (one {W}x{H} keyframe, {iters} iterations, from an empty map)",
           "value": round(world * value, 3), "unit": "iterations/s", "n_gpus": world, "steps": res["n"],
           "warmup": 1, "ms_per_step": round(1000.0 * res["wall_s"] / res["n"], 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded LiDAR-sweep world; the keyframe's own sweep and camera image)",
           "config": {"workload": args.workload, "gaussians": res["gaussians"], "iterations": iters,
                      "schedule": "levels 2,1,0 over thirds; SH degree +1 every 35 iterations",
                      "first_full_resolution_iteration": lv_first, "parallelism": f"replicas x{world}"},
           "keyframe_s": round(res["wall_s"], 4), "loss_at_iteration": res["losses"],
           "psnr_full_resolution_db_at_iteration": res["psnr"]}
    if rank == 0:
        print(json.dumps(out))


def time_map_ops(P, S, lv, params, grads, cam, stream, hbm_peak, peak_kind, workload):
    """Map maintenance on the bench's map: the Adam step over every parameter
    (HBM-bound: read parameter, gradient and both moments, write parameter and
    moments, 28 B per float), expansion by one 50,000-point sweep (with and
    without the V_p filter of the first keyframe), and opacity pruning."""
    import torch

    N = params["means"].shape[0]
    K = params["sh"].shape[1]
    gm = P.GaussianMap.from_params(params, capacity=N + 120_000)
    g = gm.grads()
    for k in P.PARAM_NAMES:
        g[k].copy_(grads[k])
    for _ in range(3):
        gm.adam_step(zero_grads=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ka = 20
    e0.record(stream)
    for _ in range(ka):
        gm.adam_step(zero_grads=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_adam = e0.elapsed_time(e1) / ka
    adam_bytes = N * (11 + 3 * K) * 28
    pts, col = S.fresh_scan(50_000, step=0)
    pts, col = torch.from_numpy(pts).cuda(), torch.from_numpy(col).cuda()
    n0 = gm.n

    def timed_append(alpha=None, cam=None):
        ts = []
        for _ in range(4):
            gm.n = n0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            added = gm.append(lv, pts, col, cam, 0, alpha)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts[1:])), added

    ms_app, added = timed_append()
    gm.n = n0
    _, _, alpha, slot = lv.render(gm.params(), cam, 0)
    lv.release(slot)
    ms_app_f, added_f = timed_append(alpha, cam)
    # pruning changes the map: every run starts from a saved copy (restored
    # outside the timed region); the first run also sizes the scratch arena
    n1 = gm.n
    saved = [{k: b[k][:n1].clone() for k in P.PARAM_NAMES} for b in (gm._p, gm._m, gm._v)]
    ts = []
    for _ in range(4):
        gm.n = n1
        for b, sv in zip((gm._p, gm._m, gm._v), saved):
            for k in P.PARAM_NAMES:
                b[k][:n1].copy_(sv[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        removed = gm.prune(lv, 0.005)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    ms_prune = float(np.median(ts[1:]))
    del saved
    return {"adam": {"ms": round(ms_adam, 4), "bytes": adam_bytes, "traffic": recorded_traffic("adam", workload),
                     "achieved_gbs": round(adam_bytes / ms_adam / 1e6, 1),
                     "frac": round(adam_bytes / ms_adam / 1e6 / hbm_peak, 3), "peak": hbm_peak,
                     "peak_source": peak_kind, "floats": N * (11 + 3 * K)},
            "append_50k_sweep_ms": round(ms_app, 3), "appended": added,
            "append_50k_filtered_ms": None if ms_app_f is None else round(ms_app_f, 3), "appended_filtered": added_f,
            "prune_ms": round(ms_prune, 3), "pruned": removed, "gaussians": N}


def cpu_baseline(wl, pix_total, budget_s=25.0):
    """The oracle as it stands, on the host cores, over a bounded sample of the step.

    Sample: the views of the step in order, each a full oracle pass (pyramid,
    render, loss, backward) at its level, until about `budget_s` of CPU work;
    the step time is extrapolated by pixel count.
    """
    import oracle as O

    t0 = time.perf_counter()
    done_px = 0
    done = []
    for i, (c, l) in enumerate(zip(wl["cams"], wl["levels"])):
        cam = O.Camera(c.R, c.t, c.fx, c.fy, c.cx, c.cy, c.W, c.H)
        O.train_step(wl["params"], [cam], [l], [wl["gts"][i]], [wl["lidars"][i]], wl["lam"], wl["lam_d"])
        done_px += (c.W >> l) * (c.H >> l)
        done.append(f"view {i} (level {l})")
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    step_s = t * pix_total / done_px
    cores = O.num_threads()
    # the same on one core: the first view of the step, extrapolated by pixel count
    one = None
    if cores > 1:
        c, l = wl["cams"][0], wl["levels"][0]
        cam = O.Camera(c.R, c.t, c.fx, c.fy, c.cx, c.cy, c.W, c.H)
        O.set_num_threads(1)
        try:
            t1 = time.perf_counter()
            O.train_step(wl["params"], [cam], [l], [wl["gts"][0]], [wl["lidars"][0]], wl["lam"], wl["lam_d"])
            t1 = time.perf_counter() - t1
        finally:
            O.set_num_threads(cores)
        one = {"value": round(1.0 / (t1 * pix_total / ((c.W >> l) * (c.H >> l))), 6), "cores": 1,
               "sample": f"view 0 (level {l}), {t1:.1f} s, extrapolated by pixel count"}
    return {"value": round(1.0 / step_s, 6), "unit": "train steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{', '.join(done)} of the {len(wl['cams'])}-view step, {t:.1f} s, extrapolated by pixel count",
            "single_core": one}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import synthetic as S

    wl = S.workload(args.workload)
    pix = sum((c.W >> l) * (c.H >> l) for c, l in zip(wl["cams"], wl["levels"]))
    vals = []
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_baseline(wl, pix, budget_s=5.0)
    cb = None
    for _ in range(max(1, min(args.steps, 3))):
        cb = cpu_baseline(wl, pix, budget_s=20.0)
        vals.append(cb["value"])
    v = float(np.median(vals))
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "train steps/s", "n_gpus": 1,
           "steps": len(vals), "warmup": min(args.warmup, 1), "ms_per_step": 1000.0 / v,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded LiDAR-sweep scene; targets: the camera image of the world and a z-buffered LiDAR sweep)",
           "config": {"workload": args.workload, "implementation": "FP64 CPU oracle (oracle/)"},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "train steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload.startswith("expand_"):
        run_expand(a)
    elif a.workload.startswith("mapping_"):
        run_mapping(a)
    else:
        run_ours(a)
