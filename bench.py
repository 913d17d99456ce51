#!/usr/bin/env python3
"""Throughput of the improved SPCN normalisation on synthetic H&E slides.

One step = the whole per-pixel path on one source image: basis estimation
(sampling, i0, sparse NMF, stain ordering, sampled P99) followed by the
two-pass normalisation (exact non-white P99 per stain, then reconstruction),
against a target whose statistics are computed once before timing (one target
serves every source).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload wsi|tile]
    python bench.py --impl reference ...     # the FP64 oracle on host cores

Workloads (synthetic; the paper's TCGA slides are not available):
  wsi   100000 x 80000 source (8 Gpx, 24 GB in + 24 GB out resident in HBM),
        basis from 200 patches of 256 x 256, 2048 x 2048 target.
  tile  8192 x 8192 source, basis from a 1% SplitMix64 sample, 2048 x 2048 target.
  batch 256 uneven tiles (32 slides x 8, sides log-uniform in [256, 4096]),
        per-slide statistics, one target: the batched persistent launch
        (autotuned, CUDA-graph replays) against 256 sequential plain calls.
  grad  forward + backward of the float form, 64 x 3 x 256 x 256.

Under torchrun (N > 1) every rank normalises its own slide (replicas: the
method has no exchange step that one GPU per slide would need); the value is
the pixels of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "wsi": dict(width=100000, height=80000, sample_mode="patches", n_patches=200,
                patch_size=256, sample_rate=0.01, tgt=2048),
    "tile": dict(width=8192, height=8192, sample_mode="hash", n_patches=200,
                 patch_size=256, sample_rate=0.01, tgt=2048),
    # differentiable form: a batch of float32 CHW images, forward + backward
    "grad": dict(batch=64, height=256, width=256, tgt=256),
    # batching: 32 slides x 8 tiles, sides log-uniform in [256, 4096], one target
    "batch": dict(slides=32, per_slide=8, side_lo=256, side_hi=4096, tgt=2048,
                  slide_sample=2048, sample_rate=0.01),
    # stain separation: basis estimation + FP32 densities of every pixel of the slide
    "separation": dict(width=100000, height=80000, sample_mode="patches", n_patches=200,
                       patch_size=256, sample_rate=0.01),
    "separation_tile": dict(width=8192, height=8192, sample_mode="hash", n_patches=200,
                            patch_size=256, sample_rate=0.01),
}
METRIC = "gigapixels/s end-to-end normalize (% of HBM roofline); batched & fwd+bwd vs plain"
# algorithmic bytes per pixel of each timed kernel (reads + writes of the image)
KERNEL_BYTES = {"pass1": 3, "pass2": 6, "density": 11}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def read_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu
    summary line 'TRAFFIC <kernel> <workload> <bytes>' under profiles/."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    pat = re.compile(rf"^TRAFFIC\s+{kernel}\s+{workload}\s+([0-9.eE+]+)\s*$")
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, name)) as f:
            for ln in f:
                m = pat.match(ln.strip())
                if m:
                    return float(m.group(1))
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = f"/tmp/spcn_clocks_{os.getpid()}.csv"

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.fh.close()
        except Exception:
            pass

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for ln in f:
                    parts = [x.strip() for x in ln.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- oracle arm
def oracle_sample_run(src_np, tgt_np, wl, seed):
    """The oracle's full path on a bounded crop: basis + exact P99 of source
    and target, then normalisation.  Returns seconds."""
    from oracle import spcn_oracle as O
    h, w, _ = src_np.shape
    if wl["sample_mode"] == "patches":
        # the slide's patch density (200 patches of 256^2 over 8 Gpx) scaled to the crop
        p = O.Params(sample_mode="patches", n_patches=max(1, min(8, int(200 * h * w / 8e9) + 1)),
                     patch_size=min(256, h, w), seed=seed)
    else:
        p = O.Params(sample_mode="hash", sample_rate=wl["sample_rate"], seed=seed)
    t0 = time.perf_counter()
    s_st = O.full_stats(src_np, p)
    t_st = O.full_stats(tgt_np, O.Params(sample_mode="hash", sample_rate=wl["sample_rate"]))
    O.normalize(src_np, s_st, t_st)
    return time.perf_counter() - t0, p


def crop_for_oracle(src, side):
    import numpy as np
    h, w = src.shape[0], src.shape[1]
    y0 = max(0, h // 2 - side // 2)
    x0 = max(0, w // 2 - side // 2)
    return np.ascontiguousarray(src[y0:y0 + side, x0:x0 + side].cpu().numpy())


def normalize_workload_desc(name, wl):
    """The normalisation workload as both arms name it in their config."""
    return (f"{name}: {wl['width']}x{wl['height']} uint8 RGB source, "
            f"{wl['tgt']}x{wl['tgt']} target, basis from "
            + (f"{wl['n_patches']} patches of {wl['patch_size']}^2"
               if wl["sample_mode"] == "patches" else f"{wl['sample_rate']:.0%} hash sample"))


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import numpy as np
    from paper_1901_03088_b300 import synth
    wl = WORKLOADS[args.workload]
    side = args.oracle_side
    src = synth.make_image(side, side, 1000, blobs=True)
    tgt = synth.make_image(512, 512, 1, blobs=True)
    for _ in range(args.warmup):
        oracle_sample_run(src, tgt, wl, 0)
    times = []
    p = None
    for _ in range(args.steps):
        t, p = oracle_sample_run(src, tgt, wl, 0)
        times.append(t)
    ms = 1e3 * statistics.mean(times)
    gpx = side * side / (ms / 1e3) / 1e9
    sample = (f"{side}x{side} synthetic crop (blobs), full oracle path per step: basis "
              f"({p.sample_mode}), exact P99 of source and a 512x512 target, normalisation")
    line = {
        "impl": "reference", "metric": METRIC, "value": gpx, "unit": "Gpx/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": (normalize_workload_desc(args.workload, wl) if "tgt" in wl
                                else args.workload), "oracle_crop": f"{side}x{side}",
                   "l2": "not applicable: the oracle runs on the host cores"},
        "cpu_baseline": {"value": gpx, "unit": "Gpx/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gpx, "unit": "Gpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- CUDA arm
def run_grad(args, world, rank, local):
    """Forward + hand-written backward of the differentiable normalisation on a
    batch of 64 float32 3x256x256 images, against forward only."""
    import numpy as np
    import torch
    from paper_1901_03088_b300 import build
    build.build()
    from paper_1901_03088_b300 import spcn, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS["grad"]
    B, H, W = wl["batch"], wl["height"], wl["width"]
    xs, stats = [], []
    for b in range(B):
        img = synth.make_image(H, W, 1000 + 64 * rank + b, as_float=True)
        xs.append(img.transpose(2, 0, 1))
        stats.append(spcn.Stats.from_values(np.float32(synth.stain_basis(1000 + b)),
                                            [252.0, 249.0, 253.0], [2.3, 2.1]))
    x = torch.from_numpy(np.ascontiguousarray(np.stack(xs)).astype(np.float32)).to(dev)
    tgt = spcn.Stats.from_values(np.float32(synth.stain_basis(1)), [255.0, 254.0, 253.0], [2.4, 2.2])
    Wt = torch.tensor(np.array(tgt.basis, np.float32), device=dev, requires_grad=True)
    gy = torch.randn_like(x)
    stats = spcn.stats_array(stats)
    ctx = spcn.Context(local)
    npx = B * H * W

    # Both steps are captured once in CUDA graphs (the binding launches on the
    # current stream, no allocation or synchronisation inside), so the timed
    # replays measure the device path, not Python and autograd overhead.
    xg = x.clone().requires_grad_(True)

    def fwd_eager():
        with torch.no_grad():
            return spcn.normalize_f32(ctx, x, Wt, stats, tgt)

    def fwdbwd_eager():
        xg.grad = None
        Wt.grad = None
        spcn.normalize_f32(ctx, xg, Wt, stats, tgt).backward(gy)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            fwd_eager()
            fwdbwd_eager()
    torch.cuda.current_stream().wait_stream(side)
    g_f, g_fb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_f):
        fwd_eager()
    xg.grad = None
    Wt.grad = None
    with torch.cuda.graph(g_fb):
        spcn.normalize_f32(ctx, xg, Wt, stats, tgt).backward(gy)
    fwd, fwdbwd = g_f.replay, g_fb.replay

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ctx.launches
        barrier(world)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev), ctx.launches - l0

    with ClockSampler(local) as clk:
        ms_f, _ = timed(fwd)
        ms_fb, _ = timed(fwdbwd)
    # kernel-level times (eager launches, CUDA events around each kernel)
    ctx.kernel_timing(True)
    l0 = ctx.launches
    for _ in range(args.steps):
        fwdbwd_eager()
    torch.cuda.synchronize()
    launches = (ctx.launches - l0) // args.steps * args.steps
    k_f, n_f = ctx.kernel_times("f32_fwd")
    k_b, n_b = ctx.kernel_times("f32_bwd")
    ctx.kernel_timing(False)
    peak, peak_kind = read_peaks()
    bytes_fb = 60 * npx          # forward 12 in + 12 out, backward 12 (x) + 12 (gy) + 12 (gx)
    kf_ms, kb_ms = k_f / max(1, n_f), k_b / max(1, n_b)
    line = {
        "metric": METRIC, "value": world * npx / (ms_fb / 1e3) / 1e9, "unit": "Gpx/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fb,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"grad: forward + backward, batch {B} x 3 x {H} x {W} float32",
                   "timing": "CUDA-graph replays of the autograd step",
                   "forward_only_gpx_s": world * npx / (ms_f / 1e3) / 1e9,
                   "forward_only_ms": ms_f, "fwd_bwd_over_fwd_time": ms_fb / ms_f,
                   "kernel_ms": {"forward": round(kf_ms, 4), "backward": round(kb_ms, 4)},
                   "l2": f"inputs {12 * npx / 1e6:.0f} MB (x) + {12 * npx / 1e6:.0f} MB (gy); "
                         "no flush"},
        "roofline": {"bound": "hbm", "kernel": "backward", "achieved": 36 * npx / (kb_ms / 1e3) / 1e9,
                     "peak": peak, "unit": "GB/s",
                     "frac": 36 * npx / (kb_ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind,
                     "bytes_per_px": 36, "traffic": None},
        "roofline_step": {"bytes_per_px": 60, "achieved": bytes_fb / (ms_fb / 1e3) / 1e9,
                          "frac": bytes_fb / (ms_fb / 1e3) / 1e9 / peak},
        "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_batch(args, world, rank, local):
    """256 uneven tiles from 32 slides (own source statistics each), one
    target: one cooperative persistent launch per step (schedule from the
    library's autotuner, replayed from a CUDA graph), against the same tiles
    normalised by 256 sequential spcn_normalize calls."""
    import numpy as np
    import torch
    from paper_1901_03088_b300 import build
    build.build()
    from paper_1901_03088_b300 import spcn, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS["batch"]
    t0 = time.time()
    n_slides = args.slides or wl["slides"]
    layout = synth.batch_layout(n_slides, wl["per_slide"], wl["side_lo"], wl["side_hi"],
                                seed=3 + rank)
    tiles = [synth.make_image_torch(h, w, 3000 + 256 * rank + k,
                                    W=synth.stain_basis(2000 + s), device=dev, blobs=True)
             for k, (s, h, w) in enumerate(layout)]
    npx = sum(h * w for (_, h, w) in layout)
    ctx = spcn.Context(local)
    p = spcn.params(sample_mode="hash", sample_rate=wl["sample_rate"], seed=0)
    slide_st = []
    for s in range(n_slides):
        smp = synth.make_image_torch(wl["slide_sample"], wl["slide_sample"], 2100 + s,
                                     W=synth.stain_basis(2000 + s), device=dev, blobs=True)
        slide_st.append(ctx.estimate_basis(smp, p))
        del smp
    stats = [slide_st[s] for (s, _, _) in layout]
    tgt_img = synth.make_image_torch(wl["tgt"], wl["tgt"], 1, device=dev, blobs=True)
    t_st = ctx.estimate_basis(tgt_img, p)
    t_st.p99[0], t_st.p99[1] = ctx.stain_percentile(tgt_img, t_st, p)
    outs = [torch.empty_like(t) for t in tiles]
    ref = [torch.empty_like(t) for t in tiles]
    torch.cuda.synchronize()
    gen_s = time.time() - t0

    # sequential plain calls (the single-image path, one tile at a time)
    def seq_step():
        for t, st, o in zip(tiles, stats, ref):
            ctx.normalize(t, st, t_st, p, out=o)

    # the batch: autotune, then capture one run into a CUDA graph
    t1 = time.perf_counter()
    b = spcn.Batch(ctx, tiles, stats, t_st, outs, p)
    create_ms = 1e3 * (time.perf_counter() - t1)
    t1 = time.perf_counter()
    trials = [] if args.no_tune else b.tune(reps=3)
    tune_s = time.perf_counter() - t1
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b.run(stream=side)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)

    with ClockSampler(local) as clk:
        ms = timed(graph.replay, args.steps)
        ms_seq = timed(seq_step, max(1, min(args.steps, 5)))
    clocks = clk.summary()
    identical = all(torch.equal(a, c) for a, c in zip(outs, ref))
    p99, status, fallback = b.results(fallback=True)

    # kernel time of the persistent launch (eager runs, CUDA events around it)
    ctx.kernel_timing(True)
    l0 = ctx.launches
    for _ in range(args.steps):
        b.run()
    torch.cuda.synchronize()
    per_run = (ctx.launches - l0) // args.steps
    k_ms, k_n = ctx.kernel_times("batch")
    ctx.kernel_timing(False)
    k_ms /= max(1, k_n)
    peak, peak_kind = read_peaks()
    achieved = 9 * npx / (k_ms / 1e3) / 1e9

    # end to end: host tiles copied in, the batch run, outputs copied out
    e2e = None
    if not args.no_e2e:
        try:
            h_in = [torch.empty(t.shape, dtype=torch.uint8, pin_memory=True) for t in tiles]
            h_out = [torch.empty(t.shape, dtype=torch.uint8, pin_memory=True) for t in tiles]
            for h, t in zip(h_in, tiles):
                h.copy_(t)

            def e2e_step():
                for h, t in zip(h_in, tiles):
                    t.copy_(h, non_blocking=True)
                b.run()
                for h, o in zip(h_out, outs):
                    h.copy_(o, non_blocking=True)
                torch.cuda.current_stream().synchronize()

            e2e_step()
            steps = max(1, min(args.steps, args.e2e_steps))
            t2 = time.perf_counter()
            for _ in range(steps):
                e2e_step()
            dt = (time.perf_counter() - t2) / steps
            e2e = {"value": npx / dt / 1e9, "unit": "Gpx/s", "h2d_bytes_per_step": 3 * npx,
                   "d2h_bytes_per_step": 3 * npx, "steps": steps, "ms_per_step": 1e3 * dt}
        except Exception as e:
            e2e = {"value": None, "unit": "Gpx/s", "unavailable": f"{e}"[:200]}

    cpu = None
    if rank == 0 and not args.no_cpu:
        from oracle import spcn_oracle as O
        crop = crop_for_oracle(tiles[0], min(1024, tiles[0].shape[0], tiles[0].shape[1]))
        W = np.asarray(np.array(stats[0].basis, np.float32), np.float64)
        i0 = np.asarray(np.array(stats[0].i0[:], np.float32), np.float64)
        Wt = np.asarray(np.array(t_st.basis, np.float32), np.float64)
        i0t = np.asarray(np.array(t_st.i0[:], np.float32), np.float64)
        t2 = time.perf_counter()
        ps = O.stain_percentile(crop, W, i0)
        O.to_uint8(O.normalize_float(crop, W, i0, ps, Wt, i0t, np.array(t_st.p99[:])))
        dt = time.perf_counter() - t2
        cpu = {"value": crop.shape[0] * crop.shape[1] / dt / 1e9, "unit": "Gpx/s", "cores": 1,
               "kind": "oracle",
               "sample": f"{crop.shape[0]}x{crop.shape[1]} crop of tile 0: oracle exact P99 + "
                         f"normalisation with the slide's statistics ({dt:.1f} s, numpy FP64)"}

    best = b.config
    line = {
        "metric": METRIC, "value": world * npx / (ms / 1e3) / 1e9, "unit": "Gpx/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": f"batch: {len(tiles)} uint8 RGB tiles from {n_slides} slides, sides "
                        f"log-uniform in [{wl['side_lo']}, {wl['side_hi']}], {npx / 1e6:.1f} Mpx, "
                        f"per-slide statistics (1% hash sample of a {wl['slide_sample']}^2 slide "
                        f"sample), {wl['tgt']}x{wl['tgt']} target",
            "pixels_per_step": npx, "parallelism": f"replicas x{world}",
            "timing": "CUDA-graph replays of one cooperative persistent launch",
            "l2": f"inputs ({3 * npx / 1e9:.2f} GB) larger than L2 (126 MB); no flush",
            "schedule": best, "tuner_trials": trials, "tune_s": round(tune_s, 2),
            "create_ms": round(create_ms, 2), "generate_s": round(gen_s, 2),
            "sequential_ms_per_step": ms_seq,
            "sequential_gpx_s": world * npx / (ms_seq / 1e3) / 1e9,
            "speedup_vs_sequential": ms_seq / ms,
            "outputs_identical_to_sequential": identical,
            "tiles_no_tissue": sum(1 for x in status if x != 0),
            "tiles_exact_fallback": sum(fallback),
            "kernel_ms": round(k_ms, 4),
        },
        "roofline": {"bound": "hbm", "kernel": "k_batch", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "bytes_per_px": 9, "traffic": read_traffic("batch", "batch")},
        "roofline_step": {"bytes_per_px": 9, "achieved": 9 * npx / (ms / 1e3) / 1e9,
                          "frac": 9 * npx / (ms / 1e3) / 1e9 / peak},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": per_run * args.steps, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    b.close()
    ctx.close()
    return 0


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    if args.workload == "grad":
        return run_grad(args, world, rank, local)
    if args.workload == "batch":
        return run_batch(args, world, rank, local)
    if args.workload in ("separation", "separation_tile"):
        return run_separation(args, world, rank, local)
    from paper_1901_03088_b300 import build
    build.build()
    from paper_1901_03088_b300 import spcn, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    Wd, Hd = wl["width"], wl["height"]
    npx = Wd * Hd
    t0 = time.time()
    src = synth.make_image_torch(Hd, Wd, 1000 + rank, device=dev, blobs=True)
    tgt = synth.make_image_torch(wl["tgt"], wl["tgt"], 1, device=dev, blobs=True)
    out = torch.empty_like(src)
    torch.cuda.synchronize()
    gen_s = time.time() - t0

    ctx = spcn.Context(local)
    flags = variant_flags(spcn, args.flags)
    sampled = bool(flags & spcn.FLAG_P99_SAMPLED)
    p = spcn.params(sample_mode=wl["sample_mode"], n_patches=wl["n_patches"],
                    patch_size=wl["patch_size"], sample_rate=wl["sample_rate"], seed=0,
                    flags=flags)
    pt = spcn.params(sample_mode="hash", sample_rate=wl["sample_rate"], seed=1,
                     flags=flags & ~spcn.FLAG_P99_PATCH_MEDIAN)
    # target statistics, computed once for every source (§3.2 item 6); the
    # sampled variant keeps the target's sampled percentile too
    t1 = time.perf_counter()
    t_st = ctx.estimate_basis(tgt, pt)
    if not sampled:
        t_st.p99[0], t_st.p99[1] = ctx.stain_percentile(tgt, t_st, pt)
    tgt_ms = 1e3 * (time.perf_counter() - t1)

    def step():
        # basis estimation + both passes, statistics kept on the device
        ctx.normalize_estimated(src, t_st, p, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ctx.kernel_timing(True)
    launches0 = ctx.launches
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = ctx.launches - launches0
    ms_local = evs[0].elapsed_time(evs[-1]) / args.steps
    per_step = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps))
    ms = max_over_ranks(ms_local, world, dev)
    ktimes = {k: ctx.kernel_times(k) for k in ("pass1", "select", "pass2")}
    ctx.kernel_timing(False)
    clocks = clk.summary()

    # the statistics of one step (bench output is not a parity test)
    _, s_st = ctx.normalize_estimated(src, t_st, p, out=out, return_stats=True)
    p99 = (s_st.p99[0], s_st.p99[1])

    # roofline of the dominant kernel
    dom = max(("pass1", "pass2"), key=lambda k: ktimes[k][0])
    dom_ms = ktimes[dom][0] / max(1, ktimes[dom][1])
    achieved = KERNEL_BYTES[dom] * npx / (dom_ms / 1e3) / 1e9
    peak, peak_kind = read_peaks()
    traffic = read_traffic(dom, args.workload)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, ctx, spcn, src, t_st, p, dev, npx)

    cpu = None
    if rank == 0 and not args.no_cpu and not flags:
        cpu = cpu_baseline(src, tgt, wl, args)

    value = world * npx / (ms / 1e3) / 1e9
    step_bytes = 6 if sampled else 9   # one pass (read + write) or two (+ the pass-1 read)
    line = {
        "metric": METRIC, "value": value, "unit": "Gpx/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": normalize_workload_desc(args.workload, wl),
            "pixels_per_step": npx, "parallelism": f"replicas x{world}",
            "l2": f"inputs ({3 * npx / 1e9:.1f} GB) larger than L2 (126 MB); no flush",
            "target_stats_ms_once": round(tgt_ms, 3), "generate_s": round(gen_s, 2),
            "ms_per_step_best": round(per_step[0], 4),
            "ms_per_step_median": round(per_step[len(per_step) // 2], 4),
            "kernel_ms_per_step": {k: round(v[0] / max(1, v[1]), 4) for k, v in ktimes.items()},
            "select_fallback_launches": ktimes["select"][1],
            "src_p99": [round(p99[0], 6), round(p99[1], 6)], "snmf_iters": s_st.iters,
            "variant": args.flags or "improved method (no flags)",
        },
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "bytes_per_px": KERNEL_BYTES[dom], "traffic": traffic},
        "roofline_step": {"bytes_per_px": step_bytes,
                          "achieved": step_bytes * npx / (ms / 1e3) / 1e9,
                          "frac": step_bytes * npx / (ms / 1e3) / 1e9 / peak},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_separation(args, world, rank, local):
    """One step = basis estimation of the 8 Gpx slide and the FP32 densities of
    every pixel (spcn_stain_densities_estimated): 3 B/px read, 8 B/px written."""
    import torch
    from paper_1901_03088_b300 import build
    build.build()
    from paper_1901_03088_b300 import spcn, synth
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    Wd, Hd = wl["width"], wl["height"]
    npx = Wd * Hd
    t0 = time.time()
    src = synth.make_image_torch(Hd, Wd, 1000 + rank, device=dev, blobs=True)
    H = torch.empty((2, npx), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    ctx = spcn.Context(local)
    p = spcn.params(sample_mode=wl["sample_mode"], n_patches=wl["n_patches"],
                    patch_size=wl["patch_size"], sample_rate=wl["sample_rate"], seed=0,
                    flags=variant_flags(spcn, args.flags))

    def step():
        ctx.stain_densities_estimated(src, p, out=H)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ctx.kernel_timing(True)
    launches0 = ctx.launches
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = ctx.launches - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    kt = ctx.kernel_times("density")
    ctx.kernel_timing(False)
    clocks = clk.summary()
    _, st = ctx.stain_densities_estimated(src, p, out=H, return_stats=True)
    dens_ms = kt[0] / max(1, kt[1])
    peak, peak_kind = read_peaks()
    achieved = 11 * npx / (dens_ms / 1e3) / 1e9
    line = {
        "metric": "gigapixels/s stain separation (basis estimation + FP32 densities)",
        "value": world * npx / (ms / 1e3) / 1e9, "unit": "Gpx/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": f"{args.workload}: {Wd}x{Hd} uint8 RGB image, basis from "
                        + (f"{wl['n_patches']} patches of {wl['patch_size']}^2"
                           if wl["sample_mode"] == "patches" else f"{wl['sample_rate']:.0%} hash sample")
                        + f", planar FP32 H ({8 * npx / 1e9:.1f} GB) written to device memory",
            "pixels_per_step": npx, "parallelism": f"replicas x{world}",
            "l2": f"inputs ({3 * npx / 1e9:.1f} GB) larger than L2 (126 MB); no flush",
            "generate_s": round(gen_s, 2), "kernel_ms_per_step": {"density": round(dens_ms, 4)},
            "snmf_iters": st.iters, "variant": args.flags or "improved method (no flags)",
        },
        "roofline": {"bound": "hbm", "kernel": "density", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "bytes_per_px": 11, "traffic": read_traffic("density", args.workload)},
        "roofline_step": {"bytes_per_px": 11, "achieved": 11 * npx / (ms / 1e3) / 1e9,
                          "frac": 11 * npx / (ms / 1e3) / 1e9 / peak},
        "cpu_baseline": None,
        "e2e": {"value": None, "unit": "Gpx/s",
                "unavailable": "the step writes 64 GB of densities; copying them to the host "
                               "is not part of this workload"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


FLAG_NAMES = ("i0_255", "order_blue", "p99_sampled", "p99_patch_median", "h_pinv", "i0_out_255")


def variant_flags(spcn, names):
    """spcn_params.flags from a comma-separated list of FLAG_NAMES."""
    flags = 0
    for n in filter(None, (names or "").split(",")):
        if n not in FLAG_NAMES:
            raise SystemExit(f"unknown flag {n!r}; choose from {', '.join(FLAG_NAMES)}")
        flags |= getattr(spcn, "FLAG_" + n.upper())
    return flags


def run_e2e(args, ctx, spcn, src, t_st, p, dev, npx):
    """Same step through the Python API with pinned host buffers: copy the
    source in, estimate its basis, normalise, copy the result out.

    Successive steps are pipelined on three streams (copy in, compute, copy
    out) with two device buffers for each direction, so that step i's copy
    out overlaps step i+1's copy in (the link is full duplex).  Within a step
    nothing can leave before the whole image is in: the exact percentile
    needs every pixel.  The compute of all steps stays on one stream (the
    context's scratch is shared by its calls).  The serial form (one step at
    a time) is reported beside it."""
    import torch
    try:
        h_src = torch.empty(src.shape, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty(src.shape, dtype=torch.uint8, pin_memory=True)
    except Exception as e:   # not enough page-lockable host memory
        return {"value": None, "unit": "Gpx/s", "unavailable": f"pinned host buffers: {e}"[:200]}
    h_src.copy_(src)
    d_in = [torch.empty_like(src) for _ in range(2)]
    d_out = [torch.empty_like(src) for _ in range(2)]
    s_in, s_comp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    steps = max(1, min(args.steps, args.e2e_steps))

    def issue(i):
        b = i % 2
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(ev_comp[b])      # step i-2 has read d_in[b]
            d_in[b].copy_(h_src, non_blocking=True)
            ev_in[b].record(s_in)
        s_comp.wait_event(ev_in[b])
        if i >= 2:
            s_comp.wait_event(ev_out[b])         # step i-2's result has left d_out[b]
        ctx.normalize_estimated(d_in[b], t_st, p, out=d_out[b], stream=s_comp)
        ev_comp[b].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[b])
            h_out.copy_(d_out[b], non_blocking=True)
            ev_out[b].record(s_out)

    issue(0)                                     # warm-up (allocations, first launches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(1, steps + 1):
        issue(i)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # serial form: one step fully before the next
    serial_steps = 2
    t1 = time.perf_counter()
    for _ in range(serial_steps):
        d_in[0].copy_(h_src, non_blocking=True)
        ctx.normalize_estimated(d_in[0], t_st, p, out=d_out[0])
        h_out.copy_(d_out[0], non_blocking=True)
        torch.cuda.current_stream().synchronize()
    dts = (time.perf_counter() - t1) / serial_steps
    del d_in, d_out, h_src, h_out
    return {"value": npx / dt / 1e9, "unit": "Gpx/s", "h2d_bytes_per_step": 3 * npx,
            "d2h_bytes_per_step": 3 * npx, "steps": steps, "ms_per_step": 1e3 * dt,
            "pipelined": "copy-out of step i overlaps copy-in of step i+1 (2 buffers each way)",
            "serial_value": npx / dts / 1e9, "serial_ms_per_step": 1e3 * dts}


def cpu_baseline(src, tgt, wl, args):
    """The oracle, as it stands, on a bounded crop of the same slide."""
    side = args.oracle_side
    s = crop_for_oracle(src, side)
    t = crop_for_oracle(tgt, 512)
    dt, p = oracle_sample_run(s, t, wl, 0)
    return {"value": side * side / dt / 1e9, "unit": "Gpx/s", "cores": 1, "kind": "oracle",
            "sample": f"{side}x{side} centre crop of the slide (+512x512 target crop), full "
                      f"oracle path: basis ({p.sample_mode}), exact P99, normalisation; "
                      f"{dt:.1f} s single-threaded numpy FP64"}


def main():
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="wsi")
    ap.add_argument("--oracle-side", type=int, default=8192)
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--slides", type=int, default=0,
                    help="batch workload: number of slides (default 32, 8 tiles each)")
    ap.add_argument("--flags", default="",
                    help="wsi/tile workloads: comma-separated variants of the method ("
                         + ", ".join(FLAG_NAMES) + "); p99_sampled is the one-pass step")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch workload: keep the default schedule (no autotuner runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if args.oracle_side == 8192:
            args.oracle_side = 1024
        return run_reference(args, world, rank)
    world, rank, local = dist_setup(args)
    rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
