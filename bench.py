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
  pair  512 x 512 source and target, basis from every pixel (the latency of one
        end-to-end normalisation).
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
    # the small pair: 512 x 512 source and target, basis from every pixel;
    # reported as the latency of one end-to-end normalisation
    "pair": dict(width=512, height=512, sample_mode="all", n_patches=200,
                 patch_size=256, sample_rate=0.01, tgt=512),
    # a profiling size: 805 MB in and out, several times L2, a few GB on the device
    "tile16k": dict(width=16384, height=16384, sample_mode="hash", n_patches=200,
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
    "separation_tile16k": dict(width=16384, height=16384, sample_mode="hash", n_patches=200,
                               patch_size=256, sample_rate=0.01),
}
METRIC = "gigapixels/s end-to-end normalize (% of HBM roofline); batched & fwd+bwd vs plain"
# algorithmic bytes per pixel of each timed kernel (reads + writes of the image)
KERNEL_BYTES = {"pass1": 3, "pass2": 6, "density": 11}
GRAPH_REPS = 10            # steps per captured graph in the differentiable workload


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
# The oracle, as it stands, timed on every host core.  Its per-pixel steps
# (densities of every pixel for the exact P99, then Eq. 3-4 and rounding) are
# elementwise, so rows of the image are split into bands and each band runs
# through the oracle's own functions in a worker process; the percentile is
# the oracle's, over the concatenated non-white densities in raster order, so
# every value equals the single-process result.  Basis estimation (sampling,
# i0, sparse NMF, ordering) is one process, as the oracle defines it.  Arrays
# travel through memory-mapped files, not pickles.
BAND_PX = 1 << 20          # pixels per band (bounds each worker's temporaries)


def _oracle_import(_):
    """Worker warm-up: the imports a band needs."""
    import numpy  # noqa: F401
    from oracle import spcn_oracle  # noqa: F401
    return os.getpid()


def _oracle_band(task):
    """Worker: one band of rows through the oracle.  kind 'dens' writes the
    band's densities (2 x n) and non-white mask; kind 'norm' writes the
    band's normalised uint8 pixels."""
    import numpy as np
    from oracle import spcn_oracle as O
    kind, d, shape, r0, r1, a, b = task
    h, w = shape
    img = np.memmap(os.path.join(d, "src.u8"), np.uint8, "r", shape=(h, w, 3))
    band = np.ascontiguousarray(img[r0:r1])
    if kind == "dens":
        W, i0, lam, thr = a
        Hs = np.memmap(os.path.join(d, "H.f64"), np.float64, "r+", shape=(2, h * w))
        nw = np.memmap(os.path.join(d, "nw.b"), np.bool_, "r+", shape=(h * w,))
        Hs[:, r0 * w:r1 * w] = O.stain_densities(band, W, i0, lam)
        nw[r0 * w:r1 * w] = O.nonwhite_mask(band.reshape(-1, 3), thr)
    else:
        out = np.memmap(os.path.join(d, "out.u8"), np.uint8, "r+", shape=(h, w, 3))
        out[r0:r1] = O.normalize(band, a, b)
    return r1 - r0   # shared file mappings: the parent sees the pages without msync


class OraclePool:
    """A spawn-started process pool over every host core (safe after CUDA is
    initialised), with a scratch directory for the shared arrays."""

    def __init__(self):
        import multiprocessing as mp
        import tempfile
        self.cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") \
            else (os.cpu_count() or 1)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                 "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"            # one thread per worker; the pool supplies the cores
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        shm = "/dev/shm"
        roomy = os.path.isdir(shm) and os.statvfs(shm).f_bavail * os.statvfs(shm).f_frsize > 4e9
        self.dir = tempfile.mkdtemp(prefix="spcn_oracle_", dir=shm if roomy else None)
        self.pool.map(_oracle_import, range(4 * self.cores), chunksize=1)   # workers imported

    def close(self):
        import shutil
        self.pool.terminate()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)

    def bands(self, h, w):
        """Row bands: at least four per worker, at most BAND_PX pixels each."""
        rows = max(1, min(BAND_PX // max(1, w), -(-h // (4 * self.cores))))
        return [(r, min(h, r + rows)) for r in range(0, h, rows)]

    def step(self, img, tgt_st, p):
        """One oracle step on the host image `img` (h x w x 3 uint8): basis
        estimation with the oracle's Params p, exact non-white P99 of the
        whole image (parallel densities), normalisation (parallel).  Returns
        the seconds of each part, the statistics and the output."""
        import numpy as np
        from oracle import spcn_oracle as O
        h, w, _ = img.shape
        src = np.memmap(os.path.join(self.dir, "src.u8"), np.uint8, "w+", shape=(h, w, 3))
        src[:] = img
        for name, dt, shp in (("H.f64", np.float64, (2, h * w)), ("nw.b", np.bool_, (h * w,)),
                              ("out.u8", np.uint8, (h, w, 3))):
            np.memmap(os.path.join(self.dir, name), dt, "w+", shape=shp)
        t0 = time.perf_counter()
        st = O.estimate_basis(img, p)
        t1 = time.perf_counter()
        bands = self.bands(h, w)
        self.pool.map(_oracle_band, [("dens", self.dir, (h, w), r0, r1,
                                      (st.W, st.i0, p.lam, p.white_thresh), None)
                                     for r0, r1 in bands], chunksize=1)
        Hs = np.memmap(os.path.join(self.dir, "H.f64"), np.float64, "r", shape=(2, h * w))
        nw = np.memmap(os.path.join(self.dir, "nw.b"), np.bool_, "r", shape=(h * w,))
        mask = np.array(nw)
        st.p99 = np.array([O.percentile(np.asarray(Hs[j])[mask], p.stain_pct) for j in range(2)])
        t2 = time.perf_counter()
        self.pool.map(_oracle_band, [("norm", self.dir, (h, w), r0, r1, st, tgt_st)
                                     for r0, r1 in bands], chunksize=1)
        t3 = time.perf_counter()
        out = np.array(np.memmap(os.path.join(self.dir, "out.u8"), np.uint8, "r", shape=(h, w, 3)))
        return {"basis_s": t1 - t0, "p99_s": t2 - t1, "normalize_s": t3 - t2}, st, out


def oracle_target_stats(tgt_np, wl):
    """The target's statistics, once, as the GPU step has them (basis from a
    hash sample, exact P99)."""
    from oracle import spcn_oracle as O
    return O.full_stats(tgt_np, O.Params(sample_mode="hash", sample_rate=wl["sample_rate"],
                                         seed=1))


def oracle_params(wl, side, n_patches):
    """The oracle's sampling for a crop of `side`^2 and the factor that scales
    its sample to the slide's: patches (n_patches of the workload's size) or
    the workload's hash rate (sample proportional to the pixels)."""
    from oracle import spcn_oracle as O
    if wl["sample_mode"] == "patches":
        ps = min(wl["patch_size"], side)      # a crop smaller than a patch takes smaller patches
        return (O.Params(sample_mode="patches", n_patches=n_patches, patch_size=ps, seed=0),
                wl["n_patches"] * wl["patch_size"] ** 2 / (n_patches * ps * ps))
    if wl["sample_mode"] == "all":
        return O.Params(sample_mode="all"), wl["width"] * wl["height"] / (side * side)
    return (O.Params(sample_mode="hash", sample_rate=wl["sample_rate"], seed=0),
            wl["width"] * wl["height"] / (side * side))


def oracle_step_rate(parts, crop_px, slide_px, basis_scale):
    """Seconds of one slide step from one timed oracle step: the basis time
    scaled to the slide's sample (the sparse NMF's work is linear in it), the
    per-pixel time scaled to the slide's pixels."""
    return (parts["basis_s"] * basis_scale
            + (parts["p99_s"] + parts["normalize_s"]) * slide_px / crop_px)


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
            + (f"{wl['n_patches']} patches of {wl['patch_size']}^2" if wl["sample_mode"] == "patches"
               else "every pixel" if wl["sample_mode"] == "all"
               else f"{wl['sample_rate']:.0%} hash sample"))


def normalize_config(name, wl, world):
    """The config object of a normalisation line, the same in both arms."""
    npx = wl["width"] * wl["height"]
    l2 = (f"inputs ({3 * npx / 1e9:.1f} GB) larger than L2 (126 MB); no flush"
          if 3 * npx > 126e6 else
          f"inputs ({3 * npx / 1e6:.2f} MB) fit in L2: a latency measurement, not flushed")
    return {"workload": normalize_workload_desc(name, wl), "pixels_per_step": npx,
            "parallelism": f"replicas x{world}", "l2": l2}


def oracle_sample_desc(side, p, basis_scale, wl, parts, cores, scaled_s):
    smp = (f"{p.n_patches} patches of {p.patch_size}^2" if p.sample_mode == "patches"
           else "every pixel of the crop" if p.sample_mode == "all"
           else f"a {p.sample_rate:.0%} hash sample of the crop")
    return (f"per step: oracle basis estimation from {smp} (one process; scaled "
            f"x{basis_scale:g} to the slide's sample), then the exact non-white P99 and the "
            f"normalisation of a "
            f"{side}x{side} centre crop of the synthetic slide in row bands over {cores} worker "
            f"processes (scaled to the slide's pixels); timed {parts['basis_s']:.2f} + "
            f"{parts['p99_s']:.2f} + {parts['normalize_s']:.2f} s -> {scaled_s:.1f} s per slide; "
            "numpy FP64")


def run_reference(args, world, rank):
    """The oracle arm: each step one bounded sample of the slide workload
    (basis from 25 of the 200 patches, per-pixel steps of a 2048^2 crop over
    every host core), scaled to one slide."""
    if rank != 0:
        return 0
    import numpy as np
    from paper_1901_03088_b300 import synth
    wl = WORKLOADS[args.workload]
    if "n_patches" not in wl or "tgt" not in wl:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the oracle arm times the normalisation workloads, not {args.workload}"}))
        return 0
    side = min(args.oracle_side, wl["width"], wl["height"])
    p, scale = oracle_params(wl, side, max(1, wl["n_patches"] // 8))
    src = synth.make_image(side, side, 1000, blobs=True)
    tgt = synth.make_image(wl["tgt"], wl["tgt"], 1, blobs=True)
    t_st = oracle_target_stats(tgt, wl)
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step(src, t_st, p)
        per = []
        parts = None
        for _ in range(args.steps):
            parts, _, _ = pool.step(src, t_st, p)
            per.append(oracle_step_rate(parts, side * side, wl["width"] * wl["height"], scale))
    finally:
        pool.close()
    npx = wl["width"] * wl["height"]
    sec = statistics.mean(per)
    gpx = npx / sec / 1e9
    sample = oracle_sample_desc(side, p, scale, wl, parts, pool.cores, sec)
    line = {
        "impl": "reference", "metric": METRIC, "value": gpx, "unit": "Gpx/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": normalize_config(args.workload, wl, world),
        "cpu_baseline": {"value": gpx, "unit": "Gpx/s", "cores": pool.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gpx, "unit": "Gpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- CUDA arm
def run_grad(args, world, rank, local, leg=False):
    """Forward + hand-written backward of the differentiable normalisation on a
    batch of 64 float32 3x256x256 images, against forward only.  As a leg of
    the default run it returns a summary instead of printing a line."""
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
    # each graph holds GRAPH_REPS steps, so that the host's graph-launch time
    # (tens of microseconds) does not hide the device time of a short step
    g_f, g_fb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_f):
        for _ in range(GRAPH_REPS):
            fwd_eager()
    with torch.cuda.graph(g_fb):
        for _ in range(GRAPH_REPS):
            xg.grad = None
            Wt.grad = None
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
        return max_over_ranks(e0.elapsed_time(e1) / (args.steps * GRAPH_REPS), world, dev), \
            ctx.launches - l0

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
    if leg:
        ctx.close()
        return {"workload": f"{B} x 3 x {H} x {W} float32, own source statistics per image",
                "fwd_ms": round(ms_f, 5), "fwd_bwd_ms": round(ms_fb, 5),
                "ratio": round(ms_fb / ms_f, 3),
                "fwd_gpx_s": world * npx / (ms_f / 1e3) / 1e9,
                "fwd_bwd_gpx_s": world * npx / (ms_fb / 1e3) / 1e9,
                "kernel_ms": {"forward": round(kf_ms, 5), "backward": round(kb_ms, 5)},
                "roofline_frac": bytes_fb / (ms_fb / 1e3) / 1e9 / peak,
                "roofline_bytes_per_px": 60,
                "backward_roofline_frac": 36 * npx / (kb_ms / 1e3) / 1e9 / peak,
                "timing": f"CUDA-graph replays of {GRAPH_REPS} autograd steps each (forward "
                          "only / forward + backward), CUDA events",
                "gpu_launches_per_step": launches // max(1, args.steps), "clocks": clk.summary()}
    line = {
        "metric": METRIC, "value": world * npx / (ms_fb / 1e3) / 1e9, "unit": "Gpx/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fb,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"grad: forward + backward, batch {B} x 3 x {H} x {W} float32",
                   "timing": f"CUDA-graph replays of {GRAPH_REPS} autograd steps each",
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


def run_batch(args, world, rank, local, leg=False):
    """256 uneven tiles from 32 slides (own source statistics each), one
    target: one batch run per step (the library's staged schedule: window
    pilot, pass 1 of every tile, per-tile selects, pass 2, and the exact
    fallback launch that returns at once when no tile missed its window),
    replayed from a CUDA graph, against the same tiles normalised by 256
    sequential spcn_normalize calls.  As a leg of the
    default run it returns a summary instead of printing a line."""
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

    if leg:
        out = {"workload": f"{len(tiles)} uint8 RGB tiles from {n_slides} slides, sides "
                           f"log-uniform in [{wl['side_lo']}, {wl['side_hi']}], {npx / 1e6:.1f} Mpx, "
                           f"one {wl['tgt']}x{wl['tgt']} target",
               "ms": round(ms, 4), "gpx_s": world * npx / (ms / 1e3) / 1e9,
               "plain_ms": round(ms_seq, 4), "plain_gpx_s": world * npx / (ms_seq / 1e3) / 1e9,
               "speedup": ms_seq / ms, "kernel_ms": round(k_ms, 4),
               "roofline_frac": achieved / peak, "roofline_bytes_per_px": 9,
               "outputs_identical_to_plain": identical,
               "tiles_exact_fallback": sum(fallback), "schedule": b.config,
               "fused_launch_ms": min((t["ms"] for t in trials
                                       if t["schedule"] in ("phased", "interleaved")),
                                      default=None),
               "persistent_launch_ms": min((t["ms"] for t in trials
                                            if t["schedule"] == "persistent"), default=None),
               "tune_s": round(tune_s, 2),
               "timing": f"CUDA-graph replays of one batch run ({per_run} launches) vs "
                         f"{len(tiles)} sequential spcn_normalize calls, CUDA events",
               "gpu_launches_per_step": per_run, "clocks": clocks}
        b.close()
        ctx.close()
        del tiles, outs, ref
        torch.cuda.empty_cache()
        return out

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
            "timing": f"CUDA-graph replays of one batch run ({per_run} launches)",
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
        "roofline": {"bound": "hbm", "kernel": "batch run (k_batch_p1, k_sel_*, k_batch_p2, k_batch)", "achieved": achieved, "peak": peak,
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
    if args.workload.startswith("separation"):
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

    if args.hint != "sample":
        # the window-miss recovery on record: the sampled percentile is dropped
        # ("none": pass 1 has no window) or scaled by a factor (a window that
        # misses the percentile), so every step takes the recovery; a host
        # round trip separates the two calls
        factor = 0.0 if args.hint == "none" else float(args.hint)

        def step():
            s_st = ctx.estimate_basis(src, p)
            s_st.p99[0] *= factor
            s_st.p99[1] *= factor
            ctx.normalize(src, s_st, t_st, p, out=out)
    else:
        def step():
            # basis estimation + both passes, statistics kept on the device
            ctx.normalize_estimated(src, t_st, p, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # --graph: the one-call step is stream-ordered and allocation-free once
    # warm, so it is captured once into a CUDA graph and replayed (no host
    # launch latency); the kernels' own times then come from eager steps
    timed_step, graph, graph_launches = step, None, 0
    if args.graph and args.hint == "sample":
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        l0 = ctx.launches
        with torch.cuda.graph(graph):
            step()
        graph_launches = ctx.launches - l0
        timed_step = graph.replay
        for _ in range(args.warmup):
            timed_step()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ctx.kernel_timing(graph is None)
    launches0 = ctx.launches
    fallbacks0 = ctx.exact_fallbacks
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(args.steps):
            timed_step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = ctx.launches - launches0 if graph is None else graph_launches * args.steps
    fallbacks = ctx.exact_fallbacks - fallbacks0
    ms_local = evs[0].elapsed_time(evs[-1]) / args.steps
    per_step = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps))
    ms = max_over_ranks(ms_local, world, dev)
    direct_ms = None
    if graph is not None:   # kernel times and the direct-call time from eager steps
        ctx.kernel_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        direct_ms = e0.elapsed_time(e1) / args.steps
    ktimes = {k: ctx.kernel_times(k) for k in ("pass1", "ladder", "select", "pass2")}
    ctx.kernel_timing(False)
    clocks = clk.summary()

    # the statistics of one step (bench output is not a parity test)
    _, s_st = ctx.normalize_estimated(src, t_st, p, out=out, return_stats=True)
    p99 = (s_st.p99[0], s_st.p99[1])
    if args.hint != "sample":
        sampled_st = ctx.estimate_basis(src, p)
        s_st.iters = sampled_st.iters

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

    # the other two legs of the metric on the same GPU: the batched launch
    # against plain calls, and forward + backward against forward only
    legs = {}
    if args.workload == "wsi" and not args.no_legs and not flags and args.hint == "sample":
        legs["batched"] = run_batch(args, world, rank, local, leg=True)
        legs["fwd_bwd"] = run_grad(args, world, rank, local, leg=True)

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
        "config": (normalize_config(args.workload, wl, world) if not flags
                   and args.hint == "sample" else dict(normalize_config(args.workload, wl, world),
                                                       variant=args.flags or "improved method",
                                                       p99_window=args.hint)),
        "details": {
            "timing": ("CUDA-graph replays of the one-call step" if graph is not None else
                       "direct calls of the one-call step, CUDA events"),
            "direct_call_ms_per_step": round(direct_ms, 4) if direct_ms is not None else None,
            "target_stats_ms_once": round(tgt_ms, 3), "generate_s": round(gen_s, 2),
            "ms_per_step_best": round(per_step[0], 4),
            "ms_per_step_median": round(per_step[len(per_step) // 2], 4),
            "kernel_ms_per_step": {k: round(v[0] / max(1, v[1]), 4) for k, v in ktimes.items()},
            "select_kernel_launches": ktimes["select"][1],
            "ladder_kernel_launches": ktimes["ladder"][1],
            "exact_fallback_steps": fallbacks,
            "p99_window": ("from the basis sample's percentile" if args.hint == "sample" else
                           "none: the sampled percentile dropped" if args.hint == "none" else
                           f"the sampled percentile x {args.hint} (a window that misses)"),
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
    line.update(legs)
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
    """The oracle, as it stands, on every host core: basis estimation at the
    slide's own sampling (200 patches of 256^2, 13.1 Mpx) and the per-pixel
    steps of an 8192^2 centre crop, scaled to the slide."""
    import numpy as np
    side = min(args.oracle_side, wl["width"], wl["height"])
    s = crop_for_oracle(src, side)
    t_st = oracle_target_stats(np.ascontiguousarray(tgt.cpu().numpy()), wl)
    p, scale = oracle_params(wl, side, wl["n_patches"])
    pool = OraclePool()
    try:
        parts, _, _ = pool.step(s, t_st, p)
    finally:
        pool.close()
    sec = oracle_step_rate(parts, side * side, wl["width"] * wl["height"], scale)
    return {"value": wl["width"] * wl["height"] / sec / 1e9, "unit": "Gpx/s",
            "cores": pool.cores, "kind": "oracle",
            "sample": oracle_sample_desc(side, p, scale, wl, parts, pool.cores, sec)}


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
    ap.add_argument("--graph", action="store_true",
                    help="wsi/tile/pair workloads: time CUDA-graph replays of the one-call step "
                         "(no host launch latency) instead of direct calls")
    ap.add_argument("--no-legs", action="store_true",
                    help="wsi workload: skip the batched and forward+backward legs")
    ap.add_argument("--hint", default="sample",
                    help="wsi/tile workloads: 'sample' (the method), 'none' (no window) or a "
                         "factor applied to the sampled percentile (a window that misses): "
                         "every step then takes the window-miss recovery (its cost on record)")
    args = ap.parse_args()
    if args.hint not in ("sample", "none"):
        try:
            float(args.hint)
        except ValueError:
            ap.error("--hint: 'sample', 'none' or a factor")
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if args.oracle_side == 8192:
            args.oracle_side = 2048     # each of the K + W steps is a bounded sample
        return run_reference(args, world, rank)
    world, rank, local = dist_setup(args)
    rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
