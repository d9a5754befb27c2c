"""Throughput of the single-pass AMR raycaster on one GB300 (or N, one process per GPU).

A step is one frame: every pixel's ray is traversed through the kD-tree leaves and
sampled, shaded and composited (the whole hot path), on the cosmology-like 5-level
hierarchy (2,219 patches, 1.33e8 cells, 602 MB of FP32 bricks) at 2048x2048 with
central-difference Phong shading.  The hierarchy, tree and bricks are built once before
timing (the paper's preprocessing).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own view (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsamples/s and frames/s at 2048² (fraction of HBM roofline); learned-skip speedup at PSNR≥45 dB"
UNIT = "Gsamples/s"
SIZE = 2048
BYTES_PER_SAMPLE = {0: 32, 1: 224}  # FP32 trilinear stencil, x7 with the six gradient stencils
CELL_BYTES = {"f32": 4, "f16": 2, "bf16": 2}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _march_sha() -> str:
    """sha1 (12 hex digits) of the sources the frame kernels compile from: every
    march*.cuh header, amr_device.h and storage16.h."""
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1212_3333_gb300", "csrc")
    names = sorted(f for f in os.listdir(d) if f.startswith("march") and f.endswith(".cuh"))
    for f in names + ["amr_device.h", "storage16.h"]:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _variant(storage: str, gradient: bool, dtype: str, halo: int = 1, maxbrick: bool = False) -> str:
    return (f"{storage}{'+grad' if gradient else ''}{'+halo2' if halo == 2 else ''}"
            f"{'+max' if maxbrick else ''}/{dtype}")


def _profiled_counters(shade: int, variant: str, size: int, schedule: int):
    """ncu counters of the frame kernel from the committed summary
    (profiles/march_counters.json), if they were taken on the current kernel sources;
    else None.  One entry per (sources hash, variant, shade, size, schedule)."""
    path = os.path.join(ROOT, "profiles", "march_counters.json")
    try:
        with open(path) as f:
            entries = json.load(f)["entries"]
    except Exception:
        return None
    sha = _march_sha()
    for e in entries:
        if (e.get("sources") == sha and e.get("variant") == variant and e.get("shade") == shade
                and e.get("size") == size and e.get("schedule", 0) == schedule):
            return e
    return None


def _l1_peak_gbs(sm_mhz):
    """L1 data throughput of the whole chip at the SM clock sampled during the timed region:
    ncu's peak rate of L1 data-pipe wavefronts per cycle over all SMs (a property of the
    chip, recorded in the counters summary) times the 128 bytes one wavefront moves;
    without that figure, the nominal 128 B per cycle per SM."""
    import torch

    per_clk, kind = None, None
    try:
        with open(os.path.join(ROOT, "profiles", "march_counters.json")) as f:
            per_clk = 128.0 * float(json.load(f)["l1_lsu_wavefronts_peak_per_cycle"])
            kind = ("ncu l1tex__data_pipe_lsu_wavefronts.sum.peak_sustained x 128 B x median "
                    "SM clock under load")
    except Exception:
        pass
    if per_clk is None:
        per_clk = 128.0 * torch.cuda.get_device_properties(0).multi_processor_count
        kind = "nominal 128 B/clk/SM x SMs x median SM clock under load"
    return per_clk * (sm_mhz or 2070.0) * 1e6 / 1e9, kind


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        from paper_1212_3333_gb300 import shard

        shard.barrier()


def _max_over_ranks(world, x: float) -> float:
    from paper_1212_3333_gb300 import shard

    return shard.all_max(x) if world > 1 else x


def _sum_over_ranks(world, x: float) -> float:
    from paper_1212_3333_gb300 import shard

    return shard.all_sum(x) if world > 1 else x


def cpu_baseline(hier, cam, tf, vmin, vmax, shade, budget_s=15.0, seed=0):
    """The FP64 oracle, as it stands, on a bounded random sample of the same frame's
    pixels; returns samples/s and how the sample was taken."""
    import oracle

    o = oracle.Oracle(hier)
    op = oracle.OracleParams(vmin=vmin, vmax=vmax, shade=shade)
    threads = oracle.max_threads()
    rng = np.random.default_rng(seed)
    n = 64
    total_s, total_samples, total_pix = 0.0, 0, 0
    while total_s < budget_s:
        pix = np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], 1)
        t = time.perf_counter()
        _, smp = o.render(cam, tf, op, pixels=pix.astype(np.int32))
        dt = time.perf_counter() - t
        total_s += dt
        total_samples += int(smp.sum())
        total_pix += n
        if dt < budget_s / 8:
            n *= 2
    # one thread on a small sample, for the per-core rate
    pix = np.stack([rng.integers(0, cam.width, 256), rng.integers(0, cam.height, 256)], 1)
    t = time.perf_counter()
    _, smp1 = o.render(cam, tf, op, pixels=pix.astype(np.int32), nthreads=1)
    one = int(smp1.sum()) / (time.perf_counter() - t)
    return {"value": total_samples / total_s / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle", "host_cpus": os.cpu_count(),
            "single_thread_msamples_s": one / 1e6,
            "sample": f"{total_pix} seeded random pixels of the {cam.width}x{cam.height} frame "
                      f"({total_samples} samples, {total_s:.1f} s), FP64 oracle, {threads} threads"}


def learned_eval(amr, ctx, hier, vmin, vmax, tf, args, taus=(1e-4, 1e-3, 1e-2)):
    """Learned segment proposal on the same hierarchy: log segments from 256 seeded poses
    (seeds 1000-1255), train the MLP with the library's kernels, then time held-out views
    (seeds 2000-2007) at the bench size: plain march, exact min/max skipping, and min/max +
    learned skipping (and 16x / 32x / 64x coarser sampling) for each tau and each minimum
    segment length the proposal is asked about, PSNR against the plain march."""
    import torch

    import synth
    from paper_1212_3333_gb300 import proposal

    t0 = time.perf_counter()
    p_log = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=0)
    poses = [synth.orbit_camera(1000 + s, args.log_size, args.log_size) for s in range(256)]
    feats, tgts, seen = proposal.log_segments(ctx, poses, tf, p_log, capacity=args.log_cap,
                                              keep_prob=args.log_keep, seed=1)
    t_log = time.perf_counter() - t0
    t0 = time.perf_counter()
    prop = proposal.Proposal(seed=0)
    losses = prop.train(feats, tgts, epochs=args.epochs, batch=16384, lr=2e-3)
    t_train = time.perf_counter() - t0
    prop.install(ctx)
    size = args.size
    out = torch.empty((size, size, 4), dtype=torch.float32, device="cuda")
    ref = torch.empty_like(out)
    stream = torch.cuda.current_stream()

    def timed(cam, params, reps=2):
        ctx.amr_render(cam, tf, params, out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            ctx.amr_render(cam, tf, params, out)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    base = dict(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert)
    configs = {"plain": {}, "minmax": {"skip": 1}}
    # the proposal is asked about segments of at least m samples (m1: every segment)
    for m in (1, 8):
        for tau in taus:
            configs[f"skip@{tau:g}/m{m}"] = {"skip": 1, "learned": 1, "tau": tau,
                                             "learned_min_samples": m}
            for cf in (16, 32, 64):
                configs[f"coarse{cf}@{tau:g}/m{m}"] = {"skip": 1, "learned": 2, "tau": tau,
                                                       "coarse_factor": cf,
                                                       "learned_min_samples": m}
    res = {k: {"ms": 0.0, "psnr_min": float("inf"), "samples": 0} for k in configs}
    views = [synth.orbit_camera(2000 + s, size, size) for s in range(args.heldout)]
    for cam in views:
        ctx.amr_render(cam, tf, amr.amr_default_params(**base), ref)
        for name, extra_p in configs.items():
            prm = amr.amr_default_params(**base, **extra_p)
            n = ctx.amr_render(cam, tf, prm, out, count_samples=True)
            res[name]["samples"] += n
            res[name]["psnr_min"] = min(res[name]["psnr_min"], proposal.psnr(out, ref))
            res[name]["ms"] += timed(cam, prm)
    t_plain, t_minmax = res["plain"]["ms"], res["minmax"]["ms"]
    best = None
    for name in configs:
        r = res[name]
        r["speedup_vs_plain"] = t_plain / r["ms"]
        r["speedup_vs_minmax"] = t_minmax / r["ms"]
        if name.startswith(("skip@", "coarse")) and r["psnr_min"] >= 45.0:
            if best is None or r["ms"] < res[best]["ms"]:
                best = name
    return {"train": {"poses": 256, "log_size": args.log_size, "segments_seen": seen,
                      "records": int(feats.shape[0]), "epochs": args.epochs,
                      "loss_per_epoch": losses, "log_s": t_log, "train_s": t_train},
            "heldout_views": len(views), "results": res, "best_at_psnr45": best,
            "learned_speedup_vs_plain": res[best]["speedup_vs_plain"] if best else None,
            "learned_speedup_vs_minmax": res[best]["speedup_vs_minmax"] if best else None,
            "minmax_speedup_vs_plain": t_plain / t_minmax}


def precision_eval(amr, hier, vmin, vmax, cam, tf, out, args, peak):
    """Cell storage precision: FP32 / FP16 / BF16 bricks (pointer table, gradient bricks and
    the bench's halo and stencil-maximum options),
    each timed plain and Phong, with PSNR and max-abs of its Phong image against the
    FP32-storage image of the same view."""
    import torch

    stream = torch.cuda.current_stream()
    res = {}
    ref = None
    for dtype, e in (("f32", 4), ("f16", 2), ("bf16", 2)):
        t0 = time.perf_counter()
        ctx = amr.from_hierarchy(hier, dtype)
        ctx.amr_build_kdtree("ptr", gradient=True, halo=args.halo, maxbrick=bool(args.maxbrick))
        r = {"brick_mb": ctx.amr_get_stats().brick_bytes / 1e6,
             "build_s": time.perf_counter() - t0}
        for shade in (0, 1):
            p = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=shade, ert_eps=args.ert)
            n = ctx.amr_render(cam, tf, p, out, count_samples=True)
            for _ in range(2):
                ctx.amr_render(cam, tf, p, out)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(5):
                ctx.amr_render(cam, tf, p, out)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 5
            bps = 8 * e * (7 if shade else 1)
            key = "phong" if shade else "plain"
            r[key] = {"gsamples_s": n / ms / 1e6, "ms": ms, "bytes_per_sample": bps,
                      "frac_hbm": n * bps / (ms * 1e-3) / 1e9 / peak}
        img = out.double().clone()  # the Phong image
        if ref is None:
            ref = img
        else:
            d = (img - ref).abs()
            mse = float((d ** 2).mean())
            r["psnr_vs_f32_storage_db"] = float("inf") if mse == 0 else 10 * math.log10(1 / mse)
            r["max_abs_vs_f32_storage"] = float(d.max())
        res[dtype] = r
        ctx.amr_destroy()
    return res


def lod_eval(amr, ctx, vmin, vmax, cam, tf, out, args, lods=(0.5, 1.0, 2.0, 4.0)):
    """Level-of-detail pruning (Sec. 3.1 type-(a) nodes) on the bench view: samples, time
    and PSNR against the unpruned image for a few thresholds (pixels)."""
    import torch

    stream = torch.cuda.current_stream()
    base = dict(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert)

    def run(prm):
        n = ctx.amr_render(cam, tf, prm, out, count_samples=True)
        ctx.amr_render(cam, tf, prm, out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            ctx.amr_render(cam, tf, prm, out)
        b.record(stream)
        torch.cuda.synchronize()
        return n, a.elapsed_time(b) / 3, out.double().clone()

    n0, ms0, ref = run(amr.amr_default_params(**base))
    res = {"off": {"samples": n0, "ms": ms0, "gsamples_s": n0 / ms0 / 1e6}}
    for lod in lods:
        n, ms, img = run(amr.amr_default_params(**base, lod_pixels=lod))
        mse = float(((img - ref) ** 2).mean())
        res[f"{lod:g}px"] = {"samples": n, "ms": ms, "gsamples_s": n / ms / 1e6,
                             "speedup": ms0 / ms,
                             "psnr_vs_unpruned_db": float("inf") if mse == 0 else
                             10 * math.log10(1 / mse)}
    return res


def shadow_eval(amr, ctx, vmin, vmax, args, size=512):
    """Secondary rays to a central point light (the paper's global-illumination example):
    frame time at `size`² without them, and with them under the per-ray loop (each lane
    marches its samples' light rays) and under deferred shading (the default for Phong:
    a warp marches each queued sample's light ray together); Phong, light step half a
    level-0 cell."""
    import torch
    import synth

    cam = synth.orbit_camera(2, size, size)
    tf = torch.as_tensor(synth.ramp_tf(), device="cuda")
    out = torch.empty((size, size, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {"size": size}
    light = {"shadow": 1, "light": (0.5, 0.5, 0.5), "light_step": 0.5 / 128,
             "light_ambient": 0.2}
    for name, kw in (("plain", {}), ("shadow_per_ray", dict(light, schedule=0)),
                     ("shadow", dict(light, schedule=3))):
        prm = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert,
                                     **kw)
        if args.shade != 1 and kw.get("schedule") == 3:
            continue
        n = ctx.amr_render(cam, tf, prm, out, count_samples=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(2):
            ctx.amr_render(cam, tf, prm, out)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 2
        res[name] = {"ms": ms, "frames_per_s": 1e3 / ms, "samples": n}
    best = "shadow" if "shadow" in res else "shadow_per_ray"
    res["slowdown"] = res[best]["ms"] / res["plain"]["ms"]
    res["slowdown_per_ray"] = res["shadow_per_ray"]["ms"] / res["plain"]["ms"]
    return res


def batch_eval(amr, ctx, vmin, vmax, args, peak, n_views=64, seed=5, lo=256, hi=2048,
               tune_views=16, schedule=0):
    """Batched multi-view rendering: 64 seeded views with square sides uniform in
    256..2048 and four 256-entry transfer functions, rendered (a) as 64 separate
    amr_render launches, (b) as one persistent amr_render_batch launch with the autotuned
    tile configuration, (c) as that launch replayed from a CUDA graph.  schedule 3: the
    batched launch marches with deferred shading (the separate renders stay per-ray)."""
    import torch
    import synth

    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=n_views)
    cams = [synth.orbit_camera(5000 + v, int(sd), int(sd)) for v, sd in enumerate(sides)]
    tfi = [v % 4 for v in range(n_views)]
    tfs = torch.as_tensor(np.stack(synth.tf_variants()), device="cuda")
    # the separate launches use the batch's schedule (like for like)
    p0 = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert,
                                schedule=schedule, samples_per_iter=16)
    p = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert,
                               schedule=schedule, samples_per_iter=16)
    views, offsets, total = amr.make_views(cams, tfi)
    out = torch.zeros((total,), dtype=torch.float32, device="cuda")
    ref = torch.zeros_like(out)
    stream = torch.cuda.current_stream()

    def separate(dst):
        for cam, t, off in zip(cams, tfi, offsets):
            ctx.amr_render(cam, tfs[t], p0, dst[off:off + 4 * cam.width * cam.height])

    def timed(fn, reps=3):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_sep = timed(lambda: separate(ref), reps=1)
    # tune on the first 16 views (a quarter of the work), then render all 64 with the winner
    t0 = time.perf_counter()
    sub = (amr._lib.amr_view * tune_views)(*views[:tune_views])
    best, table = ctx.amr_batch_autotune(sub, tfs, p, out, reps=1)
    tune_s = time.perf_counter() - t0
    samples = ctx.amr_render_batch(views, tfs, p, out, count_samples=True)
    same = bool(torch.equal(out, ref))
    ms_batch = timed(lambda: ctx.amr_render_batch(views, tfs, p, out), reps=1)
    s = torch.cuda.Stream()
    s.wait_stream(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        ctx.amr_render_batch(views, tfs, p, out, stream=s)
    ms_graph = timed(g.replay, reps=2)
    same = same and bool(torch.equal(out, ref))
    names = [f"{tw}x{th}/r{r}" for tw, th in ((8, 8), (16, 8), (16, 16)) for r in (1, 2, 4)]
    names += [f"best tile/spi{k}" for k in (4, 8, 16, 32)]
    bps = BYTES_PER_SAMPLE[args.shade]
    return {"views": n_views, "sides": [lo, hi], "schedule": schedule,
            "pixels": int(sum(int(sd) ** 2 for sd in sides)),
            "samples": samples, "identical_to_separate": same,
            "separate": {"ms": ms_sep, "gsamples_s": samples / ms_sep / 1e6},
            "batched": {"ms": ms_batch, "gsamples_s": samples / ms_batch / 1e6},
            "batched_graph": {"ms": ms_graph, "gsamples_s": samples / ms_graph / 1e6,
                              "frac_hbm": samples * bps / (ms_graph * 1e-3) / 1e9 / peak},
            "speedup_vs_separate": ms_sep / ms_graph,
            "autotune": {"best": f"{best.tile_w}x{best.tile_h}/r{best.rays_per_thread}"
                                 f"/spi{best.samples_per_iter or p.samples_per_iter}",
                         "tuned_on_views": tune_views, "ms": dict(zip(names, table)),
                         "seconds": tune_s}}


def schedules_eval(amr, ctx, vmin, vmax, tf, args, sizes=(2048, 1024, 512), spi=16):
    """The frame march under the per-ray loop (schedule 0), persistent refill (2),
    deferred shading (3) and the library's default choice (auto) at several image sizes
    (the C2 orbit view): Gsamples/s and whether each image equals the per-ray one bit for
    bit."""
    import torch
    import synth

    stream = torch.cuda.current_stream()
    res = {}
    for size in sizes:
        cam = synth.orbit_camera(2, size, size)
        ref = torch.empty((size, size, 4), dtype=torch.float32, device="cuda")
        out = torch.empty_like(ref)
        row = {}
        for sched in (0, 2, 3, -1):
            p = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert,
                                       schedule=sched, samples_per_iter=spi)
            if sched == 3 and args.shade != 1:
                continue
            dst = ref if sched == 0 else out
            n = ctx.amr_render(cam, tf, p, dst, count_samples=True)
            ctx.amr_render(cam, tf, p, dst)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                ctx.amr_render(cam, tf, p, dst)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 3
            row["auto" if sched < 0 else str(sched)] = {
                "ms": ms, "gsamples_s": n / ms / 1e6,
                "identical_to_per_ray": bool(torch.equal(dst, ref))}
        res[str(size)] = row
    return {"samples_per_iter": spi, "by_size": res}


def halo_eval(amr, hier, vmin, vmax, tf, args):
    """Bricks with a one- and a two-cell halo (the second lets gradient neighbours beyond
    faces onto the same level read the sample's brick): Phong + gradient bricks, the
    per-ray loop at 2048² and deferred shading at 1024² (the C2 orbit view)."""
    import torch
    import synth

    stream = torch.cuda.current_stream()
    res = {}
    for halo in (1, 2):
        ctx = amr.from_hierarchy(hier)
        ctx.amr_build_kdtree("ptr", gradient=True, halo=halo)
        row = {"brick_mb": ctx.amr_get_stats().brick_bytes / 1e6}
        for size, sched in ((2048, 0), (1024, 3)):
            cam = synth.orbit_camera(2, size, size)
            out = torch.empty((size, size, 4), dtype=torch.float32, device="cuda")
            p = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=1, ert_eps=args.ert,
                                       schedule=sched)
            n = ctx.amr_render(cam, tf, p, out, count_samples=True)
            ctx.amr_render(cam, tf, p, out)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                ctx.amr_render(cam, tf, p, out)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 3
            row[f"{size}/s{sched}"] = {"ms": ms, "gsamples_s": n / ms / 1e6}
        res[f"halo{halo}"] = row
        ctx.amr_destroy()
    return res


def c3_eval(amr, args, peak):
    """The deep 8-level hierarchy (1/16384 finest spacing, ~1e9 cells) at 2048², Phong:
    FP32 / FP16 / BF16 cells, throughput and PSNR of each against the FP32-cell image."""
    import torch
    import synth

    t0 = time.perf_counter()
    h = synth.amr.make_c3(device="cuda")
    gen_s = time.perf_counter() - t0
    vmin, vmax = synth.amr.percentile_range(h)
    cam = synth.orbit_camera(3, SIZE, SIZE)
    tf = torch.as_tensor(synth.ramp_tf(), device="cuda")
    out = torch.empty((SIZE, SIZE, 4), dtype=torch.float32, device="cuda")
    precision = precision_eval(amr, h, vmin, vmax, cam, tf, out, args, peak)
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True)
    lod = lod_eval(amr, ctx, vmin, vmax, cam, tf, out, args)
    st = ctx.amr_get_stats()
    ctx.amr_destroy()
    return {"patches": h.num_patches, "patches_per_level": h.patches_per_level(),
            "cells": h.n_cells(), "levels": h.num_levels, "generate_s": gen_s,
            "tree": {"nodes": st.num_nodes, "leaves": st.num_leaves, "depth": st.max_depth},
            "precision": precision, "lod": lod}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import synth

    # the same seeded inputs as the GPU arm (generated on the GPU when one is present, so
    # both arms see bit-identical hierarchies); only the oracle's rendering is timed
    hier = synth.make_c2(device=None)
    vmin, vmax = synth.amr.percentile_range(hier)
    cam = synth.orbit_camera(2, args.size, args.size)
    tf = synth.ramp_tf()
    vals = []
    cb = None
    for s in range(args.warmup + args.steps):
        cb = cpu_baseline(hier, cam, tf, vmin, vmax, args.shade,
                          budget_s=max(2.0, 60.0 / (args.warmup + args.steps)), seed=s)
        if s >= args.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(hier, args, "oracle", args.size),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(hier, args, storage, size=SIZE):
    return {"workload": (f"c2: lognormal 5-level AMR, {hier.num_patches} patches, "
                         f"{hier.n_cells():.3g} FP32 cells; {size}x{size} view; "
                         f"{'Phong' if args.shade else 'unshaded'} trilinear; step 0.5 h^l; "
                         f"ERT eps {args.ert}"),
            "storage": storage + ("+gradient bricks" if getattr(args, "gradient", 0) and
                                  storage != "oracle" else "") +
                       (", two-cell halo" if getattr(args, "halo", 1) == 2 and
                        storage != "oracle" else "") +
                       (", stencil-maximum bricks" if getattr(args, "maxbrick", 0) and
                        storage == "ptr" else ""),
            "cells": getattr(args, "dtype", "f32"),
            "image": [size, size], "shade": args.shade,
            "schedule": getattr(args, "schedule", 0),
            "l2": ("inputs larger than L2: 602-677 MB of bricks (plus gradient and "
                   "stencil-maximum bricks) vs 129 MB L2, no flush")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="ptr",
                    choices=["ptr", "texobj", "atlas_linear", "atlas_tex3d"])
    ap.add_argument("--shade", type=int, default=1)
    ap.add_argument("--ert", type=float, default=1e-4)
    ap.add_argument("--compare", type=int, default=1, help="time every storage briefly")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--e2e", type=int, default=1, help="also time the host-buffer entry point")
    ap.add_argument("--size", type=int, default=SIZE, help="image side (the metric is at 2048)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="0 per-ray loop, 1 warp wavefront, 2 refill, 3 deferred shading")
    ap.add_argument("--spi", type=int, default=16, help="samples per step, schedules 2 and 3")
    ap.add_argument("--schedules", type=int, default=1,
                    help="time schedules 0 / 2 / 3 at 2048, 1024 and 512 pixels")
    ap.add_argument("--gradient", type=int, default=1, help="build gradient bricks")
    ap.add_argument("--halo", type=int, default=2, choices=[1, 2],
                    help="brick halo cells (2: gradient neighbours beyond faces onto the "
                         "same level read the sample's brick)")
    ap.add_argument("--halos", type=int, default=1, help="time one- and two-cell halos")
    ap.add_argument("--maxbrick", type=int, default=1,
                    help="build stencil-maximum bricks (one-load test of transparent samples)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "bf16"],
                    help="brick cell storage type (interpolation and compositing stay FP32)")
    ap.add_argument("--learned", type=int, default=1, help="evaluate the learned proposal")
    ap.add_argument("--precision", type=int, default=1, help="time FP16 / BF16 cell storage")
    ap.add_argument("--batch", type=int, default=1, help="time 64-view batched rendering")
    ap.add_argument("--lod", type=int, default=1, help="time level-of-detail pruning")
    ap.add_argument("--shadow", type=int, default=1, help="time secondary rays to a point light")
    ap.add_argument("--c3", type=int, default=0,
                    help="also render the deep 8-level hierarchy (~1e9 cells; minutes)")
    ap.add_argument("--log-size", type=int, default=96)
    ap.add_argument("--log-cap", type=int, default=10_000_000)
    ap.add_argument("--log-keep", type=float, default=0.3)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--heldout", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    world, rank, local = _dist()
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_1212_3333_gb300 as amr
    import synth

    hier = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(hier)
    size = args.size
    cam = synth.orbit_camera(2 + rank, size, size)   # each rank its own view
    tf_h = synth.ramp_tf()
    tf = torch.as_tensor(tf_h, device="cuda")
    ctx = amr.from_hierarchy(hier, args.dtype)
    t0 = time.perf_counter()
    ctx.amr_build_kdtree(args.storage, gradient=bool(args.gradient), halo=args.halo,
                         maxbrick=bool(args.maxbrick) and args.storage == "ptr")
    build_s = time.perf_counter() - t0
    st = ctx.amr_get_stats()
    params = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=args.shade, ert_eps=args.ert,
                                    schedule=args.schedule, samples_per_iter=args.spi)
    out = torch.empty((size, size, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    samples = ctx.amr_render(cam, tf, params, out, count_samples=True)  # also checks status
    exact_paths = list(ctx.amr_get_stats().exact_paths)
    for _ in range(args.warmup):
        ctx.amr_render(cam, tf, params, out)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _barrier(world)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for k in range(args.steps):
        starts[k].record(stream)
        ctx.amr_render(cam, tf, params, out)
        ends[k].record(stream)
    g1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    clk = clocks.stop() if clocks else None
    total_ms = g0.elapsed_time(g1)
    kern_ms = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_ms = _max_over_ranks(world, total_ms)
    all_samples = _sum_over_ranks(world, float(samples)) * args.steps
    ms_per_step = total_ms / args.steps
    value = all_samples / (total_ms * 1e-3) / 1e9
    fps = 1e3 / ms_per_step

    # end to end through the public API with host buffers: TF in, image out, every step
    e2e = None
    if args.e2e:
        tf_pin = torch.as_tensor(tf_h).pin_memory()
        img_pin = torch.empty((size, size, 4), dtype=torch.float32).pin_memory()
        ctx.amr_render_host(cam, tf_pin, params, img_pin)
        _barrier(world)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.amr_render_host(cam, tf_pin, params, img_pin)
        e2e_s = _max_over_ranks(world, time.perf_counter() - e0)
        e2e = {"value": all_samples / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(tf_h.nbytes),
               "d2h_bytes_per_step": int(img_pin.numel() * 4)}

    if rank != 0:
        return
    peak, peak_kind = _peaks()
    bps = BYTES_PER_SAMPLE[args.shade] * CELL_BYTES[args.dtype] // 4
    variant = _variant(args.storage, bool(args.gradient), args.dtype, args.halo,
                       bool(args.maxbrick) and args.storage == "ptr")
    # the march is bound by neither HBM nor any throughput unit (ncu: L1 data pipe at a
    # fifth of its peak, issue slots half busy, under half of the lanes active): the
    # roofline is the one its gathers would hit first, L1, with the algorithmic stencil
    # bytes (8 cells per trilinear sample, 7 stencils with central-difference shading)
    stencil = samples * bps / (kern_ms * 1e-3) / 1e9
    l1_peak, l1_kind = _l1_peak_gbs(clk["sm_mhz"] if clk else None)
    prof = _profiled_counters(args.shade, variant, size, args.schedule)
    traffic = prof["dram_bytes"] if prof else None
    roof = {"bound": "l1", "achieved": stencil, "peak": l1_peak, "unit": "GB/s",
            "frac": stencil / l1_peak, "peak_kind": l1_kind, "traffic": traffic,
            "stencil_gbs": stencil, "bytes_per_sample": bps,
            "l1_frac": prof["l1tex_throughput_pct"] / 100.0 if prof else None,
            "lane_efficiency": prof["threads_per_inst"] / 32.0 if prof else None,
            "issue_active": prof["issue_active_pct"] / 100.0 if prof else None,
            "l1_bytes_per_sample": (prof["l1tex_t_bytes"] / samples
                                    if prof and prof.get("l1tex_t_bytes") else None),
            "hbm": {"peak": peak, "peak_kind": peak_kind, "stencil_frac": stencil / peak,
                    "dram_frac": (traffic / (kern_ms * 1e-3) / 1e9 / peak
                                  if traffic else None)},
            "counters": (f"profiles/march_counters.json, sources {prof['sources']}"
                         if prof else "stale or missing for the current kernel sources"),
            "kernel": {0: "march_kernel", 1: "wave_kernel", 2: "persist_kernel",
                       3: "deferred_kernel"}[args.schedule] +
                      f"<{variant}, trilinear, {'phong' if args.shade else 'plain'}>",
            "kernel_ms": kern_ms}
    extra = {"frames_per_s": fps, "samples_per_frame": samples, "build_s": build_s,
             "exact_fp64_paths_per_frame": {"descent": exact_paths[0], "count": exact_paths[1],
                                            "position": exact_paths[2]},
             "tree": {"nodes": st.num_nodes, "leaves": st.num_leaves, "depth": st.max_depth,
                      "brick_mb": st.brick_bytes / 1e6}}
    if args.compare:
        comp = {}
        for s, grad in (("ptr", 0), ("ptr", 1), ("texobj", 0), ("texobj", 1),
                        ("atlas_linear", 0), ("atlas_linear", 1), ("atlas_tex3d", 0),
                        ("atlas_tex3d", 1)):
            c2 = amr.from_hierarchy(hier)
            c2.amr_build_kdtree(s, gradient=bool(grad))
            combos = ((0, 0), (1, 0), (0, 1), (1, 1)) if not grad else ((1, 0), (1, 1))
            for shade, sched in combos:
                p2 = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=shade, ert_eps=args.ert,
                                            schedule=sched)
                n2 = c2.amr_render(cam, tf, p2, out, count_samples=True)
                for _ in range(2):
                    c2.amr_render(cam, tf, p2, out)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(3):
                    c2.amr_render(cam, tf, p2, out)
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / 3
                comp[f"{s}{'+grad' if grad else ''}/{'phong' if shade else 'plain'}/"
                     f"{'wave' if sched else 'ray'}"] = {
                    "gsamples_s": n2 / ms / 1e6, "ms": ms,
                    "frac_hbm": n2 * BYTES_PER_SAMPLE[shade] / (ms * 1e-3) / 1e9 / peak}
            if s == "atlas_linear":
                s2 = c2.amr_get_stats()
                extra["atlas"] = {"dims": list(s2.atlas_dims), "efficiency": s2.atlas_efficiency,
                                  "efficiency_with_halo": s2.atlas_efficiency_halo}
            c2.amr_destroy()
        extra["storages"] = comp
    if args.shadow and world == 1 and args.storage in ("ptr", "atlas_linear") and \
            args.dtype == "f32":
        extra["shadow"] = shadow_eval(amr, ctx, vmin, vmax, args)
    if args.lod and world == 1:
        extra["lod"] = lod_eval(amr, ctx, vmin, vmax, cam, tf, out, args)
    if args.precision and world == 1:
        extra["precision"] = precision_eval(amr, hier, vmin, vmax, cam, tf, out, args, peak)
    if args.batch and world == 1 and args.storage == "ptr" and args.dtype == "f32":
        extra["batch"] = batch_eval(amr, ctx, vmin, vmax, args, peak)
        extra["batch_small_views"] = batch_eval(amr, ctx, vmin, vmax, args, peak, lo=64, hi=256,
                                                tune_views=64)
        if args.shade == 1:
            extra["batch_deferred"] = batch_eval(amr, ctx, vmin, vmax, args, peak, schedule=3)
            extra["batch_small_views_deferred"] = batch_eval(
                amr, ctx, vmin, vmax, args, peak, lo=64, hi=256, tune_views=64, schedule=3)
    if args.schedules and world == 1:
        extra["schedules"] = schedules_eval(amr, ctx, vmin, vmax, tf, args)
    if args.halos and world == 1 and args.shade == 1 and args.dtype == "f32":
        extra["halo"] = halo_eval(amr, hier, vmin, vmax, tf, args)
    if args.c3 and world == 1:
        extra["c3"] = c3_eval(amr, args, peak)
    if args.learned and world == 1:
        extra["learned"] = learned_eval(amr, ctx, hier, vmin, vmax, tf, args)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": _config(hier, args, args.storage, size), "gpu_launches": args.steps,
            "e2e": e2e, "roofline": roof, "clocks": clk, "extra": extra}
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(hier, cam, tf_h, vmin, vmax, args.shade)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
