#!/usr/bin/env python3
"""Benchmark of the point-cloud rasterizer (arXiv 1908.02681) on one GB300 per rank.

One step = one complete frame of the hot path over the whole point cloud: atomicMin rasterization
(Section 2.1, pass 1), the basic resolve, the high-quality splatting band accumulation (Section 2.2,
pass 2) and the HQ resolve that also clears the framebuffer for the next frame. `value` is points per
second through that whole frame (Gpts/s). The points are resident in HBM when the timed region starts;
`e2e` repeats the frame through the same C ABI with the points copied from pinned host memory and both
images copied back inside the timed region.

Default workload: the 100M-point synthetic LIDAR scene (sin-sum terrain over 1 km^2 + 200 box
buildings, 1 cm noise, height-ramp RGB, coherent scan order), 1920x1080, fov 60, near 0.1, far 3000,
linear 40-bit depth, eps = 1 %. It stands in for the paper's scanned data sets (Table 1), which are not
available. Inputs are 1.6 GB, larger than the 129 MB L2, so no L2 flush is needed between steps.

After the main timed region, one GPU also reports two sub-results (each timed on its own, not part of
`value`): `batched`, 64 orbit views of a 20M-point cloud at mixed resolutions in one autotuned batched frame
against the same views rendered one view per launch; and `serving`, a Poisson request stream over 6 resident
clouds served with continuous batching (frames/s, p50/p99 latency) against one request per frame.

--impl reference times the oracle (single-threaded FP64 C++) on the workload (or a bounded sample of it).
Multi-GPU (torchrun): independent replicas, one full frame per rank per step (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s atomicMin & HQ-splat, % of HBM/atomic roofline; served frames/s, p50/p99"
BYTES_PER_POINT = 16


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload(name: str):
    import scenes
    if name == "lidar100m":
        return dict(desc="LIDAR 100M points (1 km^2 sin-sum terrain + 200 boxes, 1 cm noise, coherent order), "
                         "1920x1080, fov 60, near 0.1, far 3000, 40-bit linear depth, eps 1%",
                    n=100_000_000, gen=lambda n, out: scenes.lidar(n, 2, out=out), view=scenes.lidar_1km_view())
    if name == "lidar100m-shuffled":
        def gen(n, out):
            scenes.lidar(n, 2, out=out)
            scenes.shuffle(out, 17)
        return dict(desc="LIDAR 100M points, shuffled order, 1920x1080, 40-bit linear depth, eps 1%", n=100_000_000,
                    gen=gen, view=scenes.lidar_1km_view())
    if name == "lidar20m":  # the same recipe and view at 20M points (320 MB, above L2): for profiler captures
        return dict(desc="LIDAR 20M points (the 100M recipe at 20M points), 1920x1080, fov 60, near 0.1, far 3000, "
                         "40-bit linear depth, eps 1%",
                    n=20_000_000, gen=lambda n, out: scenes.lidar(n, 2, out=out), view=scenes.lidar_1km_view())
    if name == "city400m":  # the precision study's scene
        return dict(desc="city 400M points ([-5000, 5000]^2 m, 8000 boxes, street-level detail), 3840x2160, eye 1.7 m "
                         "above the terrain, near 0.01, far 10000, 40-bit linear depth, eps 1%",
                    n=400_000_000, gen=lambda n, out: scenes.lidar(n, 4, scenes.lidar_params_city(), out=out),
                    view=scenes.city_view(4))
    if name == "cube1m":
        return dict(desc="1M points uniform in the unit cube, 640x480, fov 60, near 0.1, far 10, 40-bit linear depth",
                    n=1_000_000, gen=lambda n, out: scenes.cube(n, 1, out=out), view=scenes.cube_1m_view())
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pcr_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _code_only(text: str) -> str:
    """C++ source without its comments and with whitespace runs collapsed (the code tokens that a build sees)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", " ", text).strip()


def _csrc_digest() -> str:
    """Digest of the code (comments and layout aside) that defines the two point-pass kernels (k_raster_cert,
    k_hq_cert)."""
    h = hashlib.sha256()
    for name in ("pcr_certified.cuh", "pcr_device.cuh", "pcr_kernels.cuh"):
        f = os.path.join(ROOT, "paper_1908_02681_gb300", "csrc", name)
        with open(f, encoding="utf-8") as fh:
            h.update(name.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic(kernel: str, workload: str, n: int, args=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernels and on this
    configuration (the exact transform with the default tuning: other transforms and options run other kernels)."""
    if args is not None and (args.transform != "exact" or getattr(args, "band_filter", False) or
                             getattr(args, "band_bounds", False)):
        return None
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel][workload]
        if e.get("csrc_digest") != _csrc_digest():
            return None
        return e["bytes_per_point"] * n
    except Exception:
        return None


def host_cpu() -> dict:
    """The host the oracle runs on: CPU model and logical core count."""
    model = None
    try:  # lscpu names Arm cores too (their /proc/cpuinfo has no model line)
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in ([] if model else open("/proc/cpuinfo")):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """Time of the slowest rank (replicas: the job ends with its last rank); ms itself without dist."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed, over the slowest rank's time (units per s)."""
    return world * units_per_rank / (ms * 1e-3)


def cpu_oracle_frame(points, view, eps=(1, 100)):
    """One full frame (both passes, both resolves) of the oracle; returns seconds."""
    import oracle
    t0 = time.perf_counter()
    fb = oracle.render_atomicmin(points, view)
    oracle.resolve_basic(fb)
    acc, _ = oracle.hq_accumulate(points, view, fb, *eps)
    oracle.resolve_hq(acc)
    return time.perf_counter() - t0


def _config(wl, args, n, world=1):
    """The workload's config block, the same for both arms (the reference arm names its own point count)."""
    view = wl["view"]
    return {"workload": wl["desc"], "points": n, "width": view.width, "height": view.height,
            "transform": args.transform,
            "step": "atomicMin pass + HQ band pass + one resolve of both images (basic and HQ) with clear",
            "band_filter": "on: pass 1 records the points that may be in the eps band, pass 2 skips the others "
                           "(exact)" if getattr(args, "band_filter", False) else "off",
            "band_bounds": "on: pass 2 tests codes against per-pixel bounds from one extra kernel (exact)"
                           if getattr(args, "band_bounds", False) else "off",
            "l2": f"inputs {wl['n'] * 16 / 1e9:.2f} GB > 129 MB L2: no flush between steps",
            "parallelism": "replicas" if world > 1 else "single GPU"}


# The reference arm's work bound: point-frames over the whole run (warm-up included), about 50 s of the
# oracle on one Grace core. The driver's short runs (about 25 frames) then take the full workload.
REFERENCE_POINT_FRAMES = 3_000_000_000


def run_reference(args, wl):
    """The oracle as it stands, on host cores: the workload's full point count when the run's frames fit the
    work bound, else a bounded sample of it (the scene generated at fewer points, same recipe and view)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cap = args.reference_sample if args.reference_sample else wl["n"]
    sample_n = min(wl["n"], cap, max(1_000_000, REFERENCE_POINT_FRAMES // max(1, args.steps + args.warmup)))
    pts = np.empty((sample_n, 4), np.uint32)
    wl["gen"](sample_n, pts)
    for _ in range(args.warmup):
        cpu_oracle_frame(pts, wl["view"])
    ts = [cpu_oracle_frame(pts, wl["view"]) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    value = sample_n / t / 1e9
    if sample_n == wl["n"]:
        sample = "the full workload (every point), full frame: both passes and resolves"
    else:
        sample = (f"the workload's scene generated at {sample_n} points (same recipe and view), full frame: both "
                  f"passes and resolves")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(wl, args, sample_n, args.gpus),
        "cpu_baseline": {"value": value, "unit": "Gpts/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def pattern_ceilings(ceil, pts, n, view, npx, eps, stream, timed):
    """The two passes' framebuffer operations replayed alone for this cloud and view (visible fragments in
    point order, no transform): the memory-side floor of each pass for its own access pattern."""
    import torch
    vp = ctypes.c_void_p
    ceil.pcr_ceiling_pattern_project.argtypes = [vp, ctypes.c_uint64, vp, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int32, ctypes.c_int32, vp, vp, vp]
    ceil.pcr_ceiling_pattern_min.argtypes = [vp, vp, ctypes.c_uint64, vp, ctypes.c_int32, vp]
    ceil.pcr_ceiling_pattern_hq.argtypes = [vp, vp, ctypes.c_uint64, vp, vp, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint64, vp]
    dev = pts.device
    pix = torch.empty(n, dtype=torch.int32, device=dev)
    key = torch.empty(n, dtype=torch.int64, device=dev)
    keys = torch.full((npx,), -1, dtype=torch.int64, device=dev)
    accum = torch.zeros(2 * npx, dtype=torch.int64, device=dev)
    m12 = np.ascontiguousarray(np.asarray(view.view_proj, dtype=np.float64)[[0, 1, 3], :].reshape(-1))
    s_ptr = vp(stream.cuda_stream)
    scale = 1099511627776.0 / (view.far - view.near)
    nq = math.floor(view.near * scale)

    def check(rc):
        if rc != 0:
            raise RuntimeError(f"roofline probe failed: CUDA error {rc}")

    check(ceil.pcr_ceiling_pattern_project(vp(pts.data_ptr()), n, m12.ctypes.data, view.near, view.far,
                                           view.width, view.height, vp(pix.data_ptr()), vp(key.data_ptr()), s_ptr))
    run_min = lambda f: check(ceil.pcr_ceiling_pattern_min(vp(pix.data_ptr()), vp(key.data_ptr()), n,
                                                           vp(keys.data_ptr()), f, s_ptr))
    run_hq = lambda: check(ceil.pcr_ceiling_pattern_hq(vp(pix.data_ptr()), vp(key.data_ptr()), n,
                                                       vp(keys.data_ptr()), vp(accum.data_ptr()), eps[0], eps[1],
                                                       nq, s_ptr))
    def fresh(f):  # from a cleared framebuffer, as in a frame (the clear is not timed)
        keys.fill_(-1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_min(f)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    fresh(0)
    t_min = min(fresh(0) for _ in range(5))
    t_min_filtered = min(fresh(1) for _ in range(5))
    accum.zero_()
    run_hq()
    torch.cuda.synchronize()
    visible = int((pix != -1).sum().item())
    accepted = int((accum.view(-1, 2)[:, 1] >> 32).sum().item())
    t_hq = timed(run_hq)
    del pix, key, keys, accum
    return {"pattern_atomicmin_ms": t_min, "pattern_atomicmin_filtered_ms": t_min_filtered, "pattern_hq_ms": t_hq,
            "visible_fragments": visible, "accepted_fragments": accepted}


def run_ours(args, wl):
    import torch
    from paper_1908_02681_gb300 import build as pcr_build
    from paper_1908_02681_gb300 import pcr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pcr.load()
    n, view = wl["n"], wl["view"]
    view.transform = {"exact": 0, "fp64": 1, "double-float": 2}[args.transform]
    W, H = view.width, view.height
    npx = W * H

    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    wl["gen"](n, host)
    pts = host.to(dev)
    stream = torch.cuda.current_stream()
    img_basic = torch.empty(npx, dtype=torch.int32, device=dev)
    img_hq = torch.empty(npx, dtype=torch.int32, device=dev)
    fb = pcr.pcr_create_framebuffer(W, H, pcr.PCR_FB_HQ)
    eps = (1, 100)
    # --band-filter: pass 1 records which points may still be in the HQ band, pass 2 skips the others (exact;
    # faster for shuffled clouds, slower for scan-ordered ones)
    pcr.pcr_set_tuning(fb, 0, 8, 0, band_filter=1 if args.band_filter else 0, band_eps=eps,
                       band_bounds=1 if args.band_bounds else 0)

    names = ["raster_atomicmin", "hq_accumulate", "resolve"]

    def frame(evs=None):
        def mark(i):
            if evs is not None:
                evs[i].record(stream)
        mark(0)
        pcr.pcr_render_atomicmin(fb, pts, view, stream)
        mark(1)
        pcr.pcr_hq_accumulate(fb, pts, view, *eps, stream)
        mark(2)
        # both images (the basic one from the keys, the HQ one from the sums) and the clear, in one pass
        pcr.pcr_resolve_both(fb, img_basic, img_hq, 0, True, stream)
        mark(3)

    # roofline probes: measured random u64 atomic rate at this framebuffer size, streaming read rate
    ceil = ctypes.CDLL(pcr_build.build_ceilings())
    ceil.pcr_ceiling_random_atomics.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                                ctypes.c_void_p]
    ceil.pcr_ceiling_stream_read.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    slots = torch.full((npx,), -1, dtype=torch.int64, device=dev)
    sink = torch.empty(torch.cuda.get_device_properties(dev).multi_processor_count * 64 * 256, dtype=torch.int32,
                       device=dev)
    n_ops = 1 << 28

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    s_ptr = ctypes.c_void_p(stream.cuda_stream)
    t_at = timed(lambda: ceil.pcr_ceiling_random_atomics(ctypes.c_void_p(slots.data_ptr()), npx, n_ops, 0, s_ptr))
    atomic_rate = n_ops / (t_at * 1e-3)
    t_rd = timed(lambda: ceil.pcr_ceiling_stream_read(ctypes.c_void_p(pts.data_ptr()), n,
                                                      ctypes.c_void_p(sink.data_ptr()), s_ptr))
    read_gbs = n * BYTES_PER_POINT / (t_rd * 1e-3) / 1e9
    # FP64 and FP32 fused multiply-add rates: the FP64 rate bounds a direct FP64 evaluation of the transform
    ceil.pcr_ceiling_fma.argtypes = [ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
    fmas = ctypes.c_uint64()

    def fma_rate(fp64, iters):
        t = timed(lambda: ceil.pcr_ceiling_fma(fp64, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fmas),
                                               s_ptr))
        return fmas.value / (t * 1e-3)

    dfma_rate = fma_rate(1, 1000)
    ffma_rate = fma_rate(0, 50000)
    del slots
    pattern = pattern_ceilings(ceil, pts, n, view, npx, eps, stream, timed)

    for _ in range(args.warmup):
        frame()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = pcr.pcr_kernel_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        start.record(stream)
        for k in range(args.steps):
            frame(evs[k])
        stop.record(stream)
        torch.cuda.synchronize()
    launches = pcr.pcr_kernel_launch_count() - launches0
    if dist:
        dist.barrier()
    ms = max_over_ranks(start.elapsed_time(stop), dist, dev)
    ms_step = ms / args.steps
    per_kernel = {nm: sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)) / args.steps
                  for i, nm in enumerate(names)}
    status = pcr.pcr_get_device_status(fb)
    tier_counts = None
    if args.transform == "exact":  # how the certified transform decided each point (one extra, untimed pass)
        counts = torch.zeros(4, dtype=torch.int64, device=dev)
        pcr.pcr_clear(fb, stream)
        pcr.pcr_render_atomicmin_stats(fb, pts, view, counts, stream)
        c = [int(x) for x in counts.cpu()]
        tier_counts = {"tier1_exact": c[0], "tier1_undecided_code": c[1], "fp64_arbiter": c[2],
                       "deferred_to_tier2": c[3]}
        pcr.pcr_clear(fb, stream)

    # end to end through the C ABI with host buffers (pcr_render_frame_host): every step copies the 1.6 GB
    # of points from pinned host memory (in chunks, pass 1 starting on each chunk as it lands) and both
    # images back. Two framebuffers on two streams alternate, so one frame's upload overlaps the other's
    # compute.
    e2e = None
    if not args.no_e2e:
        fbs2 = [fb, pcr.pcr_create_framebuffer(W, H, pcr.PCR_FB_HQ)]
        d_pts2 = [pts, torch.empty_like(pts)]
        d_img2 = [torch.empty(2 * npx, dtype=torch.int32, device=dev) for _ in range(2)]
        h_img2 = [[torch.empty(npx, dtype=torch.int32, pin_memory=True) for _ in range(2)] for _ in range(2)]
        streams2 = [stream, torch.cuda.Stream()]

        def e2e_frame(k):
            i = k % 2
            pcr.pcr_render_frame_host(fbs2[i], host, view, d_pts2[i], d_img2[i], h_img2[i][0], h_img2[i][1],
                                      *eps, stream=streams2[i])

        for k in range(2):
            e2e_frame(k)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        streams2[1].wait_event(a)
        for k in range(args.steps):
            e2e_frame(k)
        stream.wait_stream(streams2[1])
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(a.elapsed_time(b) / args.steps, dist, dev)
        # the host-to-device link rate on this machine: one plain copy of the pinned points (best of 3)
        link = 0.0
        for _ in range(3):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            d_pts2[1].copy_(host, non_blocking=True)
            c1.record(stream)
            c1.synchronize()
            link = max(link, n * BYTES_PER_POINT / (c0.elapsed_time(c1) * 1e-3) / 1e9)
        link_ms = n * BYTES_PER_POINT / (link * 1e9) * 1e3
        # the same link sustained: plain copies of the points in the frames' 8 chunks, back to back on one
        # stream for as many frames as the timed loop (what the frames' uploads get on this machine over that time)
        up = torch.cuda.Stream()
        bounds = [n * k // 8 for k in range(9)]
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        c0.record(up)
        with torch.cuda.stream(up):
            for _ in range(args.steps):
                for k in range(8):
                    d_pts2[1][bounds[k]:bounds[k + 1]].copy_(host[bounds[k]:bounds[k + 1]], non_blocking=True)
        c1.record(up)
        c1.synchronize()
        sustained_ms = c0.elapsed_time(c1) / args.steps
        e2e = {"value": job_rate(n, world, e2e_ms) / 1e9, "unit": "Gpts/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": n * BYTES_PER_POINT, "d2h_bytes_per_step": 2 * npx * 4,
               "api": "pcr_render_frame_host, 2 frames in flight",
               # bound: the points' upload at the measured pinned host-to-device copy rate
               "h2d_link_gbs": link, "h2d_link_ms": link_ms, "frac_of_link": link_ms / e2e_ms,
               "h2d_sustained_gbs": n * BYTES_PER_POINT / (sustained_ms * 1e-3) / 1e9,
               "h2d_sustained_ms": sustained_ms, "frac_of_sustained_link": sustained_ms / e2e_ms}
        fbs2[1].close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    hbm_peak, peak_kind = _peaks()
    dominant = max(("raster_atomicmin", "hq_accumulate"), key=lambda k: per_kernel[k])
    kernel_name = {"raster_atomicmin": "k_raster", "hq_accumulate": "k_hq"}[dominant]
    achieved = n * BYTES_PER_POINT / (per_kernel[dominant] * 1e-3) / 1e9
    pass1_pts = n / (per_kernel["raster_atomicmin"] * 1e-3)
    hbm_pts = hbm_peak * 1e9 / BYTES_PER_POINT
    hbm_ms = n * BYTES_PER_POINT / (hbm_peak * 1e9) * 1e3
    floor1 = max(hbm_ms, min(pattern["pattern_atomicmin_ms"], pattern["pattern_atomicmin_filtered_ms"]))
    floor2 = max(hbm_ms, pattern["pattern_hq_ms"])
    result = {
        "metric": METRIC, "value": job_rate(n, world, ms_step) / 1e9, "unit": "Gpts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"exact": "f32+i64+f64", "fp64": "f64", "double-float": "f32"}[args.transform],
        "data": "synthetic",
        "config": _config(wl, args, n, world),
        "kernels_ms": per_kernel,
        "atomicmin_gpts": pass1_pts / 1e9,
        "hq_splat_gpts": n / ((per_kernel["raster_atomicmin"] + per_kernel["hq_accumulate"] +
                                per_kernel["resolve"]) * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                     "traffic": _traffic(kernel_name, args.workload, n, args)},
        "memory_floor": {
            "floor": "max(16 B/point at the measured HBM peak, the pass's framebuffer operations for this cloud "
                     "and view replayed alone in point order without the transform; pass 1: the faster of one "
                     "atomic per fragment and a stored-key read that skips atomics which cannot lower it)",
            "random_u64_atomics_per_s": atomic_rate, "fp64_dfma_per_s": dfma_rate, "fp32_ffma_per_s": ffma_rate,
            "stream_read_gbs": read_gbs, **pattern,
            "atomicmin_floor_ms": floor1, "hq_accumulate_floor_ms": floor2,
            "atomicmin_frac_of_floor": floor1 / per_kernel["raster_atomicmin"],
            "hq_accumulate_frac_of_floor": floor2 / per_kernel["hq_accumulate"],
            # pass 1 against min(HBM points/s, random-order atomic rate at one atomic per point): the roofline
            # defined on uniform random atomics, kept beside the measured floor of this cloud's own order
            "atomicmin_frac_of_random_order_roofline": pass1_pts / min(hbm_pts, atomic_rate)},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
        "device_status": status,
        "tier_counts": tier_counts,
    }
    if e2e:
        result["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        sample_n = min(n, args.cpu_sample)
        sample = host[:sample_n].numpy().view(np.uint32)
        t = cpu_oracle_frame(sample, view)
        result["cpu_baseline"] = {"value": sample_n / t / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
                                  "host": host_cpu(),
                                  "sample": f"first {sample_n} points of the workload, one full frame "
                                            f"(both passes and resolves), {t:.1f} s"}
    # the batched and serving workloads, after the main timed region, on one GPU: their own timings, reported
    # beside the frame (sub-results, not part of `value`)
    if world == 1 and not args.no_batched:
        result["batched"] = batched_results(args, 20_000_000, 64, [(640, 480), (1920, 1080), (3840, 2160)],
                                            steps=max(4, min(args.steps, 20)), warmup=max(1, min(args.warmup, 3)))
    if world == 1 and not args.no_serving:
        result["serving"] = serving_results(args, args.requests, ("continuous_batching", "one_request_per_frame"),
                                            100)
    print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_results(args, n, nv, res, steps, warmup):
    """Batched workload: n LIDAR points (seed 3), nv seeded orbit poses cycling over the resolutions res, basic
    and HQ frames. Three ways to render the same frame, all giving the same images (checked):
      * single-view launches: per view one certified render call and one resolve (the library's own
        one-view-per-launch path, the primary comparison);
      * the plain FP64 path: the same with the depth in FP64 per point, as the paper computes it (secondary);
      * the batched frame: one pcr_batch frame (chunk culling, one persistent launch per pass, one resolve),
        autotuned (pcr_batch_autotune), replayed from a CUDA graph."""
    import torch
    import scenes
    from paper_1908_02681_gb300 import pcr
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    scenes.lidar(n, 3, out=host)
    pts = host.cuda()
    del host
    views = scenes.orbit_views(nv, 3, resolutions=res)
    stream = torch.cuda.Stream()
    results = {}
    for hq in (False, True):
        flag = pcr.PCR_FB_HQ if hq else 0
        fbs = [pcr.pcr_create_framebuffer(v.width, v.height, flag) for v in views]
        outs_plain = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]
        outs_batch = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]

        def plain_frame(vs=views, outs=outs_plain):
            for v, fb, o in zip(vs, fbs, outs):
                if hq:
                    pcr.pcr_render_hq_splat(fb, pts, v, 1, 100, stream)
                else:
                    pcr.pcr_render_atomicmin(fb, pts, v, stream)
                pcr.pcr_resolve(fb, o, 0, True, stream)

        views_fp64 = [scenes.View(v.view_proj, v.near, v.far, v.width, v.height) for v in views]
        for v in views_fp64:
            v.transform = 1
        outs_fp64 = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]

        def timed(fn, k):
            for _ in range(warmup):
                fn()
            stream.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                fn()
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b) / k

        with torch.cuda.stream(stream):
            t_plain = timed(plain_frame, max(2, steps // 4))
            t_fp64 = timed(lambda: plain_frame(views_fp64, outs_fp64), 2)
            cloud = pcr.pcr_cloud_create(pts, stream)
            batch = pcr.pcr_batch_create(cloud, fbs, outs_batch, hq=hq, clear_after=True)
            pcr.pcr_batch_set_views(batch, views)
            pcr.pcr_batch_set_tuning(batch, None)
            pcr.pcr_batch_capture(batch, stream)
            t_default = timed(lambda: pcr.pcr_batch_launch(batch, stream), max(2, steps // 4))
            tuning = pcr.pcr_batch_autotune(batch, stream, force=True)
            pcr.pcr_batch_capture(batch, stream)
            t_batch = timed(lambda: pcr.pcr_batch_launch(batch, stream), steps)
            stream.synchronize()
        same = all(bool((a == b).all()) for a, b in zip(outs_plain, outs_batch)) and \
            all(bool((a == b).all()) for a, b in zip(outs_fp64, outs_batch))
        visible = pcr.pcr_batch_visible_chunks(batch)
        mode = "hq" if hq else "basic"
        results[mode] = {"batched_ms": t_batch, "single_view_launches_ms": t_plain,
                         "speedup_vs_single_view_launches": t_plain / t_batch,
                         "plain_fp64_ms": t_fp64, "speedup_vs_plain_fp64": t_fp64 / t_batch,
                         "batched_default_tuning_ms": t_default, "autotuned": tuning,
                         "point_views_per_s": nv * n / (t_batch * 1e-3), "identical_images": same,
                         "visible_chunk_fraction": sum(visible) / (nv * ((n + 1023) // 1024))}
        batch.close()
        cloud.close()
        for fb in fbs:
            fb.close()
    return {"config": {"workload": f"LIDAR {n // 1_000_000}M points (seed 3), {nv} orbit poses (seed 3), "
                                   f"{' / '.join(f'{w}x{h}' for w, h in res)} cycling, basic and HQ (eps 1%)",
                       "primary_comparison": "single-view certified launches (one view per launch)"},
            "modes": results}


def run_batched(args):
    """The batched workload alone (--workload batched): one JSON line, value = point-views/s of the basic frame."""
    import torch
    from paper_1908_02681_gb300 import pcr
    torch.cuda.set_device(0)
    pcr.load()
    res = [tuple(int(x) for x in r.split("x")) for r in args.resolutions.split(",")]
    r = batched_results(args, args.points, args.views, res, args.steps, args.warmup)
    basic = r["modes"]["basic"]
    line = {"metric": f"batched frame: point-views/s ({args.views} views, {args.points // 1_000_000}M points), "
                      f"speedup vs one view per launch",
            "value": basic["point_views_per_s"] / 1e9, "unit": "G point-views/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": basic["batched_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64+f64",
            "data": "synthetic", "config": r["config"], "modes": r["modes"]}
    print(json.dumps(line), flush=True)


def _serve_stream(pcr, server, cids, reqs, gaps_s, outs, keep):
    """Submits `reqs` at the arrival times (open loop), polls completions, returns per-request records.
    A request reuses the output ring entry of an earlier request of its resolution: it waits for that one.
    keep: optional {request index: None}, filled with a copy of those requests' images at completion."""
    import torch
    owner, done, t0 = {}, {}, time.perf_counter()
    arrival, ids, kept_ids = 0.0, {}, {}

    def take(wait_ms):
        for c in pcr.pcr_server_poll(server, 512, wait_ms):
            done[c["id"]] = c
            if c["id"] in kept_ids:
                i, out = kept_ids.pop(c["id"])
                keep[i] = out.clone()
                torch.cuda.current_stream().synchronize()   # before the ring entry is written again

    for i, (cloud, v, hq, slot) in enumerate(reqs):
        arrival += gaps_s[i]
        while time.perf_counter() - t0 < arrival:
            take(0)
        key = (v.width, v.height, slot)
        while key in owner and owner[key] not in done:
            take(1)
        out = outs[(v.width, v.height)][slot]
        rid = pcr.pcr_server_submit(server, cids[cloud], v, out, hq=hq)
        owner[key] = rid
        ids[i] = rid
        if keep is not None and i in keep:
            kept_ids[rid] = (i, out)
    while len(done) < len(reqs):
        take(10)
    torch.cuda.synchronize()
    return [done[ids[i]] for i in range(len(reqs))]


def serving_results(args, n_req, server_modes, k_plain):
    """Serving workload: 6 resident LIDAR clouds (10M, 25M, 50M, 100M, 200M, 500M points; seeds 10..15), a
    seeded Poisson request stream (mean gap 2 ms, seed 7), resolution uniform over 1280x720 / 1920x1080 /
    2560x1440 / 3840x2160, 70 % basic / 30 % HQ (eps 1 %), a seeded orbit pose per request. Served by
    pcr_server (continuous batching, 4 streams, at most 64 views and 1e9 point-views per frame, 16 GB
    framebuffer budget), by the same server without the point-view cap, and by a server that renders one
    request per frame on one stream. Latency = completion - submission (queueing
    included). Sampled requests are re-rendered alone through the single-view entry points and compared."""
    import torch
    import scenes
    from paper_1908_02681_gb300 import pcr
    sizes = [10_000_000, 25_000_000, 50_000_000, 100_000_000, 200_000_000, 500_000_000]
    if args.serving_scale != 1.0:
        sizes = [max(1024, int(n * args.serving_scale)) for n in sizes]
    host = torch.empty((max(sizes), 4), dtype=torch.int32, pin_memory=True)
    clouds = []
    for k, n in enumerate(sizes):
        scenes.lidar(n, 10 + k, out=host[:n])
        clouds.append(host[:n].cuda())
        torch.cuda.synchronize()
    del host
    res = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    rng = np.random.default_rng(7)
    gaps = rng.exponential(2e-3, n_req)
    cl = rng.integers(0, len(sizes), n_req)
    rs = rng.integers(0, len(res), n_req)
    hqs = rng.random(n_req) < 0.3
    views = scenes.orbit_views(n_req, 7, resolutions=[res[r] for r in rs])
    ring = 96
    outs = {wh: [torch.empty(wh[0] * wh[1], dtype=torch.int32, device="cuda") for _ in range(ring)] for wh in res}
    reqs = [(int(cl[i]), views[i], bool(hqs[i]), i % ring) for i in range(n_req)]
    warm_reqs = [(k % len(sizes), views[k], k % 3 == 0, k % ring) for k in range(max(args.warmup, 1) * 4)]
    sample = set(range(0, n_req, max(1, n_req // 40)))
    results = {}
    all_modes = (("continuous_batching", 4, 64, 1_000_000_000), ("continuous_batching_uncapped", 4, 64, 0),
                 ("one_request_per_frame", 1, 1, 0))
    for name, streams, per_frame, cap in [m for m in all_modes if m[0] in server_modes]:
        server = pcr.pcr_server_create(streams, per_frame, 16 << 30, cap)
        cids = [pcr.pcr_server_add_cloud(server, c) for c in clouds]
        _serve_stream(pcr, server, cids, warm_reqs, [0.0] * len(warm_reqs), outs, None)
        kept = {i: None for i in sample} if name == "continuous_batching" else None
        with ClockSampler(0) as clk:
            recs = _serve_stream(pcr, server, cids, reqs, gaps, outs, kept)
            # saturated: the same requests submitted back to back (bounded by the output rings)
            sat = _serve_stream(pcr, server, cids, reqs, [0.0] * n_req, outs, None)
        pcr.pcr_server_destroy(server)
        lat = np.array([r["done_s"] - r["submit_s"] for r in recs]) * 1e3
        span = max(r["done_s"] for r in recs) - min(r["submit_s"] for r in recs)
        sat_span = max(r["done_s"] for r in sat) - min(r["submit_s"] for r in sat)
        results[name] = {"frames_per_s": n_req / span, "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "mean_views_per_frame":
                         float(np.mean([r["batch_views"] for r in recs])),
                         "saturated_frames_per_s": n_req / sat_span,
                         "saturated_mean_views_per_frame": float(np.mean([r["batch_views"] for r in sat])),
                         "errors": int(sum(r["status"] != 0 for r in recs + sat)), "clocks": clk.summary()}
        if kept is not None:
            same = 0
            for i in sorted(kept):
                cloud, v, hq, _ = reqs[i]
                fb = pcr.pcr_create_framebuffer(v.width, v.height, pcr.PCR_FB_HQ if hq else 0)
                alone = torch.empty(v.width * v.height, dtype=torch.int32, device="cuda")
                if hq:
                    pcr.pcr_render_hq_splat(fb, clouds[cloud], v, 1, 100)
                    pcr.pcr_resolve(fb, alone, 0)
                else:
                    pcr.pcr_render_atomicmin(fb, clouds[cloud], v)
                    pcr.pcr_resolve_basic(fb, alone, 0)
                torch.cuda.synchronize()
                same += int(bool((alone == kept[i]).all()))
                fb.close()
            results[name]["sampled_identical_to_alone"] = f"{same}/{len(kept)}"
    # The plain path: each request rendered alone, one view per launch, the depth in FP64 as the paper
    # computes it (PCR_TRANSFORM_FP64), back to back on one stream, over a sample of the same requests.
    k_plain = min(n_req, k_plain)
    fb_plain = {}

    def plain_one(cloud, v, hq, out):
        key = (v.width, v.height, hq)
        if key not in fb_plain:
            fb_plain[key] = pcr.pcr_create_framebuffer(v.width, v.height, pcr.PCR_FB_HQ if hq else 0)
        fb = fb_plain[key]
        vf = scenes.View(v.view_proj, v.near, v.far, v.width, v.height)
        vf.transform = 1
        if hq:
            pcr.pcr_render_hq_splat(fb, clouds[cloud], vf, 1, 100)
            pcr.pcr_resolve(fb, out, 0, True)
        else:
            pcr.pcr_render_atomicmin(fb, clouds[cloud], vf)
            pcr.pcr_resolve_basic(fb, out, 0, True)

    for cloud, v, hq, slot in warm_reqs:
        plain_one(cloud, v, hq, outs[(v.width, v.height)][slot])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for cloud, v, hq, slot in reqs[:k_plain]:
        plain_one(cloud, v, hq, outs[(v.width, v.height)][slot])
    torch.cuda.synchronize()
    results["plain_fp64_one_view_per_launch"] = {"saturated_frames_per_s": k_plain / (time.perf_counter() - t0),
                                                 "sample_requests": k_plain}
    for fb in fb_plain.values():
        fb.close()
    cb, one = results["continuous_batching"], results["one_request_per_frame"]
    del clouds, outs
    torch.cuda.empty_cache()
    return {"config": {"workload": f"serving: clouds {[n // 1_000_000 for n in sizes]}M LIDAR points (seeds 10-15), "
                                   f"{n_req} requests, Poisson mean gap 2 ms (seed 7), 720p-4K, 70% basic / 30% HQ"},
            "frames_per_s": cb["frames_per_s"], "p50_ms": cb["p50_ms"], "p99_ms": cb["p99_ms"],
            "saturated_frames_per_s": cb["saturated_frames_per_s"], "modes": results,
            "saturated_speedup_vs_one_request_per_frame": cb["saturated_frames_per_s"] / one["saturated_frames_per_s"],
            "saturated_speedup_vs_plain_fp64": cb["saturated_frames_per_s"] /
            results["plain_fp64_one_view_per_launch"]["saturated_frames_per_s"]}


def run_serving(args):
    """The serving workload alone (--workload serving): one JSON line, value = served frames/s (Poisson)."""
    import torch
    from paper_1908_02681_gb300 import pcr
    torch.cuda.set_device(0)
    pcr.load()
    r = serving_results(args, args.requests, ("continuous_batching", "continuous_batching_uncapped",
                                              "one_request_per_frame"), 300)
    cb = r["modes"]["continuous_batching"]
    line = {"metric": "served frames/s and latency (Poisson 2 ms mean gap, 6 resident clouds)",
            "value": r["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": args.requests,
            "warmup": max(args.warmup, 1) * 4, "ms_per_step": 1e3 / r["frames_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64+f64", "data": "synthetic",
            "config": r["config"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "modes": r["modes"],
            "saturated_speedup_vs_one_request_per_frame": r["saturated_speedup_vs_one_request_per_frame"],
            "saturated_speedup_vs_plain_fp64": r["saturated_speedup_vs_plain_fp64"], "clocks": cb["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)  # about 1 s of timed frames: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lidar100m")
    ap.add_argument("--transform", choices=["exact", "fp64", "double-float"], default="exact")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="default run: skip the batched sub-result")
    ap.add_argument("--band-filter", action="store_true",
                    help="pass 1 records which points may be in the HQ band; pass 2 skips the others")
    ap.add_argument("--band-bounds", action="store_true",
                    help="pass 2 tests codes against per-pixel bounds computed by one extra kernel")
    ap.add_argument("--no-serving", action="store_true", help="default run: skip the serving sub-result")
    ap.add_argument("--cpu-sample", type=int, default=100_000_000)
    ap.add_argument("--reference-sample", type=int, default=0,
                    help="reference arm: at most this many points per frame (0: the workload's own count)")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: number of requests")
    ap.add_argument("--views", type=int, default=64, help="batched workload: number of orbit poses")
    ap.add_argument("--points", type=int, default=20_000_000, help="batched workload: cloud size")
    ap.add_argument("--resolutions", default="640x480,1920x1080,3840x2160",
                    help="batched workload: resolutions cycled by pose index")
    ap.add_argument("--serving-scale", type=float, default=1.0, help="serving workload: cloud size factor")
    args = ap.parse_args()
    if args.workload in ("batched", "batched64"):
        run_batched(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    wl = _workload(args.workload)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
