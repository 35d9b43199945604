#!/usr/bin/env python3
"""Benchmark: recolour + render frames/s of a 3M-Gaussian SH3 scene at 1080p.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--sh-dtype f32|f16|bf16] [--no-cpu-baseline] [--no-e2e]

One step is one frame through the C ABI (recogs_render with the fused edit):
select the Gaussians whose centres fall in a 12-vertex polygon covering 15%
of the view, recolour their SH coefficients with a 90-degree hue rotation,
project, bin, sort and blend into a 1920x1080 HWC float32 image. Inputs are
seeded synthetic scenes (the paper's MipNeRF360 captures are not available).
The scene (708 MB of float32 attributes) is larger than the 126 MB L2, so no
explicit flush is needed between frames.

With N > 1 (torchrun, one process per GPU) every rank renders its own replica
of the workload; the path has no cross-GPU exchange. ``--impl reference``
times the FP64 CPU oracle on the same workload instead (rank 0 only).
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

METRIC = "recolor+render frames/s at 1080p, 3M SH3 splats; % HBM roofline; vs plain FP32"
N_SPLATS = 3_000_000  # --gaussians overrides it for small profiling cases
SEED = 2
WIDTH, HEIGHT = 1920, 1080
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}


def workload_config(sh_dtype, readback=False):
    return {
        "workload": (f"recolor+render, {N_SPLATS / 1e6:g}M SH3 Gaussians ({sh_dtype} SH), "
                     f"{WIDTH}x{HEIGHT}, 12-gon selection covering 15%, 90 deg hue rotation"),
        "n_gaussians": N_SPLATS, "width": WIDTH, "height": HEIGHT, "seed": SEED,
        "sh_dtype": sh_dtype,
        "generator": "40 spheres + 20 planes in a 10^3 box, camera at distance 14, fovy 60",
        "l2": "inputs larger than L2 (708 MB scene vs 126 MB L2); no flush",
        "parallelism": "replicas (one independent frame stream per GPU)",
        "frame": ("recogs_render, fused select+recolour edit, with the mid-frame read back"
                  if readback else
                  "recogs_render, fused select+recolour edit, no mid-frame read back "
                  "(pair buffers preset from a first frame; overflow checked after the run)"),
    }


def pair_capacity(n_pairs: int) -> int:
    """Pair buffers for frames without the read back: 1/16 headroom."""
    return n_pairs + n_pairs // 16 + 4096


def make_workload():
    from paper_2511_18441_b300 import scenegen as sg
    return sg.paper_scale_workload(n=N_SPLATS, seed=SEED, width=WIDTH, height=HEIGHT)


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("RECOGS_DIST_BACKEND")
        if backend is None:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(steps: int, world: int, max_ms: float) -> float:
    """Whole-job frames/s: frames of all ranks over the slowest rank's time."""
    return steps * world / (max_ms / 1000.0)


# ---------------------------------------------------------------------------
# clocks during the timed region

class _Nvml:
    """The few read-only NVML queries the clock sampler needs, through the
    driver's libnvidia-ml (no Python package required)."""

    CLOCK_SM = 1

    def __init__(self):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")

    def handle(self, device):
        C = self.C
        import torch
        h = C.c_void_p()
        props = torch.cuda.get_device_properties(device)
        bus = getattr(props, "pci_bus_id", None)
        dom = getattr(props, "pci_domain_id", None)
        dev = getattr(props, "pci_device_id", None)
        if bus is not None and dom is not None and dev is not None:
            pci = f"{dom:08x}:{bus:02x}:{dev:02x}.0".encode()
            if self.lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(pci), C.byref(h)) == 0:
                return h
        count = C.c_uint()
        self.lib.nvmlDeviceGetCount_v2(C.byref(count))
        idx = 0 if count.value == 1 else int(device)
        if self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(idx), C.byref(h)) != 0:
            raise RuntimeError("no NVML handle for the device")
        return h

    def _u(self, fn, *args):
        v = self.C.c_uint()
        if fn(*args, self.C.byref(v)) != 0:
            raise RuntimeError(fn.__name__)
        return v.value

    def sm_mhz(self, h):
        return self._u(self.lib.nvmlDeviceGetClockInfo, h, self.C.c_int(self.CLOCK_SM))

    def sm_max_mhz(self, h):
        return self._u(self.lib.nvmlDeviceGetMaxClockInfo, h, self.C.c_int(self.CLOCK_SM))

    def power_w(self, h):
        return self._u(self.lib.nvmlDeviceGetPowerUsage, h) / 1000.0

    def reasons(self, h):
        v = self.C.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        if fn(h, self.C.byref(v)) != 0:
            raise RuntimeError("clock event reasons")
        return v.value


class ClockSampler:
    """SM clock, power and clock-event reasons of the bench's GPU, sampled
    through NVML every 50 ms on a thread while the bench runs (read-only
    queries)."""

    # NVML clock-event reason bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40}

    def __init__(self, device):
        self.device = device
        self.samples = []
        self.t0 = self.t1 = None
        self.error = None
        self._stop = threading.Event()
        self.th = None

    def start(self):
        try:
            nv = _Nvml()
            h = nv.handle(self.device)
            self.max_mhz = nv.sm_max_mhz(h)
        except Exception as e:   # no NVML: report why instead of clocks
            self.error = f"{type(e).__name__}: {e}"
            return

        def run():
            while not self._stop.is_set():
                try:
                    self.samples.append((time.time(), nv.sm_mhz(h), nv.power_w(h), nv.reasons(h)))
                except Exception as e:
                    self.error = f"{type(e).__name__}: {e}"
                    return
                self._stop.wait(0.05)

        self.th = threading.Thread(target=run, daemon=True)
        self.th.start()

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        self._stop.set()
        if self.th is not None:
            self.th.join(timeout=5)
        if not self.samples:
            return {"unavailable": self.error or "no NVML samples"}
        # samples within 0.2 s of the timed region (the region itself may be
        # shorter than the sampling period), else all of them
        near = [s for s in self.samples
                if self.t0 is not None and self.t0 - 0.2 <= s[0] <= self.t1 + 0.2]
        use = near or self.samples
        reasons = sorted({k for s in use for k, bit in self.REASONS.items() if s[3] & bit})
        return {"sm_mhz": statistics.median(s[1] for s in use), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(use), "power_w_max": max(s[2] for s in use),
                "source": "NVML, 50 ms period, samples within 0.2 s of the timed region"}


# ---------------------------------------------------------------------------
# roofline bookkeeping

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def issue_roofline(kernel, inst, ms, dev, clocks=None):
    """Warp instructions per launch over the launch time, against one warp
    instruction per cycle per SM sub-partition at the highest SM clock (the
    sampled clocks' maximum, else NVML's, else 2032 MHz)."""
    if inst is None or not ms or ms <= 0:
        return None
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz")
    if not mhz:
        try:
            nv = _Nvml()
            mhz = nv.sm_max_mhz(nv.handle(dev.index if hasattr(dev, "index") else dev))
        except Exception:
            mhz = 2032
    peak = 4.0 * sms * mhz * 1e6
    ach = inst / (ms / 1000.0)
    return {"kernel": kernel, "bound": "issue", "achieved": ach, "peak": peak,
            "unit": "warp instructions/s", "frac": ach / peak,
            "warp_instructions_per_launch": inst, "ms_per_launch": ms,
            "peak_source": f"4 issue slots x {sms} SMs x {mhz} MHz"}


def kernel_source_sha(kernel_file):
    with open(os.path.join(ROOT, "paper_2511_18441_b300", "csrc", kernel_file), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(stage):
    """DRAM bytes per launch from a committed ncu summary, or None if absent
    or taken on a different version of the kernel's source."""
    files = {"blend": "blend.cu", "preprocess": "preprocess.cu", "refit": "refit.cu",
             "blend_grad": "blend.cu"}
    if stage not in files:
        return None
    path = os.path.join(ROOT, "profiles", f"traffic_{stage}_3m_1080p.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != kernel_source_sha(files[stage]):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def profiled_instructions(stage):
    """Warp instructions per launch from a committed ncu summary, or None if
    absent or taken on a different version of the kernel's source."""
    files = {"blend": ("blend.cu", "issue_blend_3m_1080p.txt"),
             "mlp_select": ("mlp.cu", "issue_mlp_select_6m.txt")}
    if stage not in files:
        return None
    src, name = files[stage]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != kernel_source_sha(src):
        return None
    try:
        return float(kv["warp_instructions_per_launch"])
    except (KeyError, ValueError):
        return None


def algorithmic_bytes(stage, stats, n, sh_bytes):
    """Bytes a launch of `stage` must move at minimum (per-unit figures of the
    design notes x units per launch)."""
    W, H = WIDTH, HEIGHT
    tiles = stats["n_tiles"]
    n_vis = stats["n_visible"]
    pairs = stats["n_pairs"]
    if stage == "blend":
        # per consumed pair: 4 B index + 36 B record; image 12 B/pixel; 8 B range per tile
        return stats["n_pairs_read"] * 40 + 12 * W * H + 8 * tiles
    if stage == "preprocess":
        # per Gaussian: 44 B geometry read, 4 B tile count written; per
        # visible Gaussian: 48 SH coefficients read, 40 B of its 2D record
        # written (mean 8, conic 12, opacity 4, colour 12, depth 4)
        return n * (44 + 4) + n_vis * (48 * sh_bytes + 40)
    if stage == "scatter":
        # per visible Gaussian 16 B read (count, rectangle, depth key); per
        # pair one 8-byte key written
        return n_vis * 16 + pairs * 8
    if stage == "tile_sort":
        # per pair: the 8-byte key read, the 4-byte index written
        return pairs * 12
    return None


FRAME_STAGES = ("preprocess", "scatter", "tile_sort", "blend")


def frame_algorithmic_bytes(stats, n, sh_bytes):
    """The frame's minimum traffic: the sum over the stages that move the
    per-Gaussian and per-pair data."""
    return sum(algorithmic_bytes(k, stats, n, sh_bytes) for k in FRAME_STAGES)


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline leg)

def oracle_frame(w, threads=None):
    """One whole FP64 oracle frame of the workload: the per-Gaussian pass
    (selection, recolour, projection, colour), depth order, tile lists and
    every tile blended. Returns (seconds, image dict)."""
    import oracle
    t0 = time.perf_counter()
    img, *_ = oracle.render_image(w.scene, w.camera, w.edit, threads=threads)
    return time.perf_counter() - t0, img


def cpu_baseline(w, budget_s=20.0):
    """Whole oracle frames on all host cores until about budget_s / 2 of
    wall time is spent (at least one). Returns (the cpu_baseline entry, the
    last frame's image)."""
    cores = os.cpu_count() or 1
    times = []
    img = None
    while not times or sum(times) < budget_s * 0.5:
        t, img = oracle_frame(w, threads=cores)
        times.append(t)
    spent = sum(times)
    return ({"value": len(times) / spent, "unit": "frames/s", "cores": cores, "kind": "oracle",
             "sample": (f"{len(times)} whole FP64 oracle frame(s) of the workload ({N_SPLATS} "
                        f"Gaussians, all {((WIDTH + 15) // 16) * ((HEIGHT + 15) // 16)} tiles "
                        f"blended) on {cores} threads: {spent:.1f} s of wall time")}, img)


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, each step one whole frame of the
    workload on all host cores (rank 0 only)."""
    if rank != 0:
        return
    w = make_workload()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_frame(w, threads=cores)
    times = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        times.append(oracle_frame(w, threads=cores)[0])
    spent = time.perf_counter() - t0
    value = args.steps / spent
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * spent / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config("f32"),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": (f"each step one whole FP64 oracle frame of the workload "
                                    f"({N_SPLATS} Gaussians, every tile blended) on {cores} "
                                    f"threads; {args.steps} steps in {spent:.1f} s, slowest "
                                    f"{max(times):.2f} s")},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm

def run_ours(args, rank, world, local):
    import torch
    from paper_2511_18441_b300 import binding, build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_workload()
    ds = binding.DeviceScene.from_numpy(w.scene, dev, args.sh_dtype)
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream(dev)
    img = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device=dev)

    def frame():
        ctx.render(ds, w.camera, w.edit, image_out=img, stream=stream)

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        frame()
    torch.cuda.synchronize(dev)
    _, stats = ctx.render(ds, w.camera, w.edit, image_out=img, stats=True, stream=stream)
    # frames without the mid-frame read back: pair buffers sized from this
    # frame with 1/16 headroom; an overflow would be reported by check()
    capacity = pair_capacity(stats["n_pairs"])
    if not args.readback:
        ctx.set_pair_capacity(capacity)
        for _ in range(3):
            frame()
        ctx.check(stream)

    # stage breakdown (every stage timed) outside the timed region; it names
    # the dominant kernel, the only stage timed inside the timed region
    k_breakdown = max(20, args.steps // 4)
    ctx.set_timing(True)
    ctx.stage_times(reset=True)
    for _ in range(k_breakdown):
        frame()
    torch.cuda.synchronize(dev)
    breakdown = {k: v for k, v in ctx.stage_times(reset=True).items()
                 if v[1] > 0 and k not in ("h2d", "d2h")}
    ctx.set_timing(False)
    dom = max(breakdown, key=lambda k: breakdown[k][0])

    barrier(world)
    torch.cuda.synchronize(dev)
    ctx.set_timing(True, stages=[dom])
    ctx.stage_times(reset=True)
    l0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler.mark_begin()
    e0.record(stream)
    for _ in range(args.steps):
        frame()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sampler.mark_end()
    barrier(world)
    ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - l0
    stages = ctx.stage_times(reset=True)
    ctx.set_timing(False, stages=None)
    clocks = sampler.stop()
    ctx.check(stream)   # raises if any timed frame overflowed its buffers
    max_ms = max_over_ranks(ms, world, dev)
    value = aggregate_value(args.steps, world, max_ms)

    # roofline of the dominant kernel: its events (recorded on `stream`)
    # bracket each of its launches inside the timed region
    peaks, peaks_src = load_peaks()
    dom_ms = stages[dom][0] / max(stages[dom][1], 1)
    sh_bytes = 4 if args.sh_dtype == "f32" else 2
    alg = algorithmic_bytes(dom, stats, N_SPLATS, sh_bytes)
    roof = None
    if alg is not None:
        achieved = alg / (dom_ms / 1000.0) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"{peaks_src} copy bandwidth", "traffic": profiled_traffic(dom),
                "algorithmic_bytes": alg, "ms_per_launch": dom_ms,
                "timed": f"CUDA events around each {dom} launch of the {args.steps} timed frames"}
    stage_ms = {k: round(v[0] / k_breakdown, 4) for k, v in breakdown.items()}

    # the blend is bound by instruction issue, not by HBM: its warp
    # instructions per launch (a committed ncu count of this source) over its
    # measured launch time, against one warp instruction per cycle per SM
    # sub-partition at the highest SM clock seen
    roof_issue = issue_roofline(dom, profiled_instructions(dom), dom_ms, dev, clocks)

    # other stages' HBM fractions for context (from the breakdown frames)
    other = {}
    for k in FRAME_STAGES:
        if k in breakdown and k != dom:
            # bytes of the stage per frame over its time per frame (the tile
            # sort is one launch per size class)
            a = algorithmic_bytes(k, stats, N_SPLATS, sh_bytes)
            t = breakdown[k][0] / k_breakdown
            other[k] = {"achieved_gbs": a / (t / 1000.0) / 1e9,
                        "frac": a / (t / 1000.0) / 1e9 / peaks["hbm_gbs"], "ms_per_frame": t,
                        "launches_per_frame": breakdown[k][1] / k_breakdown,
                        "algorithmic_bytes": a}
    # the whole frame: the stages' algorithmic bytes over the timed frame time
    fb = frame_algorithmic_bytes(stats, N_SPLATS, sh_bytes)
    frame_ms = max_ms / args.steps
    whole = {"achieved_gbs": fb / (frame_ms / 1000.0) / 1e9,
             "frac": fb / (frame_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
             "algorithmic_bytes": fb, "ms_per_frame": frame_ms,
             "stages": list(FRAME_STAGES), "peak_source": f"{peaks_src} copy bandwidth"}

    # end to end through the public API: pinned host scene in, host image out
    def e2e_run(sh_dtype, pipelined=True):
        # every step uploads the whole scene from pinned host memory and
        # reads its image back; pipelined, step k + 1's upload overlaps step
        # k's render and read back (one recogs_render_host_frames call for
        # all steps), otherwise one recogs_render_host call per step
        hs = binding.DeviceScene.from_numpy(w.scene, "cpu", sh_dtype, pin=True)
        himg = [torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32).pin_memory()
                for _ in range(2)]
        n_e2e = max(3, min(args.steps, 20))
        if pipelined:
            frames = [(hs, w.camera, w.edit)] * n_e2e
            outs = [himg[i % 2] for i in range(n_e2e)]
            ctx.render_host_frames(frames[:2], images_out=outs[:2], stream=stream)
        else:
            ctx.render_host(hs, w.camera, w.edit, image_out=himg[0], stream=stream)
        barrier(world)
        t0 = time.perf_counter()
        if pipelined:
            ctx.render_host_frames(frames, images_out=outs, stream=stream)
        else:
            for _ in range(n_e2e):
                ctx.render_host(hs, w.camera, w.edit, image_out=himg[0], stream=stream)
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world, dev)
        h2d = sum(t.numel() * t.element_size() for t in (hs.xyz, hs.log_scale, hs.quat,
                                                          hs.opacity_logit, hs.sh))
        return {"value": n_e2e * world / el, "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": himg[0].numel() * 4, "steps": n_e2e,
                "api": ("recogs_render_host_frames (pinned host buffers; one call for all "
                        "steps, step k + 1's upload during step k's render and read back)"
                        if pipelined else "recogs_render_host (pinned host buffers), one call "
                        "per step")}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(args.sh_dtype)
        if args.sh_dtype == "f32" and not args.no_variants:
            # the same through the host with 16-bit SH storage: the
            # upload, which bounds this number, shrinks from 236 to 140 B per
            # Gaussian
            e2e["variants"] = {"bf16": e2e_run("bf16"),
                               "one_call_per_step": e2e_run("f32", pipelined=False)}

    # context: 16-bit SH storage, the frame with the read back, and the frame
    # replayed as a one-view CUDA graph (recogs_render_batch)
    variants = {}
    variant_images = {}
    if not args.no_variants:
        k = max(10, args.steps // 2)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(k):
                fn()
            a1.record(stream)
            torch.cuda.synchronize(dev)
            ctx.check(stream)
            t = a0.elapsed_time(a1) / k
            return {"frames_per_s": 1000.0 / t, "ms_per_step": t}

        if args.sh_dtype == "f32":
            for kind in ("bf16", "f16"):
                dv = binding.DeviceScene.from_numpy(w.scene, dev, kind)
                variants[kind] = timed(
                    lambda: ctx.render(dv, w.camera, w.edit, image_out=img, stream=stream))
                torch.cuda.synchronize(dev)
                variant_images[kind] = img.cpu().numpy()
                del dv
        ctx.set_pair_capacity(0)
        variants["with_readback"] = timed(frame)
        b = ctx.batch([ds], [dict(scene=0, camera=w.camera, edit=w.edit, image_out=img)],
                      graph=True)
        b(stream=stream)
        variants["graph_replay"] = timed(lambda: b(nowait=True, stream=stream))
        variants["graph_replay"]["kernel_nodes"] = ctx.batch_info()["graph_launches"]

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ctx.render(ds, w.camera, w.edit, image_out=img, stream=stream)
        torch.cuda.synchronize(dev)
        ours = img.cpu().numpy()
        cpu, ref_img = cpu_baseline(w)
        # the error of each measured form against the FP64 oracle frame
        for kind, im in [("f32", ours)] + sorted(variant_images.items()):
            d = im.astype(np.float64) - ref_img["rgb"]
            mse = float(np.mean(d ** 2))
            e = {"max_abs_error": float(np.abs(d).max()),
                 "psnr_db": 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf"),
                 "vs": "FP64 oracle frame of the float32 scene"}
            if kind == "f32":
                e["pixels_over_2e-4"] = int((np.abs(d).max(-1) > 2e-4).sum())
                e["oracle_flagged_pixels"] = int((ref_img["flag"] > 0).sum())
                # blended contributors per pixel (alpha >= 1/255, before the stop)
                e["mean_contributors_per_pixel"] = float(ref_img["ncontrib"].mean())
                accuracy = e
            else:
                variants[kind]["error"] = e

    # the batched workload and the benchmark spec's combined form (BF16 SH,
    # learned selection, one graph replay) on one GPU, so that the default
    # run records them too (each is also a workload of its own)
    if rank == 0 and world == 1 and not args.no_variants and not args.readback:
        from paper_2511_18441_b300 import scenegen as sg
        bw = sg.batched_workload(sizes=BATCH_SIZES, views_per_scene=BATCH_VIEWS_PER_SCENE)
        sub = argparse.Namespace(**vars(args))
        sub.sh_dtype, sub.steps, sub.warmup = "f32", 10, 3
        bl = run_batch(sub, rank, world, local, emit=False, bw=bw)
        variants["batch_64_views"] = {
            "views_per_s": bl["value"], "ms_per_step": bl["ms_per_step"],
            "per_view_views_per_s": bl["per_view_renders"]["views_per_s"],
            "workload": bl["config"]["workload"], "api": "recogs_render_batch, one graph replay"}
        sub.steps = 5
        cl = run_combined(sub, rank, world, local, emit=False, bw=bw)
        variants["combined_bf16_learned_batched"] = {
            "views_per_s": cl["value"], "ms_per_step": cl["ms_per_step"],
            "plain_f32_views_per_s": cl["plain_f32_form"]["views_per_s"],
            "speedup_vs_plain_f32": cl["speedup_vs_plain_f32"],
            "psnr_db_vs_fp64_oracle": {q["size"]: q["psnr_combined_db"]
                                       for q in cl["quality_vs_fp64_oracle_of_the_plain_edit"]},
            "workload": cl["config"]["workload"], "step": cl["config"]["step"]}
        torch.cuda.set_device(local)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.sh_dtype if args.sh_dtype != "f32" else "f32",
            "data": "synthetic (seeded generator; MipNeRF360 captures unavailable)",
            "config": workload_config(args.sh_dtype, args.readback),
            "gaussians_per_s": value * N_SPLATS,
            "frame_stats": stats,
            "stage_ms_per_step": stage_ms,
            "stage_ms_note": f"every stage timed by events over {k_breakdown} extra frames",
            "roofline": roof,
            "roofline_issue": roof_issue,
            "roofline_other": other,
            "roofline_frame": whole,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# the batched workload: many scenes and views in one graph replay

BATCH_SIZES = (500_000, 1_000_000, 2_000_000, 4_000_000)
BATCH_VIEWS_PER_SCENE = 16


def run_batch(args, rank, world, local, emit=True, bw=None):
    """4 scenes (0.5M, 1M, 2M, 4M Gaussians, different seeds), 16 ring views
    each at resolutions drawn from 720p/1080p/1440p/2160p, each scene with its
    own selection box and tint; one step renders all 64 views through one
    replay of the planned, autotuned batch graph (recogs_render_batch)."""
    import torch
    from paper_2511_18441_b300 import binding, build
    from paper_2511_18441_b300 import scenegen as sg
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if bw is None:
        bw = sg.batched_workload(sizes=BATCH_SIZES, views_per_scene=BATCH_VIEWS_PER_SCENE)
    scenes = [binding.DeviceScene.from_numpy(sc, dev, args.sh_dtype) for sc in bw.scenes]
    views = [dict(scene=si, camera=cam, edit=edit) for si, cam, edit in bw.views]
    pixels = sum(cam.width * cam.height for _, cam, _ in bw.views)
    splat_views = sum(bw.scenes[si].n for si, _, _ in bw.views)
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream(dev)
    b = ctx.batch(scenes, views, graph=True, tune=True)
    t0 = time.perf_counter()
    b(stream=stream)                      # plans, tunes, captures
    plan_s = time.perf_counter() - t0
    info = ctx.batch_info()

    def per_view_pass():
        for v, img in zip(views, b.images):
            ctx.render(scenes[v["scene"]], v["camera"], v["edit"], image_out=img, stream=stream)

    def timed(fn, k):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        return e0.elapsed_time(e1)

    sampler = ClockSampler(local)
    sampler.start()
    steps = args.steps
    sampler.mark_begin()
    l0 = ctx.launch_count()
    ms = timed(lambda: b(nowait=True, stream=stream), steps)
    launches = ctx.launch_count() - l0
    sampler.mark_end()
    clocks = sampler.stop()
    ctx.check(stream)
    max_ms = max_over_ranks(ms, world, dev)
    value = steps * len(views) * world / (max_ms / 1000.0)
    seq_ms = timed(per_view_pass, max(2, steps // 4)) / max(2, steps // 4)
    if rank == 0:
        line = {
            "metric": "views/s of the batched recolor+render workload (64 views, 4 scenes)",
            "value": value, "unit": "views/s", "n_gpus": world, "steps": steps,
            "warmup": max(3, args.warmup), "ms_per_step": max_ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.sh_dtype, "data": "synthetic (seeded generator)",
            "config": {"workload": (f"{len(bw.scenes)} scenes of "
                                    f"{'/'.join(f'{n / 1e6:g}M' for n in BATCH_SIZES)} Gaussians, "
                                    f"{BATCH_VIEWS_PER_SCENE} ring views each, resolutions drawn "
                                    "from 1280x720/1920x1080/2560x1440/3840x2160, per-scene box "
                                    "selection and tint"),
                       "views": len(views), "pixels_per_step": pixels,
                       "gaussian_views_per_step": splat_views, "sh_dtype": args.sh_dtype,
                       "l2": "inputs larger than L2; no flush"},
            "megapixels_per_s": pixels * steps * world / (max_ms / 1000.0) / 1e6,
            "plan": {**info, "plan_seconds": plan_s},
            "per_view_renders": {"views_per_s": len(views) / (seq_ms / 1000.0),
                                 "ms_per_step": seq_ms,
                                 "api": "recogs_render per view, with the read back"},
            "gpu_launches": launches, "clocks": clocks,
        }
        if emit:
            print(json.dumps(line), flush=True)
    ctx.close()
    return line if rank == 0 else None


# ---------------------------------------------------------------------------
# the refit tail: median depth (Sec. 3.2.2) and the SH-only refit (Sec. 3.3)

REFIT_LR = 0.005


def refit_algorithmic_bytes(stage, stats, n, n_vis):
    """Minimum bytes of one launch of the refit's own kernels."""
    W, H = WIDTH, HEIGHT
    if stage == "refit":
        # per Gaussian: 4 B count, SH, m and v (48 float32 each) read and
        # written; per visible Gaussian: 12 B position, 16 B colour record,
        # 12 B colour gradient
        return n * (4 + 6 * 48 * 4) + n_vis * (12 + 16 + 12)
    if stage == "blend_grad":
        # per consumed pair 40 B; image and target 24 B/pixel; 8 B range per
        # tile; the colour gradient of every visible Gaussian written once
        return stats["n_pairs_read"] * 40 + 24 * W * H + 8 * stats["n_tiles"] + 12 * n_vis
    return None


def oracle_refit_step(w, lr, threads):
    """One FP64 oracle refit step of the whole workload on the host cores:
    per-Gaussian pass, depth order, tile lists, full render, L1 gradient,
    colour gradient, SH gradient and an Adam step. Returns seconds."""
    import oracle
    t0 = time.perf_counter()
    sp = oracle.preprocess(w.scene, w.camera, None, threads=threads)
    order = oracle.depth_order(sp)
    tx, ty = (WIDTH + 15) // 16, (HEIGHT + 15) // 16
    off, ids = oracle.tile_lists(sp, order, tx, ty)
    y = oracle.render_tiles(sp, off, ids, threads=threads)
    target = np.clip(y["rgb"][:, :, ::-1], 0.0, None)   # any fixed target: channels swapped
    _, g = oracle.l1_loss_grad(y["rgb"], target)
    grgb = oracle.color_grad(sp, off, ids, g)
    gsh = oracle.sh_grad(w.scene, sp, grgb)
    C = np.asarray(w.scene.sh, np.float64)
    oracle.adam_step(C, gsh, np.zeros_like(gsh), np.zeros_like(gsh), 1, lr)
    return time.perf_counter() - t0


def run_refit(args, rank, world, local):
    """The refit tail at the headline workload (3M SH3 Gaussians, 1920x1080,
    polygon selection and hue rotation). (1) The median-depth render
    (Sec. 3.2.2) against the plain render, frames/s. (2) SH-only refit steps
    (Sec. 3.3) towards the edited render of the same view: forward render, L1
    colour gradient, SH gradient and Adam on every coefficient; steps/s, stage
    times, the dominant kernel's roofline, the loss before and after, and one
    FP64 oracle step on the host cores."""
    import torch
    from paper_2511_18441_b300 import binding, build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_workload()
    cam = w.camera
    n = N_SPLATS
    ds = binding.DeviceScene.from_numpy(w.scene, dev, "f32")
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream(dev)
    img = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device=dev)
    depth = torch.empty((HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    warm = max(3, args.warmup)

    def timed(fn, k):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world, dev) / k

    def stage_breakdown(fn, k):
        ctx.set_timing(True)
        ctx.stage_times(reset=True)
        for _ in range(k):
            fn()
        torch.cuda.synchronize(dev)
        b = {s: v for s, v in ctx.stage_times(reset=True).items()
             if v[1] > 0 and s not in ("h2d", "d2h")}
        ctx.set_timing(False)
        return b

    # (1) median depth: frames without the read back, like the headline frame
    _, stats_e = ctx.render(ds, cam, w.edit, image_out=img, stats=True, stream=stream)
    ctx.set_pair_capacity(pair_capacity(stats_e["n_pairs"]))
    k_depth = max(20, args.steps // 2)
    plain_ms = timed(lambda: ctx.render(ds, cam, w.edit, image_out=img, stream=stream), k_depth)
    depth_ms = timed(lambda: ctx.render_depth(ds, cam, w.edit, tau=0.5, image_out=img,
                                              depth_out=depth, stream=stream), k_depth)
    ctx.check(stream)
    bd_plain = stage_breakdown(lambda: ctx.render(ds, cam, w.edit, image_out=img,
                                                  stream=stream), 20)
    bd_depth = stage_breakdown(lambda: ctx.render_depth(ds, cam, w.edit, tau=0.5, image_out=img,
                                                        depth_out=depth, stream=stream), 20)
    covered = float((depth > 0).float().mean())

    # (2) the refit: the target is the edited render; the fitted scene starts
    # from the unedited SH coefficients; the pair capacity stays preset (the
    # geometry, hence the pairs, are those of the depth frames), so a step has
    # no mid-frame read back
    target = ctx.render(ds, cam, w.edit, stream=stream).clone()
    fit = binding.DeviceScene.from_numpy(w.scene, dev, "f32")
    m = torch.zeros((16, 3, n), dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    step = [0]

    def refit_step(want_loss=False):
        step[0] += 1
        return ctx.refit_step(fit, cam, target, m, v, step=step[0], lr=REFIT_LR,
                              want_loss=want_loss, stream=stream)

    loss_first = refit_step(want_loss=True)
    for _ in range(warm):
        refit_step()
    k_breakdown = max(10, args.steps // 4)
    breakdown = stage_breakdown(refit_step, k_breakdown)
    dom = max(breakdown, key=lambda s: breakdown[s][0])

    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize(dev)
    barrier(world)
    ctx.set_timing(True, stages=[dom])
    ctx.stage_times(reset=True)
    l0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler.mark_begin()
    e0.record(stream)
    for _ in range(args.steps):
        refit_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sampler.mark_end()
    barrier(world)
    ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - l0
    stages = ctx.stage_times(reset=True)
    ctx.set_timing(False, stages=None)
    clocks = sampler.stop()
    ctx.check(stream)   # raises if any timed step overflowed its pair buffers
    max_ms = max_over_ranks(ms, world, dev)
    loss_last = refit_step(want_loss=True)
    fitted = ctx.render(fit, cam, stream=stream)
    mse = float(((fitted - target) ** 2).mean())
    start_img = ctx.render(ds, cam, stream=stream)
    mse0 = float(((start_img - target) ** 2).mean())
    psnr = lambda e: 10.0 * math.log10(1.0 / e) if e > 0 else float("inf")
    _, stats_r = ctx.render(fit, cam, image_out=img, stats=True, stream=stream)
    n_vis = stats_r["n_visible"]

    peaks, peaks_src = load_peaks()

    def roof_of(stage, ms_launch):
        alg = refit_algorithmic_bytes(stage, stats_r, n, n_vis)
        if alg is None:
            alg = algorithmic_bytes(stage, stats_r, n, 4)
        if alg is None:
            return None
        a = alg / (ms_launch / 1000.0) / 1e9
        return {"kernel": stage, "bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                "peak_source": f"{peaks_src} copy bandwidth", "algorithmic_bytes": alg,
                "ms_per_launch": ms_launch}

    dom_ms = stages[dom][0] / max(stages[dom][1], 1)
    roof = roof_of(dom, dom_ms)
    if roof is not None:
        roof["traffic"] = profiled_traffic(dom)
        roof["timed"] = f"CUDA events around each {dom} launch of the {args.steps} timed steps"
    other = {}
    for s_ in ("refit", "blend_grad", "blend", "preprocess"):
        if s_ in breakdown and s_ != dom:
            r = roof_of(s_, breakdown[s_][0] / max(breakdown[s_][1], 1))
            if r is not None:
                other[s_] = {"achieved_gbs": r["achieved"], "frac": r["frac"],
                             "ms_per_launch": r["ms_per_launch"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sec = oracle_refit_step(w, REFIT_LR, cores)
        cpu = {"value": 1.0 / sec, "unit": "steps/s", "cores": cores, "kind": "oracle",
               "sample": (f"one whole FP64 oracle refit step of the workload ({n} Gaussians, "
                          f"{WIDTH}x{HEIGHT}: render on {cores} threads, colour gradient on one "
                          f"thread, SH gradient, numpy Adam): {sec:.1f} s")}

    if rank == 0:
        line = {
            "metric": ("SH refit steps/s at 1080p, 3M SH3 splats (render, L1 colour and SH "
                       "gradients, Adam)"),
            "value": args.steps * world / (max_ms / 1000.0), "unit": "steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": warm,
            "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator)",
            "config": {"workload": (f"SH-only refit of {n / 1e6:g}M SH3 Gaussians at "
                                    f"{WIDTH}x{HEIGHT} towards the render of the 12-gon + "
                                    f"90 deg hue edit, Adam lr {REFIT_LR}; median depth "
                                    "(tau 0.5) of the edited frame"),
                       "n_gaussians": n, "width": WIDTH, "height": HEIGHT, "seed": SEED,
                       "l2": (f"inputs larger than L2 (SH, m and v {3 * 192 * n / 1e9:.2f} GB); "
                              "no flush"),
                       "step": ("recogs_refit_step: render (pair capacity preset, no mid-frame "
                                "read back), gradient blend, SH gradient + Adam; no loss read "
                                "back")},
            "frame_stats": stats_r,
            "stage_ms_per_step": {s_: round(v_[0] / k_breakdown, 4) for s_, v_ in breakdown.items()},
            "stage_ms_note": f"every stage timed by events over {k_breakdown} extra steps",
            "roofline": roof,
            "roofline_other": other,
            "quality": {"loss_step1": loss_first, "loss_after": loss_last,
                        "steps_taken": step[0], "psnr_start_vs_target": psnr(mse0),
                        "psnr_fitted_vs_target": psnr(mse)},
            "median_depth": {
                "frames_per_s": 1000.0 / depth_ms, "ms_per_frame": depth_ms,
                "plain_frames_per_s": 1000.0 / plain_ms, "plain_ms_per_frame": plain_ms,
                "overhead_ms": depth_ms - plain_ms, "pixels_with_depth": covered,
                "blend_ms": bd_depth.get("blend", (0, 1))[0] / 20,
                "plain_blend_ms": bd_plain.get("blend", (0, 1))[0] / 20,
                "api": "recogs_render_depth (tau 0.5) vs recogs_render, pair capacity preset"},
            "cpu_baseline": cpu,
            "e2e": None,
            "e2e_note": "the refit entry points take device buffers only",
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# the learned selection workload

MLP_SPLATS = 6_000_000
MLP_TRAIN_POLYGONS = 32
MLP_EVAL_POLYGONS = 8


def run_mlp(args, rank, world, local):
    """6M Gaussians at 1920x1080: labels of 32 random polygons train the
    59-64-64-4 selection MLP on the GPU; 8 held-out polygons compare the
    learned selection (features + network + fallback decisions) with the
    plain selection: mask disagreement, PSNR of the learned render against
    the plain one and against the pixel-tinted target, fallback rate, and
    the timings (learned selection, plain selection, labels, the network's
    forward pass with its tensor-core rate)."""
    import torch
    from paper_2511_18441_b300 import binding, build
    from paper_2511_18441_b300 import scenegen as sg
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.gaussians or MLP_SPLATS
    w = sg.paper_scale_workload(n=n, seed=SEED, width=WIDTH, height=HEIGHT)
    cam = w.camera
    ds = binding.DeviceScene.from_numpy(w.scene, dev, "f32")
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream(dev)
    polys = sg.random_polygons(MLP_TRAIN_POLYGONS + MLP_EVAL_POLYGONS, WIDTH, HEIGHT, 17)
    rng = np.random.default_rng(SEED)

    def event_ms(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    # training set: features and labels of the training polygons, 1M
    # random Gaussians of each (inside the learned domain)
    feats, labs = [], []
    per_poly = min(1_000_000, n)
    for reg in polys[:MLP_TRAIN_POLYGONS]:
        F, L, V = ctx.mlp_features(ds, cam, reg, stream=stream)
        idx = torch.nonzero(V.bool()).squeeze(1)
        pick = idx[torch.from_numpy(rng.integers(0, idx.numel(), per_poly)).to(dev)]
        feats.append(F[pick])
        labs.append(L[pick])
        del F, L, V
    F = torch.cat(feats)
    L = torch.cat(labs)
    del feats, labs
    N = F.shape[0]
    net = ctx.mlp(sg.mlp_init(SEED))
    steps, B = args.mlp_steps, 16384
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    first = last = None
    for k in range(steps):
        rows = torch.from_numpy(rng.integers(0, N, B).astype(np.uint32)).to(dev)
        l = net.train_step(F, L, rows, lr=2e-3, want_loss=(k == 0 or k == steps - 1),
                           stream=stream)
        if k == 0:
            first = l
        if k == steps - 1:
            last = l
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    flop_fwd = 2 * (64 * 64 + 64 * 64 + 64 * 8)       # per sample, padded shapes
    # evaluation on held-out polygons
    tint = (0.3, 0.9, 1.4)
    M = sg.tint_matrix(tint)
    base = ctx.render(ds, cam, stream=stream).cpu().numpy()
    py, px = np.mgrid[0:HEIGHT, 0:WIDTH]
    evals = []
    for reg in polys[MLP_TRAIN_POLYGONS:]:
        xy = np.asarray(reg.xy, np.float64)
        inside = np.zeros(HEIGHT * WIDTH, bool)
        u, v = px.ravel().astype(np.float64), py.ravel().astype(np.float64)
        for i in range(len(xy)):
            (xi, yi), (xj, yj) = xy[i], xy[i - 1]
            cond = (yi > v) != (yj > v)
            with np.errstate(divide="ignore", invalid="ignore"):
                xc = xi + (v - yi) * (xj - xi) / (yj - yi)
            inside ^= cond & (u < xc)
        target = np.where(inside.reshape(HEIGHT, WIDTH)[..., None], base * np.asarray(tint), base)
        p = binding.DeviceScene.from_numpy(w.scene, dev, "f32")
        mask = torch.zeros((binding.mask_words(n),), dtype=torch.int32, device=dev)
        ctx.select(p, cam, reg, mask, stream=stream)
        ctx.recolor(p, mask, M, stream=stream)
        plain_img = ctx.render(p, cam, stream=stream).cpu().numpy()
        del p
        q = binding.DeviceScene.from_numpy(w.scene, dev, "f32")
        m2, wts, nfb = net.select(q, cam, reg, delta=0.1, stream=stream)
        ctx.recolor_weighted(q, wts, M, stream=stream)
        mlp_img = ctx.render(q, cam, stream=stream).cpu().numpy()
        del q
        b1 = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:n]
        b2 = np.unpackbits(m2.cpu().numpy().view(np.uint8), bitorder="little")[:n]

        def psnr(a, b):
            mse = float(np.mean((a.astype(np.float64) - b) ** 2))
            return 10 * math.log10(1.0 / max(mse, 1e-20))
        evals.append(dict(disagreement=float((b1 != b2).mean()), fallback=nfb / n,
                          psnr_vs_plain=psnr(mlp_img, plain_img),
                          psnr_plain_vs_target=psnr(plain_img, target),
                          psnr_learned_vs_target=psnr(mlp_img, target)))
    reg = polys[MLP_TRAIN_POLYGONS]
    mask = torch.zeros((binding.mask_words(n),), dtype=torch.int32, device=dev)
    Fe = torch.empty((n, 64), dtype=torch.bfloat16, device=dev)
    out = torch.empty((n, 4), dtype=torch.float32, device=dev)
    t_learned = event_ms(lambda: net.select(ds, cam, reg, delta=0.1, stream=stream))
    t_plain = event_ms(lambda: ctx.select(ds, cam, reg, mask, stream=stream))
    t_labels = event_ms(lambda: ctx.mlp_features(ds, cam, reg, stream=stream), reps=2)
    Fe = ctx.mlp_features(ds, cam, reg, labels=False, stream=stream)[0]
    t_fwd = event_ms(lambda: net.forward(Fe, out=out, stream=stream))
    peaks, src = load_peaks()
    tflops = n * flop_fwd / (t_fwd / 1000.0) / 1e12
    flop_sel = 2 * (64 * 64 + 64 * 64 + 64 * 16)      # per row, the tcgen05 shapes
    sel_tflops = n * flop_sel / (t_learned / 1000.0) / 1e12
    issue_roof = issue_roofline("mlp_select_tc_kernel", profiled_instructions("mlp_select")
                                if n == 6_000_000 else None, t_learned, dev)
    E = {k: float(np.mean([e[k] for e in evals])) for k in evals[0]}
    if rank == 0:
        line = {
            "metric": "learned selection Gaussians/s at 6M, 1080p (features + MLP + fallback)",
            "value": n / (t_learned / 1000.0), "unit": "Gaussians/s", "n_gpus": world,
            "steps": MLP_EVAL_POLYGONS, "warmup": 2, "ms_per_step": t_learned,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded generator)",
            "config": {"workload": (f"{n / 1e6:g}M Gaussians, {WIDTH}x{HEIGHT}, MLP 59-64-64-4 "
                                    f"GELU trained on {MLP_TRAIN_POLYGONS} random 12-gons, "
                                    f"evaluated on {MLP_EVAL_POLYGONS} held-out ones, tint "
                                    f"{tint}"),
                       "train_samples": N, "train_steps": steps, "batch": B},
            "quality_mean_over_heldout": E, "quality_per_polygon": evals,
            "training": {"seconds": train_s, "samples_per_s": steps * B / train_s,
                         "loss_first": first, "loss_last": last},
            "timings_ms": {"learned_selection": t_learned, "plain_selection": t_plain,
                           "labels_render_and_cover": t_labels, "mlp_forward": t_fwd},
            "roofline": {"kernel": ("mlp_select_tc_kernel (features + tcgen05 network + "
                                    "decisions in one kernel)"),
                         "bound": "tensor", "achieved": sel_tflops, "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": sel_tflops / peaks["bf16_tflops"],
                         "peak_source": f"{src} cuBLAS bf16 burst", "traffic": None,
                         "note": ("the tensor pipe is far from busy: the kernel is bound by "
                                  "CUDA-core issue (128 GELUs and the features per row)")},
            "roofline_issue": issue_roof,
            "forward_only_mma_sync": {"kernel": "mlp_forward_kernel (mma.sync bf16, features "
                                                "read from HBM)",
                                      "achieved_tflops": tflops, "ms": t_fwd},
        }
        print(json.dumps(line), flush=True)
    net.close()
    ctx.close()


# ---------------------------------------------------------------------------
# the combined form: BF16 SH + learned selection + batched graph launch

COMBINED_TRAIN_POLYGONS = 16


def psnr_db(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf")


def run_combined(args, rank, world, local, emit=True, bw=None):
    """The batched workload (4 scenes of 0.5/1/2/4M Gaussians, 16 ring views
    each at 720p-2160p, a box selection and tint per scene) in two forms in
    the same run. Plain FP32: float32 SH, every view through recogs_render
    with the fused plain edit. Combined: BF16 SH; per scene the learned
    selection (its box as a 4-vertex polygon, plain fallback) and the
    weighted recolour of the unedited coefficients, then all 64 views in one
    replay of the planned, tuned batch graph. Both in views/s; each form's
    PSNR on sampled views against the FP64 oracle of the plain edit."""
    import torch
    import oracle
    from paper_2511_18441_b300 import binding, build
    from paper_2511_18441_b300 import scenegen as sg
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if bw is None:
        bw = sg.batched_workload(sizes=BATCH_SIZES, views_per_scene=BATCH_VIEWS_PER_SCENE)
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream(dev)
    nv = len(bw.views)
    first = {si: k for k, (si, _, _) in reversed(list(enumerate(bw.views)))}

    # the plain FP32 form
    f32 = [binding.DeviceScene.from_numpy(sc, dev, "f32") for sc in bw.scenes]
    img_p = [torch.empty((cam.height, cam.width, 3), device=dev) for _, cam, _ in bw.views]

    def plain_step():
        for (si, cam, edit), img in zip(bw.views, img_p):
            ctx.render(f32[si], cam, edit, image_out=img, stream=stream)

    # the selection network: labels of random polygons in the 1M scene's first view
    tsi = 1
    tcam = bw.views[first[tsi]][1]
    net = ctx.mlp(sg.mlp_init(SEED))
    feats, labs = [], []
    for reg in sg.random_polygons(COMBINED_TRAIN_POLYGONS, tcam.width, tcam.height, 23):
        F, L, V = ctx.mlp_features(f32[tsi], tcam, reg, stream=stream)
        keep = V.bool()
        feats.append(F[keep])
        labs.append(L[keep])
    F = torch.cat(feats)
    L = torch.cat(labs)
    del feats, labs
    rng = np.random.default_rng(SEED)
    t0 = time.perf_counter()
    for k in range(args.mlp_steps):
        rows = torch.from_numpy(rng.integers(0, F.shape[0], 16384).astype(np.uint32)).to(dev)
        net.train_step(F, L, rows, lr=2e-3, stream=stream)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    del F, L

    # the combined form
    orig = [binding.DeviceScene.from_numpy(sc, dev, "bf16") for sc in bw.scenes]
    work = [binding.DeviceScene.from_numpy(sc, dev, "bf16") for sc in bw.scenes]
    edits = []
    for si in range(len(bw.scenes)):
        e = bw.views[first[si]][2]
        n = bw.scenes[si].n
        edits.append(dict(cam=e.select_camera, poly=sg.box_as_polygon(e.region), M=e.color_matrix,
                          mask=torch.zeros((binding.mask_words(n),), dtype=torch.int32, device=dev),
                          w=torch.empty((n, 3), dtype=torch.float32, device=dev)))
    img_c = [torch.empty((cam.height, cam.width, 3), device=dev) for _, cam, _ in bw.views]
    views_c = [dict(scene=si, camera=cam, edit=None, image_out=img)
               for (si, cam, _), img in zip(bw.views, img_c)]

    def edit_all():
        for si, e in enumerate(edits):
            work[si].sh.copy_(orig[si].sh)             # the unedited coefficients
            net.select(work[si], e["cam"], e["poly"], delta=0.1, mask_out=e["mask"],
                       weights_out=e["w"], count_fallbacks=False, stream=stream)
            ctx.recolor_weighted(work[si], e["w"], e["M"], stream=stream)

    edit_all()
    b = ctx.batch(work, views_c, graph=True, tune=True)
    b(stream=stream)                                   # plans, tunes, captures

    def combined_step():
        edit_all()
        b(nowait=True, stream=stream)

    def timed(fn, k):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world, dev) / k

    sampler = ClockSampler(local)
    sampler.start()
    sampler.mark_begin()
    l0 = ctx.launch_count()
    comb_ms = timed(combined_step, args.steps)
    launches = (ctx.launch_count() - l0) // (args.steps + max(3, args.warmup))
    sampler.mark_end()
    clocks = sampler.stop()
    ctx.check(stream)
    plain_ms = timed(plain_step, max(3, args.steps // 2))
    edit_ms = timed(edit_all, max(3, args.steps // 2))

    # quality: sampled views of the 1M scene against the FP64 oracle of the plain edit
    combined_step()
    plain_step()
    torch.cuda.synchronize(dev)
    quality = []
    fallbacks = []
    for si, e in enumerate(edits):
        _, _, nfb = net.select(work[si], e["cam"], e["poly"], delta=0.1, stream=stream)
        fallbacks.append(nfb / bw.scenes[si].n)
    edit_all()
    b(stream=stream)
    torch.cuda.synchronize(dev)
    picked = {}
    for k, (si, cam, edit) in enumerate(bw.views):
        if si == tsi and (cam.width, cam.height) in ((1280, 720), (1920, 1080)):
            picked.setdefault((cam.width, cam.height), k)
    for (W, H), k in sorted(picked.items()):
        si, cam, edit = bw.views[k]
        ref, *_ = oracle.render_image(bw.scenes[si], cam, edit)
        quality.append({"view": k, "size": f"{W}x{H}",
                        "psnr_combined_db": psnr_db(img_c[k].cpu().numpy(), ref["rgb"]),
                        "psnr_plain_f32_db": psnr_db(img_p[k].cpu().numpy(), ref["rgb"])})
    if rank == 0:
        line = {
            "metric": ("views/s of the batched recolor+render workload: BF16 SH + learned "
                       "selection + one graph replay, against the plain FP32 form"),
            "value": nv * world / (comb_ms / 1000.0), "unit": "views/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": comb_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded generator)",
            "config": {"workload": (f"{len(bw.scenes)} scenes of "
                                    f"{'/'.join(f'{n / 1e6:g}M' for n in BATCH_SIZES)} Gaussians, "
                                    f"{BATCH_VIEWS_PER_SCENE} ring views each (1280x720 to "
                                    "3840x2160), per-scene box selection (as a 4-gon) and tint"),
                       "step": ("per scene: restore the unedited BF16 SH, learned selection "
                                "(features + tcgen05 network + decisions, plain fallback at "
                                "|p - 1/2| < 0.1), weighted recolour; then one replay of the "
                                "64-view batch graph"),
                       "network": (f"59-64-64-4 GELU trained on the GPU for {args.mlp_steps} "
                                   f"steps on labels of {COMBINED_TRAIN_POLYGONS} random "
                                   "polygons of the 1M scene's first view"),
                       "l2": "inputs larger than L2; no flush"},
            "plain_f32_form": {"views_per_s": nv * world / (plain_ms / 1000.0),
                               "ms_per_step": plain_ms,
                               "api": "recogs_render per view with the fused plain edit"},
            "speedup_vs_plain_f32": plain_ms / comb_ms,
            "edit_ms_per_step": edit_ms,
            "quality_vs_fp64_oracle_of_the_plain_edit": quality,
            "fallback_fraction_per_scene": fallbacks,
            "training_seconds": train_s,
            "gpu_launches": launches, "clocks": clocks,
        }
        if emit:
            print(json.dumps(line), flush=True)
    net.close()
    ctx.close()
    return line if rank == 0 else None


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sh-dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--readback", action="store_true",
                    help="time frames with the mid-frame read back (default: pair capacity preset)")
    ap.add_argument("--workload", choices=["frame", "batch", "mlp", "refit", "combined"],
                    default="frame",
                    help="frame: the 3M/1080p headline; batch: 64 views of 4 scenes; "
                         "mlp: the learned selection at 6M Gaussians; refit: median depth "
                         "and SH-only refit steps at 3M/1080p; combined: BF16 + learned "
                         "selection + batched graph against the plain FP32 form")
    ap.add_argument("--mlp-steps", type=int, default=4000,
                    help="training steps of the mlp workload (batch 16384)")
    ap.add_argument("--gaussians", type=int, default=None,
                    help="scene size for small profiling cases (default 3,000,000)")
    args = ap.parse_args(argv)
    if args.gaussians is not None:
        global N_SPLATS
        N_SPLATS = args.gaussians
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_init()
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.workload == "batch":
            run_batch(args, rank, world, local)
        elif args.workload == "mlp":
            run_mlp(args, rank, world, local)
        elif args.workload == "refit":
            run_refit(args, rank, world, local)
        elif args.workload == "combined":
            run_combined(args, rank, world, local)
        else:
            run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
