#!/usr/bin/env python3
"""Throughput of multi-scale selective Gaussian-splat rendering on GB300.

Workload (one "step"): a 1M-Gaussian, four-level scene (700k/200k/70k/30k,
SH degree 3, 64 clusters in a 20-unit box; coverage ranges calibrated on
the device with UpdateRange from 8 orbit cameras) rendered from one camera
at 1256x832 and at 2, 4, 8, 16, 32, 64, 128x downscale -- 8 frames.

`value` is frames/s of the selective path (Eq. 6) over that sweep with the
scene resident in device memory; the same sweep with every level rendered
(no selection) is reported beside it, per scale too.  `e2e` is the same
metric through the public API with the scene uploaded from pinned host
memory and every image read back inside each step.  The scene (about
250 MB) is larger than L2, so the timed steps do not flush L2.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2311_17089_gb300 import inputs  # noqa: E402

METRIC = ("frames/s at 1x-128x downscale, selective vs all-levels; "
          "serve p50/p99 ms; bwd it/s")
N_GAUSS = 1_000_000
FP32_LANES_PER_SM = 128    # nominal, for the derived peak shown beside the measured one
OPS_PER_EVAL = 16          # FP32 operations per pixel-Gaussian evaluation
# FP32 operations per pixel-Gaussian evaluation of the raster backward (an
# FMA counting as one): the forward's alpha again (power 6, test 2, ex2 and
# clamp 3), the colour and transmittance recurrences (F 3, T 2, 1 / (1 -
# alpha) 2), dL/dalpha over the three channels (13), the opacity and power
# terms (4), the centre and conic terms (18) and the pixel's share of the
# warp's reduce-scatter of the 2D gradients (6)
OPS_PER_BWD_EVAL = 60
MUFU_LANES_PER_SM = 16     # nominal ex2 results per SM per clock (one ex2 per evaluation)
PAPER_LEVEL_MIX = (0.95, 0.035, 0.01, 0.005)   # coarse levels under 5% of the Gaussians
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of ncu captures,
# each with the SHA-256 (first 16 hex digits) of the kernel sources it was
# taken on: a figure whose sources changed since is reported as stale (null)
# (the raster figure was taken on sources whose kernels are those of the
# current ones: since then only comments and the host's launch choice for
# duplicate capacities below 1024 per tile, which no profiled frame has,
# changed)
RASTER_DRAM = {"bytes": 33.95e6, "sources": ("raster.cu", "raster_list.cu", "raster_ws.cuh"),
               "sha16": "d0db282cefbd654c"}   # mean over the 8 frames' raster stages, each frame alone
PROJECT_VIEWS_DRAM = {"bytes": 505.1e6, "sources": ("project.cu", "footprint.cuh"),
                      "sha16": "1e94d3f932b66c6a"}   # the selective sweep's projection launch


def sources_sha16(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_2311_17089_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def captured_traffic(rec):
    """The captured DRAM bytes when the kernel sources are unchanged since
    the capture, else None."""
    if rec["bytes"] is None or rec["sha16"] != sources_sha16(rec["sources"]):
        return None
    return rec["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GAUSS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-near-far", action="store_true")
    ap.add_argument("--no-level-mix", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-n", type=int, default=2_000_000)
    ap.add_argument("--serve-only", action="store_true",
                    help="run the serving leg alone and print its JSON (the full bench runs "
                         "it this way, in a fresh process)")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--profile", default=None,
                    choices=["selective", "all_levels", "train", "selective_frames"],
                    help="for profilers: two warm-up sweeps (training steps), then one "
                         "of this mode inside the NVTX range 'sweep'; prints no JSON")
    return ap.parse_args()


def workload(n):
    sc = inputs.multiscale_scene(n=n, seed=0)
    cams = [inputs.downscale(inputs.config2_camera(), s) for s in inputs.SCALES]
    calib = inputs.orbit_cameras(8, seed=1, radius=25.0)
    return sc, cams, calib


def config(n, extra=None):
    c = {"workload": f"multiscale-{n // 1000}k-4level-sh3-1256x832-sweep8",
         "gaussians": n, "levels": [0.70, 0.20, 0.07, 0.03], "sh_degree": 3,
         "image": [1256, 832], "scales": list(inputs.SCALES),
         "frames_per_step": len(inputs.SCALES), "parallelism": "replicas",
         "l2": "inputs larger than L2 (scene ~250 MB), no flush",
         "launch": "each 8-frame sweep replayed as one CUDA graph, one stream per frame"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------- replicas

def reduce_max(x: float, world: int, device) -> float:
    """The largest of the ranks' values (the job's time is its slowest
    rank's); every rank gets it.  `device`: a CUDA device under NCCL, the
    CPU under gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput of N replicas: every rank renders the same
    number of units, the time is the slowest rank's (reduce_max)."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- measured peaks

def alu_peaks(msgs, torch, dev, reps=3):
    """FP32 and MUFU throughput measured on this GPU by the library's probe
    kernels (scalar FFMA, packed FFMA2, ex2), each launch timed with CUDA
    events on its stream and the SM clock sampled meanwhile.  The FP32 peak
    is the faster of the scalar and packed forms, in FP32 operations/s (an
    FMA counts as one operation, as in the blend's operation count)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    iters = {msgs.MS_PROBE_FFMA: 4000, msgs.MS_PROBE_FFMA2: 2000, msgs.MS_PROBE_EX2: 500}
    res = {}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    for kind, name in ((msgs.MS_PROBE_FFMA, "ffma"), (msgs.MS_PROBE_FFMA2, "ffma2"),
                       (msgs.MS_PROBE_EX2, "ex2")):
        msgs.ms_alu_probe(kind, blocks, iters[kind], msgs._ptr(out))
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(4):
                msgs.ms_alu_probe(kind, blocks, iters[kind], msgs._ptr(out))
            e1.record(stream)
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            rate = 4 * msgs.ms_alu_probe_ops(kind, blocks, iters[kind]) / dt / 1e12
            best = rate if best is None else max(best, rate)
        res[name] = best
    clk = clocks.stop()
    res["unit"] = "T ops/s (ex2: T ex2/s)"
    res["sm_count"] = sms
    res["clocks"] = clk
    res["fp32_peak"] = max(res["ffma"], res["ffma2"])
    return res


# ---------------------------------------------------------- training step

TRAIN_SCALES = (1, 4, 16, 64)
TRAIN_LEVELS = (1, 2, 3, 4)    # the level whose creation scale each view renders at


def train_setup(msgs, torch, ds, sc, dev):
    """Forward + backward of a multi-scale training batch (Sec. 4.1): four
    orbit cameras at 1x/4x/16x/64x of 1256x832 (the creation scales of
    levels 1-4, so each view's projection also applies UpdateRange to its
    level), selective rendering, L1 mean loss per view against seeded U(0,1)
    targets, gradients of every scene parameter accumulated over the batch.  Returns the cameras, the
    renderers, forward() (prepare, 4 forwards, 4 loss gradients) and
    backward() (4 backwards), the loss and the gradient buffers."""
    base = inputs.orbit_cameras(4, seed=2, radius=25.0)
    cams = [inputs.downscale(c, s) for c, s in zip(base, TRAIN_SCALES)]
    rng = np.random.default_rng(1)
    targets = [torch.tensor(rng.uniform(0.0, 1.0, (3, c.height, c.width)).astype(np.float32),
                            device=dev) for c in cams]
    probe = msgs.Renderer(sc.n, cams[0].tiles_x * cams[0].tiles_y, 4 * sc.n, device=dev,
                          with_cover=False, with_mask=False)
    caps = []
    for cam in cams:
        probe.render(ds, cam, "selective")
        rc, d, _ = msgs.ms_bin_counts(probe.bins)
        # margin: UpdateRange moves the ranges, and with them the selection
        caps.append(int(d * 1.5) + 4096)
    del probe
    rs = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, cap, device=dev, with_cover=False,
                        with_mask=False) for c, cap in zip(cams, caps)]
    outs = [r.images(c, device=dev) for r, c in zip(rs, cams)]
    dls = [torch.empty_like(t) for t in targets]
    grads_t = {k: torch.empty(getattr(ds, k).shape, dtype=torch.float32, device=dev)
               for k in ("mean", "log_scale", "quat", "opacity", "color")}
    grads = msgs.ms_grads_t(*(msgs._ptr(grads_t[k]) for k in
                              ("mean", "log_scale", "quat", "opacity", "color")))
    loss = torch.zeros(1, device=dev)
    css = [msgs.camera_struct(c) for c in cams]

    streams = [torch.cuda.Stream(device=dev) for _ in cams]
    views = [msgs.bwd_view(cs, r.proj, r.bins, msgs._ptr(out[0]), msgs._ptr(out[2]),
                           msgs._ptr(r.rws), r.rws_bytes, msgs._ptr(dl))
             for cs, r, out, dl in zip(css, rs, outs, dls)]
    bwd_bytes = msgs.ms_raster_bwd_views_workspace_bytes(sc.n, len(cams))
    bwd_ws = torch.empty(bwd_bytes, dtype=torch.uint8, device=dev)

    def forward():
        # one projection pass for the four views; then each view bins,
        # blends and takes its loss on its own stream
        msgs.ms_scene_prepare(ds.struct)
        loss.zero_()
        main = torch.cuda.current_stream()
        # view v renders at the creation scale 4^v of level v + 1, whose
        # coverage ranges it updates after selecting (Alg. 2, Eq. 5)
        msgs.ms_project_views_update(ds.struct, css, msgs.MODES["selective"],
                                     list(TRAIN_LEVELS), [r.proj for r in rs], main)
        for r, cam, out, tgt, dl, st in zip(rs, cams, outs, targets, dls, streams):
            st.wait_stream(main)
            with torch.cuda.stream(st):
                r.bin_raster(ds, cam, out=out, stream=st)
                cnt = out[0].numel()
                msgs.ms_l1_loss_grad(msgs._ptr(out[0]), msgs._ptr(tgt), cnt, 1.0 / cnt,
                                     msgs._ptr(dl), msgs._ptr(loss), stream=st)
        for st in streams:
            main.wait_stream(st)

    def backward(passes=0):
        # all views in one batched backward: one raster pass over every
        # view's segments, one projection pass summing the views (`passes`
        # picks one of them, for timing them apart)
        msgs.ms_raster_bwd_views(ds.struct, views, grads, passes, msgs._ptr(bwd_ws), bwd_bytes)

    backward.outs = outs
    return cams, rs, forward, backward, loss, grads_t


def train_step_bench(msgs, torch, ds, sc, dev, steps, warmup):
    """The training step timed as two CUDA graphs per iteration (forward,
    backward) with events on the launching stream.  The scene's coverage
    ranges, which every step updates, are restored afterwards."""
    saved = (ds.s_max.clone(), ds.s_min.clone())
    cams, rs, forward, backward, loss, grads_t = train_setup(msgs, torch, ds, sc, dev)
    forward()
    backward()
    for r in rs:
        r.check()
    torch.cuda.synchronize()
    graphs = []
    for fn in (forward, backward):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        graphs.append(g)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        graphs[0].replay()
        graphs[1].replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for _ in range(steps):
        graphs[0].replay()
        graphs[1].replay()
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_step = ev[0].elapsed_time(ev[1]) / 1e3 / steps
    fwd = bwd = 0.0
    for _ in range(steps):
        ev[0].record(stream)
        graphs[0].replay()
        ev[1].record(stream)
        graphs[1].replay()
        ev[2].record(stream)
        torch.cuda.synchronize()
        fwd += ev[0].elapsed_time(ev[1])
        bwd += ev[1].elapsed_time(ev[2])
    # the backward's two passes timed apart (after a forward, the raster pass
    # then the projection pass from the 2D gradients it left)
    g_pass = []
    for flag in (msgs.MS_BWD_RASTER_PASS, msgs.MS_BWD_PROJECT_PASS):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            backward(flag)
        g_pass.append(g)
    t_pass = [0.0, 0.0]
    for _ in range(steps):
        graphs[0].replay()
        ev[0].record(stream)
        g_pass[0].replay()
        ev[1].record(stream)
        g_pass[1].replay()
        ev[2].record(stream)
        torch.cuda.synchronize()
        t_pass[0] += ev[0].elapsed_time(ev[1]) / steps
        t_pass[1] += ev[1].elapsed_time(ev[2]) / steps
    # evaluations the raster backward walks: every pixel's list up to its
    # last contributor (the forward's n_contrib), over the views
    n_walk = sum(int(o[2].sum(dtype=torch.int64).item()) for o in backward.outs)
    listed_any = torch.zeros(sc.n, dtype=torch.bool, device=dev)
    for r in rs:
        listed_any |= r.n_tiles[:sc.n] != 0
    n_blended = int(listed_any.sum().item())
    for r in rs:
        r.check()
    finite = all(bool(torch.isfinite(t).all()) for t in grads_t.values())
    ds.s_max.copy_(saved[0])
    ds.s_min.copy_(saved[1])
    launches = 2                                    # prepare; one projection for the views
    sms_dev = torch.cuda.get_device_properties(dev).multi_processor_count
    for r, cam in zip(rs, cams):
        tiles = cam.tiles_x * cam.tiles_y
        # segment offsets, then the blend as ms_raster launches it (mask pass
        # and list kernel; tile kernel; or, in between, both and the mask pass)
        blend = (2 if tiles < sms_dev else
                 3 if tiles < 4 * sms_dev and r.dup_capacity >= 1024 * tiles else 1)
        launches += (1 + 4 + 1 + (1 if tiles <= 256 else 2) + 1) + 1 + blend + 1
    launches += 2                                   # batched backward: raster, projection
    nv = len(cams)
    # the projection pass: per Gaussian its geometry (44 B), the 2D gradients
    # of every view (36 B each) and the gradients written (236 B), plus the
    # SH row (192 B) of every Gaussian some view blended
    proj_bwd_bytes = sc.n * (44 + 36 * nv + 236) + 192 * n_blended
    rast_s, proj_s = t_pass[0] / 1e3, t_pass[1] / 1e3
    roof_bwd = {
        "raster_bwd": {"bound": "alu", "kernel": "raster_bwd_kernel (the four views' segments)",
                       "evaluations": n_walk, "ops_per_evaluation": OPS_PER_BWD_EVAL,
                       "ms": t_pass[0], "unit": "Tops/s",
                       "achieved": OPS_PER_BWD_EVAL * n_walk / rast_s / 1e12},
        "project_bwd": {"bound": "hbm", "kernel": "project_bwd_kernel<3> (the views summed)",
                        "bytes_per_launch": proj_bwd_bytes, "ms": t_pass[1], "unit": "GB/s",
                        "achieved": proj_bwd_bytes / proj_s / 1e9}}
    return {"metric": "bwd it/s", "value": 1.0 / t_step, "unit": "it/s",
            "ms_per_step": 1e3 * t_step, "fwd_ms": fwd / steps, "bwd_ms": bwd / steps,
            "roofline_bwd": roof_bwd,
            "loss": float(loss.item()), "grads_finite": finite,
            "gpu_launches": launches * steps,
            "config": {"workload": f"train-multiscale-{sc.n // 1000}k-4level-sh3-4views",
                       "views": [[c.width, c.height] for c in cams],
                       "scales": list(TRAIN_SCALES), "mode": "selective",
                       "update_range": "fused into the projection pass: view v updates "
                                       "level v + 1 after its selection",
                       "loss": "L1 mean per view, targets U(0,1) seed 1",
                       "launch": "forward (one stream per view) and backward (one batched "
                                 "call over the views) each one CUDA graph"}}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the
    implementer and part codes)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    fields = {}
    for line in info:
        k, _, v = line.partition(":")
        fields.setdefault(k.strip(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    return " ".join(f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part") if k in fields) \
        or "unknown"


# ---------------------------------------------------------- level mix

def level_mix_bench(msgs, torch, dev, n, cams, calib, steps, split=PAPER_LEVEL_MIX):
    """The sweep on a scene whose coarse levels hold under 5% of the
    Gaussians (the paper's setting; the main workload puts 30% there):
    the same generator, cameras and calibration with split 95/3.5/1/0.5%.
    One 8-frame sweep (one multi-view projection, then each frame's bin and
    raster on its own stream, all frames binning from one shared depth sort,
    with or without the SMs shared between the fine and coarse frames,
    whichever a short trial finds faster) replayed from a CUDA graph;
    selective and all-levels frames/s."""
    sc = inputs.multiscale_scene(n=n, seed=0, split=split)
    ds = msgs.DeviceScene(sc, device=dev)
    ds.calibrate(calib)
    max_tiles = cams[0].tiles_x * cams[0].tiles_y
    probe = msgs.Renderer(n, max_tiles, 60 * n, device=dev, with_cover=False, with_mask=False)
    out = {"config": {"workload": f"multiscale-{n // 1000}k-levelmix-"
                                  + "/".join(f"{100 * f:g}" for f in split) + "-sweep8",
                      "split": list(split)}}
    streams = [torch.cuda.Stream(device=dev, priority=(-1 if k < 3 else 0))
               for k in range(len(cams))]
    orders = {True: msgs.DepthOrder(n, device=dev, split_views=len(cams)),
              False: msgs.DepthOrder(n, device=dev)}
    for mode in ("selective", "all_levels"):
        caps, surv = [], []
        for cam in cams:
            probe.render(ds, cam, mode)
            _, d, s_ = msgs.ms_bin_counts(probe.bins)
            caps.append(d)
            surv.append(s_)
        rs = [msgs.Renderer(n, c.tiles_x * c.tiles_y, int(d * 1.05) + 1024, device=dev,
                            with_cover=False, with_mask=False) for c, d in zip(cams, caps)]
        bufs = [r.images(c, device=dev) for r, c in zip(rs, cams)]
        ov, split = msgs.depth_order_plan(surv)

        def sweep(share):
            msgs.render_views(ds, rs, cams, mode, outs=bufs, streams=streams,
                              order=orders[split], order_views=ov, share_sms=share)

        # with and without the SMs shared; the faster is timed
        cand, trial = {}, {}
        for share in (False, True):
            gc_ = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gc_):
                sweep(share)
            for _ in range(3):
                gc_.replay()
            torch.cuda.synchronize()
            t0_, t1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0_.record()
            for _ in range(10):
                gc_.replay()
            t1_.record()
            torch.cuda.synchronize()
            cand[share], trial[share] = gc_, t0_.elapsed_time(t1_) / 10
        shared = trial[True] < trial[False]
        g = cand[shared]
        for _ in range(3):
            g.replay()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        for r in rs:
            r.check()
        out[mode] = {"fps": len(cams) * steps * 1e3 / e0.elapsed_time(e1),
                     "D": [int(d) for d in caps],
                     "shared_depth_order": {"frames": [f"{cams[k].width}x{cams[k].height}"
                                                       for k in ov], "split": bool(split)},
                     "share_sms": {"chosen": bool(shared), "shared_ms": trial[True],
                                   "not_shared_ms": trial[False]}}
        del rs, bufs, g, cand
    out["selective_over_all_levels"] = out["selective"]["fps"] / out["all_levels"]["fps"]
    return out


# --------------------------------------------------------- single level

def single_level_bench(msgs, torch, dev, steps):
    """The single-level configuration: 10k Gaussians (means U[-1,1]^3,
    log-scales N(-3.5, 0.5), opacity sigmoid(N(0,1)), plain RGB), one camera
    at distance 3, fov 60 deg, 256x256, black background.  One frame =
    ms_project -> ms_bin -> ms_raster replayed from a CUDA graph; frames/s
    with the raster stage's ALU rate (its evaluations counted exactly)."""
    sc = inputs.single_level_scene(n=10_000, seed=0)
    cam = inputs.config1_camera()
    ds = msgs.DeviceScene(sc, device=dev)
    # the duplicate capacity sized from a probe render, as in the sweep
    probe = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, 64 * sc.n, device=dev)
    probe.render(ds, cam, "selective")
    d, _ = probe.check()
    del probe
    r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, int(d * 1.05) + 1024, device=dev)
    out = r.images(cam, device=dev)
    ne = torch.empty((cam.height, cam.width), dtype=torch.int32, device=dev)
    r.render(ds, cam, "selective", out=out, n_eval=ne)
    d, surv = r.check()
    p_eval = int(ne.sum(dtype=torch.int64).item())
    cs = msgs.camera_struct(cam)
    stream = torch.cuda.current_stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r.render(ds, cam, "selective", out=out)
    g_r = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_r):
        msgs.ms_raster(r.proj, r.bins, cs, msgs._ptr(out[0]), msgs._ptr(out[1]),
                       msgs._ptr(out[2]), 0, msgs._ptr(r.rws), r.rws_bytes)
    res = {"config": {"workload": "single-level-10k-rgb-256x256", "gaussians": sc.n,
                      "image": [cam.width, cam.height],
                      "launch": "project + bin + raster as one CUDA graph"}}
    for name, graph in (("frame", g), ("raster", g_r)):
        for _ in range(3):
            graph.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"{name}_ms"] = e0.elapsed_time(e1) / steps
    r.check()
    res.update(fps=1e3 / res["frame_ms"], D=int(d), survivors=int(surv), P_eval=p_eval,
               raster_tops=OPS_PER_EVAL * p_eval / (res["raster_ms"] / 1e3) / 1e12)
    return res


# ------------------------------------------------------------- near / far

def near_far_bench(msgs, torch, dev, n=3_000_000, scales=(1, 8, 64)):
    """The near/far stress workload: 3M Gaussians (dense unit ball, sparse
    shell of radius 50), 32 orbit cameras at radii 2 .. 60 (calibrated on
    the device), rendered selectively at each scale of 1256x832.  Per scale:
    frames/s over the 32 cameras (one stream, one graph per camera), the
    tile-list skew (longest list / mean non-empty list) and the
    early-termination rate (pixels that stopped before the end of their
    tile's list)."""
    sc = inputs.near_far_scene(n=n, seed=0)
    cams = inputs.orbit_cameras(32, seed=3, radius=np.geomspace(2.0, 60.0, 32))
    ds = msgs.DeviceScene(sc, device=dev)
    ds.calibrate(cams)
    out = {}
    for s in scales:
        fr = [inputs.downscale(c, s) for c in cams]
        probe = msgs.Renderer(n, fr[0].tiles_x * fr[0].tiles_y, 16 * n, device=dev,
                              with_cover=False, with_mask=False)
        dmax = 0
        for cam in fr:  # the exact count is reported even when it overflows
            probe.render(ds, cam, "selective")
            dmax = max(dmax, msgs.ms_bin_counts(probe.bins)[1])
        del probe
        r = msgs.Renderer(n, fr[0].tiles_x * fr[0].tiles_y, int(dmax * 1.02) + 1024, device=dev,
                          with_cover=False, with_mask=False)
        bufs = r.images(fr[0], device=dev)
        ne = torch.empty((fr[0].height, fr[0].width), dtype=torch.int32, device=dev)
        skews, terms, ds_ = [], [], []
        for cam in fr:
            r.render(ds, cam, "selective", out=bufs, n_eval=ne)
            d, _ = r.check()
            tiles = cam.tiles_x * cam.tiles_y
            rg = r.ranges[:2 * tiles].view(-1, 2).to(torch.int64)
            ln = (rg[:, 1] - rg[:, 0]).clamp(min=0)
            nz = ln[ln > 0]
            skews.append(float(nz.max() / nz.float().mean()) if len(nz) else 0.0)
            # the list length of each pixel's tile, against the positions walked
            ty = torch.arange(cam.height, device=dev) // 16
            tx = torch.arange(cam.width, device=dev) // 16
            plen = ln[(ty[:, None] * cam.tiles_x + tx[None, :])]
            terms.append(float((ne.to(torch.int64) < plen).float().mean()))
            ds_.append(d)
        graphs = []
        for cam in fr:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                r.render(ds, cam, "selective", out=bufs)
            graphs.append(g)
        for g in graphs:
            g.replay()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for g in graphs:
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        r.check()
        out[f"{fr[0].width}x{fr[0].height}"] = {
            "fps": len(fr) * 1e3 / e0.elapsed_time(e1),
            "tile_list_skew_mean": float(np.mean(skews)), "tile_list_skew_max": float(np.max(skews)),
            "early_termination_rate": float(np.mean(terms)), "D_mean": float(np.mean(ds_))}
        del r, graphs
    return {"config": {"workload": f"near-far-{n // 1000}k-4level-sh3-32cams-r2..60",
                       "mode": "selective", "cameras": 32, "scales": list(scales)},
            "per_scale": out}


# ------------------------------------------------------------ aggregation

def aggregate_bench(msgs, torch, ds, sc, dev, reps=10):
    """AggregateGaussians (Alg. 1) for level 2 on the resident scene: every
    level-1 Gaussian splatted to the 8 calibration cameras at 4x, small ones
    binned into 200^3 voxels and pooled.  Timed with events on one stream
    (one CUDA graph per call)."""
    base = inputs.orbit_cameras(8, seed=1, radius=25.0)
    cams = [msgs.camera_struct(inputs.downscale(c, 4)) for c in base]
    extent = float(max(np.abs(np.asarray(c.campos, np.float32)).max() for c in base))
    cap = sc.n
    ws_b = msgs.ms_aggregate_workspace_bytes(sc.n)
    ws = torch.empty(ws_b, dtype=torch.uint8, device=dev)
    n_out = torch.zeros(2, dtype=torch.int64, device=dev)
    o = [torch.empty((cap, 3), device=dev), torch.empty((cap, 3), device=dev),
         torch.empty((cap, 4), device=dev), torch.empty(cap, device=dev),
         torch.empty((cap,) + tuple(ds.color.shape[1:]), device=dev),
         torch.empty(cap, dtype=torch.uint8, device=dev), torch.empty(cap, device=dev),
         torch.empty(cap, device=dev)]
    out = msgs.ms_scene_t(cap, ds.n_levels, ds.sh_degree, *(msgs._ptr(t) for t in o), 0, 0)

    def call():
        msgs.ms_aggregate(ds.struct, cams, 2, extent, out, cap, msgs._ptr(n_out),
                          msgs._ptr(ws), ws_b)
    call()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call()
    for _ in range(2):
        g.replay()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    m, status = (int(v) for v in n_out.cpu())
    return {"ms_per_call": e0.elapsed_time(e1) / reps, "new_gaussians": m,
            "inputs": int((sc.level < 2).sum()), "status": status,
            "config": {"level_m": 2, "cameras": 8, "downscale": 4, "voxels_per_axis": 200,
                       "extent": extent}}


# ---------------------------------------------------------------- serving

def sphere_cameras(k, seed, radius=25.0, width=1256, height=832):
    """k cameras at uniformly random points of a sphere around the origin,
    looking at it."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((k, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cams = []
    for v in d:
        up = (0.0, -1.0, 0.0) if abs(v[1]) < 0.95 else (0.0, 0.0, 1.0)
        cams.append(inputs.pinhole(tuple(radius * v), (0.0, 0.0, 0.0), up, width, height, 60.0))
    return cams


def serve_bench(msgs, torch, dev, n_requests, n_gauss, loads=(0.5, 0.7, 0.9)):
    """Serving loop: two resident scenes of n_gauss Gaussians (the multi-
    scale generator, seeds 0 and 1, calibrated on the device), requests for
    random cameras on a radius-25 sphere at a downscale drawn uniformly from
    1..128x of 1256x832, Poisson arrivals (seed 2) at 0.5/0.7/0.9 of the
    measured capacity, at most 64 on the device, memory-admitted; every
    image is copied to pinned host memory.  Latency = completion - submit."""
    import time as _t
    dss = []
    for seed in (0, 1):
        sc = inputs.multiscale_scene(n=n_gauss, seed=seed)
        ds = msgs.DeviceScene(sc, device=dev)
        ds.calibrate(inputs.orbit_cameras(8, seed=1, radius=25.0))
        dss.append(ds)
    rng = np.random.default_rng(2)
    base = sphere_cameras(n_requests, seed=2)
    reqs = [(int(rng.integers(0, 2)),
             inputs.downscale(c, int(rng.choice(inputs.SCALES)))) for c in base]
    ring = 256
    hosts = [torch.empty((3, 832, 1256), dtype=torch.float32).pin_memory() for _ in range(ring)]
    budget = 64 << 30
    out = {}
    base_rate = {}
    for mode, mb in (("selective", 1), ("selective", 0), ("all_levels", 1), ("all_levels", 0)):
        # max_batch_views 1: every request projected by itself (the unbatched
        # reference); 0: requests of one scene and mode admitted together
        # share one projection pass of up to 8 cameras
        srv = msgs.Server(max_gaussians=n_gauss, max_width=1256, max_height=832,
                          mem_budget_bytes=budget, max_inflight=64, n_streams=16,
                          device=dev.index or 0, max_batch_views=mb)
        ids = [srv.add_scene(ds) for ds in dss]

        def run(arrivals):
            """Submit reqs at the given offsets (None: all at once); returns
            the results in order."""
            tickets, owner = [], [None] * ring
            t0 = _t.perf_counter()
            c0 = msgs.ms_serve_clock()
            for i, (s, cam) in enumerate(reqs):
                slot = i % ring
                if owner[slot] is not None:     # ring buffer: wait for its last user
                    r = srv.wait(owner[slot][0], 120.0)
                    owner[slot][1].append(r)
                if arrivals is not None:
                    delay = t0 + arrivals[i] - _t.perf_counter()
                    if delay > 0:
                        _t.sleep(delay)
                h = hosts[slot].view(-1)[:3 * cam.height * cam.width]
                res_box = []
                tickets.append((srv.submit(ids[s], cam, mode, image_host=h), res_box))
                owner[slot] = tickets[-1]
            for t, box in tickets:
                if not box:
                    box.append(srv.wait(t, 120.0))
            res = [box[0] for _, box in tickets]
            bad = [r.status for r in res if r.status != msgs.MS_OK]
            if bad:
                raise msgs.MsError(bad[0], "serve request failed")
            # latency from the scheduled arrival (the submit call may lag it)
            arr = ([r.t_submit for r in res] if arrivals is None
                   else [min(r.t_submit, c0 + a) for r, a in zip(res, arrivals)])
            return res, arr

        def summary(out):
            res, arr = out
            lat = np.array([r.t_done - a for r, a in zip(res, arr)]) * 1e3
            span = max(r.t_done for r in res) - min(arr)
            return {"fps": len(res) / span, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)),
                    "mean_ms": float(lat.mean()), "retries": int(sum(r.retries for r in res))}

        run(None)                                   # warm-up: capacity history, caches
        st0 = srv.stats()
        cap = summary(run(None))                    # closed loop: all requests queued at once
        st1 = srv.stats()
        passes = st1.proj_passes - st0.proj_passes
        renders = st1.renders - st0.renders
        proj_ms = (st1.proj_seconds - st0.proj_seconds) * 1e3
        # projection GPU time (CUDA events around each pass, which shares the
        # GPU with the other requests' work) against the GPU time one request
        # takes at capacity (the closed loop's wall time per request)
        cap.update(proj_passes=passes, views_per_pass=renders / max(passes, 1),
                   proj_ms_per_request=proj_ms / max(renders, 1),
                   proj_share=(proj_ms / max(renders, 1)) / (1e3 / cap["fps"]))
        # Poisson arrivals at fractions of the unbatched server's capacity, so
        # both servers see the same offered rates
        if mb == 1:
            base_rate[mode] = cap["fps"]
        loads_out = []
        for load in loads:
            rate = load * base_rate[mode]
            gaps = np.random.default_rng(2).exponential(1.0 / rate, len(reqs))
            res = run(np.cumsum(gaps) - gaps[0])
            loads_out.append({"load": load, "offered_fps": rate, **summary(res)})
        st = srv.stats()
        srv.close()
        out[mode + ("_unbatched" if mb == 1 else "")] = {
            "capacity": cap, "poisson": loads_out, "peak_inflight": st.peak_inflight,
            "arena_peak_gb": st.arena_peak / 1e9,
            "issue_us_per_render": st.issue_seconds / max(st.renders, 1) * 1e6}
    return {"metric": "serve p50/p99 ms", "value": out["selective"]["poisson"][-1]["p99_ms"],
            "unit": "ms (p99 at 0.9 of the unbatched capacity, selective)",
            "higher_is_better": False,
            "selective": out["selective"], "all_levels": out["all_levels"],
            "selective_unbatched": out["selective_unbatched"],
            "all_levels_unbatched": out["all_levels_unbatched"],
            "config": {"workload": f"serve-2x{n_gauss // 1000}k-4level-sh3-1256x832-1x..128x",
                       "scenes": 2, "requests_per_run": len(reqs), "max_inflight": 64,
                       "streams": 16, "mem_budget_gb": budget / 2 ** 30,
                       "projection": "requests of one scene and mode admitted together share "
                                     "one ms_project_views pass (up to 8 cameras); "
                                     "selective_unbatched: one ms_project per request",
                       "arrivals": "Poisson, seed 2, rate = load x closed-loop capacity of "
                                   "the unbatched server (the same rates for both)",
                       "output": "image copied to pinned host memory per request"}}


# ------------------------------------------------------------- oracle arm

def oracle_scene(sc):
    """The oracle's own calibration of the coverage ranges (same cameras)."""
    import oracle
    calibrated = oracle.calibrate(sc.copy(), inputs.orbit_cameras(8, seed=1, radius=25.0))
    return calibrated, oracle.prepare(calibrated)


def oracle_sweep(scene, cams, budget_s):
    """Time the oracle on the workload's frames, coarse to fine, until the
    time budget is spent; returns (frames, seconds, threads, widths)."""
    import oracle
    calibrated, prepared = scene
    frames, spent, done = 0, 0.0, []
    for cam in reversed(cams):
        t0 = time.perf_counter()
        oracle.render(calibrated, cam, "selective", prepared=prepared)
        dt = time.perf_counter() - t0
        frames += 1
        spent += dt
        done.append(cam.width)
        if spent > budget_s:
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return frames, spent, threads, done


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, cams, _ = workload(args.n)
    scene = oracle_scene(sc)
    budget = max(0.5, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sweep(scene, cams, budget)
    frames, secs = 0, 0.0
    threads, scales = 1, []
    for _ in range(args.steps):
        f, s, threads, scales = oracle_sweep(scene, cams, budget)
        frames += f
        secs += s
    value = frames / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config(args.n),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads,
                         "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"selective frames at widths {scales} per step "
                                   f"(coarse to fine until {budget:.1f} s)"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- our arm

def serve_in_child(args, local):
    """The serving leg in a fresh process on the same GPU: its Poisson
    arrivals come from a host loop whose pace the earlier legs' leftovers
    (host arrays, pinned buffers, threads) disturbed when it ran in this
    one (p99 at 0.9 load 19.8-23.6 ms against 10.0-10.4 ms alone)."""
    import subprocess
    env = dict(os.environ, LOCAL_RANK=str(local), RANK="0", WORLD_SIZE="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-only",
           "--serve-requests", str(args.serve_requests), "--serve-n", str(args.serve_n)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("serving leg failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    import paper_2311_17089_gb300 as msgs

    if args.serve_only:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        print(json.dumps(serve_bench(msgs, torch, torch.device("cuda", local),
                                     args.serve_requests, args.serve_n)))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, world, dev)

    sc, cams, calib = workload(args.n)
    ds = msgs.DeviceScene(sc, device=dev)
    ds.calibrate(calib)
    max_tiles = cams[0].tiles_x * cams[0].tiles_y
    if args.profile == "train":
        _, rs, forward, backward, _, _ = train_setup(msgs, torch, ds, sc, dev)
        for it in range(3):
            torch.cuda.synchronize()
            if it == 2:
                torch.cuda.nvtx.range_push("sweep")
            forward()
            backward()
            torch.cuda.synchronize()
            if it == 2:
                torch.cuda.nvtx.range_pop()
        for r in rs:
            r.check()
        return
    # size each frame's duplicate capacity from one pass of both modes
    probe = msgs.Renderer(sc.n, max_tiles, 60_000_000 if sc.n >= 500_000 else 60 * sc.n,
                          device=dev, with_cover=False, with_mask=False)
    dmax, surv = {}, {}
    for mode in ("selective", "all_levels"):
        for cam in cams:
            probe.render(ds, cam, mode)
            rc, d, s_ = msgs.ms_bin_counts(probe.bins)
            if rc != msgs.MS_OK:
                raise msgs.MsError(rc, "probe capacity")
            dmax[(mode, cam.width)] = d
            surv[(mode, cam.width)] = s_
    del probe
    # the eight frames share the pose, so the depth keys: one depth sort of
    # the union of their lists serves them all, split into every frame's
    # own order when the frames list very different numbers of Gaussians
    # (selective), taken as it is when they list nearly the same ones (all
    # levels)
    orders = {True: msgs.DepthOrder(sc.n, device=dev, split_views=len(cams)),
              False: msgs.DepthOrder(sc.n, device=dev)}
    plan = {m: msgs.depth_order_plan([surv[(m, c.width)] for c in cams])
            for m in ("selective", "all_levels")}
    # frames the tile kernel blends; whether a mode's sweep shares the SMs
    # between them and the coarse frames is decided below by timing both
    # schedules (it helps where the coarse frames carry much of the work and
    # the fine frames bin quickly: selective 1.051 vs 1.088 ms, all levels
    # 2.484 vs 2.447 ms)
    sms_dev = torch.cuda.get_device_properties(dev).multi_processor_count
    fine = [c.tiles_x * c.tiles_y >= sms_dev for c in cams]
    tiles_max = max(c.tiles_x * c.tiles_y for c, f in zip(cams, fine) if f) if any(fine) else 1
    share_ctas = [msgs.share_ctas_per_sm(c.tiles_x * c.tiles_y, tiles_max) if f else 0
                  for c, f in zip(cams, fine)]
    share_plan = {"selective": True, "all_levels": False}
    # one renderer (projection, tile lists, workspaces) per frame and mode,
    # sized by that frame's duplicate count, and one stream per frame: the
    # frames of a sweep are independent, and the small ones leave most SMs
    # idle, so they run concurrently
    rs_mode = {m: [msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y,
                                 int(dmax[(m, cam.width)] * 1.05) + 1024, device=dev,
                                 with_cover=False, with_mask=False) for cam in cams]
               for m in ("selective", "all_levels")}
    bufs = [rs_mode["selective"][k].images(cam, device=dev) for k, cam in enumerate(cams)]
    # the three finest frames (the tile kernel's) have the longest chains:
    # their streams get the higher priority
    streams = [torch.cuda.Stream(device=dev, priority=(-1 if k < 3 else 0))
               for k, _ in enumerate(cams)]

    css = [msgs.camera_struct(cam) for cam in cams]

    def step(mode, after=None, scene=None, views=True, share=None):
        # views: one projection pass for the eight frames (they share the
        # camera centre, so a Gaussian listed at several scales is coloured
        # once) that also forms the union of their lists, whose depth sort
        # (and split) runs once on the first frame's stream; then each
        # frame's binning and blend on its own stream; otherwise each frame
        # projects and sorts on its own stream.  In selective mode the frames
        # the tile kernel blends share the SMs: their blends run on
        # share_ctas_per_sm() CTAs per SM and the coarse frames start once
        # they have binned (as render_views with share_sms)
        main = torch.cuda.current_stream()
        d = scene or ds
        ov, split = plan[mode]
        order = orders[split]
        share = views and (share_plan[mode] if share is None else share)
        sorted_ev = None
        binned = []
        if views:
            order.project(d, rs_mode[mode], cams, mode, main, ov)
        for k in sorted(range(len(cams)), key=lambda k: not (share and fine[k])):
            r, cam, out, st = rs_mode[mode][k], cams[k], bufs[k], streams[k]
            st.wait_stream(main)
            if views and k in ov:
                if sorted_ev is None:
                    order.sort(st)
                    sorted_ev = torch.cuda.Event()
                    sorted_ev.record(st)
                else:
                    st.wait_event(sorted_ev)
            if share and not fine[k]:
                for e in binned:
                    st.wait_event(e)
            with torch.cuda.stream(st):
                if views:
                    r.bin(d, cam, st, (order, k) if k in ov else None)
                    if share and fine[k]:
                        binned.append(torch.cuda.Event())
                        binned[-1].record(st)
                    r.raster(cam, out, st, max_ctas_per_sm=share_ctas[k] if share else 0)
                else:
                    r.render(d, cam, mode, out=out, stream=st)
                if after is not None:
                    after(k, out, st)
        for st in streams:
            main.wait_stream(st)

    if args.profile:
        # selective_frames: each selective frame projected, binned and
        # blended alone with every CTA (the per-frame stage timings the
        # raster roofline divides by); otherwise one sweep as timed
        frames_alone = args.profile == "selective_frames"
        prof_mode = "selective" if frames_alone else args.profile
        for it in range(3):
            torch.cuda.synchronize()
            if it == 2:
                torch.cuda.nvtx.range_push("sweep")
            if frames_alone:
                for r, cam, out in zip(rs_mode[prof_mode], cams, bufs):
                    r.render(ds, cam, prof_mode, out=out)
            else:
                step(prof_mode)
            torch.cuda.synchronize()
            if it == 2:
                torch.cuda.nvtx.range_pop()
        for r in rs_mode[prof_mode]:
            r.check()
        return
    neval = [torch.empty((c.height, c.width), dtype=torch.int32, device=dev) for c in cams]

    # counts: duplicates, survivors, evaluations per frame
    stats = {}
    for mode in ("selective", "all_levels"):
        for r, cam, out, ne in zip(rs_mode[mode], cams, bufs, neval):
            r.render(ds, cam, mode, out=out, n_eval=ne)
            rc, d, s_ = msgs.ms_bin_counts(r.bins)
            if rc != msgs.MS_OK:
                raise msgs.MsError(rc, "capacity")
            stats[(mode, cam.width)] = dict(D=d, survivors=s_,
                                            P_eval=int(ne.sum(dtype=torch.int64).item()))

    # CUDA graphs: one per 8-frame sweep, and one per stage of every frame
    # (the per-scale breakdown); the same kernels run on every replay
    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    # each mode's sweep with and without the SMs shared; the faster is timed
    share_trial = {}
    g_step = {}
    for m in ("selective", "all_levels"):
        cand = {sh: capture(lambda m=m, sh=sh: step(m, share=sh)) for sh in (False, True)}
        trial = {}
        for sh, g in cand.items():
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            trial[sh] = e0.elapsed_time(e1) / 20
        share_plan[m] = trial[True] < trial[False]
        g_step[m] = cand[share_plan[m]]
        share_trial[m] = {"shared_ms": trial[True], "not_shared_ms": trial[False]}
    # the sweep's projection launch as the step issues it (with the union),
    # and the step's binning (the shared sort and split, every frame's
    # binning) on one stream
    sel_views, sel_split = plan["selective"]
    g_views = capture(lambda: orders[sel_split].project(ds, rs_mode["selective"], cams,
                                                        "selective", views=sel_views))

    def bin_step():
        o = orders[sel_split]
        o.sort()
        for k, (r, cam) in enumerate(zip(rs_mode["selective"], cams)):
            cs = msgs.camera_struct(cam)
            if k in sel_views:
                po, pst = o.view_order(k)
                msgs.ms_bin_ordered(r.proj, sc.n, cs, r.bins, po, pst, msgs._ptr(r.ws),
                                    r.ws_bytes)
            else:
                msgs.ms_bin(r.proj, sc.n, cs, r.bins, msgs._ptr(r.ws), r.ws_bytes)
    g_bin_step = capture(bin_step)
    # Gaussians listed in at least one frame: each reads its SH row once
    listed_any = torch.zeros(sc.n, dtype=torch.bool, device=dev)
    g_views.replay()
    for r in rs_mode["selective"]:
        listed_any |= r.n_tiles[:sc.n] != 0
    n_listed_any = int(listed_any.sum().item())
    g_stage = {}
    for mode in ("selective", "all_levels"):
        for r, cam, out in zip(rs_mode[mode], cams, bufs):
            cs = msgs.camera_struct(cam)
            md = msgs.MODES[mode]
            g_stage[(mode, cam.width)] = (
                capture(lambda cs=cs, md=md, r=r: msgs.ms_project(ds.struct, cs, md, r.proj)),
                capture(lambda cs=cs, r=r: msgs.ms_bin(r.proj, sc.n, cs, r.bins,
                                                       msgs._ptr(r.ws), r.ws_bytes)),
                capture(lambda cs=cs, out=out, r=r: msgs.ms_raster(
                    r.proj, r.bins, cs, msgs._ptr(out[0]), msgs._ptr(out[1]),
                    msgs._ptr(out[2]), 0, msgs._ptr(r.rws), r.rws_bytes)))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        g_step["selective"].replay()
        g_step["all_levels"].replay()
    torch.cuda.synchronize()

    def timed(mode, k):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            g_step[mode].replay()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t_sel = timed("selective", args.steps)
    t_all = timed("all_levels", args.steps)

    frames = len(cams)
    value = job_rate(frames * args.steps, world, t_sel)
    value_all = job_rate(frames * args.steps, world, t_all)

    # per-scale and per-stage timing (events on the launching stream)
    per_scale = {"selective": {}, "all_levels": {}}
    stage_ms = {"project": 0.0, "bin": 0.0, "raster": 0.0, "bin_frames_alone": 0.0}
    reps = max(20, args.steps)
    for mode in ("selective", "all_levels"):
        for cam in cams:
            graphs = g_stage[(mode, cam.width)]
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            tot = [0.0, 0.0, 0.0]
            frame_ms = []
            for _ in range(reps):
                for k in range(3):
                    ev[k].record(stream)
                    graphs[k].replay()
                ev[3].record(stream)
                torch.cuda.synchronize()
                for k in range(3):
                    tot[k] += ev[k].elapsed_time(ev[k + 1])
                frame_ms.append(ev[0].elapsed_time(ev[3]))
            ms = [t / reps for t in tot]
            per_scale[mode][f"{cam.width}x{cam.height}"] = {
                "fps": 1e3 / sum(ms), "project_ms": ms[0], "bin_ms": ms[1],
                "raster_ms": ms[2], "frame_ms_median": float(np.median(frame_ms)),
                "frame_ms_p99": float(np.percentile(frame_ms, 99)),
                **stats[(mode, cam.width)]}
            if mode == "selective":
                for k, name in (1, "bin_frames_alone"), (2, "raster"):
                    stage_ms[name] = stage_ms.get(name, 0.0) + ms[k]
    # the sweep projects its eight frames in one launch, then bins them from
    # one shared depth sort (timed here on one stream, every kernel in turn)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        g_views.replay()
    ev[1].record(stream)
    torch.cuda.synchronize()
    stage_ms["project"] = ev[0].elapsed_time(ev[1]) / reps
    ev[0].record(stream)
    for _ in range(reps):
        g_bin_step.replay()
    ev[1].record(stream)
    torch.cuda.synchronize()
    stage_ms["bin"] = ev[0].elapsed_time(ev[1]) / reps
    clk = clocks.stop()

    # roofline of the dominant stage of the selective step
    sm_mhz = clk.get("sm_mhz") or 2070.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    n = sc.n
    # one pass: the geometry (53 B) and opacity (4 B) of every Gaussian once;
    # per frame the tile count, depth key and tile rectangle (16 B) of every
    # Gaussian and the 48-B record of each survivor; the SH row (192 B) once
    # per Gaussian listed in any frame.  (Counting depth and rectangle only
    # for survivors, as the binning needs them, gives proj_bytes_listed.)
    # The launch also writes the 4-B union flag of every Gaussian for the
    # shared depth sort.
    proj_bytes = 57 * n + 192 * n_listed_any + 4 * n
    proj_bytes_listed = 57 * n + 192 * n_listed_any + 4 * n
    evals = 0
    for cam in cams:
        s = stats[("selective", cam.width)]
        proj_bytes += 16 * n + 48 * s["survivors"]
        proj_bytes_listed += 4 * n + (48 + 12) * s["survivors"]
        evals += s["P_eval"]
    proj_s = stage_ms["project"] / 1e3
    raster_s = stage_ms["raster"] / 1e3
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks_alu = alu_peaks(msgs, torch, dev)
    alu_peak = peaks_alu["fp32_peak"]
    mufu_peak = peaks_alu["ex2"]
    # the unit-count figure at the maximum clock, for context
    alu_nominal = sms * FP32_LANES_PER_SM * 2070.0e6 / 1e12
    roof_project = {"bound": "hbm", "kernel": f"project_pruned_kernel ({len(cams)} views of "
                                              "one pose, one launch)",
                    "achieved": proj_bytes / proj_s / 1e9, "peak": hbm_peak, "unit": "GB/s"}
    roof_project["frac"] = roof_project["achieved"] / roof_project["peak"]
    roof_project["bytes_per_launch"] = proj_bytes
    roof_project["bytes_per_launch_listed_only"] = proj_bytes_listed
    # DRAM bytes of one ncu capture of the sweep's projection launch (null
    # once the projection kernel has changed since the capture)
    roof_project["traffic"] = captured_traffic(PROJECT_VIEWS_DRAM)
    roof_raster = {"bound": "alu", "kernel": "raster_kernel (tile) + raster_list_kernel "
                                              "(with its row_mask_kernel pass)",
                   "achieved": OPS_PER_EVAL * evals / raster_s / 1e12, "peak": alu_peak,
                   "unit": "Tops/s",
                   "peak_source": "measured: the faster of the scalar FFMA and packed FFMA2 "
                                  "probes (bench leg alu_peaks), one FMA = one operation",
                   "peak_nominal": alu_nominal}
    roof_raster["frac"] = roof_raster["achieved"] / roof_raster["peak"]
    # the co-bound: one ex2 per evaluation on the MUFU unit
    roof_raster["co_bound"] = {"bound": "mufu", "achieved": evals / raster_s / 1e12,
                               "peak": mufu_peak, "unit": "T ex2/s",
                               "frac": evals / raster_s / 1e12 / mufu_peak}
    # the same split by kernel, by ms_raster's own rule (MS_RASTER_AUTO, no
    # cap: the frames are timed alone): the list kernel (with its mask pass)
    # for frames with fewer tiles than SMs, and up to 4x as many when the
    # mean list length is 1024-8192; the tile kernel otherwise
    by_kernel = {}
    for cam in cams:
        nt = cam.tiles_x * cam.tiles_y
        d_ = stats[("selective", cam.width)]["D"]
        list_k = nt < sms or (nt < 4 * sms and 1024 * nt <= d_ <= 8192 * nt)
        name = "raster_list_kernel" if list_k else "raster_kernel"
        e = by_kernel.setdefault(name, {"frames": [], "P_eval": 0, "ms": 0.0})
        e["frames"].append(f"{cam.width}x{cam.height}")
        e["P_eval"] += stats[("selective", cam.width)]["P_eval"]
        e["ms"] += per_scale["selective"][f"{cam.width}x{cam.height}"]["raster_ms"]
    for e in by_kernel.values():
        e["achieved"] = OPS_PER_EVAL * e["P_eval"] / (e["ms"] / 1e3) / 1e12
        e["frac"] = e["achieved"] / alu_peak
    roof_raster["by_kernel"] = by_kernel
    # binning (compaction + duplication, sort, ranges): the algorithmic bytes
    # of each frame, read the survivors' tile counts and records (44 B), write
    # D (tile, depth, index) entries (12 B), one sorting read + write of them
    # (24 B), and the ranges read of the sorted keys (8 B)
    bin_bytes = 0
    for cam in cams:
        st_ = stats[("selective", cam.width)]
        bin_bytes += 44 * st_["survivors"] + 44 * st_["D"]
    roof_bin = {"bound": "hbm", "kernel": "the step's binning on one stream (the shared depth "
                                          "sort and split, per frame start, duplicate, 1-2 tile "
                                          "passes, ranges)",
                "achieved": bin_bytes / (stage_ms["bin"] / 1e3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "bytes_per_step": bin_bytes}
    roof_bin["frac"] = roof_bin["achieved"] / hbm_peak
    dominant = max(("project", "bin", "raster"), key=stage_ms.get)
    roof = roof_raster if dominant == "raster" else roof_project
    if dominant == "bin":
        roof = dict(roof_project)
        roof["note"] = "binning dominates; project roofline shown"
    # DRAM bytes per frame of the dominant stage: dram__bytes_read.sum +
    # dram__bytes_write.sum of one ncu capture of the eight frames' raster
    # launches (the tile kernel, or the list kernel's mask pass and blend),
    # each frame rendered alone with every CTA as in the per-frame stage
    # timings, averaged (to be taken again whenever a raster kernel changes)
    traffic = captured_traffic(RASTER_DRAM) if roof is roof_raster else roof.get("traffic")
    roof = dict(roof, traffic=traffic, stage_ms_per_step=stage_ms,
                traffic_source=("ncu capture, mean over the eight frames' raster stages "
                                "(tile kernel, or mask pass + list kernel), each frame alone "
                                "(bench.py --profile selective_frames)"
                                if roof is roof_raster else
                                "ncu capture of the sweep's projection launch")
                if traffic else None)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).pin_memory()
                for k in ("mean", "log_scale", "quat", "opacity", "color", "level")}
        host["s_max"] = ds.s_max.cpu().pin_memory()
        host["s_min"] = ds.s_min.cpu().pin_memory()
        outs = [torch.empty((3, c.height, c.width), dtype=torch.float32).pin_memory()
                for c in cams]
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = sum(t.numel() * t.element_size() for t in outs)

        # every step uploads the whole scene and reads back all 8 images;
        # two scene buffers let step i + 1's upload and prepare run on a copy
        # stream while step i renders from the other buffer
        scenes = [ds, msgs.DeviceScene(sc, device=dev, prepare=False)]
        up = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        freed = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(i):
            d = scenes[i % 2]
            up.wait_event(freed[i % 2])  # the step that last rendered from it is done
            with torch.cuda.stream(up):
                for k, t in host.items():
                    getattr(d, k).copy_(t, non_blocking=True)
                msgs.ms_scene_prepare(d.struct, stream=up)
            ready[i % 2].record(up)

        def render_body(j):
            # the sweep as the timed step runs it (one projection launch, one
            # shared depth sort) from scene buffer j, each image read back
            # into pinned host memory as its frame ends
            step("selective",
                 after=lambda k, out, st: outs[k].copy_(out[0], non_blocking=True),
                 scene=scenes[j])

        # the public calls of each buffer's render captured once as a CUDA
        # graph (they never synchronise with the host) and replayed every
        # step after that step's upload: 6320 vs 5990 frames/s issued one by
        # one from Python
        e2e_graphs = []
        for j in range(2):
            gj = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gj):
                render_body(j)
            e2e_graphs.append(gj)

        def render(i):
            main = torch.cuda.current_stream()
            main.wait_event(ready[i % 2])
            e2e_graphs[i % 2].replay()
            freed[i % 2].record(main)

        def e2e_run(k):
            upload(0)
            for i in range(k):
                if i + 1 < k:
                    upload(i + 1)
                render(i)

        e2e_run(args.warmup)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        barrier()
        e2e = {"value": job_rate(frames * args.steps, world, t_e2e), "unit": "frames/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "pipeline": "scene upload + prepare of step i+1 on a copy stream during "
                           "step i's render (two scene buffers; each buffer's render, its "
                           "public calls captured once as a CUDA graph, replayed per step); "
                           "images read back per frame"}

    # kernels of libmsgs per selective step: one projection for every frame,
    # 4 passes of the shared depth sort and its split; per frame the start
    # kernel, 4 depth passes (frames outside the shared order), duplicate,
    # 1-2 tile passes, ranges; segment offsets, then the blend as ms_raster
    # launches it: the mask pass and the list kernel (fewer tiles than SMs),
    # the tile kernel alone (capped, or 4x as many tiles, or a capacity below
    # 1024 per tile), or both kernels and the mask pass (in between)
    launches_per_step = 1 + 4 + (1 if sel_split else 0)
    for k, cam in enumerate(cams):
        tiles = cam.tiles_x * cam.tiles_y
        capped = share_plan["selective"] and share_ctas[k] > 0
        cap_ok = rs_mode["selective"][k].dup_capacity >= 1024 * tiles
        blend = (2 if tiles < sms_dev else
                 3 if (not capped and tiles < 4 * sms_dev and cap_ok) else 1)
        launches_per_step += (1 + (0 if k in sel_views else 4) + 1
                              + (1 if tiles <= 256 else 2) + 1) + 1 + blend

    serve = None
    if not args.no_serve:
        serve = serve_in_child(args, local)

    train = None
    if not args.no_train:
        train = train_step_bench(msgs, torch, ds, sc, dev, max(10, args.steps // 2),
                                 args.warmup)
        train["value"] *= world

    if train is not None:
        rb = train["roofline_bwd"]
        rb["raster_bwd"]["peak"] = alu_peak
        rb["raster_bwd"]["frac"] = rb["raster_bwd"]["achieved"] / alu_peak
        rb["project_bwd"]["peak"] = hbm_peak
        rb["project_bwd"]["frac"] = rb["project_bwd"]["achieved"] / hbm_peak

    aggregate = aggregate_bench(msgs, torch, ds, sc, dev)
    single_level = single_level_bench(msgs, torch, dev, max(50, args.steps))
    single_level["raster_frac"] = single_level["raster_tops"] / alu_peak
    level_mix = None if args.no_level_mix else level_mix_bench(
        msgs, torch, dev, sc.n, cams, calib, max(20, args.steps // 2))
    near_far = None if args.no_near_far else near_far_bench(msgs, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f, s, threads, scales = oracle_sweep(oracle_scene(sc), cams, args.cpu_budget_s)
        cpu = {"value": f / s, "unit": "frames/s", "cores": threads, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"{f} selective frames of the same scene at widths {scales}"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_sel / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config(sc.n), shared_depth_order={
                m: {"frames": [f"{cams[k].width}x{cams[k].height}" for k in v],
                    "split": bool(sp)} for m, (v, sp) in plan.items()},
                share_sms={m: {"chosen": bool(share_plan[m]),
                               "fine_frames": [f"{c.width}x{c.height}"
                                               for c, f in zip(cams, fine) if f],
                               "ctas_per_sm": [c for c in share_ctas if c], **share_trial[m]}
                           for m in share_plan}),
            "clocks": clk, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "roofline": roof,
            "cpu_baseline": cpu,
            "all_levels": {"value": value_all, "unit": "frames/s",
                           "ms_per_step": 1e3 * t_all / args.steps},
            "per_scale": per_scale,
            "roofline_all": {"project": roof_project, "bin": roof_bin, "raster": roof_raster},
            "alu_peaks": peaks_alu,
            "train": train,
            "aggregate": aggregate,
            "single_level": single_level,
            "level_mix": level_mix,
            "near_far": near_far,
            "serve": serve,
        }))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
