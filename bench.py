#!/usr/bin/env python3
"""Throughput of one 3DGS training step on the city-scale single-view workload.

Workload (the paper's aerial datasets are replaced by a synthetic city): 5M
Gaussians over 2 km x 2 km (ground plane + 200 buildings), degree-3 SH, one
1920x1080 aerial camera at 45 degree pitch, LOD gate (d0 = 1600 m, Lmax = 5)
and the importance cull column enabled.  One step runs every stage of the hot
path through the C ABI on resident device data:

  preprocess (gate + projection + SH; Gaussians culled in the view are kept
  and marked) -> bin_sort -> one walk of the tile lists that composites the
  image (marked records composite nowhere) and the importance sweep's raster
  (every record, as without the Cull column) -> L1 + 0.2 D-SSIM loss against
  a target -> render backward (+ scale regulariser) into compact per-Gaussian
  gradient rows -> Adam over all 59 parameters of all Gaussians
  (zero-gradient steps deferred and replayed exactly); beside them, on a
  second stream forked after the walk, the importance sweep's selection (w,
  a, s, c^rad, c^vis and the next Cull column); the step ends when both
  streams have.  (--overlap picks other arrangements: the whole sweep on the
  second stream after bin_sort, or all on one stream.)

The timed steps are replays of one CUDA graph of the whole step (captured
after eager warm-up steps; cameras from the workspace's device table, the Adam
step number from its device counter), followed by the flush of the deferred
Adam steps.

value = rendered pixels per second of whole steps (Mpix/s); the line also
carries Mgaussian/s.  All inputs (1.2 GB of parameters, Adam state, the
workspace) exceed the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsblitz|reference]

With N > 1 (under torchrun) every rank renders its own replica on its own GPU
(weak scaling, no data-path collective); value is the sum over ranks.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s and Mgaussian/s at 5M Gaussians 1080p; render p50/p99 ms"
WORKLOAD = "city-5M-1080p-single-view-train-step"
N_GAUSS = 5_000_000
W_IMG, H_IMG = 1920, 1080
SCENE_SEED, CAM_SEED, TARGET_SEED = 3, 4, 5
LOD = dict(lod_d0=1600.0, lod_Lmax=5)
LAMBDA, BETA = 0.2, 10.0
# learning rates of standard 3DGS training (position lr scaled for a city extent)
LRS = dict(mean=1.6e-4 * 100.0, log_scale=5e-3, quat=1e-3, opacity_logit=5e-2, sh=2.5e-3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gsblitz", choices=["gsblitz", "reference"])
    ap.add_argument("--n", type=int, default=N_GAUSS, help="Gaussians (default: the 5M workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving run of the default line")
    ap.add_argument("--no-train8", action="store_true",
                    help="skip the multi-view training figures (8 views of 1600x1200, 20M Gaussians) of the default line")
    ap.add_argument("--workload", default="city5M", choices=["city5M", "train8-city20M", "batch64-city10M",
                                                              "serve-city30M"],
                    help="city5M: the single-view training step (the default line); the others run the "
                         "multi-view graph-captured training loop, the 64-camera mixed-resolution batched "
                         "render and the serving loop")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file for batch64-city10M")
    ap.add_argument("--tile", default="16x16", choices=["16x16", "32x8", "8x32", "32x16", "16x8", "8x16"],
                    help="render tile shape of the city5M step")
    ap.add_argument("--dense-adam", action="store_true",
                    help="update every Gaussian every step instead of deferring zero-gradient steps (same results)")
    ap.add_argument("--overlap", default="fused", choices=["fwd", "step", "late", "fused", "off"],
                    help="city5M: the importance sweep on a second stream beside the forward and loss (fwd), "
                         "beside the whole training pass (step), its raster fused into the forward's walk and "
                         "its selection on a second stream (fused), or on the one stream (off)")
    return ap.parse_args()


# ---- clocks ---------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons at 50 ms.  Only
    samples whose timestamps fall inside the marked load windows count."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        self.path = None
        self.windows = []

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # the timed region starts only once sampling runs
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def mark(self, t0: float, t1: float):
        self.windows.append((t0, t1))

    @staticmethod
    def _epoch(stamp: str):
        try:
            base, _, frac = stamp.strip().partition(".")
            return time.mktime(time.strptime(base, "%Y/%m/%d %H:%M:%S")) + (float("0." + frac) if frac else 0.0)
        except ValueError:
            return None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        rows = [r for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        inside = [r for r in rows if (t := self._epoch(r[0])) is not None and
                  any(a - 0.05 <= t <= b + 0.05 for a, b in self.windows)]
        use = inside if inside else rows
        sm = [float(r[1]) for r in use]
        mx = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm), "in_timed_window": bool(inside)}


# ---- workload ---------------------------------------------------------------------

def make_host_inputs(n):
    from paper_2605_13794_gb300 import synth
    g = synth.city_scene(n, seed=SCENE_SEED)
    cam = synth.aerial_camera(seed=CAM_SEED, width=W_IMG, height=H_IMG)
    target = synth.noise_target(W_IMG, H_IMG, seed=TARGET_SEED)
    return g, cam, target


class Step:
    """Device state and the sequence of C-ABI calls of one training step."""

    def __init__(self, g, cam, target, tile=(16, 16), lazy=True, overlap="fwd"):
        import torch
        from paper_2605_13794_gb300 import binding as B
        self.B, self.torch = B, torch
        self.cam = cam
        self.n = g.n
        self.gt = B.GaussianTensors.from_host(g)
        for t in self.gt.params():
            t.requires_grad_(False)
        self.m = self.gt.zeros_like()
        self.v = self.gt.zeros_like()
        self.target = torch.from_numpy(target).cuda().unsqueeze(0).contiguous()
        self.P = cam.width * cam.height
        self.rgb = torch.empty(3 * self.P, device="cuda")
        self.T = torch.empty(self.P, device="cuda")
        self.dL = torch.empty(3 * self.P, device="cuda")
        self.loss = torch.zeros(1, device="cuda")
        self.reg = torch.zeros(1, device="cuda")
        words = (self.n + 31) // 32
        self.cull = torch.zeros(words, device="cuda", dtype=torch.int32)
        self.s = torch.zeros(self.n, device="cuda")
        self.crad = torch.zeros(self.n, device="cuda", dtype=torch.int32)
        self.cvis = torch.zeros(self.n, device="cuda", dtype=torch.int32)
        tw, th = tile
        # one binning per step: culled Gaussians stay in the lists, marked, so the training render
        # skips them and the importance sweep of the same view scores them
        self.params_train = B.RenderParams(lod_enable=True, cull_enable=B.GS_CULL_MARK, tile_w=tw, tile_h=th,
                                           **LOD)
        # the scoring sweep after density control (the paper's T2 pass) renders with the LOD gate
        # engaged and never applies the Cull mask it recomputes
        self.params_imp = B.RenderParams(lod_enable=True, cull_enable=False, tile_w=tw, tile_h=th, **LOD)
        self.graph = None
        # the captured step runs the importance sweep on a second stream, forked after the
        # binning: "fwd" joins it before the adjoint, "step" at the end of the step, "off"
        # keeps the single stream (the sweep shares no scratch with the training pass)
        self.overlap = overlap
        # both streams at the same priority: a higher one for the training pass was
        # measured slower (the sweep's raster then runs into the adjoint)
        self.cap_stream = torch.cuda.Stream()
        self.side = torch.cuda.Stream() if overlap != "off" else None
        # capacities from a dry run of the importance configuration (no Cull column)
        tiles = B.tiles_of(cam, tw, th)
        probe = B.Workspace(max_gaussians=self.n, max_records=self.n, max_instances=min((1 << 30) - 1, 32 * self.n),
                            max_tiles=tiles, max_pixels=self.P)
        probe.preprocess(self.gt, [cam], self.params_imp)
        probe.bin_sort()
        c = probe.counts()
        probe.close()
        del probe
        # headroom for the training itself: the Gaussians' footprints drift over the steps
        # (measured against the noise target: 1.25x the initial instances after ~210 steps,
        # 1.66x after ~420)
        self.inst_cap = min((1 << 30) - 1, int(c["instances_needed"] * 2.5) + 4096)
        self.rec_cap = min(self.n, int(c["records_needed"] * 1.5) + 4096)
        self.ws = B.Workspace(max_gaussians=self.n, max_records=self.rec_cap, max_instances=self.inst_cap,
                              max_tiles=tiles, max_pixels=self.P)
        # initial Cull column from an importance sweep of this view
        self.ws.preprocess(self.gt, [cam], self.params_imp)
        self.ws.bin_sort()
        self.ws.importance(cull_out=self.cull)
        self.ws.sync_status()
        self.lr = [LRS[k] for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")]
        self.stage_names = ["preprocess", "bin_sort", "render_fwd", "loss", "render_bwd", "adam", "importance"]
        self.lazy = lazy
        if lazy:
            # Adam with deferred zero-gradient steps: bit-identical to dense Adam, touching only the
            # Gaussians in use; flush() brings every Gaussian to the current step
            self.last = torch.zeros(self.n, dtype=torch.int32, device="cuda")
            self.drift = torch.zeros(2, self.n, device="cuda")
            self.ws.adam_lazy_enable(self.m, self.v, self.last, self.drift, max_steps=1 << 16)

    def flush(self):
        if self.lazy:
            self.ws.adam_flush(self.gt)

    def run(self, ev=None):
        """One eager step; ev, if given, is a list of 8 CUDA events recorded between stages."""
        self._body(ev)

    def capture(self):
        """The step as a CUDA graph (cameras in the workspace's device table,
        the Adam step number from its device counter); returns the number of
        kernels of this library in it."""
        torch = self.torch
        self.ws.upload_cameras([self.cam], self.params_train)
        torch.cuda.synchronize()
        n0 = self.B.kernel_launches()
        self.graph = self.capture_with(self.target)
        torch.cuda.synchronize()
        return self.B.kernel_launches() - n0

    def capture_with(self, target):
        """A graph of the step whose loss reads the target image from `target`."""
        saved, self.target = self.target, target
        graph = self.B.Graph()
        try:
            with graph.capture(self.cap_stream):
                self._body(None, uploaded=True)
        finally:
            self.target = saved
        return graph

    def replay(self):
        self.graph.launch()

    def _importance(self, stream=None):
        # importance sweep of the view on the step's binning; its Cull column gates the next step
        self.ws.importance(s_accum=self.s, crad=self.crad, cvis=self.cvis, cull_out=self.cull, stream=stream)

    def _body(self, ev, uploaded=False):
        B, ws, torch = self.B, self.ws, self.torch
        rec = (lambda k: ev[k].record()) if ev is not None else (lambda k: None)
        # the eager diagnostic steps (stage events) keep one stream
        side = self.side if ev is None else None
        main = torch.cuda.current_stream()
        rec(0)
        if uploaded:
            ws.preprocess_uploaded(self.gt, self.params_train, self.cull)
        else:
            ws.preprocess(self.gt, [self.cam], self.params_train, self.cull)
        rec(1)
        ws.bin_sort()
        rec(2)
        if self.overlap == "fused":
            # one walk of the lists: the image and the importance raster; the
            # selection follows on the side stream
            ws.render_fwd_importance(self.rgb, self.T)
            if side is not None:
                side.wait_stream(main)
                self._importance(stream=side)
        else:
            if side is not None and self.overlap != "late":
                side.wait_stream(main)
                self._importance(stream=side)
            ws.render_fwd(self.rgb, self.T)
        rec(3)
        if side is not None and self.overlap == "late":
            side.wait_stream(main)
            self._importance(stream=side)
        ws.photometric_loss(self.rgb.view(1, 3, self.cam.height, self.cam.width), self.target, LAMBDA, self.loss,
                            self.dL)
        rec(4)
        if side is not None and self.overlap == "fwd":
            main.wait_stream(side)
        ws.render_bwd_compact(self.gt, self.dL, scale_reg_beta=BETA, scale_reg_value=self.reg)
        rec(5)
        # Adam on all Gaussians with the compact gradients (zero for Gaussians without a
        # record); step 0: one past the workspace's device step counter
        ws.adam_step_compact(self.gt, self.m, self.v, self.lr, 0)
        rec(6)
        if side is None:
            self._importance()
        elif self.overlap in ("step", "late", "fused"):
            main.wait_stream(side)
        rec(7)


# ---- roofline bookkeeping --------------------------------------------------------


# Algorithmic FP32 operations of the compositing adjoint (App. A's compositing,
# differentiated), counted per (pixel, list entry) pair of the reverse walk (an
# FMA is two, a special-function op one).  Every pair re-evaluates the entry's
# exponent, alpha and the skip test; a pair that composites adds the adjoint.
BWD_FLOP_EVAL = 13
BWD_FLOP_COMPOSITE = 59
# Algorithmic FP32 operations of the forward compositing and of the colourless
# importance walk per (pixel, entry) pair: the same 13 to evaluate the entry's
# alpha, then per composited pair the forward's T (1 - alpha), alpha T, three
# colour FMAs and the T update (11), the importance walk's T (1 - alpha),
# alpha T, the w and a sums and the T update (8).
FWD_FLOP_COMPOSITE = 11
IMP_FLOP_COMPOSITE = 8
# Algorithmic DRAM bytes of the adjoint: per list entry its sorted index, the
# staged record (3 x 16 B), the record's slot offset and rectangle and its
# 9-float slot written back; per pixel dL/dC, T_final and n_contrib.
BWD_BYTES_ENTRY = 4 + 48 + 4 + 8 + 36
BWD_BYTES_PIXEL = 12 + 4 + 4


def alu_roofline(kernel, flops, sfu_ops, kernel_ms, alu, peaks, sm_mhz):
    """FP32 roofline of one compositing kernel: achieved FLOP/s against the
    measured FP32 FMA peak of this GPU (gs_alu_peaks), with the
    special-function fraction beside it."""
    sec = kernel_ms * 1e-3
    achieved = flops / sec / 1e12
    peak = max(alu["fp32_fma_flops"], alu["fp32x2_fma_flops"]) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "measured on this GPU (gs_alu_peaks: FP32 FMA chains on all %d SMs, best of scalar "
                           "and FP32x2)" % alu["sms"],
            "algorithmic_flops_per_launch": flops, "kernel_ms": kernel_ms,
            "sfu_frac": sfu_ops / sec / alu["ex2_per_s"], "sm_mhz_median": sm_mhz}


def bwd_roofline(fragments, composited, instances, pixels, kernel_ms, sm_mhz, peaks, alu):
    """Roofline of the compositing adjoint: achieved FP32 rate against the
    measured FP32 FMA peak, with the special-function and DRAM fractions
    beside it."""
    flops = BWD_FLOP_EVAL * fragments + BWD_FLOP_COMPOSITE * composited
    sfu_ops = fragments + composited        # ex2 per pair, reciprocal per composited pair
    r = alu_roofline("render_bwd_kernel", flops, sfu_ops, kernel_ms, alu, peaks, sm_mhz)
    sec = kernel_ms * 1e-3
    nbytes = BWD_BYTES_ENTRY * instances + BWD_BYTES_PIXEL * pixels
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    r.update({"fragments_per_launch": fragments, "composited_per_launch": composited,
              "hbm": {"algorithmic_bytes_per_launch": nbytes, "achieved_gbs": nbytes / sec / 1e9, "peak": hbm,
                      "frac": nbytes / sec / 1e9 / hbm,
                      "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}})
    return r


# Algorithmic bytes of the memory-bound kernels of the step (each read or
# written once; the units are the view's counts):
#   view gate: per Gaussian its mean 12 B, level 1 B and mean drift 4 B; per
#     candidate its log-scales 12 B and their drift 4 B read, its id 4 B and
#     camera mask 8 B written
#   binning, count pass: per record 18 B (tile count, rectangle, camera read,
#     first instance written), per instance 4 B (its tile's count)
#   binning, ranges, scatter and per-tile sort: per tile 20 B (count read,
#     range and cursor written), per record 18 B (read again), per instance
#     28 B (cursor, depth key read; key and record written; both read and the
#     record written by the per-tile sort)
#   slot reduction: per instance 36 B (its slot); per record 16 B of indices
#     and 36 B of summed gradient written
#   projection adjoint: per visible Gaussian 44 B of shape and opacity and
#     192 B of SH read and its 236 B gradient row written; per record 64 B
#     (ids, record, gradient)
#   SSIM statistics / gradient: per pixel and channel 20 B (image and target
#     read, three coefficient maps written) / 24 B (maps, image and target
#     read, the gradient written)
#   deferred Adam's step: per visible Gaussian 59 parameters x 24 B (p, m, v
#     read and written) and its 236 B gradient row
HBM_KERNELS = {
    "gate_count_kernel": ("GS_KT_GATE", lambda c: 17 * c["n"] + 28 * c["n_candidates"]),
    "bin_count": ("GS_KT_BIN_COUNT", lambda c: 18 * c["n_records"] + 4 * c["n_instances"]),
    "bin_sort": ("GS_KT_BIN_SORT", lambda c: 20 * c["tiles"] + 18 * c["n_records"] + 28 * c["n_instances"]),
    "reduce_slots_kernel": ("GS_KT_REDUCE_SLOTS", lambda c: 36 * c["n_instances"] + 52 * c["n_records"]),
    "preprocess_bwd_kernel": ("GS_KT_PREPROCESS_BWD", lambda c: 472 * c["n_visible"] + 64 * c["n_records"]),
    "ssim_fwd_kernel": ("GS_KT_SSIM_FWD", lambda c: 20 * 3 * c["pixels"]),
    "ssim_bwd_kernel": ("GS_KT_SSIM_BWD", lambda c: 24 * 3 * c["pixels"]),
    "lazy_list_vec_kernel (gradient step)": ("GS_KT_ADAM_GRAD", lambda c: (59 * 24 + 236) * c["n_visible"]),
}


def hbm_rooflines(kernel_ms, c, peaks):
    """Each memory-bound kernel's algorithmic bytes over its mean launch time,
    against the measured copy bandwidth."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    for name, (_, nbytes) in HBM_KERNELS.items():
        ms = kernel_ms.get(name)
        if not ms:
            continue
        b = nbytes(c)
        gbs = b / (ms * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "kernel_ms": round(ms, 4), "algorithmic_bytes_per_launch": int(b),
                     "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "traffic": None}
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def traffic_from_profile(profile, kernel_file):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if the
    summary was taken on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", profile)
    src = os.path.join(ROOT, "paper_2605_13794_gb300", "csrc", kernel_file)
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in text.splitlines() if l.startswith(("source_sha:", "dram_bytes_per_launch:")))
    if vals.get("source_sha", "").strip() != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


# ---- latency ------------------------------------------------------------------------

LATENCY_VIEWS = 40


def render_latency(step, g, B, torch):
    """Forward-only render of single 1920x1080 views of the resident scene
    (preprocess with the LOD gate, bin_sort, render_fwd), LATENCY_VIEWS random
    aerial poses one after another: per view the device time between events
    around the three calls, and the host time from the first call to the
    image being complete."""
    from paper_2605_13794_gb300 import synth
    cams = [synth.aerial_camera(seed=1000 + k, width=W_IMG, height=H_IMG) for k in range(LATENCY_VIEWS)]
    params = B.RenderParams(lod_enable=True, **LOD)
    ws = B.Workspace(max_gaussians=step.n, max_records=min(step.n, 1 << 21), max_instances=1 << 25,
                     max_tiles=B.tiles_of(cams[0]), max_pixels=W_IMG * H_IMG, forward_only=True)
    rgb = torch.empty(3 * W_IMG * H_IMG, device="cuda")
    dev, host = [], []
    for k in range(-3, LATENCY_VIEWS):  # three warm-up views
        cam = cams[k % LATENCY_VIEWS]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        e0.record()
        ws.preprocess(step.gt, [cam], params)
        ws.bin_sort()
        ws.render_fwd(rgb)
        e1.record()
        e1.synchronize()
        h1 = time.perf_counter()
        if k >= 0:
            dev.append(e0.elapsed_time(e1))
            host.append((h1 - h0) * 1e3)
    ws.sync_status()
    ws.close()
    q = lambda a, f: float(np.quantile(np.asarray(a), f))
    return {"views": LATENCY_VIEWS, "resolution": f"{W_IMG}x{H_IMG}", "gaussians": step.n,
            "p50_ms": q(dev, 0.5), "p99_ms": q(dev, 0.99), "host_p50_ms": q(host, 0.5), "host_p99_ms": q(host, 0.99),
            "what": "forward-only render of one view: preprocess (LOD gate) + bin_sort + render_fwd"}


SERVE_RATE, SERVE_SECONDS = 200.0, 3.0


def serving_short(step, torch):
    """A short run of the serving loop (continuous batching, three batches in
    flight at most) against the resident scene: Poisson arrivals at
    SERVE_RATE per second for SERVE_SECONDS, resolutions 720p-4K."""
    from paper_2605_13794_gb300 import workloads as WL
    r = WL.serve_run(step.gt, SERVE_RATE, SERVE_SECONDS, seed=5, key_budget=12e9, slots=3, check_alone=False)
    keep = ("requests", "p50_ms", "p99_ms", "max_ms", "req_per_s", "mpix_per_s", "mean_batch", "mean_in_flight",
            "overlap_frac", "max_in_flight", "slots", "rate", "duration_s")
    out = {k: r[k] for k in keep}
    out["what"] = (f"serving loop against the {step.n // 1_000_000}M-Gaussian scene: Poisson {SERVE_RATE:.0f} req/s "
                   f"for {SERVE_SECONDS:.0f} s, 720p-4K, latency from arrival to the image complete on the device")
    return out


TRAIN8_STEPS, TRAIN8_LFL_STEPS = 10, 3


def train8_figures(torch):
    """The realistic training step: 8 views of 1600x1200 per step cycling
    through a pool of 64 aerial views of a 20M-Gaussian city, the whole step a
    CUDA graph (Adam with deferred zero-gradient steps, scale regulariser),
    and the batched step against the plain per-view path with the same
    arithmetic (dense gradients, dense Adam, no regulariser) and their losses."""
    from paper_2605_13794_gb300 import workloads as WL
    r = WL.train_batch_workload(steps=TRAIN8_STEPS, warmup=2, per_view_steps=TRAIN8_LFL_STEPS)
    keep = ("n", "views", "width", "height", "steps", "graph_ms", "graph_mpix_per_s", "eager_ms", "eager_mpix_per_s",
            "graph_equals_eager", "graph_step", "loss_first", "loss_last", "like_for_like")
    return {k: r[k] for k in keep}


# ---- CPU oracle on a bounded sample ------------------------------------------------

class OracleSample:
    """The FP64 oracle timed on a bounded sample of one step, each part scaled
    by the units it covers: per-Gaussian work (projection with and without the
    gate, Adam) on a random Gaussian sample; per-pixel work (binning,
    compositing, loss, backward, importance) on a centred window rendered with
    every Gaussian that touches it, so the window keeps the scene's depth
    complexity.  The window's Gaussian set is found once, untimed."""

    def __init__(self, g, cam, target, window):
        import oracle as O
        from paper_2605_13794_gb300 import synth
        self.O, self.g, self.cam = O, g, cam
        ww, wh = window
        x0, y0 = (cam.width - ww) // 2, (cam.height - wh) // 2
        self.wcam = synth.Camera(R=cam.R, t=cam.t, fx=cam.fx, fy=cam.fy, cx=cam.cx - x0, cy=cam.cy - y0,
                                 width=ww, height=wh, campos=cam.campos)
        self.target = np.ascontiguousarray(target[:, y0:y0 + wh, x0:x0 + ww])
        self.Pt = O.Params(lod_enable=True, lod_d0=LOD["lod_d0"], lod_Lmax=LOD["lod_Lmax"])
        self.Pi = O.Params(lod_enable=True, lod_d0=LOD["lod_d0"], lod_Lmax=LOD["lod_Lmax"])
        pw = O.project(O.gaussians64(g), self.wcam, self.Pi)
        sel = np.nonzero(pw["status"] == O.ACTIVE)[0]
        self.gw = O.gaussians64(g.subset(sel if len(sel) else np.arange(1)))
        self.frac_pix = (ww * wh) / (cam.width * cam.height)

    def step(self, proj_sample, seed):
        O, g = self.O, self.g
        n = g.n
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(n, size=min(proj_sample, n), replace=False))
        g64s = O.gaussians64(g.subset(idx))
        t = {}
        t0 = time.perf_counter()
        O.project(g64s, self.cam, self.Pt)
        O.project(g64s, self.cam, self.Pi)
        t["projection"] = (time.perf_counter() - t0) * n / len(idx)
        t0 = time.perf_counter()
        fwd = O.forward_view(self.gw, self.wcam, self.Pt)
        _, dL = O.photometric_loss(fwd["image"][None], self.target[None], LAMBDA)
        O.backward_view(self.gw, fwd, self.wcam, self.Pt, dL[0])
        imp = O.forward_view(self.gw, self.wcam, self.Pi)
        O.visible_top_mass(imp["w"])
        t["per_pixel_stages"] = (time.perf_counter() - t0) / self.frac_pix
        k = min(proj_sample, n)
        p = rng.standard_normal(k)
        t0 = time.perf_counter()
        for _ in range(59):
            O.adam_step(p, p, p, np.abs(p), 1, 1e-3)
        t["adam"] = (time.perf_counter() - t0) * n / k
        return sum(t.values()), t


def cpu_baseline(g, cam, target):
    sample = OracleSample(g, cam, target, window=(240, 136))
    total, parts = sample.step(proj_sample=200_000, seed=0)
    P = cam.width * cam.height
    return {"value": P / total / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": ("FP64 C/numpy oracle, one thread: projection (gated and ungated) and Adam on a random "
                       "200k-Gaussian sample scaled by N; binning, compositing, L1+SSIM loss, backward and the "
                       "importance sweep on a centred 240x136 window with every Gaussian touching it, scaled by "
                       "the pixel ratio"),
            "seconds_per_step": total, "parts_s": {k: round(v, 3) for k, v in parts.items()}}


# The small scene (10k Gaussians in front of one 256x256 camera): the oracle's
# whole step in full, at one thread and on every host core.
SMALL_N, SMALL_W, SMALL_F = 10_000, 256, 300.0


def _small_inputs():
    from paper_2605_13794_gb300 import synth
    g = synth.plain_scene(SMALL_N, seed=1)
    cam = synth.plain_camera(SMALL_W, SMALL_W, SMALL_F)
    target = synth.noise_target(SMALL_W, SMALL_W, seed=2)
    return g, cam, target


def _small_step(inputs):
    """One full oracle step of the small scene: forward, loss, backward, the
    importance sweep and its visible set; returns its seconds."""
    import oracle as O
    g, cam, target = inputs
    P = O.Params()
    g64 = O.gaussians64(g)
    t0 = time.perf_counter()
    fwd = O.forward_view(g64, cam, P)
    _, dL = O.photometric_loss(fwd["image"][None], target[None], LAMBDA)
    O.backward_view(g64, fwd, cam, P, dL[0])
    imp = O.forward_view(g64, cam, P)
    O.visible_top_mass(imp["w"])
    return time.perf_counter() - t0


_small_barrier = None


def _small_init(barrier):
    global _small_barrier
    _small_barrier = barrier


def _small_worker(steps):
    """A spawned process: inputs built before the common start, then `steps`
    full steps; returns (start, end) wall times."""
    inputs = _small_inputs()
    _small_step(inputs)  # warm-up: the oracle library loaded and its pages touched
    _small_barrier.wait()
    t0 = time.time()
    for _ in range(steps):
        _small_step(inputs)
    return t0, time.time()


def cpu_small_scene(steps=3):
    """The oracle on the small scene at one thread (a full step, best of
    `steps`) and on all host cores (one spawned process per core, each running
    `steps` full steps at once; throughput over the wall time from the common
    start to the last finish)."""
    import multiprocessing as mp
    inputs = _small_inputs()
    _small_step(inputs)
    one = min(_small_step(inputs) for _ in range(steps))
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")  # never fork a process that has used the GPU
    barrier = ctx.Barrier(cores)
    with ctx.Pool(cores, initializer=_small_init, initargs=(barrier,)) as pool:
        spans = pool.map(_small_worker, [steps] * cores)
    wall = max(e for _, e in spans) - min(t for t, _ in spans)
    pix = SMALL_W * SMALL_W
    return {"workload": f"{SMALL_N // 1000}k Gaussians, {SMALL_W}x{SMALL_W}, full step (forward, L1 + D-SSIM, "
                        "backward, importance sweep and visible set)",
            "unit": "Mpix/s", "kind": "oracle",
            "one_thread": {"value": pix / one / 1e6, "seconds_per_step": one, "cores": 1},
            "all_cores": {"value": cores * steps * pix / wall / 1e6, "cores": cores,
                          "what": f"{cores} spawned processes, {steps} steps each, at once"}}


# ---- main -------------------------------------------------------------------------------

def dist_backend():
    """NCCL between GPUs; gloo where there is no GPU (the CPU tests of the
    multi-rank path)."""
    import torch
    return "nccl" if torch.cuda.is_available() else "gloo"


def dist_setup(args=None):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if dist_backend() == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def build_once(world, local):
    """Builds the library on local rank 0 only (the others wait), so that ranks
    of one node never compile into the same in-tree files at once."""
    if local == 0:
        __import__("__graft_entry__").build()
    barrier(world)
    if local != 0:
        __import__("__graft_entry__").build()  # up to date by now: checks only


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest of the ranks' x (each rank's time for the same K steps)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ms_max, world):
    """Whole-job throughput of weak-scaled replicas: every rank processes
    units_per_rank per step; the job's step time is the slowest rank's."""
    return world * units_per_rank / (ms_max * 1e-3)


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    g, cam, target = make_host_inputs(args.n)
    # the sample per step shrinks with the number of steps, so that the whole
    # run stays within a few minutes of host time
    nsteps = args.warmup + args.steps
    window, proj = ((120, 68), 50_000) if nsteps <= 12 else ((64, 36), 20_000)
    sample = OracleSample(g, cam, target, window=window)
    samples = []
    for k in range(nsteps):
        s, _ = sample.step(proj_sample=proj, seed=k)
        if k >= args.warmup:
            samples.append(s)
    sec = statistics.mean(samples)
    P = cam.width * cam.height
    value = P / sec / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": args.n, "width": W_IMG, "height": H_IMG, "lod": True,
                       "cull": True, "importance_pass": True,
                       "execution": "FP64 oracle on one host core, a bounded sample per step scaled to the view"},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step: {proj // 1000}k-Gaussian projection sample and a "
                                       f"{window[0]}x{window[1]} window, scaled"},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_workload(args, world, rank, local):
    """The batched workloads: one JSON line each (device-timed; clocks sampled
    over the whole run)."""
    import torch
    build_once(world, local)
    from paper_2605_13794_gb300 import workloads as WL
    torch.cuda.set_device(local)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    w0 = time.time()
    if args.workload == "train8-city20M":
        r = WL.train_batch_workload(steps=args.steps, warmup=args.warmup)
        line = {"metric": "multi-view training step Mpix/s (8 views 1600x1200, 20M city Gaussians, graph-captured)",
                "value": r["graph_mpix_per_s"], "unit": "Mpix/s", "higher_is_better": True,
                "ms_per_step": r["graph_ms"], "detail": r}
    elif args.workload == "batch64-city10M":
        r = WL.batched_render_workload(reps=args.steps, warmup=args.warmup, tune_cache=args.tune_cache)
        line = {"metric": "batched render Mpix/s (64 cameras of mixed resolution, 10M city Gaussians, one pass)",
                "value": r["mpix_per_s"], "unit": "Mpix/s", "higher_is_better": True, "ms_per_step": r["ms"],
                "detail": r}
    else:
        r = WL.serving_workload()
        line = {"metric": "serving p99 latency ms (Poisson 200 req/s, 60 s, 720p-4K, 30M resident Gaussians)",
                "value": r["p99_ms"], "unit": "ms", "higher_is_better": False, "detail": r}
    sampler.mark(w0, time.time())
    line.update({"workload": args.workload, "n_gpus": world, "dtype": "f32", "data": "synthetic",
                 "clocks": sampler.stop(), "gpu_launches": None})
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload != "city5M":
        run_workload(args, world, rank, local)
        return
    import torch
    build_once(world, local)
    from paper_2605_13794_gb300 import binding as B
    torch.cuda.set_device(local)
    g, cam, target = make_host_inputs(args.n)
    # measured FP32 FMA and special-function throughput of this GPU: the roofline peaks
    alu = B.alu_peaks()
    step = Step(g, cam, target, tile=tuple(int(x) for x in args.tile.split("x")), lazy=not args.dense_adam,
                overlap=args.overlap)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize()
    step.ws.sync_status()
    # per-launch device time of the compositing adjoint: the library brackets each
    # launch with events on its stream, as event nodes inside the captured step
    # (only this kernel: an event pair between two kernels costs their
    # programmatic-launch overlap)
    step.ws.kernel_timing(True, kernels=[B.GS_KT_RENDER_BWD])
    launches_per_step = step.capture()
    for _ in range(args.warmup):
        step.replay()
    torch.cuda.synchronize()
    step.ws.sync_status()

    # ---- device-timed region: K whole steps, inputs resident in HBM
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    launches0 = B.kernel_launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    torch.cuda.nvtx.range_push("timed_region")  # lets a profiler select the timed launches
    start.record(stream)
    for k in range(args.steps):
        step.replay()
    # the deferred Adam steps of every Gaussian not yet brought up to date, inside the timed region
    fl0, fl1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fl0.record(stream)
    step.flush()
    fl1.record(stream)
    end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    sampler.mark(w0, time.time())
    # graph replays launch the captured kernels without host calls
    launches = launches_per_step * args.steps + (B.kernel_launches() - launches0)
    barrier(world)
    step.ws.sync_status()
    # the captured event nodes hold the last timed replay's kernel durations
    kt = {"render_bwd_kernel": step.ws.kernel_time(B.GS_KT_RENDER_BWD)}
    step.ws.kernel_timing(False)
    kernel_ms = {name: max_over_ranks(t / max(n, 1), world) for name, (t, n) in kt.items()}
    ms = start.elapsed_time(end) / args.steps
    ms = max_over_ranks(ms, world)

    # ---- end to end through the public API with host buffers: every step's
    # target image comes from pinned host memory, and its loss and new Cull
    # column go back to pinned host memory.  The copies run on their own
    # streams through double-buffered device staging, overlapped with the
    # neighbouring steps; the timed region ends when the last read-back lands.
    K = args.steps
    tgt_host = torch.from_numpy(target).pin_memory()
    loss_host = torch.empty(K).pin_memory()
    cull_host = torch.empty((K, step.cull.numel()), dtype=torch.int32).pin_memory()
    h2d = tgt_host.numel() * 4
    d2h = 4 + step.cull.numel() * 4
    h2d_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
    stage_t = [torch.empty_like(step.target) for _ in range(2)]
    stage_o = [(torch.empty(1, device="cuda"), torch.empty_like(step.cull)) for _ in range(2)]
    t_ready, t_free = [torch.cuda.Event() for _ in range(2)], [torch.cuda.Event() for _ in range(2)]
    o_ready, o_free = [torch.cuda.Event() for _ in range(2)], [torch.cuda.Event() for _ in range(2)]
    # one graph of the step per staging buffer: each upload lands where its step reads it
    e2e_graphs = [step.capture_with(stage_t[b]) for b in range(2)]
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    h2d_stream.wait_event(e0)
    with torch.cuda.stream(h2d_stream):
        stage_t[0].copy_(tgt_host, non_blocking=True)
        t_ready[0].record(h2d_stream)
    for k in range(K):
        b, nb = k % 2, (k + 1) % 2
        if k + 1 < K:  # the next step's target, into the buffer the previous step read
            h2d_stream.wait_event(t_free[nb])
            with torch.cuda.stream(h2d_stream):
                stage_t[nb].copy_(tgt_host, non_blocking=True)
                t_ready[nb].record(h2d_stream)
        stream.wait_event(t_ready[b])
        e2e_graphs[b].launch(stream)
        t_free[b].record(stream)
        stream.wait_event(o_free[b])
        stage_o[b][0].copy_(step.loss)
        stage_o[b][1].copy_(step.cull)
        o_ready[b].record(stream)
        d2h_stream.wait_event(o_ready[b])
        with torch.cuda.stream(d2h_stream):
            loss_host[k:k + 1].copy_(stage_o[b][0], non_blocking=True)
            cull_host[k].copy_(stage_o[b][1], non_blocking=True)
            o_free[b].record(d2h_stream)
    step.flush()
    stream.wait_stream(d2h_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(w0, time.time())
    clocks = sampler.stop()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    assert bool(torch.isfinite(loss_host).all()), "non-finite loss read back"

    # stage breakdown (diagnostic, outside the timed regions): eager steps with
    # events between the stages
    diag = max(1, min(args.steps, 10))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(diag)]
    # and the per-launch device time of the forward and the importance raster in
    # these one-stream steps (event pairs around each launch)
    # (the breakdown runs the forward and the importance raster as separate
    # launches; with --overlap fused, a few more steps time the fused walk)
    timed = [("render_fwd_kernel", B.GS_KT_RENDER_FWD), ("importance_raster_kernel", B.GS_KT_IMPORTANCE)] + \
        [(name, getattr(B, kid)) for name, (kid, _) in HBM_KERNELS.items()] + [("project_kernel", B.GS_KT_PROJECT)]
    mode, step.overlap = step.overlap, "step"
    step.ws.kernel_timing(True, kernels=[kid for _, kid in timed])
    for k in range(diag):
        step.run(evs[k])
    torch.cuda.synchronize()
    for name, kid in timed:
        t, n_l = step.ws.kernel_time(kid)
        if n_l:
            kernel_ms[name] = max_over_ranks(t / n_l, world)
    step.ws.kernel_timing(False)
    step.overlap = mode
    if mode == "fused":
        step.ws.kernel_timing(True, kernels=[B.GS_KT_RENDER_FWD])
        for k in range(min(diag, 3)):
            step.run([torch.cuda.Event(enable_timing=True) for _ in range(8)])
        torch.cuda.synchronize()
        t, n_l = step.ws.kernel_time(B.GS_KT_RENDER_FWD)
        kernel_ms["render_fwd_importance_kernel"] = max_over_ranks(t / max(n_l, 1), world)
        step.ws.kernel_timing(False)
    stage_ms = {name: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(diag))
                for i, name in enumerate(step.stage_names)}
    stage_ms["adam_flush_per_step"] = fl0.elapsed_time(fl1) / args.steps

    P = cam.width * cam.height
    value = job_rate(P, ms, world) / 1e6
    # the render's forward and backward alone (gate and projection, sorts,
    # compositing, its adjoint and the projection adjoint), without the loss,
    # Adam and the importance sweep
    fb_ms = max_over_ranks(sum(stage_ms[k] for k in ("preprocess", "bin_sort", "render_fwd", "render_bwd")), world)
    fwd_bwd = {"ms": fb_ms, "mpix_per_s": job_rate(P, fb_ms, world) / 1e6,
               "mgaussian_per_s": job_rate(g.n, fb_ms, world) / 1e6,
               "stages": ["preprocess", "bin_sort", "render_fwd", "render_bwd"]}
    gauss = job_rate(g.n, ms, world) / 1e6
    peaks = measured_peaks()
    dom = max(stage_ms, key=stage_ms.get)
    # the counts of one more untimed forward and backward of this view
    step.ws.preprocess(step.gt, [cam], step.params_train, step.cull)
    step.ws.bin_sort()
    step.ws.render_fwd(step.rgb, step.T)
    step.ws.photometric_loss(step.rgb.view(1, 3, cam.height, cam.width), step.target, LAMBDA, step.loss, step.dL)
    step.ws.render_bwd_compact(step.gt, step.dL, scale_reg_beta=BETA, scale_reg_value=step.reg)
    counts = step.ws.counts()
    # the importance walk's composited pairs: the sum of its per-Gaussian a
    a_imp = torch.zeros(g.n, device="cuda", dtype=torch.int32)
    step.ws.importance(a=a_imp)
    imp_composited = int(a_imp.sum().item())
    # the dominant kernel of the step is the compositing adjoint: FP32-issue bound
    sm_mhz = clocks.get("sm_mhz")
    roof = bwd_roofline(counts["fragments"], counts["composited"], counts["n_instances"], P,
                        kernel_ms["render_bwd_kernel"], sm_mhz, peaks, alu)
    roof["traffic"] = traffic_from_profile("render_bwd_kernel_city5M_1080p.md", "render.cu")
    roof["dominant_stage"] = dom
    # the forward and the importance raster against the same peak; their pairs are
    # counted as the adjoint's (the entries up to each pixel's last composited one, a
    # lower bound of the pairs they evaluate)
    frag = counts["fragments"]
    roof_comp = {
        "render_fwd_kernel": alu_roofline("render_fwd_kernel",
                                          BWD_FLOP_EVAL * frag + FWD_FLOP_COMPOSITE * counts["composited"],
                                          frag, kernel_ms["render_fwd_kernel"], alu, peaks, sm_mhz),
        "importance_raster_kernel": alu_roofline("importance_raster_kernel",
                                                 BWD_FLOP_EVAL * frag + IMP_FLOP_COMPOSITE * imp_composited,
                                                 frag, kernel_ms["importance_raster_kernel"], alu, peaks, sm_mhz)}
    if "render_fwd_importance_kernel" in kernel_ms:
        # one walk: the pairs' alpha once, then the forward's and the importance's sums
        roof_comp["render_fwd_importance_kernel"] = alu_roofline(
            "render_fwd_importance_kernel",
            BWD_FLOP_EVAL * frag + FWD_FLOP_COMPOSITE * counts["composited"] + IMP_FLOP_COMPOSITE * imp_composited,
            frag, kernel_ms["render_fwd_importance_kernel"], alu, peaks, sm_mhz)
    roof_comp["importance_raster_kernel"]["composited_per_launch"] = imp_composited
    tw, th = (int(x) for x in args.tile.split("x"))
    tiles = ((cam.width + tw - 1) // tw) * ((cam.height + th - 1) // th)
    roof_hbm = hbm_rooflines(kernel_ms, dict(counts, n=g.n, pixels=P, tiles=tiles), peaks)
    latency = render_latency(step, g, B, torch)
    serving = serving_short(step, torch) if not args.no_serving else None
    train8 = train8_figures(torch) if not args.no_train8 else None
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": g.n, "width": W_IMG, "height": H_IMG, "tile": args.tile,
                       "lod": True, "cull": True, "importance_pass": True,
                       "optimizer": "adam (dense)" if args.dense_adam else "adam, zero-gradient steps deferred (exact)",
                       "l2": "inputs larger than L2 (no flush)", "execution": "CUDA graph of the whole step",
                       "importance_stream": {"fwd": "second stream beside forward and loss",
                                             "step": "second stream beside the training pass",
                                             "late": "second stream beside loss and adjoint",
                                             "fused": "raster in the forward's walk, selection on a second stream "
                                                      "beside the training pass",
                                             "off": "one stream"}[args.overlap],
                       "parallelism": f"replicas{world}"},
            "mgaussian_per_s": gauss,
            "fwd_bwd": fwd_bwd,
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "stage_ms_source": "eager steps with events between stages, outside the timed region",
            "counts": {k: counts[k] for k in ("n_records", "n_instances", "n_visible")},
            "kernel_ms": {k: round(v, 4) for k, v in kernel_ms.items()},
            "roofline": roof,
            "roofline_other": {**roof_comp, **roof_hbm},
            "alu_peaks": {k: (round(v / 1e12, 3) if k != "sms" else v) for k, v in alu.items()},
            "alu_peaks_unit": "TFLOP/s (FMA) and T results/s (ex2)",
            "render_latency": latency,
            "serving": serving,
            "train8": train8,
            "e2e": {"value": job_rate(P, e2e_ms, world) / 1e6, "unit": "Mpix/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, cam, target)
        line["cpu_small_scene"] = cpu_small_scene()
    if rank == 0:
        print(json.dumps(line), flush=True)
    # the graphs name the workspace's buffers and events: release them first
    for gr in e2e_graphs:
        gr.close()
    step.graph.close()
    step.graph = None
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
