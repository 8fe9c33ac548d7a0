"""Drivers of the batched workloads beside the single-view training step:

* a multi-view training loop (several equal-size views per step, the whole
  step captured once as a CUDA graph), against the same steps run eagerly and
  against the plain per-view path (one view at a time, dense gradients
  accumulated, then a dense Adam step);
* one batched render of many cameras of mixed resolution, its tile shape and
  sort chunk chosen by the autotuner;
* the serving loop under Poisson arrivals.

Each returns a dict of measured figures; bench.py prints them.  Scenes and
cameras come from synth (seeded, city-shaped)."""
from __future__ import annotations

import statistics

import numpy as np
import torch

from . import binding as B
from . import synth
from .autotune import Autotuner, max_tiles
from .serve import Server, poisson_requests
from .train import TrainStep

LOD = dict(lod_d0=1600.0, lod_Lmax=5)
LRS = [1.6e-4 * 100.0, 5e-3, 1e-3, 5e-2, 2.5e-3]


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _capacity_probe(gt, cams, params):
    """Records and instances a batch needs, from one preprocess + bin_sort."""
    n = gt.n
    probe = B.Workspace(max_gaussians=n, max_records=min(n * len(cams), 1 << 27),
                        max_instances=(1 << 30) - 1, max_tiles=max_tiles(cams),
                        max_pixels=sum(c.width * c.height for c in cams), max_cameras=len(cams), forward_only=True)
    probe.preprocess(gt, cams, params)
    probe.bin_sort()
    c = probe.counts()  # *_needed hold the full counts even past the probe's capacity
    probe.close()
    if c["records_needed"] > (1 << 27):
        raise RuntimeError("batch needs more than 2^27 records")
    return c


# ---- multi-view training loop -------------------------------------------------------

def view_pool(n_views: int, seed: int, width: int, height: int):
    cams = []
    for k in range(n_views):
        cams.append(synth.aerial_camera(seed * 1000 + k, width=width, height=height))
    return cams


def train_batch_workload(n: int = 20_000_000, views: int = 8, width: int = 1600, height: int = 1200,
                         steps: int = 50, warmup: int = 3, pool: int = 64, per_view_steps: int = 5) -> dict:
    g = synth.city_scene(n, seed=3)
    target_scene = synth.perturbed_copy(g, seed=4)
    cams = view_pool(pool, 4, width, height)
    params = B.RenderParams(lod_enable=True, **LOD)
    gt_target = B.GaussianTensors.from_host(target_scene)
    # targets: the perturbed scene rendered through the same path
    cap = _capacity_probe(gt_target, cams[:views], params)
    rec = min(n * views, int(cap["records_needed"] * 1.5) + 8192)
    inst = min((1 << 30) - 1, int(cap["instances_needed"] * 1.5) + 65536)
    rws = B.Workspace(max_gaussians=n, max_records=rec, max_instances=inst,
                      max_tiles=views * B.tiles_of(cams[0]), max_pixels=views * width * height, max_cameras=views,
                      forward_only=True)
    targets = torch.empty(pool, 3, height, width, device="cuda")
    for k in range(0, pool, views):
        rws.preprocess(gt_target, cams[k:k + views], params)
        rws.bin_sort()
        rws.render_fwd(targets[k:k + views].view(-1))
    rws.sync_status()
    rws.close()
    del gt_target

    def batch(k):
        idx = [(k * views + j) % pool for j in range(views)]
        return [cams[i] for i in idx], targets[idx]

    capd = dict(max_records=rec, max_instances=inst)
    ga, gb = B.GaussianTensors.from_host(g), B.GaussianTensors.from_host(g)
    c0, t0 = batch(0)
    # Adam with deferred zero-gradient steps (exact): each timed region ends with the flush
    eager = TrainStep(ga, c0, t0, params, LRS, capacity=capd, lazy=True)
    graph = TrainStep(gb, c0, t0, params, LRS, capacity=capd, lazy=True)
    eager.run(step=1)
    graph.run(step=1)
    graph.capture()
    for k in range(1, 1 + warmup):
        cm, tg = batch(k)
        eager.set_views(cm, tg)
        eager.run()
        graph.set_views(cm, tg)
        graph.replay()
    torch.cuda.synchronize()
    # timed: the same steps, eager then replayed (uploads included in both)
    losses_e, losses_g = [], []
    e0, e1 = _events()
    e0.record()
    for k in range(1 + warmup, 1 + warmup + steps):
        cm, tg = batch(k)
        eager.set_views(cm, tg)
        eager.run()
        losses_e.append(eager.loss.clone())
    eager.flush()
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / steps
    g0, g1 = _events()
    torch.cuda.nvtx.range_push("timed_region")  # lets a profiler select the replayed steps
    g0.record()
    for k in range(1 + warmup, 1 + warmup + steps):
        cm, tg = batch(k)
        graph.set_views(cm, tg)
        graph.replay()
        losses_g.append(graph.loss.clone())
    graph.flush()
    g1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / steps
    eager.ws.sync_status()
    graph.ws.sync_status()
    le = torch.cat(losses_e).cpu().numpy()
    lg = torch.cat(losses_g).cpu().numpy()
    same_params = all(torch.equal(a, b) for a, b in zip(ga.params(), gb.params()))
    eager.ws.close()
    graph.ws.close()
    del eager, graph, ga, gb
    # batched against the plain per-view path, like for like
    lfl = _like_for_like(g, cams, targets, params, views, per_view_steps, capd)
    pix = views * width * height
    lfl.update({"batched_mpix_per_s": pix / lfl["batched_ms"] / 1e3,
                "per_view_mpix_per_s": pix / lfl["per_view_ms"] / 1e3,
                "speedup": lfl["per_view_ms"] / lfl["batched_ms"],
                "arithmetic": "dense gradients, dense Adam, no scale regulariser, eager, in both arms"})
    return {"n": n, "views": views, "width": width, "height": height, "steps": steps,
            "graph_ms": graph_ms, "eager_ms": eager_ms, "graph_mpix_per_s": pix / graph_ms / 1e3,
            "eager_mpix_per_s": pix / eager_ms / 1e3,
            "graph_step": "views cycling through a pool of 64, L1 + 0.2 D-SSIM, scale regulariser, Adam with "
                          "deferred zero-gradient steps (exact), flush inside the timed region",
            "graph_equals_eager": bool(np.array_equal(le, lg)) and same_params,
            "loss_first": float(le[0]), "loss_last": float(le[-1]),
            "like_for_like": lfl}


class _PerViewPath:
    """The plain per-view path: one view at a time (preprocess, sort, render,
    loss, dense backward accumulated over the views), then a dense Adam step.
    No scale regulariser: like the batched arm it is compared with."""

    def __init__(self, g, cams, targets, params, views, capd):
        n = g.n
        self.H, self.W = targets.shape[2], targets.shape[3]
        self.cams, self.targets, self.params, self.views = cams, targets, params, views
        self.ws = B.Workspace(max_gaussians=n, max_records=capd["max_records"], max_instances=capd["max_instances"],
                              max_tiles=B.tiles_of(cams[0]), max_pixels=self.W * self.H)
        self.rgb = torch.empty(3 * self.H * self.W, device="cuda")
        self.dL = torch.empty_like(self.rgb)
        self.l1 = torch.zeros(1, device="cuda")
        self.loss = torch.zeros(1, device="cuda")

    def step(self, gt, m, v, grads, idx, step_no):
        ws, H, W, views = self.ws, self.H, self.W, self.views
        self.loss.zero_()
        for j, i in enumerate(idx):
            ws.preprocess(gt, [self.cams[i]], self.params)
            ws.bin_sort()
            ws.render_fwd(self.rgb)
            ws.photometric_loss(self.rgb.view(1, 3, H, W), self.targets[i:i + 1], 0.2, self.l1, self.dL)
            self.dL.mul_(1.0 / views)  # the batch loss is the mean over its views
            self.loss.add_(self.l1, alpha=1.0 / views)
            ws.render_bwd(gt, self.dL, grads, accumulate=j > 0)
        B.adam_step([(p, gr, mm, vv, LRS[q], 0.9, 0.999, 1e-15) for q, (p, gr, mm, vv) in
                     enumerate(zip(gt.params(), grads.params(), m.params(), v.params()))], step=step_no)
        return self.loss


class _BatchedDense:
    """The batched step with the per-view path's arithmetic: one preprocess /
    bin_sort / render / loss / backward over all views of the step, dense
    gradients, a dense Adam step, no scale regulariser."""

    def __init__(self, g, cams, targets, params, views, capd):
        n = g.n
        self.H, self.W = targets.shape[2], targets.shape[3]
        self.cams, self.targets, self.params, self.views = cams, targets, params, views
        self.ws = B.Workspace(max_gaussians=n, max_records=capd["max_records"], max_instances=capd["max_instances"],
                              max_tiles=views * B.tiles_of(cams[0]), max_pixels=views * self.W * self.H,
                              max_cameras=views)
        self.rgb = torch.empty(views * 3 * self.H * self.W, device="cuda")
        self.dL = torch.empty_like(self.rgb)
        self.loss = torch.zeros(1, device="cuda")

    def step(self, gt, m, v, grads, idx, step_no):
        ws, H, W, V = self.ws, self.H, self.W, self.views
        ws.preprocess(gt, [self.cams[i] for i in idx], self.params)
        ws.bin_sort()
        ws.render_fwd(self.rgb)
        ws.photometric_loss(self.rgb.view(V, 3, H, W), self.targets[idx], 0.2, self.loss, self.dL)
        ws.render_bwd(gt, self.dL, grads, accumulate=False)
        B.adam_step([(p, gr, mm, vv, LRS[q], 0.9, 0.999, 1e-15) for q, (p, gr, mm, vv) in
                     enumerate(zip(gt.params(), grads.params(), m.params(), v.params()))], step=step_no)
        return self.loss


def _like_for_like(g, cams, targets, params, views, steps, capd):
    """Batched against per-view at the same accuracy: both arms run the same
    `steps` steps (views cycling through the pool) from the same start with
    the same arithmetic -- dense gradients, a dense Adam step, no scale
    regulariser -- so their losses must agree step by step.  Returns each
    arm's ms per step and the largest relative difference of their losses."""
    pool = targets.shape[0]
    out = {}
    losses = {}
    for name, cls in (("batched", _BatchedDense), ("per_view", _PerViewPath)):
        path = cls(g, cams, targets, params, views, capd)
        # warm-up on scratch state: every kernel of the path is loaded before timing
        scratch = B.GaussianTensors.from_host(g)
        path.step(scratch, scratch.zeros_like(), scratch.zeros_like(), scratch.zeros_like(), list(range(views)), 1)
        torch.cuda.synchronize()
        del scratch
        gt = B.GaussianTensors.from_host(g)
        m, v, grads = gt.zeros_like(), gt.zeros_like(), gt.zeros_like()
        ls = []
        e0, e1 = _events()
        e0.record()
        for k in range(steps):
            idx = [(k * views + j) % pool for j in range(views)]
            ls.append(path.step(gt, m, v, grads, idx, k + 1).clone())
        e1.record()
        torch.cuda.synchronize()
        path.ws.sync_status()
        path.ws.close()
        out[name + "_ms"] = e0.elapsed_time(e1) / steps
        losses[name] = torch.cat(ls).double().cpu().numpy()
        del gt, m, v, grads
    out["loss_rel_max"] = float(np.max(np.abs(losses["per_view"] - losses["batched"]) / np.abs(losses["batched"])))
    out["steps"] = steps
    return out


# ---- batched render of many cameras -------------------------------------------------

def batched_render_workload(n: int = 10_000_000, n_cams: int = 64, reps: int = 10, warmup: int = 2,
                            tune_cache: str | None = None) -> dict:
    g = synth.city_scene(n, seed=3)
    cams = synth.mixed_cameras(n_cams, seed=7)
    gt = B.GaussianTensors.from_host(g)
    params = B.RenderParams(lod_enable=True, **LOD)
    cap = _capacity_probe(gt, cams, params)
    rec = min(n * n_cams, int(cap["records_needed"] * 1.3) + 8192, (1 << 30) - 1)
    inst = min((1 << 30) - 1, int(cap["instances_needed"] * 1.3) + 65536)
    pix = sum(c.width * c.height for c in cams)
    ws = B.Workspace(max_gaussians=n, max_records=rec, max_instances=inst, max_tiles=max_tiles(cams),
                     max_pixels=pix, max_cameras=n_cams)
    choice = Autotuner(tune_cache).tune(ws, gt, cams, params, backward=False, reps=2)
    p = choice.apply(ws, params)
    rgb = torch.empty(3 * pix, device="cuda")
    for _ in range(warmup):
        ws.preprocess(gt, cams, p)
        ws.bin_sort()
        ws.render_fwd(rgb)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = _events()
        e0.record()
        ws.preprocess(gt, cams, p)
        ws.bin_sort()
        ws.render_fwd(rgb)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    counts = ws.counts()
    # every view of the batch equals its render alone (checked for a few views)
    same = True
    offs = np.cumsum([0] + [c.width * c.height for c in cams])
    solo = B.Workspace(max_gaussians=n, max_records=min(n, rec), max_instances=inst,
                       max_tiles=max_tiles(cams[:1] + [max(cams, key=lambda c: c.width * c.height)]),
                       max_pixels=max(c.width * c.height for c in cams), forward_only=True)
    solo.set_sort_chunk(choice.sort_chunk)
    for k in (0, n_cams // 2, n_cams - 1):
        one = torch.empty(3 * cams[k].width * cams[k].height, device="cuda")
        solo.preprocess(gt, [cams[k]], p)
        solo.bin_sort()
        solo.render_fwd(one)
        same &= bool(torch.equal(one, rgb[3 * offs[k]:3 * offs[k + 1]]))
    solo.close()
    ms = statistics.median(times)
    return {"n": n, "cameras": n_cams, "pixels": int(pix), "ms": ms, "mpix_per_s": pix / ms / 1e3,
            "mgaussian_views_per_s": n * n_cams / ms / 1e3, "records": counts["n_records"],
            "instances": counts["n_instances"], "tile": f"{choice.tile_w}x{choice.tile_h}",
            "sort_chunk": choice.sort_chunk, "tuning_ms": choice.trials, "views_equal_alone": same,
            "resolutions": sorted({f"{c.width}x{c.height}" for c in cams})}


# ---- serving -------------------------------------------------------------------------

SERVE_SIZES = ((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def serve_camera(rng):
    """A serving request's view: a random aerial pose at 720p, 1080p, 1440p or 4K."""
    w, h = SERVE_SIZES[rng.integers(len(SERVE_SIZES))]
    return synth.aerial_camera(int(rng.integers(1 << 30)), width=w, height=h)


def serve_run(gt, rate: float, duration: float, seed: int = 5, key_budget: float = 40e9, max_batch: int = 64,
              slots: int = 3, check_alone: bool = True) -> dict:
    """Poisson arrivals at `rate` for `duration` seconds against resident
    Gaussians gt, with `slots` batches in flight at most (1: one batch at a
    time, the control without overlap)."""
    params = B.RenderParams(lod_enable=True, **LOD)
    reqs = poisson_requests(rate, duration, serve_camera, seed=seed)
    server = Server(gt, params, key_budget_bytes=key_budget, max_batch=max_batch,
                    max_pixels=16 * 3840 * 2160, slots=slots)
    # warm-up on a few requests outside the timed run
    warm = poisson_requests(rate, 0.2, serve_camera, seed=seed + 1)
    server.run(warm, realtime=False)
    server.batches.clear()
    stats = server.run(reqs, realtime=True)
    server.close()
    stats.update({"rate": rate, "duration_s": duration, "key_budget_gb": key_budget / 1e9})
    if check_alone:
        # a request renders the same image in an overlapped mix of batches as alone
        mix = Server(gt, params, key_budget_bytes=8e9, max_batch=4, max_pixels=4 * 3840 * 2160, keep_images=True,
                     slots=3)
        few = [dataclasses_replace(r) for r in reqs[:12]]
        mstats = mix.run(few, realtime=False)
        mix.close()
        alone = Server(gt, params, key_budget_bytes=4e9, max_batch=1, max_pixels=3840 * 2160, keep_images=True,
                       slots=1)
        solo = [dataclasses_replace(r) for r in few[:4]]
        alone.run(solo, realtime=False)
        alone.close()
        stats["alone_equals_in_mix"] = all(torch.equal(a.image, b.image) for a, b in zip(few[:4], solo))
        stats["mix_max_in_flight"] = mstats["max_in_flight"]
    return stats


def serving_workload(n: int = 30_000_000, rate: float = 200.0, duration: float = 60.0, seed: int = 5,
                     key_budget: float = 40e9, max_batch: int = 64) -> dict:
    g = synth.city_scene(n, seed=3)
    gt = B.GaussianTensors.from_host(g)
    stats = serve_run(gt, rate, duration, seed, key_budget, max_batch, slots=3)
    # the control: one batch at a time
    off = serve_run(gt, rate, duration, seed, key_budget, max_batch, slots=1, check_alone=False)
    stats.update({"n": n, "overlap_off": {k: off[k] for k in ("p50_ms", "p99_ms", "mean_batch", "req_per_s",
                                                              "mean_in_flight")}})
    return stats


def dataclasses_replace(r):
    import dataclasses
    return dataclasses.replace(r, start=None, done=None, image=None, batch=-1)
