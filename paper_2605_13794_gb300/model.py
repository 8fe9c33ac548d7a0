"""Model-level passes of the method on the device (Sec. 3.2, Sec. 3.3):

* importance_sweep: the instrumented sweep over all training views, up to
  GS_MAX_CAMERAS views per launch sequence, accumulating s, c^rad, c^vis and
  writing the bit-packed N x V Cull matrix (row v = Cull column of view v);
* simplify: Pass 1 (importance-weighted sampling without replacement of a
  fixed fraction) or Pass 2 (the 99 %-mass cut of s), then an
  order-preserving compaction of parameters, Adam moments and LOD labels;
* densify: clone / split with the phi_i reweighting and LOD inheritance.

Random numbers (the exponential clocks of Pass 1, the split offsets) are drawn
here with a seeded torch generator and passed to the kernels."""
from __future__ import annotations

import torch

from . import binding as B


def importance_sweep(ws: B.Workspace, g: B.GaussianTensors, cams, params: B.RenderParams, chunk: int | None = None):
    """One scoring pass over `cams` (never applying a Cull column).  Returns
    dict(s, crad, cvis, cull): s float32 [n], crad / cvis int32 [n] (views
    with a record / in the view's top-vis_mass of w), cull int32
    [len(cams)][ceil(n/32)] (bit set = Cull)."""
    n, V = g.n, len(cams)
    chunk = chunk or ws.cap.max_cameras
    words = (n + 31) // 32
    out = dict(s=torch.zeros(n, device="cuda"), crad=torch.zeros(n, dtype=torch.int32, device="cuda"),
               cvis=torch.zeros(n, dtype=torch.int32, device="cuda"),
               cull=torch.zeros(V, words, dtype=torch.int32, device="cuda"))
    for c0 in range(0, V, chunk):
        part = cams[c0:c0 + chunk]
        ws.preprocess(g, part, params)
        ws.bin_sort()
        ws.importance(s_accum=out["s"], crad=out["crad"], cvis=out["cvis"], cull_out=out["cull"][c0:c0 + len(part)])
    return out


def _bits(n):
    return torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")


def compact(ws: B.Workspace, model: B.ModelTensors, keep_bits) -> B.ModelTensors:
    """The rows of `model` whose keep bit is set, in order, as a new model."""
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    dst = B.ModelTensors.empty(model.n, with_moments=model.m is not None)
    ws.compact(model, keep_bits, dst, n_out)
    ws.sync_status()
    return dst.head(int(n_out.item()))


def simplify(ws: B.Workspace, model: B.ModelTensors, s, pass_no: int, keep_fraction: float = 0.7,
             mass: float = 0.99, seed: int = 0) -> B.ModelTensors:
    """Pass 1 (stochastic, keeps keep_fraction of the Gaussians) or Pass 2
    (deterministic, keeps the 99 %-mass prefix of s)."""
    keep = _bits(model.n)
    if pass_no == 1:
        gen = torch.Generator(device="cuda").manual_seed(seed)
        expo = torch.empty(model.n, device="cuda").exponential_(1.0, generator=gen)
        ws.prune_sample(s, expo, int(round(keep_fraction * model.n)), keep)
    else:
        ws.prune_mass(s, keep, mass)
    return compact(ws, model, keep)


def densify(ws: B.Workspace, model: B.ModelTensors, absgrad, denom, cvis, crad, seed: int = 0,
            **params) -> B.ModelTensors:
    """One density-control step; params: grad_threshold, dense_scale,
    min_opacity, split_shrink, eps, n_levels (see gs_densify)."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    noise = torch.randn(model.n, 2, 3, device="cuda", generator=gen)
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    dst = B.ModelTensors.empty(2 * model.n, with_moments=model.m is not None)
    ws.densify(model, absgrad, denom, cvis, crad, noise, dst, n_out, **params)
    ws.sync_status()
    return dst.head(int(n_out.item()))
