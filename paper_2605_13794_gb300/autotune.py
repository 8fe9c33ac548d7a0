"""A small autotuner for the render path: it times every tile shape the
kernels support (16x16, 32x8, 8x32, 32x16, 16x8, 8x16) with the radix-sort chunkings
(1024, 2048 and 4096 keys per block) on the caller's own workload and keeps the
fastest, cached per workload class (Gaussian count and camera resolutions).

The sort chunk (1024, 2048 or 4096 keys per block) leaves every result
unchanged.  The tile shape decides which
Gaussians are listed for which pixels (through the 3-sigma tile rectangle), so
images from different shapes agree to rounding except where a fragment of
opacity above 0.35 falls just outside one shape's rectangle."""
from __future__ import annotations

import collections
import dataclasses
import json
import os
import statistics

import torch

from . import binding as B

TILE_SHAPES = ((16, 16), (32, 8), (8, 32), (32, 16), (16, 8), (8, 16))
SORT_CHUNKS = (1024, 2048, 4096)


def max_tiles(cams) -> int:
    """Tiles of the cameras under the tile shape that needs the most."""
    return max(sum(B.tiles_of(c, tw, th) for c in cams) for tw, th in TILE_SHAPES)


def workload_key(n: int, cams) -> str:
    res = sorted(collections.Counter((c.width, c.height) for c in cams).items())
    return f"n={float(f'{n:.2g}'):.0f};" + ",".join(f"{w}x{h}:{k}" for (w, h), k in res)


@dataclasses.dataclass
class Choice:
    tile_w: int
    tile_h: int
    sort_chunk: int
    ms: float
    trials: dict

    def apply(self, ws: B.Workspace, params: B.RenderParams) -> B.RenderParams:
        ws.set_sort_chunk(self.sort_chunk)
        return dataclasses.replace(params, tile_w=self.tile_w, tile_h=self.tile_h)


class Autotuner:
    def __init__(self, cache_path: str | None = None):
        self.path = cache_path
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def _save(self):
        if self.path:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            with open(self.path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)

    def tune(self, ws: B.Workspace, g: B.GaussianTensors, cams, params: B.RenderParams, cull=None,
             backward: bool = True, reps: int = 3) -> Choice:
        """The fastest (tile shape, sort chunk) for preprocess + bin_sort +
        render_fwd (+ the compact backward) of this workload; `ws` must hold
        max_tiles(cams) tiles.  A shape whose binning needs more records or
        instances than `ws` holds is skipped (its capacity error cleared), so
        the choice fits the workspace.  A cached choice is returned without
        timing."""
        key = workload_key(g.n, cams) + f";bwd={int(backward)}"
        if key in self.cache:
            c = self.cache[key]
            return Choice(c["tile_w"], c["tile_h"], c["sort_chunk"], c["ms"], c["trials"])
        npix = sum(c.width * c.height for c in cams)
        rgb = torch.empty(3 * npix, device="cuda")
        dL = torch.full_like(rgb, 1e-3)
        trials, skipped = {}, []
        for tw, th in TILE_SHAPES:
            p = dataclasses.replace(params, tile_w=tw, tile_h=th)
            # the binning of this shape must fit the workspace (the sort chunk changes no count)
            ws.preprocess(g, cams, p, cull)
            ws.bin_sort()
            try:
                ws.sync_status()
            except B.GSError as e:
                if e.code != B.GS_ERR_CAPACITY:
                    raise
                ws.clear_error()
                skipped.append(f"{tw}x{th}")
                continue
            for chunk in SORT_CHUNKS:
                ws.set_sort_chunk(chunk)
                times = []
                for r in range(reps + 1):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    ws.preprocess(g, cams, p, cull)
                    ws.bin_sort()
                    ws.render_fwd(rgb)
                    if backward:
                        ws.render_bwd_compact(g, dL)
                    e1.record()
                    e1.synchronize()
                    if r > 0:  # the first run warms caches and clocks
                        times.append(e0.elapsed_time(e1))
                ws.sync_status()
                trials[f"{tw}x{th}/{chunk}"] = statistics.median(times)
        if not trials:
            raise RuntimeError("autotune: no tile shape fits the workspace's capacity")
        best = min(trials, key=trials.get)
        shape, chunk = best.split("/")
        tw, th = (int(x) for x in shape.split("x"))
        choice = Choice(tw, th, int(chunk), trials[best], dict(trials, skipped=skipped) if skipped else trials)
        self.cache[key] = dataclasses.asdict(choice)
        self._save()
        ws.set_sort_chunk(choice.sort_chunk)
        return choice
