"""A serving loop for novel-view renders against resident Gaussians.

Requests (a camera each, any of several resolutions) arrive over time and wait
in a FIFO queue.  Whenever the GPU is free the loop admits the oldest waiting
requests into one batch -- as many as fit the batch limits and the memory
budget of their sort keys -- and renders the whole batch with one
preprocess / bin_sort / render_fwd sequence (one launch per stage for all
cameras of the batch, each at its own resolution).  A request's latency runs
from its arrival to the moment its image is complete on the device.

Admission: the key buffers of a batch take 24 bytes per (record, tile)
instance (tile key and record id, double-buffered, plus the sorted copy), and
a request's instance count is predicted from its pixel count with a running
estimate of instances per pixel, updated from every rendered batch.  A batch
whose real count overflows the workspace anyway is split in two and retried.
Rendering is deterministic and every view's tile lists keep the same order in
any batch, so a request's image does not depend on what it was batched with.
"""
from __future__ import annotations

import dataclasses
import statistics
import time

import numpy as np
import torch

from . import binding as B

KEY_BYTES_PER_INSTANCE = 24


@dataclasses.dataclass
class Request:
    rid: int
    cam: object
    arrival: float                 # seconds after the start of the run
    start: float | None = None     # when latency starts: the arrival, or 0 when all wait from the start
    done: float | None = None      # seconds after the start of the run
    batch: int = -1
    image: torch.Tensor | None = None

    @property
    def latency(self) -> float:
        return self.done - self.start


def poisson_requests(rate: float, duration: float, cameras, seed: int = 5):
    """Arrivals of a Poisson process of `rate` per second over `duration`
    seconds; request k renders cameras(rng) (a callable drawing one camera)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append(Request(len(out), cameras(rng), t))


class Server:
    def __init__(self, g: B.GaussianTensors, params: B.RenderParams, key_budget_bytes: float = 40e9,
                 max_batch: int = 64, max_pixels: int = 64 * 3840 * 2160, max_tiles: int | None = None,
                 max_records: int | None = None, inst_per_pixel: float = 8.0, keep_images: bool = False):
        self.g, self.params = g, params
        self.max_batch = min(max_batch, B.GS_MAX_CAMERAS)
        self.max_instances = int(min(key_budget_bytes // KEY_BYTES_PER_INSTANCE, (1 << 30) - 1))
        self.max_pixels = max_pixels
        tw, th = params.tile_w, params.tile_h
        self.max_tiles = max_tiles or (max_pixels // (tw * th) + self.max_batch * (3840 // tw + 2160 // th + 2))
        records = max_records or int(min(g.n * self.max_batch, key_budget_bytes // 200, (1 << 30) - 1))
        self.ws = B.Workspace(max_gaussians=g.n, max_records=records,
                              max_instances=self.max_instances, max_tiles=self.max_tiles, max_pixels=max_pixels,
                              max_cameras=self.max_batch, forward_only=True)
        self.rgb = torch.empty(3 * max_pixels, device="cuda")
        self.ipp = inst_per_pixel
        self.keep_images = keep_images
        self.batches = []
        self.overflows = 0

    def predicted_instances(self, cam) -> float:
        return self.ipp * cam.width * cam.height

    def admit(self, queue):
        """The longest prefix of the queue that fits one batch."""
        n, pix, tiles, inst = 0, 0, 0, 0.0
        tw, th = self.params.tile_w, self.params.tile_h
        for r in queue:
            p = r.cam.width * r.cam.height
            t = B.tiles_of(r.cam, tw, th)
            i = self.predicted_instances(r.cam)
            if n == self.max_batch or pix + p > self.max_pixels or tiles + t > self.max_tiles or \
                    (n > 0 and inst + i > self.max_instances):
                break
            n, pix, tiles, inst = n + 1, pix + p, tiles + t, inst + i
        return queue[:n]

    def render(self, reqs) -> bool:
        """Renders one batch; False if it overflowed the workspace."""
        cams = [r.cam for r in reqs]
        ws = self.ws
        ws.preprocess(self.g, cams, self.params)
        ws.bin_sort()
        ws.render_fwd(self.rgb)
        c = ws.counts()  # synchronises: the batch is complete
        if c["error"] == B.GS_ERR_CAPACITY:
            ws.clear_error()
            self.overflows += 1
            return False
        if c["error"] != 0:
            ws.sync_status()  # raises with the library's message
        pix = sum(cm.width * cm.height for cm in cams)
        self.ipp = 0.7 * self.ipp + 0.3 * c["n_instances"] / max(pix, 1) * 1.15  # running estimate, 15 % margin
        if self.keep_images:
            off = 0
            for r in reqs:
                n = r.cam.width * r.cam.height
                r.image = self.rgb[3 * off:3 * (off + n)].clone()
                off += n
        return True

    def run(self, requests, realtime: bool = True) -> dict:
        """Serves `requests` (sorted by arrival).  realtime: arrivals follow
        the wall clock and latency counts from arrival; otherwise every
        request is waiting at t = 0 and latency counts from there."""
        pending = list(requests)
        queue = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        k = 0
        while pending or queue:
            t = now()
            while pending and (not realtime or pending[0].arrival <= t):
                r = pending.pop(0)
                r.start = r.arrival if realtime else 0.0
                queue.append(r)
            if not queue:
                time.sleep(max(0.0, min(pending[0].arrival - t, 1e-3)))
                continue
            batch = self.admit(queue)
            while not self.render(batch):
                if len(batch) == 1:
                    raise RuntimeError("a single request exceeds the workspace")
                batch = batch[:len(batch) // 2]
            done = now()
            for r in batch:
                r.done, r.batch = done, k
            self.batches.append(len(batch))
            queue = queue[len(batch):]
            k += 1
        wall = now()
        lat = sorted(r.latency for r in requests)
        pix = sum(r.cam.width * r.cam.height for r in requests)
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
        return {"requests": len(requests), "batches": len(self.batches), "overflow_retries": self.overflows,
                "mean_batch": statistics.mean(self.batches) if self.batches else 0.0,
                "p50_ms": 1e3 * q(0.50), "p99_ms": 1e3 * q(0.99), "max_ms": 1e3 * lat[-1] if lat else 0.0,
                "wall_s": wall, "req_per_s": len(requests) / wall, "mpix_per_s": pix / wall / 1e6}
