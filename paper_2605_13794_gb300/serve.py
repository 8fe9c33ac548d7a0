"""A serving loop for novel-view renders against resident Gaussians, with
continuous batching.

Requests (a camera each, any of several resolutions) arrive over time and wait
in a FIFO queue.  The server keeps up to `slots` batches in flight, each slot
with its own forward-only workspace, CUDA stream, output buffer and
completion event.  Whenever a slot is free the loop admits the oldest waiting
requests into one batch -- as many as fit the batch limits and the key-buffer
memory of that slot -- and launches the whole batch with one preprocess /
bin_sort / render_fwd sequence on the slot's stream (one launch per stage for
all cameras of the batch, each at its own resolution), without waiting for
it: the batches of different slots overlap on the device.  The loop polls the
slots' completion events; a finished slot's requests are marked done and the
slot takes the next batch.  A request's latency runs from its arrival to the
moment the loop sees its batch complete on the device.

Admission: the key buffers of a batch take 24 bytes per (record, tile)
instance (tile key and record id, double-buffered, plus the sorted copy); the
key budget is split evenly over the slots.  A request's instance count is
predicted from its pixel count with a running estimate of instances per
pixel, updated from every completed batch.  A batch whose real count
overflows its slot's workspace anyway is put back at the head of the queue
and admitted again with a larger estimate (so in smaller batches).  Rendering
is deterministic and every view's tile lists keep the same order in any
batch, so a request's image does not depend on what it was batched or
overlapped with.
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


class _Slot:
    """One batch in flight: its workspace, stream, output and completion event."""

    def __init__(self, g, max_records, max_instances, max_tiles, max_pixels, max_cameras):
        self.ws = B.Workspace(max_gaussians=g.n, max_records=max_records, max_instances=max_instances,
                              max_tiles=max_tiles, max_pixels=max_pixels, max_cameras=max_cameras, forward_only=True)
        self.stream = torch.cuda.Stream()
        self.rgb = torch.empty(3 * max_pixels, device="cuda")
        self.done = torch.cuda.Event()
        self.batch = None      # requests in flight
        self.index = -1        # batch number


class Server:
    def __init__(self, g: B.GaussianTensors, params: B.RenderParams, key_budget_bytes: float = 40e9,
                 max_batch: int = 64, max_pixels: int = 64 * 3840 * 2160, max_tiles: int | None = None,
                 max_records: int | None = None, inst_per_pixel: float = 8.0, keep_images: bool = False,
                 slots: int = 3):
        self.g, self.params = g, params
        self.max_batch = min(max_batch, B.GS_MAX_CAMERAS)
        self.n_slots = max(1, int(slots))
        per_slot = key_budget_bytes / self.n_slots
        self.max_instances = int(min(per_slot // KEY_BYTES_PER_INSTANCE, (1 << 30) - 1))
        self.max_pixels = max_pixels
        tw, th = params.tile_w, params.tile_h
        self.max_tiles = max_tiles or (max_pixels // (tw * th) + self.max_batch * (3840 // tw + 2160 // th + 2))
        records = max_records or int(min(g.n * self.max_batch, per_slot // 200, (1 << 30) - 1))
        self.slots = [_Slot(g, records, self.max_instances, self.max_tiles, max_pixels, self.max_batch)
                      for _ in range(self.n_slots)]
        self.ipp = inst_per_pixel
        self.keep_images = keep_images
        self.batches = []
        self.overflows = 0

    def predicted_instances(self, cam) -> float:
        return self.ipp * cam.width * cam.height

    def admit(self, queue):
        """The longest prefix of the queue that fits one slot."""
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

    def launch(self, slot: _Slot, reqs, index: int):
        """Enqueues one batch on the slot's stream; returns at once."""
        cams = [r.cam for r in reqs]
        ws, st = slot.ws, slot.stream
        ws.preprocess(self.g, cams, self.params, stream=st)
        ws.bin_sort(stream=st)
        ws.render_fwd(slot.rgb, stream=st)
        slot.done.record(st)
        slot.batch, slot.index = list(reqs), index

    def finish(self, slot: _Slot) -> bool:
        """Collects a completed slot; False if its batch overflowed the workspace."""
        ws, st = slot.ws, slot.stream
        c = ws.counts(stream=st)  # the stream's work is complete: no wait
        reqs, slot.batch = slot.batch, None
        if c["error"] == B.GS_ERR_CAPACITY:
            ws.clear_error(stream=st)
            self.overflows += 1
            if len(reqs) == 1:
                raise RuntimeError("a single request exceeds the workspace")
            # admitted again with a larger estimate, so in a smaller batch
            pix = sum(r.cam.width * r.cam.height for r in reqs)
            self.ipp = max(2.0 * self.ipp, 1.15 * c["instances_needed"] / max(pix, 1))
            return False
        if c["error"] != 0:
            ws.sync_status(stream=st)  # raises with the library's message
        pix = sum(r.cam.width * r.cam.height for r in reqs)
        self.ipp = 0.7 * self.ipp + 0.3 * c["n_instances"] / max(pix, 1) * 1.15  # running estimate, 15 % margin
        if self.keep_images:
            # copied on the slot's stream, so the slot's next batch writes its buffer after the copy
            with torch.cuda.stream(st):
                off = 0
                for r in reqs:
                    n = r.cam.width * r.cam.height
                    r.image = slot.rgb[3 * off:3 * (off + n)].clone()
                    off += n
            torch.cuda.current_stream().wait_stream(st)
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
        busy_time = [0.0] * (self.n_slots + 1)  # seconds spent with j batches in flight
        t_last, in_flight, max_in_flight = 0.0, 0, 0
        while pending or queue or in_flight:
            t = now()
            busy_time[in_flight] += t - t_last
            t_last = t
            progressed = False
            while pending and (not realtime or pending[0].arrival <= t):
                r = pending.pop(0)
                r.start = r.arrival if realtime else 0.0
                queue.append(r)
                progressed = True
            # completed slots
            for slot in self.slots:
                if slot.batch is not None and slot.done.query():
                    done = now()
                    reqs, index = slot.batch, slot.index
                    in_flight -= 1
                    progressed = True
                    if self.finish(slot):
                        for r in reqs:
                            r.done, r.batch = done, index
                        self.batches.append(len(reqs))
                    else:
                        queue = reqs + queue
            # free slots take the next batches
            for slot in self.slots:
                if slot.batch is None and queue:
                    batch = self.admit(queue)
                    queue = queue[len(batch):]
                    self.launch(slot, batch, k)
                    k += 1
                    in_flight += 1
                    progressed = True
            max_in_flight = max(max_in_flight, in_flight)
            if not progressed:
                if in_flight == 0 and pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now(), 1e-3)))
                else:
                    time.sleep(20e-6)
        wall = now()
        busy_time[in_flight] += wall - t_last
        lat = sorted(r.latency for r in requests)
        pix = sum(r.cam.width * r.cam.height for r in requests)
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
        tot = max(sum(busy_time), 1e-12)
        busy = sum(busy_time[1:])
        return {"requests": len(requests), "batches": len(self.batches), "overflow_retries": self.overflows,
                "mean_batch": statistics.mean(self.batches) if self.batches else 0.0,
                "p50_ms": 1e3 * q(0.50), "p99_ms": 1e3 * q(0.99), "max_ms": 1e3 * lat[-1] if lat else 0.0,
                "wall_s": wall, "req_per_s": len(requests) / wall, "mpix_per_s": pix / wall / 1e6,
                "slots": self.n_slots, "max_in_flight": max_in_flight,
                # time-averaged batches in flight while any is, and the share of that time with two or more
                "mean_in_flight": sum(j * busy_time[j] for j in range(len(busy_time))) / max(busy, 1e-12),
                "overlap_frac": sum(busy_time[2:]) / max(busy, 1e-12), "busy_frac": busy / tot}

    def close(self):
        for s in self.slots:
            s.ws.close()
