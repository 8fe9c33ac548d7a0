"""One training step of the method over a batch of views, eager or as a
captured CUDA graph.

A step renders every view of the batch in one pass (view gate, projection,
sorts, compositing), takes the loss of Eq. 4 (L1 + lambda D-SSIM, batch mean)
plus the scale regulariser of Eq. 5, runs the adjoint into compact gradient
rows and applies one Adam step to every Gaussian.  Nothing in the step reads
a value back to the host, so the whole step can be captured once and replayed:
the cameras come from the workspace's device table (set_views uploads them
before a replay) and the Adam step number from its device counter.
"""
from __future__ import annotations

import torch

from . import binding as B


class TrainStep:
    """Static buffers and the call sequence of one step.

    g: the Gaussians (updated in place by each step); cams: the views of a
    batch (all of one width and height); targets: (V, 3, H, W) float32 CUDA
    tensor of the views' ground-truth images; lr: the five learning rates
    (mean, log-scale, quaternion, opacity, SH)."""

    def __init__(self, g: B.GaussianTensors, cams, targets: torch.Tensor, params: B.RenderParams, lr,
                 lam: float = 0.2, beta: float = 10.0, ws: B.Workspace | None = None, cull=None,
                 capacity: dict | None = None, betas=(0.9, 0.999), eps: float = 1e-15, lazy: bool = False):
        V, C, H, W = targets.shape
        assert C == 3 and len(cams) == V and all(c.width == W and c.height == H for c in cams)
        self.g, self.params, self.lr, self.lam, self.beta = g, params, list(lr), lam, beta
        self.betas, self.eps = betas, eps
        self.V, self.H, self.W = V, H, W
        if ws is None:
            cap = capacity or {}
            tiles = V * B.tiles_of(cams[0], params.tile_w, params.tile_h)
            ws = B.Workspace(max_gaussians=g.n, max_records=cap.get("max_records", g.n * V),
                             max_instances=cap.get("max_instances", 64 * g.n * V), max_tiles=tiles,
                             max_pixels=V * H * W, max_cameras=V)
        self.ws = ws
        self.cull = cull
        self.m, self.v = g.zeros_like(), g.zeros_like()
        self.target = torch.empty_like(targets)
        self.rgb = torch.empty(V * 3 * H * W, device=targets.device)
        self.dL = torch.empty_like(self.rgb)
        self.loss = torch.zeros(1, device=targets.device)
        self.reg = torch.zeros(1, device=targets.device)
        self.graph = None
        self.lazy = lazy
        if lazy:
            # deferred zero-gradient steps: exact, but only Gaussians in use are touched
            self.last = torch.zeros(g.n, dtype=torch.int32, device=targets.device)
            self.drift = torch.zeros(2, g.n, device=targets.device)
            self.ws.adam_lazy_enable(self.m, self.v, self.last, self.drift, betas[0], betas[1], eps)
        self.set_views(cams, targets)

    def set_views(self, cams, targets: torch.Tensor | None = None):
        """Uploads the views of the next step (same width and height as at
        construction) and copies their targets into the static buffer."""
        assert len(cams) == self.V and all(c.width == self.W and c.height == self.H for c in cams)
        self.ws.upload_cameras(cams, self.params)
        if targets is not None:
            self.target.copy_(targets, non_blocking=True)

    def _body(self, step: int):
        ws = self.ws
        ws.preprocess_uploaded(self.g, self.params, self.cull)
        ws.bin_sort()
        ws.render_fwd(self.rgb)
        ws.photometric_loss(self.rgb.view(self.V, 3, self.H, self.W), self.target, self.lam, self.loss, self.dL)
        ws.render_bwd_compact(self.g, self.dL, scale_reg_beta=self.beta, scale_reg_value=self.reg)
        ws.adam_step_compact(self.g, self.m, self.v, self.lr, step, beta1=self.betas[0], beta2=self.betas[1],
                             eps=self.eps)

    def flush(self):
        """Brings every Gaussian up to the current step (deferred steps only)."""
        if self.lazy:
            self.ws.adam_flush(self.g)

    def run(self, step: int = 0):
        """One eager step; step >= 1 sets the step number, 0 continues the
        device counter."""
        self._body(step)

    def capture(self) -> torch.cuda.CUDAGraph:
        """Captures one step (continuing the device step counter) as a CUDA graph."""
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self._body(0)
        self.graph = graph
        return graph

    def replay(self):
        assert self.graph is not None, "capture() first"
        self.graph.replay()
