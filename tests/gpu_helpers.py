"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and bring its outputs back in the oracle's layout."""
from __future__ import annotations

import numpy as np
import torch

from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth


def capacity_for(n, cams, records=None, instances=None, tile=(16, 16)):
    tiles = sum(B.tiles_of(c, *tile) for c in cams)
    pix = sum(c.width * c.height for c in cams)
    return dict(max_gaussians=max(n, 1), max_records=records or max(n * len(cams), 1),
                max_instances=instances or max(64 * n * len(cams), 1024), max_tiles=tiles, max_pixels=pix,
                max_cameras=len(cams))


def gpu_params(P, **over):
    """Binding params equal to oracle Params P."""
    d = dict(bg=tuple(P.bg), tile_w=P.tile_w, tile_h=P.tile_h, alpha_min=P.alpha_min, alpha_max=P.alpha_max, T_min=P.T_min, dilation=P.dilation,
             znear=P.znear, fov_clamp=P.fov_clamp, lod_enable=P.lod_enable, lod_d0=P.lod_d0, lod_f=P.lod_f,
             lod_Lmax=P.lod_Lmax, cull_enable=P.cull_enable, eps_score=P.eps_score, vis_mass=P.vis_mass)
    d.update(over)
    return B.RenderParams(**d)


class GpuRun:
    """One preprocess + bin_sort + render_fwd of a scene, with readbacks."""

    def __init__(self, g: synth.GaussianSet, cams, P, cull=None, ws=None, cap=None):
        self.cams = cams
        self.tile = (P.tile_w, P.tile_h)
        self.gt = B.GaussianTensors.from_host(g)
        self.ws = ws or B.Workspace(**(cap or capacity_for(g.n, cams, tile=self.tile)))
        self.cull = None if cull is None else torch.from_numpy(np.ascontiguousarray(cull, np.uint32).view(np.int32)).cuda()
        self.ws.preprocess(self.gt, cams, gpu_params(P), self.cull)
        c = self.ws.counts()
        self.n_records = c["n_records"]
        self.depth_bits = self.ws.read_buffer(B.GS_BUF_REC_DEPTH, np.uint32, self.n_records)
        self.ws.bin_sort()
        self.P = sum(cm.width * cm.height for cm in cams)
        self.rgb = torch.empty(3 * self.P, device="cuda")
        self.T = torch.empty(self.P, device="cuda")
        self.ws.render_fwd(self.rgb, self.T)
        self.ws.sync_status()
        self.counts = self.ws.counts()
        n = self.n_records
        self.rec_g = self.ws.read_buffer(B.GS_BUF_REC_GAUSSIAN, np.uint32, n)
        self.rec_cam = self.ws.read_buffer(B.GS_BUF_REC_CAMERA, np.uint16, n)
        self.rect = self.ws.read_buffer(B.GS_BUF_REC_RECT, np.uint32, n, 2)
        self.tt = self.ws.read_buffer(B.GS_BUF_REC_TILES, np.uint32, n)
        self.rd0 = self.ws.read_buffer(B.GS_BUF_REC_XY_CONIC, np.float32, n, 4)
        self.rd1 = self.ws.read_buffer(B.GS_BUF_REC_C_OPAC_RG, np.float32, n, 4)
        self.rd2 = self.ws.read_buffer(B.GS_BUF_REC_B_LO, np.float32, n, 4)
        ntiles = sum(B.tiles_of(cm, *self.tile) for cm in cams)
        self.ranges = self.ws.read_buffer(B.GS_BUF_TILE_RANGES, np.uint32, ntiles, 2)
        self.sorted_vals = self.ws.read_buffer(B.GS_BUF_SORTED_VALUES, np.uint32, self.counts["n_instances"])
        self.n_contrib = self.ws.read_buffer(B.GS_BUF_N_CONTRIB, np.uint32, self.P)

    # per-camera views -----------------------------------------------------------
    def pix_base(self, c):
        return sum(cm.width * cm.height for cm in self.cams[:c])

    def tile_base(self, c):
        return sum(B.tiles_of(cm, *self.tile) for cm in self.cams[:c])

    def image(self, c):
        cam = self.cams[c]
        p0, n = self.pix_base(c), cam.width * cam.height
        return self.rgb[3 * p0:3 * (p0 + n)].view(3, cam.height, cam.width).double().cpu().numpy()

    def T_final(self, c):
        cam = self.cams[c]
        p0, n = self.pix_base(c), cam.width * cam.height
        return self.T[p0:p0 + n].view(cam.height, cam.width).double().cpu().numpy()

    def n_contrib_img(self, c):
        cam = self.cams[c]
        p0, n = self.pix_base(c), cam.width * cam.height
        return self.n_contrib[p0:p0 + n].reshape(cam.height, cam.width).astype(np.int64)

    def records_of(self, c):
        """Dict Gaussian -> record index for camera c."""
        idx = np.nonzero(self.rec_cam == c)[0]
        return dict(zip(self.rec_g[idx].tolist(), idx.tolist()))

    def tile_lists(self, c):
        """Per local tile of camera c, the ordered list of Gaussian ids."""
        tb = self.tile_base(c)
        out = []
        for t in range(B.tiles_of(self.cams[c], *self.tile)):
            s, e = self.ranges[tb + t]
            out.append(self.rec_g[self.sorted_vals[s:e]].astype(np.int64))
        return out


def unpack_rect(r):
    r = np.asarray(r, np.uint32)
    return np.stack([r[..., 0] & 0xFFFF, r[..., 0] >> 16, r[..., 1] & 0xFFFF, r[..., 1] >> 16], -1).astype(np.int32)


def grads_to_host(gr: B.GaussianTensors) -> dict:
    f = lambda t: t.double().cpu().numpy()
    return dict(mean=f(gr.mean), log_scale=f(gr.log_scale), quat=f(gr.quat), opacity_logit=f(gr.opacity_logit),
                sh=f(gr.sh))


def assert_grad_close(name, g, ref, rtol=1e-3, big=1e-2):
    """Gradient parity rule: max|g - ref| <= rtol * max|ref| over the tensor, and
    elementwise relative error <= rtol where |ref| >= big * max|ref|."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    m = np.abs(ref).max()
    if m == 0:
        assert np.abs(g).max() == 0, name
        return
    err = np.abs(g - ref)
    assert err.max() <= rtol * m, f"{name}: max err {err.max():.3e} > {rtol} * {m:.3e}"
    sel = np.abs(ref) >= big * m
    rel = err[sel] / np.abs(ref[sel])
    assert rel.max() <= rtol, f"{name}: elementwise rel err {rel.max():.3e} (index {np.nonzero(sel)[0][rel.argmax()]})"


def assert_param_grad_close(name, g, ref, rtol=1e-3, big=1e-2):
    """Parameter-gradient parity rule, per Gaussian: with e_i = |g_i - ref_i|
    and r_i = |ref_i| the Euclidean norms of Gaussian i's gradient for this
    parameter (its row: 3 for the mean, 48 for the SH coefficients, ...),
    max e_i <= rtol * max r_i, and e_i <= rtol * r_i wherever r_i >= big * max r_i.
    A row is compared as a vector because its coordinates are tied to an
    arbitrary frame (world axes for the mean): a coordinate can be small only
    because the gradient points along another axis."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    n = ref.shape[0]
    e = np.linalg.norm((g - ref).reshape(n, -1), axis=1)
    r = np.linalg.norm(ref.reshape(n, -1), axis=1)
    m = r.max() if n else 0.0
    if m == 0:
        assert e.max(initial=0.0) == 0, name
        return
    assert e.max() <= rtol * m, f"{name}: max err {e.max():.3e} > {rtol} * {m:.3e}"
    sel = r >= big * m
    rel = e[sel] / r[sel]
    assert rel.max() <= rtol, f"{name}: per-Gaussian rel err {rel.max():.3e} (Gaussian {np.nonzero(sel)[0][rel.argmax()]})"


def record_mean(rd0, rd2):
    """Projected mean of GPU records: the float pair u + u_lo, in double."""
    return rd0[:, :2].astype(np.float64) + rd2[:, 1:3].astype(np.float64)


def footprint_power_err(rd0, rd1, rd2, conic, uv):
    """Largest error of the GPU records' exponent -1/2 (A (dx + k dy)^2 + D dy^2)
    on the 1-sigma and 3-sigma ellipses of the exact conic (conic rows A, B, C,
    exact mean uv), where the exact exponent is -1/2 and -9/2."""
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    det = A * C - B * B
    cov = np.stack([C / det, -B / det, A / det], 1)
    l00 = np.sqrt(cov[:, 0])
    l10 = cov[:, 1] / l00
    l11 = np.sqrt(np.maximum(cov[:, 2] - l10 ** 2, 0.0))
    mg = record_mean(rd0, rd2)
    gA, gk, gD = (rd0[:, 2:3].astype(np.float64), rd0[:, 3:4].astype(np.float64), rd1[:, 0:1].astype(np.float64))
    th = np.linspace(0.0, 2.0 * np.pi, 16, endpoint=False)[None]
    err = np.zeros(len(A))
    for r in (1.0, 3.0):
        dx = l00[:, None] * r * np.cos(th)
        dy = l10[:, None] * r * np.cos(th) + l11[:, None] * r * np.sin(th)
        ddx = uv[:, 0:1] + dx - mg[:, 0:1]
        ddy = uv[:, 1:2] + dy - mg[:, 1:2]
        e = ddx + gk * ddy
        pg = -0.5 * (gA * e * e + gD * ddy * ddy)
        err = np.maximum(err, np.abs(pg + 0.5 * r * r).max(1))
    return err

