"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and bring its outputs back in the oracle's layout."""
from __future__ import annotations

import numpy as np
import torch

from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth


def tiles_xy(cam):
    return (cam.width + 15) // 16, (cam.height + 15) // 16


def capacity_for(n, cams, records=None, instances=None):
    tiles = sum(B.tiles_of(c) for c in cams)
    pix = sum(c.width * c.height for c in cams)
    return dict(max_gaussians=max(n, 1), max_records=records or max(n * len(cams), 1),
                max_instances=instances or max(64 * n * len(cams), 1024), max_tiles=tiles, max_pixels=pix,
                max_cameras=len(cams))


def gpu_params(P, **over):
    """Binding params equal to oracle Params P."""
    d = dict(bg=tuple(P.bg), alpha_min=P.alpha_min, alpha_max=P.alpha_max, T_min=P.T_min, dilation=P.dilation,
             znear=P.znear, fov_clamp=P.fov_clamp, lod_enable=P.lod_enable, lod_d0=P.lod_d0, lod_f=P.lod_f,
             lod_Lmax=P.lod_Lmax, cull_enable=P.cull_enable, eps_score=P.eps_score, vis_mass=P.vis_mass)
    d.update(over)
    return B.RenderParams(**d)


class GpuRun:
    """One preprocess + bin_sort + render_fwd of a scene, with readbacks."""

    def __init__(self, g: synth.GaussianSet, cams, P, cull=None, ws=None, cap=None):
        self.cams = cams
        self.gt = B.GaussianTensors.from_host(g)
        self.ws = ws or B.Workspace(**(cap or capacity_for(g.n, cams)))
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
        self.rd2 = self.ws.read_buffer(B.GS_BUF_REC_B, np.float32, n)
        ntiles = sum(B.tiles_of(cm) for cm in cams)
        self.ranges = self.ws.read_buffer(B.GS_BUF_TILE_RANGES, np.uint32, ntiles, 2)
        self.sorted_vals = self.ws.read_buffer(B.GS_BUF_SORTED_VALUES, np.uint32, self.counts["n_instances"])
        self.n_contrib = self.ws.read_buffer(B.GS_BUF_N_CONTRIB, np.uint32, self.P)

    # per-camera views -----------------------------------------------------------
    def pix_base(self, c):
        return sum(cm.width * cm.height for cm in self.cams[:c])

    def tile_base(self, c):
        return sum(B.tiles_of(cm) for cm in self.cams[:c])

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
        for t in range(B.tiles_of(self.cams[c])):
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
