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


class ViewRun:
    """One preprocess + bin_sort + render_fwd of a scene, with readbacks."""

    def __init__(self, g: synth.GaussianSet, cams, P, cull=None, ws=None, cap=None):
        self.cams = cams
        self.tile = (P.tile_w, P.tile_h)
        self.gt = B.GaussianTensors.from_host(g)
        self.ws = ws or B.Workspace(**(cap or capacity_for(g.n, cams, tile=self.tile)))
        self.cull = None if cull is None else torch.from_numpy(np.ascontiguousarray(cull, np.uint32).view(np.int32)).cuda()
        self.ws.preprocess(self.gt, cams, gpu_params(P), self.cull)
        self.P = sum(cm.width * cm.height for cm in cams)
        self.rgb = torch.empty(3 * self.P, device="cuda")
        self.T = torch.empty(self.P, device="cuda")
        self.readback(render=True)

    def readback(self, render=False):
        """Bins the last preprocess (and renders it when asked), then reads the
        records, lists and counters back."""
        c = self.ws.counts()
        self.n_records = c["n_records"]
        self.depth_bits = self.ws.read_buffer(B.GS_BUF_REC_DEPTH, np.uint32, self.n_records)
        self.ws.bin_sort()
        if render:
            self.ws.render_fwd(self.rgb, self.T)
        self.ws.sync_status()
        self.counts = self.ws.counts()
        cams = self.cams
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


def assert_grad_close(name, g, ref, rtol=1e-3, big=1e-2, bound=None):
    """Gradient parity rule: max|g - ref| <= rtol * max|ref| over the tensor, and
    elementwise relative error <= rtol where |ref| >= big * max|ref|.  bound
    (same shape, optional): per element, how far any FP32 evaluation can be
    from the exact value through the element's own conditioning (the oracle's
    grad_bounds); it is added to both allowances."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    b = np.zeros_like(ref) if bound is None else np.asarray(bound, np.float64).ravel()
    m = np.abs(ref).max()
    if m == 0:
        assert np.all(np.abs(g) <= b), name
        return
    err = np.abs(g - ref)
    over = err - b
    assert over.max() <= rtol * m, f"{name}: max err {err[over.argmax()]:.3e} > {rtol} * {m:.3e} + {b[over.argmax()]:.3e}"
    sel = np.nonzero(np.abs(ref) >= big * m)[0]
    rel = (err[sel] - b[sel]) / np.abs(ref[sel])
    assert rel.max() <= rtol, f"{name}: elementwise rel err {rel.max():.3e} beyond its bound (index {sel[rel.argmax()]})"


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



# ---- projection decisions: exact outside the oracle's tie flags -----------------

PROJ_TIES = (1 | 2 | 4 | 8 | 16 | 64)  # oracle TIE_LOD | NEAR | DET | RADIUS | RECT | DEPTH


def _ulp32(x):
    return np.spacing(np.abs(np.asarray(x, np.float32))).astype(np.float64)


def allowed_rect_ranges(pr, idx, tile_w, tile_h, tiles_x, tiles_y):
    """Per Gaussian in idx, the range [lo, hi] of each rectangle edge over the
    outcomes an FP32 renderer may reach where the oracle flags a tie: radius
    ceil(extent +- 2 * its error bound), mean within 2 (1/2 ulp + 2^-38 |u|).
    For an unflagged Gaussian the ranges are single values (the oracle's own)."""
    ext, err = pr["extent"][idx, 0], pr["extent"][idx, 1]
    u, v = pr["uv"][idx, 0], pr["uv"][idx, 1]
    tied = (pr["tie"][idx] & (8 | 16)) != 0
    er = np.where(tied, 2.0 * err, 0.0)
    rmin = np.ceil(ext - er).astype(np.int64)
    rmax = np.ceil(ext + er).astype(np.int64)
    bu = np.where(tied, 2.0 * (0.5 * _ulp32(u) + 2.0 ** -38 * np.abs(u)), 0.0)
    bv = np.where(tied, 2.0 * (0.5 * _ulp32(v) + 2.0 ** -38 * np.abs(v)), 0.0)
    cx = lambda a: np.clip(a, 0, tiles_x)
    cy = lambda a: np.clip(a, 0, tiles_y)
    x0 = (cx(np.floor((u - bu - rmax) / tile_w)), cx(np.floor((u + bu - rmin) / tile_w)))
    y0 = (cy(np.floor((v - bv - rmax) / tile_h)), cy(np.floor((v + bv - rmin) / tile_h)))
    x1 = (cx(np.floor((u - bu + rmin) / tile_w) + 1), cx(np.floor((u + bu + rmax) / tile_w) + 1))
    y1 = (cy(np.floor((v - bv + rmin) / tile_h) + 1), cy(np.floor((v + bv + rmax) / tile_h) + 1))
    lo = np.stack([x0[0], y0[0], x1[0], y1[0]], 1).astype(np.int64)
    hi = np.stack([x0[1], y0[1], x1[1], y1[1]], 1).astype(np.int64)
    return lo, hi


def adopt_tied_decisions(O, pr, run, c, cam, P, max_tied_frac=1e-3):
    """Checks the GPU's projection decisions for camera c against the oracle's
    FP64 ones, and takes the GPU's outcome into the oracle's projection where
    the oracle flags both outcomes as correct (a tie).

    Exact outside the flags: the active set, every rectangle, tile count and
    depth key.  At a flagged Gaussian the GPU's outcome must be one the flag
    allows: active or not (an inactive outcome needs a flagged gate, near-plane
    or determinant test, or an allowed rectangle that is empty), rectangle
    edges within allowed_rect_ranges, depth key within one float of the
    oracle's.  Returns the number of flagged Gaussians among those active on
    either side."""
    n = pr["status"].shape[0]
    recs = run.records_of(c)
    gpu_active = np.zeros(n, bool)
    gi = np.fromiter(recs.keys(), np.int64, len(recs))
    ri = np.fromiter(recs.values(), np.int64, len(recs))
    gpu_active[gi] = True
    gpu_rect = np.zeros((n, 4), np.int64)
    gpu_rect[gi] = unpack_rect(run.rect[ri])
    gpu_depth = np.zeros(n, np.uint32)
    gpu_depth[gi] = run.depth_bits[ri]
    ora_active = pr["status"] == O.ACTIVE
    tie = (pr["tie"] & PROJ_TIES) != 0
    # unflagged: identical decisions
    mism = np.nonzero((gpu_active != ora_active) & ~tie)[0]
    assert len(mism) == 0, f"active-set mismatch outside the flags: {mism[:10]}"
    both = np.nonzero(gpu_active & ora_active & ~tie)[0]
    assert np.array_equal(gpu_rect[both], pr["rect"][both].astype(np.int64)), "rectangle differs outside the flags"
    assert np.array_equal(gpu_depth[both], pr["depth32"][both].view(np.uint32)), "depth key differs outside the flags"
    # flagged: an allowed outcome, then adopted
    tiles_x, tiles_y = (cam.width + P.tile_w - 1) // P.tile_w, (cam.height + P.tile_h - 1) // P.tile_h
    tidx = np.nonzero(tie & (gpu_active | ora_active))[0]
    assert len(tidx) <= max(3, max_tied_frac * max(int(ora_active.sum()), 1)), len(tidx)
    if len(tidx):
        lo, hi = allowed_rect_ranges(pr, tidx, P.tile_w, P.tile_h, tiles_x, tiles_y)
        for k, i in enumerate(tidx):
            if gpu_active[i]:
                r = gpu_rect[i]
                assert np.all(lo[k] <= r) and np.all(r <= hi[k]), (i, r, lo[k], hi[k])
                dg = np.float32(gpu_depth[i:i + 1].view(np.float32)[0])
                assert abs(float(dg) - pr["depth"][i]) <= 1.5 * _ulp32(pr["depth"][i]), i
                pr["status"][i] = O.ACTIVE
                pr["rect"][i] = r
                pr["tiles"][i] = (r[2] - r[0]) * (r[3] - r[1])
                pr["depth32"][i] = dg
            else:
                gate = (pr["tie"][i] & (1 | 2 | 4)) != 0
                can_empty = np.any(lo[k][2:] <= lo[k][:2]) or not ora_active[i]
                assert gate or can_empty or not ora_active[i], i
                if ora_active[i]:
                    pr["status"][i] = O.EMPTY
                    pr["tiles"][i] = 0
    return len(tidx)


def oracle_view_matched(O, run, c, g64, cam, P, cull=None):
    """The oracle's forward of camera c, with the decisions it flags as ties
    taken from the GPU run once checked (adopt_tied_decisions)."""
    pr = O.project(g64, cam, P, cull)
    adopt_tied_decisions(O, pr, run, c, cam, P)
    bins = O.bin_tiles(pr, cam, P)
    out = O.render(pr, bins, cam, P)
    out["proj"], out["bins"] = pr, bins
    return out


def assert_record_precision(run, ridx, pr, gidx, P):
    """The GPU records meet the precision the oracle's compositing flags allow
    for: projected mean within prec_mean pixels; the exponent form's A and D
    within prec_conic relative, k within prec_conic (|k| + sqrt(D / A))."""
    mg = record_mean(run.rd0[ridx], run.rd2[ridx])
    assert np.abs(mg - pr["uv"][gidx]).max(initial=0.0) <= P.prec_mean
    A, Bc, C = pr["conic"][gidx, 0], pr["conic"][gidx, 1], pr["conic"][gidx, 2]
    k = Bc / A
    D = C - Bc * k
    gA = run.rd0[ridx, 2].astype(np.float64)
    gk = run.rd0[ridx, 3].astype(np.float64)
    gD = run.rd1[ridx, 0].astype(np.float64)
    pc = P.prec_conic
    assert np.all(np.abs(gA - A) <= pc * A), np.max(np.abs(gA - A) / A)
    assert np.all(np.abs(gD - D) <= pc * D), np.max(np.abs(gD - D) / D)
    kb = np.abs(k) + np.sqrt(D / A)
    assert np.all(np.abs(gk - k) <= pc * kb), np.max(np.abs(gk - k) / kb)


PARAM_NAMES = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def assert_gaussian_grads_close(gg, og, rtol=1e-3, big=1e-2):
    """The gradient parity rule per parameter tensor: element-wise
    (assert_grad_close) for the log-scales, quaternions, opacity logits and SH
    coefficients; per Gaussian row for the mean (assert_param_grad_close),
    whose three coordinates are in an arbitrary world frame.  The log-scale and
    quaternion elements take the oracle's FP32 conditioning bound on top (a
    short axis of a long thin footprint is a nearly cancelling sum of pixel
    terms: og["bounds"], from grad_bounds)."""
    bounds = og.get("bounds", {})
    for k in PARAM_NAMES:
        if k == "mean":
            assert_param_grad_close(k, gg[k], og[k], rtol, big)
        else:
            assert_grad_close(k, gg[k], og[k], rtol, big, bound=bounds.get(k))
