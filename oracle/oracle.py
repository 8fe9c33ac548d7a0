"""FP64 CPU oracle for the 3DGS render hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never imports the CUDA package and
the CUDA package never imports it; both consume the seeded inputs of
``paper_2605_13794_gb300.synth``.

The heavy loops (projection, binning, compositing and their adjoints) live in
``gs_oracle.c``; this module marshals numpy arrays and adds the parts that are
plain array code:

* importance aggregation (Sec. 3.2, Fig. 2): s_i += w/(a+eps) over views with
  a > 0, c^rad, and c^vis = membership in the smallest set of largest w that
  carries ``vis_mass`` (99 %) of the view's total, ties by lower index;
  Cull = 1 - c^vis (Sec. 3.2, Sec. 3.3 Eq. 3);
* the photometric loss of Eq. 4 (L1 + lambda (1 - SSIM), SSIM with an 11x11
  Gaussian window, sigma 1.5, zero "same" padding) and the scale regulariser of
  Eq. 5, with their gradients;
* Adam (Kingma and Ba), the optimizer the paper's "standard 3DGS" training uses;
* the model-level operations of Sec. 3.2 and 3.3: the two pruning passes
  (importance-weighted sampling without replacement, the 99 %-mass cut of s),
  density control (clone / split) with the phi_i reweighting and the LOD
  inheritance rule, and order-preserving compaction.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_gs_oracle.so")
_SRC = [os.path.join(_HERE, "gs_oracle.c")]

ACTIVE, GATED_LOD, GATED_CULL, NEAR, DEGENERATE, EMPTY = range(6)
TIE_LOD, TIE_NEAR, TIE_DET, TIE_RADIUS, TIE_RECT, TIE_CLAMP, TIE_DEPTH = 1, 2, 4, 8, 16, 32, 64
PIX_ALPHA_MIN, PIX_T_MIN, PIX_ALPHA_MAX, PIX_POWER = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the C oracle (plain C; -ffp-contract=off keeps every FP64
    operation one IEEE operation on every host)."""
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in _SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", _SO + ".tmp", _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(_SO + ".tmp", _SO)
    return _SO


_lib = None


class ORCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("campos", ctypes.c_double * 3), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class ORParams(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("lod_enable", ctypes.c_int32), ("lod_Lmax", ctypes.c_int32),
                ("cull_enable", ctypes.c_int32), ("bg", ctypes.c_double * 3),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double), ("T_min", ctypes.c_double),
                ("dilation", ctypes.c_double), ("znear", ctypes.c_double), ("fov_clamp", ctypes.c_double),
                ("lod_d0", ctypes.c_double), ("lod_f", ctypes.c_double),
                ("prec_mean", ctypes.c_double), ("prec_conic", ctypes.c_double), ("comp_band", ctypes.c_double)]


class ORProjOut(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("status", "tie", "uv", "depth", "depth32", "conic", "opacity", "rgb", "clamp", "radius", "rect", "tiles",
                 "extent")]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        _lib.or_project.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.or_bin.argtypes = [i64, vp, vp, vp, i32, i32, vp, vp, i64]
        _lib.or_bin.restype = i64
        _lib.or_render.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.or_render_brute.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.or_render_pixels.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.or_render_bwd.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.or_grad_bounds.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, ctypes.c_double, vp, vp]
        _lib.or_project_bwd.argtypes = [i64] + [vp] * 18
        _lib.or_sh_basis.argtypes = [vp, i64, vp, vp]
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


@dataclasses.dataclass
class Params:
    """Render parameters (values of the standard 3DGS renderer unless noted)."""

    tile_w: int = 16
    tile_h: int = 16
    bg: tuple = (0.0, 0.0, 0.0)
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    dilation: float = 0.3
    znear: float = 0.2
    fov_clamp: float = 1.3
    lod_enable: bool = False
    lod_d0: float = 1600.0
    lod_f: float = 2.0
    lod_Lmax: int = 5
    cull_enable: bool = False
    # Precision of the renderer the decision flags allow for (compositing): its
    # projected mean within prec_mean pixels, the coefficients of its exponent
    # form A (x + k y)^2 + D y^2 within prec_conic (relative; k relative to
    # |k| + sqrt(D / A)).  The GPU parity tests check the CUDA records against
    # both bounds.  comp_band is a further log-space margin on every threshold.
    prec_mean: float = 1e-6
    prec_conic: float = 8e-6
    comp_band: float = 2e-6
    eps_score: float = 1e-6
    vis_mass: float = 0.99

    def c(self) -> ORParams:
        # The thresholds are FP32 constants on the GPU; the oracle compares
        # against the same FP32 values so that the two definitions agree.
        f = lambda x: float(np.float32(x))
        return ORParams(self.tile_w, self.tile_h, int(self.lod_enable), self.lod_Lmax, int(self.cull_enable),
                        (ctypes.c_double * 3)(*[f(b) for b in self.bg]), f(self.alpha_min), f(self.alpha_max),
                        f(self.T_min), f(self.dilation), f(self.znear), f(self.fov_clamp), f(self.lod_d0),
                        f(self.lod_f), self.prec_mean, self.prec_conic, self.comp_band)


def camera_c(cam) -> ORCamera:
    return ORCamera((ctypes.c_double * 9)(*np.asarray(cam.R, np.float64).ravel()),
                    (ctypes.c_double * 3)(*np.asarray(cam.t, np.float64)),
                    float(np.float32(cam.fx)), float(np.float32(cam.fy)),
                    float(np.float32(cam.cx)), float(np.float32(cam.cy)),
                    (ctypes.c_double * 3)(*np.asarray(cam.campos, np.float64)), cam.width, cam.height)


def _d(a):
    return np.ascontiguousarray(np.asarray(a, np.float64))


def gaussians64(g) -> dict:
    """FP64 copies of a GaussianSet's arrays (exact: the inputs are FP32) in
    the oracle's own attribute-major layout: mean (3, n), log_scale (3, n),
    quat (4, n), opacity_logit (n,), sh (16, 3, n)."""
    return dict(mean=_d(np.asarray(g.mean).T), log_scale=_d(np.asarray(g.log_scale).T),
                quat=_d(np.asarray(g.quat).T), opacity_logit=_d(g.opacity_logit),
                sh=_d(np.asarray(g.sh).transpose(1, 2, 0)), lod=np.ascontiguousarray(g.lod, np.uint8))


def grads_per_gaussian(grads: dict) -> dict:
    """The oracle's attribute-major gradients in the per-Gaussian row layout
    of the inputs: mean (n, 3), log_scale (n, 3), quat (n, 4), sh (n, 16, 3);
    with "bounds" (the same layout) where backward_view computed them."""
    out = dict(mean=grads["mean"].T, log_scale=grads["log_scale"].T, quat=grads["quat"].T,
               opacity_logit=grads["opacity_logit"], sh=grads["sh"].transpose(2, 0, 1))
    if "_bounds" in grads:
        out["bounds"] = dict(log_scale=grads["_bounds"]["log_scale"].T, quat=grads["_bounds"]["quat"].T)
    return out


def project(g64: dict, cam, params: Params, cull=None) -> dict:
    """Per-Gaussian gate, projection and colour for one camera."""
    n = g64["opacity_logit"].shape[0]
    out = dict(status=np.zeros(n, np.int8), tie=np.zeros(n, np.uint8), uv=np.zeros((n, 2)),
               depth=np.zeros(n), depth32=np.zeros(n, np.float32), conic=np.zeros((n, 3)),
               opacity=np.zeros(n), rgb=np.zeros((n, 3)), clamp=np.zeros(n, np.uint8),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32),
               extent=np.zeros((n, 2)))
    po = ORProjOut(*[out[f[0]].ctypes.data for f in ORProjOut._fields_])
    cull_arr = None if cull is None else np.ascontiguousarray(cull, np.uint32)
    cam_c, par_c = camera_c(cam), params.c()
    lib().or_project(n, _p(g64["mean"]), _p(g64["log_scale"]), _p(g64["quat"]), _p(g64["opacity_logit"]),
                     _p(g64["sh"]), _p(g64["lod"]), _p(cull_arr), ctypes.byref(cam_c), ctypes.byref(par_c),
                     ctypes.byref(po))
    return out


def tiles_of(cam, params: Params):
    return (cam.width + params.tile_w - 1) // params.tile_w, (cam.height + params.tile_h - 1) // params.tile_h


def bin_tiles(proj: dict, cam, params: Params):
    """Per-tile lists of active Gaussians ordered by (FP32 depth bits, index)."""
    tx, ty = tiles_of(cam, params)
    n = proj["status"].shape[0]
    tile_start = np.zeros(tx * ty + 1, np.int64)
    cap = int(proj["tiles"].astype(np.int64).sum())
    lst = np.zeros(max(cap, 1), np.int32)
    total = lib().or_bin(n, _p(proj["status"]), _p(proj["rect"]), _p(proj["depth32"]), tx, ty,
                         _p(tile_start), _p(lst), cap)
    assert total == cap
    return tile_start, lst[:cap]


def render(proj: dict, bins, cam, params: Params) -> dict:
    tile_start, lst = bins
    n = proj["status"].shape[0]
    W, H = cam.width, cam.height
    out = dict(image=np.zeros((3, H, W)), T=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32),
               flags=np.zeros((H, W), np.uint8), w=np.zeros(n), a=np.zeros(n), gcount=np.zeros(n, np.int32))
    lst = np.ascontiguousarray(lst, np.int32) if lst.size else np.zeros(1, np.int32)
    lib().or_render(ctypes.byref(camera_c(cam)), ctypes.byref(params.c()), n, _p(proj["uv"]), _p(proj["conic"]),
                    _p(proj["opacity"]), _p(proj["rgb"]), _p(tile_start), _p(lst), _p(out["image"]), _p(out["T"]),
                    _p(out["n_contrib"]), _p(out["flags"]), _p(out["w"]), _p(out["a"]), _p(out["gcount"]))
    return out


def render_brute(proj: dict, cam, params: Params):
    n = proj["status"].shape[0]
    W, H = cam.width, cam.height
    image, T = np.zeros((3, H, W)), np.zeros((H, W))
    lib().or_render_brute(ctypes.byref(camera_c(cam)), ctypes.byref(params.c()), n, _p(proj["status"]),
                          _p(proj["depth32"]), _p(proj["uv"]), _p(proj["conic"]), _p(proj["opacity"]),
                          _p(proj["rgb"]), _p(image), _p(T))
    return image, T


def render_pixels(proj: dict, pixels, lists, params: Params) -> dict:
    """Composites explicit pixels; ``lists[k]`` is pixel k's ordered Gaussian list."""
    pixels = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    npix = pixels.shape[0]
    starts = np.zeros(npix + 1, np.int64)
    starts[1:] = np.cumsum([len(l) for l in lists])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(l, np.int32) for l in lists]) if npix else
                                np.zeros(1, np.int32))
    if flat.size == 0:
        flat = np.zeros(1, np.int32)
    out = dict(C=np.zeros((npix, 3)), T=np.zeros(npix), n_contrib=np.zeros(npix, np.int32),
               flags=np.zeros(npix, np.uint8))
    lib().or_render_pixels(ctypes.byref(params.c()), npix, _p(pixels), _p(starts), _p(flat), _p(proj["uv"]),
                           _p(proj["conic"]), _p(proj["opacity"]), _p(proj["rgb"]), _p(out["C"]), _p(out["T"]),
                           _p(out["n_contrib"]), _p(out["flags"]))
    return out


def render_bwd(proj: dict, bins, cam, params: Params, dL_dimage) -> dict:
    """Gradients of the projected quantities; conic_abs holds, per Gaussian, the
    sums of the magnitudes of the pixel terms of dL/dconic."""
    tile_start, lst = bins
    n = proj["status"].shape[0]
    out = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               conic_abs=np.zeros((n, 3)))
    lst = np.ascontiguousarray(lst, np.int32) if lst.size else np.zeros(1, np.int32)
    lib().or_render_bwd(ctypes.byref(camera_c(cam)), ctypes.byref(params.c()), n, _p(proj["uv"]),
                        _p(proj["conic"]), _p(proj["opacity"]), _p(proj["rgb"]), _p(tile_start), _p(lst),
                        _p(_d(dL_dimage)), _p(out["uv"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]),
                        _p(out["conic_abs"]))
    return out


# FP32 error of a renderer's summed conic gradient, relative to the sum of the
# magnitudes of its pixel terms: a budget of 64 roundings (the per-pixel chain
# through alpha, T and dL/dalpha, and the tree sums over the pixels)
EPS_CONIC_SUM = 64 * 2.0 ** -24


def grad_bounds(g64: dict, proj: dict, cam, params: Params, pgrad: dict, bounds=None) -> dict:
    """Accumulates, per Gaussian, how far an FP32 renderer's log-scale and
    quaternion gradients can be from the exact ones through the conditioning of
    the bilinear forms they are (see or_grad_bounds in gs_oracle.c)."""
    n = g64["opacity_logit"].shape[0]
    if bounds is None:
        bounds = dict(log_scale=np.zeros((3, n)), quat=np.zeros((4, n)))
    lib().or_grad_bounds(n, _p(g64["mean"]), _p(g64["log_scale"]), _p(g64["quat"]), _p(proj["status"]),
                         ctypes.byref(camera_c(cam)), ctypes.byref(params.c()), _p(pgrad["conic_abs"]),
                         EPS_CONIC_SUM, _p(bounds["log_scale"]), _p(bounds["quat"]))
    return bounds


def zero_grads(n: int) -> dict:
    return dict(mean=np.zeros((3, n)), log_scale=np.zeros((3, n)), quat=np.zeros((4, n)),
                opacity_logit=np.zeros(n), sh=np.zeros((16, 3, n)))


def project_bwd(g64: dict, proj: dict, cam, params: Params, pgrad: dict, grads: dict) -> dict:
    """Accumulates parameter gradients into ``grads`` (FP64 arrays)."""
    n = g64["opacity_logit"].shape[0]
    lib().or_project_bwd(n, _p(g64["mean"]), _p(g64["log_scale"]), _p(g64["quat"]), _p(g64["opacity_logit"]),
                         _p(g64["sh"]), _p(proj["status"]), _p(proj["clamp"]), ctypes.byref(camera_c(cam)),
                         ctypes.byref(params.c()), _p(pgrad["uv"]), _p(pgrad["conic"]), _p(pgrad["opacity"]),
                         _p(pgrad["rgb"]), _p(grads["mean"]), _p(grads["log_scale"]), _p(grads["quat"]),
                         _p(grads["opacity_logit"]), _p(grads["sh"]))
    return grads


def sh_basis(dirs, with_grad: bool = False):
    dirs = _d(np.asarray(dirs).reshape(-1, 3))
    m = dirs.shape[0]
    Y = np.zeros((m, 16))
    dY = np.zeros((m, 16, 3)) if with_grad else None
    lib().or_sh_basis(_p(dirs), m, _p(Y), _p(dY))
    return (Y, dY) if with_grad else Y


# ---- whole-view helpers -------------------------------------------------

def forward_view(g64: dict, cam, params: Params, cull=None) -> dict:
    proj = project(g64, cam, params, cull)
    bins = bin_tiles(proj, cam, params)
    out = render(proj, bins, cam, params)
    out["proj"], out["bins"] = proj, bins
    return out


def backward_view(g64: dict, fwd: dict, cam, params: Params, dL_dimage, grads=None) -> dict:
    if grads is None:
        grads = zero_grads(g64["opacity_logit"].shape[0])
    pg = render_bwd(fwd["proj"], fwd["bins"], cam, params, dL_dimage)
    project_bwd(g64, fwd["proj"], cam, params, pg, grads)
    grads["_projected"] = pg
    grads["_bounds"] = grad_bounds(g64, fwd["proj"], cam, params, pg, grads.get("_bounds"))
    return grads


# ---- importance (Sec. 3.2, Fig. 2) ------------------------------------------

def visible_top_mass(w, vis_mass: float = 0.99) -> np.ndarray:
    """c^vis for one view: the smallest prefix of Gaussians sorted by w
    (descending, ties by lower index) whose summed w reaches vis_mass of the
    total.  Gaussians with w = 0 are never visible."""
    w = np.asarray(w, np.float64)
    vis = np.zeros(w.shape[0], bool)
    pos = np.nonzero(w > 0)[0]
    if pos.size == 0:
        return vis
    order = pos[np.lexsort((pos, -w[pos]))]
    cum = np.cumsum(w[order])
    k = int(np.searchsorted(cum, vis_mass * cum[-1], side="left"))
    vis[order[:k + 1]] = True
    return vis


def importance_update(acc: dict, w, a, proj: dict, vis_mass=0.99, eps=1e-6) -> dict:
    """Adds one view to the running score s, c^rad and c^vis; returns this
    view's c^vis and Cull bits."""
    w = np.asarray(w, np.float64)
    a = np.asarray(a, np.float64)
    hit = a > 0
    acc["s"][hit] += w[hit] / (a[hit] + eps)
    crad = (proj["status"] == ACTIVE)
    acc["crad"] += crad.astype(np.int64)
    vis = visible_top_mass(w, vis_mass)
    acc["cvis"] += vis.astype(np.int64)
    return dict(cvis=vis, cull=~vis)


def new_importance(n: int) -> dict:
    return dict(s=np.zeros(n), crad=np.zeros(n, np.int64), cvis=np.zeros(n, np.int64))


# ---- loss (Sec. 3.4, Eq. 4 and Eq. 5) -----------------------------------------

def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    x = np.arange(size) - size // 2
    g = np.exp(-(x ** 2) / (2.0 * sigma ** 2))
    g /= g.sum()
    return np.outer(g, g)


def window_sum(img, win):
    """Zero-padded 'same' weighted window sum over the last two axes."""
    img = np.asarray(img, np.float64)
    k = win.shape[0]
    r = k // 2
    H, W = img.shape[-2:]
    pad = np.zeros(img.shape[:-2] + (H + 2 * r, W + 2 * r))
    pad[..., r:r + H, r:r + W] = img
    out = np.zeros_like(img)
    for i in range(k):
        for j in range(k):
            out += win[i, j] * pad[..., i:i + H, j:j + W]
    return out


def ssim_and_grad(x, y, C1=0.01 ** 2, C2=0.03 ** 2, win=None):
    """Mean SSIM over channels and pixels and its gradient with respect to x."""
    if win is None:
        win = gaussian_window()
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = window_sum(x, win), window_sum(y, win)
    exx, eyy, exy = window_sum(x * x, win), window_sum(y * y, win), window_sum(x * y, win)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
    B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
    S = A1 * A2 / (B1 * B2)
    npx = S.size
    dS_dmx = 2 * my * A2 / (B1 * B2) - S * 2 * mx / B1
    dS_dsxx = -S / B2
    dS_dsxy = 2 * A1 / (B1 * B2)
    # S depends on x through mx = w*x, E[x^2] = w*x^2 and E[xy] = w*(xy)
    g = (window_sum(dS_dmx - 2 * mx * dS_dsxx - my * dS_dsxy, win)
         + 2 * x * window_sum(dS_dsxx, win) + y * window_sum(dS_dsxy, win)) / npx
    return float(S.mean()), g


def photometric_loss(images, targets, lam=0.2):
    """Eq. 4 over a batch (B, 3, H, W): mean over views of
    (1 - lambda) mean|I - I*| + lambda (1 - SSIM); returns (loss, dL/dimages)."""
    images = np.asarray(images, np.float64)
    targets = np.asarray(targets, np.float64)
    B = images.shape[0]
    loss = 0.0
    grad = np.zeros_like(images)
    for b in range(B):
        d = images[b] - targets[b]
        l1 = np.abs(d).mean()
        s, gs = ssim_and_grad(images[b], targets[b])
        loss += ((1 - lam) * l1 + lam * (1 - s)) / B
        grad[b] = ((1 - lam) * np.sign(d) / d.size - lam * gs) / B
    return loss, grad


def scale_regulariser(log_scale, visible, beta=10.0):
    """Eq. 5: beta * mean over visible Gaussians of the smallest scale; returns
    (value, dL/dlog_scale).  log_scale is (3, n); the derivative goes to the
    first smallest axis."""
    ls = np.asarray(log_scale, np.float64)
    vis = np.asarray(visible, bool)
    g = np.zeros_like(ls)
    nv = int(vis.sum())
    if nv == 0:
        return 0.0, g
    s = np.exp(ls[:, vis])
    j = np.argmin(s, axis=0)
    smin = s[j, np.arange(s.shape[1])]
    cols = np.nonzero(vis)[0]
    g[j, cols] = beta * smin / nv
    return float(beta * smin.mean()), g


# ---- Adam (Kingma and Ba) ---------------------------------------------------------

def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v


# ---- model level: simplification passes and density control --------------------
#
# Sec. 3.2: an importance pass yields s_i; Pass 1 keeps a fixed fraction by
# importance-weighted sampling without replacement, Pass 2 keeps the smallest
# prefix of Gaussians by descending s carrying 99 % of the total s.  Density
# control (standard 3DGS adaptive density control, Sec. 3) tests the averaged
# view-space positional gradient, reweighted by phi_i = c^vis_i / (c^rad_i + eps)
# (Sec. 3.2), clones small selected Gaussians and splits large ones; the LOD
# label follows the inheritance rule of Sec. 3.3 (clone keeps the parent's
# level, split increments it by one).

def prune_mass(s, mass: float = 0.99) -> np.ndarray:
    """Pass 2: keep mask of the smallest prefix by descending s (ties by lower
    index) whose summed s reaches `mass` of the total; s = 0 is never kept."""
    return visible_top_mass(s, mass)


def prune_sample(s, expo, k: int, with_ties: bool = False):
    """Pass 1: importance-weighted sampling of k Gaussians without replacement,
    with probability proportional to s at every draw.  Drawn as exponential
    clocks: Gaussian i fires at expo_i / s_i (expo_i ~ Exp(1), given), and the
    k earliest are kept (ties by lower index; s_i = 0 never fires before a
    Gaussian with s > 0).  The times are exact quotients (FP64 of the FP32
    inputs).

    with_ties: also returns the Gaussians a renderer forming the times in FP32
    may put on the other side of the cut: an FP32 quotient is within 2^-24 of
    the exact one, so two times less than 2^-22 apart (relative) may swap; the
    flagged set is every time within that of the k-th or (k+1)-th smallest when
    those two are that close."""
    s64 = np.asarray(s, np.float32).astype(np.float64)
    e64 = np.asarray(expo, np.float32).astype(np.float64)
    with np.errstate(divide="ignore"):
        t = np.where(s64 > 0, e64 / np.where(s64 > 0, s64, 1.0), np.inf)
    n = len(t)
    order = np.lexsort((np.arange(n), t))
    keep = np.zeros(n, bool)
    keep[order[:k]] = True
    if not with_ties:
        return keep
    tie = np.zeros(n, bool)
    if 0 < k < n:
        lo, hi = t[order[k - 1]], t[order[k]]
        band = 2.0 ** -22
        if np.isfinite(hi) and hi <= lo * (1 + 2 * band):
            tie = (t >= lo * (1 - band)) & (t <= hi * (1 + band))
    return keep, tie


def successive_sampling_probs(s, k: int) -> np.ndarray:
    """Exact inclusion probabilities of drawing k of len(s) items without
    replacement with probability proportional to s at every draw (enumeration
    of ordered draws; tiny inputs only)."""
    s = np.asarray(s, np.float64)
    n = len(s)
    incl = np.zeros(n)

    def rec(chosen, p):
        if len(chosen) == k:
            for i in chosen:
                incl[i] += p
            return
        rest = [i for i in range(n) if i not in chosen]
        tot = s[rest].sum()
        for i in rest:
            rec(chosen + [i], p * s[i] / tot)

    rec([], 1.0)
    return incl


@dataclasses.dataclass
class DensifyParams:
    grad_threshold: float = 0.0002  # on the averaged |dL/d(u,v)| (pixels), after phi reweighting
    dense_scale: float = 0.01       # largest axis at or below: clone; above: split
    min_opacity: float = 0.005      # Gaussians below are removed
    split_shrink: float = 1.6       # a split child's scales are the parent's / 1.6 (two children)
    n_levels: int = 6               # LOD labels 0..n_levels-1
    eps: float = 1e-6


def densify(g: dict, absgrad, denom, cvis, crad, noise, P: DensifyParams):
    """One density-control step on per-Gaussian rows (the layout of synth:
    mean (n,3), log_scale (n,3), quat (n,4), opacity_logit (n,), sh (n,16,3),
    lod (n,), m and v: dicts of the same rows).  noise: (n, 2, 3) N(0,1)
    samples, used for the two children of a split parent.

    Output rows in parent order; per parent: removed (opacity < min_opacity):
    none; kept: itself; clone: itself then its copy; split: its two children
    mu + R(q) (s * z), log_scale - log(1.6), same q, opacity and SH, level + 1
    (capped at n_levels - 1).  A kept or cloned parent keeps its Adam moments,
    every new Gaussian starts from zero moments.  Returns (rows, m, v, kind)
    with kind per input: 0 removed, 1 kept, 2 cloned, 3 split."""
    n = len(g["opacity_logit"])
    kind = densify_kinds(g["opacity_logit"], g["log_scale"], absgrad, denom, cvis, crad, P)
    names = ("mean", "log_scale", "quat", "opacity_logit", "sh")
    out = []  # (row, m, v) per output Gaussian, in order

    def zeros(row):
        return {k: np.zeros_like(row[k]) for k in names}

    for i in range(n):
        if kind[i] == 0:
            continue
        row = {k: np.asarray(g[k][i], np.float64) for k in names}
        row["lod"] = int(g["lod"][i])
        mi = {k: np.asarray(g["m"][k][i], np.float64) for k in names}
        vi = {k: np.asarray(g["v"][k][i], np.float64) for k in names}
        if kind[i] in (1, 2):
            out.append((row, mi, vi))
        if kind[i] == 2:
            out.append((dict(row), zeros(row), zeros(row)))
        if kind[i] == 3:
            R = _quat_to_rot(row["quat"] / np.linalg.norm(row["quat"]))
            s = np.exp(row["log_scale"])
            for c in range(2):
                child = dict(row)
                child["mean"] = row["mean"] + R @ (s * np.asarray(noise[i, c], np.float64))
                child["log_scale"] = row["log_scale"] - np.log(P.split_shrink)
                child["lod"] = min(row["lod"] + 1, P.n_levels - 1)
                out.append((child, zeros(row), zeros(row)))

    def stack(j, key):
        shape = (0,) + np.shape(g[key])[1:]
        return np.array([o[j][key] for o in out]) if out else np.zeros(shape)

    rows = {k: stack(0, k) for k in names}
    rows["lod"] = np.array([o[0]["lod"] for o in out], np.int64)
    return rows, {k: stack(1, k) for k in names}, {k: stack(2, k) for k in names}, kind


def densify_kinds(opacity_logit, log_scale, absgrad, denom, cvis, crad, P: DensifyParams, with_ties: bool = False):
    """The branch of every Gaussian: 0 removed (opacity < min_opacity), 1 kept,
    2 cloned, 3 split, decided in FP64 on the FP32 inputs: the averaged
    gradient absgrad / denom (0 without a view) times phi = c^vis / (c^rad + eps)
    against the threshold (Sec. 3.2); opacity below min_opacity, as the logit
    against logit(min_opacity); the largest scale against dense_scale, as the
    largest log-scale against log(dense_scale).

    with_ties: also returns the Gaussians whose decision an FP32 renderer may
    take the other way: a score within 10 x 2^-24 (relative) of the threshold
    (its FP32 evaluation -- two quotients, a sum and a product -- is within
    5 x 2^-24), a logit or largest log-scale within one float spacing of its
    threshold (the thresholds held as floats)."""
    f32 = lambda x: float(np.float32(x))
    absgrad = np.asarray(absgrad, np.float32).astype(np.float64)
    denom = np.asarray(denom, np.int64)
    grad = np.where(denom > 0, absgrad / np.where(denom > 0, denom, 1), 0.0)
    eps = f32(P.eps)
    phi = np.asarray(cvis, np.int64) / (np.asarray(crad, np.int64) + eps)
    score = grad * phi
    thr = f32(P.grad_threshold)
    sel = score >= thr
    logit = np.asarray(opacity_logit, np.float32).astype(np.float64)
    lthr = math.log(P.min_opacity / (1.0 - P.min_opacity))
    low = logit < lthr
    mls = np.asarray(log_scale, np.float32).astype(np.float64).max(axis=1)
    sthr = math.log(P.dense_scale)
    small = mls <= sthr
    kind = np.where(low, 0, np.where(~sel, 1, np.where(small, 2, 3))).astype(np.int64)
    if not with_ties:
        return kind
    u = 2.0 ** -24
    sp = lambda x: float(np.spacing(np.float32(abs(x))))
    tie = (np.abs(score - thr) <= 10 * u * thr) & ~low
    tie |= np.abs(logit - lthr) <= sp(lthr)
    tie |= (np.abs(mls - sthr) <= sp(sthr)) & sel & ~low
    return kind, tie


def _quat_to_rot(q):
    """Rotation matrix of the unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def compact(rows: dict, keep) -> dict:
    """The rows whose keep bit is set, in order."""
    keep = np.asarray(keep, bool)
    return {k: np.asarray(v)[keep] for k, v in rows.items()}
