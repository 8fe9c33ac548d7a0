"""ctypes binding of libgsblitz.so (include/gsblitz.h), argument marshalling only.

Every compute step runs in the CUDA library; this module converts torch CUDA
tensors and Python objects into the C structs and passes device pointers and
the current CUDA stream.  If the library is missing the import of its symbols
fails loudly: there is no fallback implementation.
"""
from __future__ import annotations

import contextlib
import ctypes
import dataclasses
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsblitz.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_OOM, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_DEVICE = 0, -1, -2, -3, -4, -5, -6
GS_MAX_CAMERAS = 64
GS_TILE = 16
GS_CAP_FORWARD_ONLY = 1
GS_CAP_MODEL_OPS = 2
(GS_BUF_REC_GAUSSIAN, GS_BUF_REC_CAMERA, GS_BUF_REC_RECT, GS_BUF_REC_TILES, GS_BUF_REC_DEPTH, GS_BUF_REC_XY_CONIC,
 GS_BUF_REC_C_OPAC_RG, GS_BUF_REC_B_LO, GS_BUF_SORTED_VALUES, GS_BUF_TILE_RANGES, GS_BUF_N_CONTRIB) = range(11)

EXPORTS = ("gs_default_params", "gs_last_error", "gs_workspace_create", "gs_workspace_destroy", "gs_workspace_bytes",
           "gs_preprocess", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_importance", "gs_photometric_loss",
           "gs_adam_step", "gs_sync_status", "gs_workspace_counts", "gs_clear_error", "gs_workspace_buffer",
           "gs_kernel_launches", "gs_render_bwd_adam", "gs_render_bwd_compact", "gs_adam_step_compact",
           "gs_visible_set_static", "gs_upload_cameras", "gs_preprocess_uploaded", "gs_workspace_set_sort_chunk",
           "gs_prune_sample", "gs_prune_mass", "gs_compact", "gs_densify", "gs_count_views", "gs_adam_lazy_enable",
           "gs_adam_lazy_disable", "gs_adam_flush", "gs_kernel_timing", "gs_kernel_time",
           "gs_render_fwd_importance", "gs_graph_capture_begin", "gs_graph_capture_end", "gs_graph_launch",
           "gs_graph_destroy", "gs_alu_peaks", "gs_workspace_set_spin_limit")

# Cull modes of RenderParams.cull_enable (include/gsblitz.h)
GS_CULL_OFF, GS_CULL_DROP, GS_CULL_MARK = 0, 1, 2

# kernels gs_kernel_timing brackets with events (include/gsblitz.h)
(GS_KT_RENDER_FWD, GS_KT_RENDER_BWD, GS_KT_IMPORTANCE, GS_KT_GATE, GS_KT_PROJECT, GS_KT_BIN_COUNT, GS_KT_BIN_SORT,
 GS_KT_REDUCE_SLOTS, GS_KT_PREPROCESS_BWD, GS_KT_SSIM_FWD, GS_KT_SSIM_BWD, GS_KT_ADAM_GRAD) = range(12)
GS_KT_COUNT = 12
GS_KT_ALL = (1 << GS_KT_COUNT) - 1


class GSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gsblitz error {code}: {msg}")
        self.code = code


class GSCapacity(ctypes.Structure):
    _fields_ = [("max_gaussians", ctypes.c_int64), ("max_records", ctypes.c_int64),
                ("max_instances", ctypes.c_int64), ("max_tiles", ctypes.c_int64), ("max_pixels", ctypes.c_int64),
                ("max_cameras", ctypes.c_int32), ("flags", ctypes.c_int32)]


class GSGaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("quat", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("lod", ctypes.c_void_p)]


class GSGaussianGrads(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("log_scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class GSModel(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("quat", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("lod", ctypes.c_void_p), ("m", GSGaussianGrads), ("v", GSGaussianGrads)]


class GSDensifyParams(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("dense_scale", ctypes.c_float), ("min_opacity", ctypes.c_float),
                ("split_shrink", ctypes.c_float), ("eps", ctypes.c_float), ("n_levels", ctypes.c_int32)]


class GSCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("campos", ctypes.c_float * 3), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class GSRenderParams(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("lod_enable", ctypes.c_int32), ("lod_Lmax", ctypes.c_int32),
                ("cull_enable", ctypes.c_int32), ("bg", ctypes.c_float * 3), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("T_min", ctypes.c_float), ("dilation", ctypes.c_float),
                ("znear", ctypes.c_float), ("fov_clamp", ctypes.c_float), ("lod_d0", ctypes.c_float),
                ("lod_f", ctypes.c_float), ("eps_score", ctypes.c_float), ("vis_mass", ctypes.c_float)]


class GSCounts(ctypes.Structure):
    _fields_ = [("n_records", ctypes.c_int64), ("n_instances", ctypes.c_int64), ("n_visible", ctypes.c_int64),
                ("records_needed", ctypes.c_int64), ("instances_needed", ctypes.c_int64),
                ("error", ctypes.c_int32), ("error_site", ctypes.c_int32), ("fragments", ctypes.c_int64),
                ("composited", ctypes.c_int64), ("n_candidates", ctypes.c_int64)]


class GSAluPeak(ctypes.Structure):
    _fields_ = [("fp32_fma_flops", ctypes.c_double), ("fp32x2_fma_flops", ctypes.c_double),
                ("ex2_per_s", ctypes.c_double), ("sms", ctypes.c_int32)]


class GSAdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("n", ctypes.c_int64), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libgsblitz.so from the package directory (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2605_13794_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.gs_default_params.argtypes = [vp]
        L.gs_default_params.restype = None
        L.gs_last_error.restype = ctypes.c_char_p
        L.gs_workspace_create.argtypes = [vp, vp]
        L.gs_workspace_destroy.argtypes = [vp]
        L.gs_workspace_bytes.argtypes = [vp]
        L.gs_workspace_bytes.restype = i64
        L.gs_kernel_launches.argtypes = []
        L.gs_kernel_launches.restype = i64
        L.gs_preprocess.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.gs_upload_cameras.argtypes = [vp, vp, i32, vp, vp]
        L.gs_workspace_set_sort_chunk.argtypes = [vp, i32]
        L.gs_prune_sample.argtypes = [vp, vp, vp, i64, i64, vp, vp]
        L.gs_prune_mass.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp]
        L.gs_compact.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.gs_densify.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp]
        L.gs_count_views.argtypes = [vp, vp, vp]
        L.gs_adam_lazy_enable.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32]
        L.gs_adam_lazy_disable.argtypes = [vp]
        L.gs_adam_flush.argtypes = [vp, vp, vp]
        L.gs_preprocess_uploaded.argtypes = [vp, vp, vp, vp, vp]
        L.gs_bin_sort.argtypes = [vp, vp]
        L.gs_render_fwd.argtypes = [vp, vp, vp, vp]
        L.gs_render_fwd_importance.argtypes = [vp, vp, vp, vp]
        L.gs_render_bwd.argtypes = [vp, vp, vp, vp, i32, vp, ctypes.c_float, vp, vp]
        f32 = ctypes.c_float
        L.gs_render_bwd_adam.argtypes = [vp, vp, vp, vp, vp, vp, f32, f32, f32, i32, vp, f32, vp, vp]
        L.gs_render_bwd_compact.argtypes = [vp, vp, vp, vp, f32, vp, vp]
        L.gs_adam_step_compact.argtypes = [vp, vp, vp, vp, vp, f32, f32, f32, i32, vp]
        L.gs_visible_set_static.argtypes = [vp, i64, f32, vp, vp, vp, vp]
        L.gs_alu_peaks.argtypes = [vp, vp]
        L.gs_workspace_set_spin_limit.argtypes = [vp, ctypes.c_uint64]
        L.gs_importance.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.gs_photometric_loss.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.c_float, vp, vp, vp]
        L.gs_adam_step.argtypes = [vp, i32, i32, vp]
        L.gs_sync_status.argtypes = [vp, vp]
        L.gs_workspace_counts.argtypes = [vp, vp, vp]
        L.gs_clear_error.argtypes = [vp, vp]
        L.gs_workspace_buffer.argtypes = [vp, i32, vp, vp]
        L.gs_kernel_timing.argtypes = [vp, i32]
        L.gs_kernel_time.argtypes = [vp, i32, vp, vp]
        L.gs_graph_capture_begin.argtypes = [vp]
        L.gs_graph_capture_end.argtypes = [vp, vp]
        L.gs_graph_launch.argtypes = [vp, vp]
        L.gs_graph_destroy.argtypes = [vp]
        for name in EXPORTS:
            if name not in ("gs_default_params", "gs_last_error", "gs_workspace_bytes", "gs_kernel_launches"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != GS_OK:
        raise GSError(rc, lib().gs_last_error().decode(errors="replace"))


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclasses.dataclass
class RenderParams:
    """Mirror of gs_render_params; defaults come from gs_default_params."""

    bg: tuple = (0.0, 0.0, 0.0)
    tile_w: int = GS_TILE
    tile_h: int = GS_TILE
    alpha_min: float | None = None
    alpha_max: float | None = None
    T_min: float | None = None
    dilation: float | None = None
    znear: float | None = None
    fov_clamp: float | None = None
    lod_enable: bool = False
    lod_d0: float | None = None
    lod_f: float | None = None
    lod_Lmax: int | None = None
    cull_enable: int = 0  # GS_CULL_OFF / GS_CULL_DROP (or True) / GS_CULL_MARK
    eps_score: float | None = None
    vis_mass: float | None = None

    def c(self) -> GSRenderParams:
        p = GSRenderParams()
        lib().gs_default_params(ctypes.byref(p))
        p.bg = (ctypes.c_float * 3)(*self.bg)
        p.tile_w, p.tile_h = int(self.tile_w), int(self.tile_h)
        p.lod_enable = int(self.lod_enable)
        p.cull_enable = int(self.cull_enable)
        for name in ("alpha_min", "alpha_max", "T_min", "dilation", "znear", "fov_clamp", "lod_d0", "lod_f",
                     "lod_Lmax", "eps_score", "vis_mass"):
            v = getattr(self, name)
            if v is not None:
                setattr(p, name, v)
        return p


@dataclasses.dataclass
class GaussianTensors:
    """Gaussian parameters as CUDA tensors in the library's row layout."""

    mean: torch.Tensor          # (N, 3) float32
    log_scale: torch.Tensor     # (N, 3)
    quat: torch.Tensor          # (N, 4) w, x, y, z
    opacity_logit: torch.Tensor # (N,)
    sh: torch.Tensor            # (N, 16, 3)
    lod: torch.Tensor | None    # (N,) uint8

    @property
    def n(self) -> int:
        return int(self.opacity_logit.shape[0])

    @staticmethod
    def from_host(g, device="cuda") -> "GaussianTensors":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return GaussianTensors(t(g.mean), t(g.log_scale), t(g.quat), t(g.opacity_logit), t(g.sh),
                               t(g.lod) if g.lod is not None else None)

    def zeros_like(self) -> "GaussianTensors":
        z = torch.zeros_like
        return GaussianTensors(z(self.mean), z(self.log_scale), z(self.quat), z(self.opacity_logit), z(self.sh), None)

    def params(self):
        return [self.mean, self.log_scale, self.quat, self.opacity_logit, self.sh]

    def c(self) -> GSGaussians:
        return GSGaussians(self.n, _ptr(self.mean), _ptr(self.log_scale), _ptr(self.quat), _ptr(self.opacity_logit),
                           _ptr(self.sh), _ptr(self.lod))

    def c_grads(self) -> GSGaussianGrads:
        return GSGaussianGrads(_ptr(self.mean), _ptr(self.log_scale), _ptr(self.quat), _ptr(self.opacity_logit),
                               _ptr(self.sh))


@dataclasses.dataclass
class ModelTensors:
    """A whole model on the device: parameters, Adam moments and LOD labels."""

    g: GaussianTensors
    m: GaussianTensors | None
    v: GaussianTensors | None

    @property
    def n(self) -> int:
        return self.g.n

    @staticmethod
    def empty(n: int, with_moments: bool = True, device="cuda") -> "ModelTensors":
        e = lambda *shape: torch.empty(*shape, device=device)
        mk = lambda: GaussianTensors(e(n, 3), e(n, 3), e(n, 4), e(n), e(n, 16, 3), None)
        g = mk()
        g.lod = torch.empty(n, dtype=torch.uint8, device=device)
        return ModelTensors(g, mk() if with_moments else None, mk() if with_moments else None)

    def head(self, k: int) -> "ModelTensors":
        """The first k rows (views, no copy)."""
        cut = lambda t: None if t is None else GaussianTensors(t.mean[:k], t.log_scale[:k], t.quat[:k],
                                                              t.opacity_logit[:k], t.sh[:k],
                                                              None if t.lod is None else t.lod[:k])
        return ModelTensors(cut(self.g), cut(self.m), cut(self.v))

    def c(self) -> GSModel:
        g = self.g
        none = GSGaussianGrads(None, None, None, None, None)
        return GSModel(g.n, _ptr(g.mean), _ptr(g.log_scale), _ptr(g.quat), _ptr(g.opacity_logit), _ptr(g.sh),
                       _ptr(g.lod), self.m.c_grads() if self.m is not None else none,
                       self.v.c_grads() if self.v is not None else none)


def camera_c(cam) -> GSCamera:
    c = GSCamera()
    c.R = (ctypes.c_float * 9)(*np.asarray(cam.R, np.float32).ravel())
    c.t = (ctypes.c_float * 3)(*np.asarray(cam.t, np.float32))
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.campos = (ctypes.c_float * 3)(*np.asarray(cam.campos, np.float32))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def tiles_of(cam, tile_w: int = GS_TILE, tile_h: int = GS_TILE) -> int:
    return ((cam.width + tile_w - 1) // tile_w) * ((cam.height + tile_h - 1) // tile_h)


class Workspace:
    """Owns a gs_workspace (all scratch of the render path) on the current device."""

    def __init__(self, max_gaussians: int, max_records: int, max_instances: int, max_tiles: int,
                 max_pixels: int, max_cameras: int = 1, forward_only: bool = False, model_ops: bool = False):
        self.cap = GSCapacity(max_gaussians, max_records, max_instances, max_tiles, max_pixels, max_cameras,
                              (GS_CAP_FORWARD_ONLY if forward_only else 0) | (GS_CAP_MODEL_OPS if model_ops else 0))
        self._ws = ctypes.c_void_p()
        _check(lib().gs_workspace_create(ctypes.byref(self.cap), ctypes.byref(self._ws)))
        self.cams = []
        # forwards started on this workspace; a differentiable render remembers
        # the one its backward belongs to
        self.generation = 0

    @staticmethod
    def bytes_for(**cap) -> int:
        c = GSCapacity(cap["max_gaussians"], cap["max_records"], cap["max_instances"], cap["max_tiles"],
                       cap["max_pixels"], cap.get("max_cameras", 1), GS_CAP_FORWARD_ONLY if cap.get("forward_only") else 0)
        return int(lib().gs_workspace_bytes(ctypes.byref(c)))

    def close(self):
        if self._ws:
            _check(lib().gs_workspace_destroy(self._ws))
            self._ws = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def preprocess(self, g: GaussianTensors, cams, params: RenderParams, cull=None, stream=None):
        arr = (GSCamera * len(cams))(*[camera_c(c) for c in cams])
        self.cams = list(cams)
        self.tile = (params.tile_w, params.tile_h)
        self._g = g  # keep the parameter tensors alive until the backward
        gc, pc = g.c(), params.c()
        self.generation += 1
        _check(lib().gs_preprocess(self._ws, ctypes.byref(gc), arr, len(cams), _ptr(cull), ctypes.byref(pc),
                                   _stream(stream)))

    def upload_cameras(self, cams, params: RenderParams, stream=None):
        """Copies the cameras to the workspace's device table (not while the
        stream is being captured); kernels read them from there."""
        arr = (GSCamera * len(cams))(*[camera_c(c) for c in cams])
        self.cams = list(cams)
        self.tile = (params.tile_w, params.tile_h)
        pc = params.c()
        _check(lib().gs_upload_cameras(self._ws, arr, len(cams), ctypes.byref(pc), _stream(stream)))

    def preprocess_uploaded(self, g: GaussianTensors, params: RenderParams, cull=None, stream=None):
        """gs_preprocess with the cameras of the last upload (graph-capturable)."""
        self._g = g
        gc, pc = g.c(), params.c()
        self.generation += 1
        _check(lib().gs_preprocess_uploaded(self._ws, ctypes.byref(gc), _ptr(cull), ctypes.byref(pc),
                                            _stream(stream)))

    def set_sort_chunk(self, keys_per_block: int):
        """Keys per block of the radix passes (1024, 2048, 4096, or 0 to pick by
        size); results are unchanged."""
        _check(lib().gs_workspace_set_sort_chunk(self._ws, int(keys_per_block)))
        self.sort_chunk = int(keys_per_block)

    def set_spin_limit(self, spins: int):
        """Bound on the look-back waits of importance()'s selection sorts (0:
        the default); see gs_workspace_set_spin_limit."""
        _check(lib().gs_workspace_set_spin_limit(self._ws, int(spins)))

    def bin_sort(self, stream=None):
        _check(lib().gs_bin_sort(self._ws, _stream(stream)))

    @property
    def total_pixels(self) -> int:
        return sum(c.width * c.height for c in self.cams)

    def render_fwd(self, rgb_out, T_out=None, stream=None):
        _check(lib().gs_render_fwd(self._ws, _ptr(rgb_out), _ptr(T_out), _stream(stream)))

    def render_fwd_importance(self, rgb_out, T_out=None, stream=None):
        """render_fwd and the importance raster in one pass; the next importance() only selects."""
        _check(lib().gs_render_fwd_importance(self._ws, _ptr(rgb_out), _ptr(T_out), _stream(stream)))

    def render_bwd(self, g: GaussianTensors, dL_drgb, grads: GaussianTensors, accumulate=False, absgrad=None,
                   scale_reg_beta=0.0, scale_reg_value=None, stream=None):
        gc, gr = g.c(), grads.c_grads()
        _check(lib().gs_render_bwd(self._ws, ctypes.byref(gc), _ptr(dL_drgb), ctypes.byref(gr), int(accumulate),
                                   _ptr(absgrad), float(scale_reg_beta), _ptr(scale_reg_value), _stream(stream)))

    def render_bwd_adam(self, g: GaussianTensors, dL_drgb, m: GaussianTensors, v: GaussianTensors, lr, step,
                        beta1=0.9, beta2=0.999, eps=1e-15, absgrad=None, scale_reg_beta=0.0, scale_reg_value=None,
                        stream=None):
        """Backward fused with an Adam step: g's arrays are updated in place.
        lr: five learning rates (mean, log-scale, quat, opacity, SH)."""
        gc, mc, vc = g.c(), m.c_grads(), v.c_grads()
        lrs = (ctypes.c_float * 5)(*lr)
        _check(lib().gs_render_bwd_adam(self._ws, ctypes.byref(gc), _ptr(dL_drgb), ctypes.byref(mc), ctypes.byref(vc),
                                        lrs, float(beta1), float(beta2), float(eps), int(step), _ptr(absgrad),
                                        float(scale_reg_beta), _ptr(scale_reg_value), _stream(stream)))

    def render_bwd_compact(self, g: GaussianTensors, dL_drgb, absgrad=None, scale_reg_beta=0.0, scale_reg_value=None,
                           stream=None):
        gc = g.c()
        _check(lib().gs_render_bwd_compact(self._ws, ctypes.byref(gc), _ptr(dL_drgb), _ptr(absgrad),
                                           float(scale_reg_beta), _ptr(scale_reg_value), _stream(stream)))

    def adam_step_compact(self, g: GaussianTensors, m: GaussianTensors, v: GaussianTensors, lr, step, beta1=0.9,
                          beta2=0.999, eps=1e-15, stream=None):
        gc, mc, vc = g.c(), m.c_grads(), v.c_grads()
        lrs = (ctypes.c_float * 5)(*lr)
        _check(lib().gs_adam_step_compact(self._ws, ctypes.byref(gc), ctypes.byref(mc), ctypes.byref(vc), lrs,
                                          float(beta1), float(beta2), float(eps), int(step), _stream(stream)))

    def importance(self, w=None, a=None, s_accum=None, crad=None, cvis=None, cull_out=None, stream=None):
        _check(lib().gs_importance(self._ws, _ptr(w), _ptr(a), _ptr(s_accum), _ptr(crad), _ptr(cvis), _ptr(cull_out),
                                   _stream(stream)))

    def photometric_loss(self, image, target, lam, loss_out, dL_dimage, stream=None):
        B, C, H, W = image.shape
        assert C == 3
        _check(lib().gs_photometric_loss(self._ws, _ptr(image), _ptr(target), B, H, W, float(lam), _ptr(loss_out),
                                         _ptr(dL_dimage), _stream(stream)))

    # ---- model level ----------------------------------------------------------------
    def prune_sample(self, s, expo, k: int, keep_bits, stream=None):
        """Pass 1: keep k Gaussians, importance-weighted sampling without
        replacement (exponential clocks expo / s; expo ~ Exp(1))."""
        _check(lib().gs_prune_sample(self._ws, _ptr(s), _ptr(expo), s.numel(), int(k), _ptr(keep_bits),
                                     _stream(stream)))

    def prune_mass(self, s, keep_bits, mass: float = 0.99, stream=None):
        """Pass 2: keep the smallest prefix by descending s carrying `mass` of it."""
        _check(lib().gs_prune_mass(self._ws, _ptr(s), s.numel(), float(mass), _ptr(keep_bits), _stream(stream)))

    def compact(self, src: "ModelTensors", keep_bits, dst: "ModelTensors", n_out, stream=None):
        sc, dc = src.c(), dst.c()
        _check(lib().gs_compact(self._ws, ctypes.byref(sc), _ptr(keep_bits), ctypes.byref(dc), dst.n, _ptr(n_out),
                                _stream(stream)))

    def densify(self, src: "ModelTensors", absgrad, denom, cvis, crad, noise, dst: "ModelTensors", n_out,
                grad_threshold=0.0002, dense_scale=0.01, min_opacity=0.005, split_shrink=1.6, eps=1e-6,
                n_levels=6, stream=None):
        sc, dc = src.c(), dst.c()
        p = GSDensifyParams(grad_threshold, dense_scale, min_opacity, split_shrink, eps, n_levels)
        _check(lib().gs_densify(self._ws, ctypes.byref(sc), _ptr(absgrad), _ptr(denom), _ptr(cvis), _ptr(crad),
                                _ptr(noise), ctypes.byref(p), ctypes.byref(dc), dst.n, _ptr(n_out),
                                _stream(stream)))

    def adam_lazy_enable(self, m: GaussianTensors, v: GaussianTensors, last_step, drift, beta1=0.9, beta2=0.999,
                         eps=1e-15, max_steps=1 << 20):
        """Deferred zero-gradient Adam steps (see gs_adam_lazy_enable).  last_step: (n,)
        int32; drift: (2, n) float32, zeroed (mean and log-scale drift bounds)."""
        assert drift.numel() == 2 * last_step.numel(), "drift must hold 2 * n floats"
        self._lazy = (m, v, last_step, drift)  # keep them alive
        mc, vc = m.c_grads(), v.c_grads()
        _check(lib().gs_adam_lazy_enable(self._ws, ctypes.byref(mc), ctypes.byref(vc), _ptr(last_step), _ptr(drift),
                                         float(beta1), float(beta2), float(eps), int(max_steps)))

    def adam_lazy_disable(self):
        _check(lib().gs_adam_lazy_disable(self._ws))

    def adam_flush(self, g: GaussianTensors, stream=None):
        gc = g.c()
        _check(lib().gs_adam_flush(self._ws, ctypes.byref(gc), _stream(stream)))

    def count_views(self, counts, stream=None):
        _check(lib().gs_count_views(self._ws, _ptr(counts), _stream(stream)))

    def counts(self, stream=None) -> dict:
        c = GSCounts()
        _check(lib().gs_workspace_counts(self._ws, ctypes.byref(c), _stream(stream)))
        return {f[0]: getattr(c, f[0]) for f in GSCounts._fields_}

    def sync_status(self, stream=None):
        _check(lib().gs_sync_status(self._ws, _stream(stream)))

    def kernel_timing(self, enable: bool = True, kernels=None):
        """Turns event timing of the rasterisers' launches on (discarding older
        records) or off; kernels: the GS_KT_* ids to time (default: all)."""
        mask = 0
        if enable:
            mask = GS_KT_ALL if kernels is None else sum(1 << int(k) for k in set(kernels))
        _check(lib().gs_kernel_timing(self._ws, mask))

    def kernel_time(self, kernel: int):
        """(summed device ms, timed launches) of one kernel since timing was turned on."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().gs_kernel_time(self._ws, int(kernel), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def clear_error(self, stream=None):
        _check(lib().gs_clear_error(self._ws, _stream(stream)))

    def buffer(self, which: int):
        p, n = ctypes.c_void_p(), ctypes.c_int64()
        _check(lib().gs_workspace_buffer(self._ws, which, ctypes.byref(p), ctypes.byref(n)))
        return p.value, n.value

    def read_buffer(self, which: int, dtype, count: int, width: int = 1) -> np.ndarray:
        """Copies `count` entries (each `width` items of `dtype`) of an internal
        buffer to the host, after synchronising the device (debug/tests)."""
        ptr, cap = self.buffer(which)
        assert count <= cap
        out = np.empty((count, width) if width > 1 else count, dtype=dtype)
        if count:
            torch.cuda.synchronize()
            _memcpy_d2h(out.ctypes.data, ptr, out.nbytes)
        return out


_cudart = None


def _memcpy_d2h(dst: int, src: int, nbytes: int):
    """Device-to-host copy through the CUDA runtime libgsblitz.so is linked with."""
    global _cudart
    if _cudart is None:
        _cudart = ctypes.CDLL("libcudart.so.13")
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    rc = _cudart.cudaMemcpy(ctypes.c_void_p(dst), ctypes.c_void_p(src), nbytes, 2)  # cudaMemcpyDeviceToHost
    if rc != 0:
        raise RuntimeError(f"cudaMemcpy failed with {rc}")


def visible_set_static(w, vis_mass, cull_out, cvis_accum=None, error_out=None, stream=None):
    """Cull column of one view from its per-Gaussian w without any allocation
    (fixed library scratch, n <= 2^20; see gs_visible_set_static).  error_out:
    an int32 device tensor of one element receiving the device error code."""
    _check(lib().gs_visible_set_static(_ptr(w), int(w.numel()), float(vis_mass), _ptr(cull_out), _ptr(cvis_accum),
                                       _ptr(error_out), _stream(stream)))


class Graph:
    """A CUDA graph of library calls (gs_graph_*): kernels keep the priority of
    the stream they were captured from.

        g = Graph()
        with g.capture(stream):      # a non-default torch stream
            ...calls on stream, and on streams that join it...
        g.launch()
    """

    def __init__(self):
        self._g = ctypes.c_void_p(0)

    @contextlib.contextmanager
    def capture(self, stream):
        assert stream.cuda_stream != 0, "capture needs a non-default stream"
        self.close()
        with torch.cuda.stream(stream):
            _check(lib().gs_graph_capture_begin(_stream(stream)))
            ok = False
            try:
                yield self
                ok = True
            finally:
                g = ctypes.c_void_p(0)
                rc = lib().gs_graph_capture_end(_stream(stream), ctypes.byref(g))
                if ok:
                    _check(rc)
                self._g = g

    def launch(self, stream=None):
        assert self._g.value, "no captured graph"
        _check(lib().gs_graph_launch(self._g, _stream(stream)))

    def close(self):
        if self._g.value:
            _check(lib().gs_graph_destroy(self._g))
            self._g = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alu_peaks(stream=None) -> dict:
    """Measured FP32 FMA (scalar, FP32x2) FLOP/s and ex2 results/s of the
    current device (gs_alu_peaks; synchronises)."""
    out = GSAluPeak()
    _check(lib().gs_alu_peaks(ctypes.byref(out), _stream(stream)))
    return {f[0]: getattr(out, f[0]) for f in GSAluPeak._fields_}


def kernel_launches() -> int:
    """Kernels the library has launched so far in this process."""
    return int(lib().gs_kernel_launches())


def adam_step(groups, step: int, stream=None):
    """groups: list of (param, grad, m, v, lr, beta1, beta2, eps) CUDA tensors/floats."""
    arr = (GSAdamGroup * len(groups))()
    for k, (p, g, m, v, lr, b1, b2, eps) in enumerate(groups):
        arr[k] = GSAdamGroup(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), lr, b1, b2, eps)
    _check(lib().gs_adam_step(arr, len(groups), int(step), _stream(stream)))


class RenderFunction(torch.autograd.Function):
    """Differentiable render through the library: forward = preprocess +
    bin_sort + render_fwd, backward = render_bwd (the hand-written adjoint).

    The backward reads the binning, T_final and n_contrib the forward left in
    the workspace; a later forward on the same workspace replaces them, so the
    backward checks the workspace's forward generation and raises if another
    forward ran in between."""

    @staticmethod
    def forward(ctx, ws, cams, params, cull, lod, mean, log_scale, quat, opacity_logit, sh):
        g = GaussianTensors(mean.detach().contiguous(), log_scale.detach().contiguous(), quat.detach().contiguous(),
                            opacity_logit.detach().contiguous(), sh.detach().contiguous(), lod)
        ws.preprocess(g, cams, params, cull)
        ws.bin_sort()
        P = ws.total_pixels
        rgb = torch.empty(3 * P, device=mean.device, dtype=torch.float32)
        T = torch.empty(P, device=mean.device, dtype=torch.float32)
        ws.render_fwd(rgb, T)
        ctx.ws, ctx.g, ctx.generation = ws, g, ws.generation
        ctx.mark_non_differentiable(T)
        return rgb, T

    @staticmethod
    def backward(ctx, dL_drgb, dL_dT):
        if ctx.ws.generation != ctx.generation:
            raise RuntimeError("render backward: the workspace has run another forward since this render's; "
                               "its binning and per-pixel state are gone (use one workspace per pending backward)")
        g = ctx.g
        grads = g.zeros_like()
        ctx.ws.render_bwd(g, dL_drgb.contiguous(), grads, accumulate=False)
        return (None, None, None, None, None, grads.mean, grads.log_scale, grads.quat, grads.opacity_logit, grads.sh)


def render(ws: Workspace, g: GaussianTensors, cams, params: RenderParams, cull=None):
    """Differentiable render of g (tensors may require grad) into the cameras.
    Returns (rgb [3*sum(H*W)] planar per camera, T_final [sum(H*W)])."""
    return RenderFunction.apply(ws, cams, params, cull, g.lod, g.mean, g.log_scale, g.quat, g.opacity_logit, g.sh)
