"""Seeded synthetic scenes, cameras and targets for the 3DGS render hot path.

This module draws inputs only: Gaussian parameter arrays in the storage
convention of the library (log-scales, unnormalised quaternions, opacity
logits, degree-3 SH), pinhole cameras and target images.  It holds none of the
method's arithmetic (no projection, shading, compositing, gating or scoring),
so both the CUDA path and the FP64 oracle may consume what it produces.

Workload recipes (the paper's datasets are aerial city captures; these scenes
stand in for them):

* ``plain_scene``  -- 10k Gaussians in front of one 256x256 camera (means in
  [-1,1]^2 x [2,6], log-uniform scales 1e-3..5e-2, random unit quaternions,
  opacity sigmoid(N(0,1)), SH coefficients N(0,0.2) with +0.5 on the DC terms).
* ``city_scene``   -- ground plane (60 %) plus the faces of 200 axis-aligned
  buildings (40 %, 10-80 m tall) over 2 km x 2 km; scales log-normal with
  median 0.3 m and sigma 1; LOD labels from the mean scale.
* ``aerial_camera`` -- 45 degree pitch, altitude 150-400 m, random yaw, aimed
  at a ground point inside the area.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SH_COEFFS = 16  # degree 3


@dataclasses.dataclass
class GaussianSet:
    """Gaussian parameters, float32, C-contiguous, one row per Gaussian:

    mean (N, 3), log_scale (N, 3), quat (N, 4) as (w, x, y, z),
    opacity_logit (N,), sh (N, 16, 3) coefficient then channel, lod (N,) uint8.
    """

    mean: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    lod: np.ndarray

    @property
    def n(self) -> int:
        return int(self.opacity_logit.shape[0])

    def arrays(self):
        return dict(mean=self.mean, log_scale=self.log_scale, quat=self.quat,
                    opacity_logit=self.opacity_logit, sh=self.sh, lod=self.lod)

    def subset(self, idx) -> "GaussianSet":
        idx = np.asarray(idx)
        return GaussianSet(**{k: np.ascontiguousarray(v[idx]) for k, v in self.arrays().items()})

    def copy(self) -> "GaussianSet":
        return GaussianSet(**{k: v.copy() for k, v in self.arrays().items()})


@dataclasses.dataclass
class Camera:
    """Pinhole camera.  x_cam = R @ x_world + t; the camera looks along +z,
    image x to the right, image y down.  Pixel (px, py) has its centre at
    (px + 0.5, py + 0.5) in image coordinates; the principal point is (cx, cy).
    ``campos`` is the camera centre in world coordinates (-R^T t)."""

    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    campos: np.ndarray

    @property
    def pixels(self) -> int:
        return self.width * self.height


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _random_quats(rng, n):
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return _f32(q.T)


def _sh(rng, n, dc=0.5, sigma=0.2):
    sh = rng.normal(0.0, sigma, size=(SH_COEFFS, 3, n))
    sh[0] += dc
    return _f32(sh.transpose(2, 0, 1))


def _logit(p):
    return np.log(p) - np.log1p(-p)


def plain_scene(n: int = 10_000, seed: int = 1) -> GaussianSet:
    """10k-Gaussian scene in front of ``plain_camera`` (uniform means, log-uniform scales)."""
    rng = np.random.default_rng(seed)
    mean = np.empty((3, n))
    mean[0] = rng.uniform(-1.0, 1.0, n)
    mean[1] = rng.uniform(-1.0, 1.0, n)
    mean[2] = rng.uniform(2.0, 6.0, n)
    log_scale = rng.uniform(math.log(1e-3), math.log(5e-2), size=(3, n))
    quat = _random_quats(rng, n)
    opacity_logit = rng.standard_normal(n)  # opacity = sigmoid(N(0,1))
    sh = _sh(rng, n)
    lod = np.zeros(n, np.uint8)
    return GaussianSet(_f32(mean.T), _f32(log_scale.T), quat, _f32(opacity_logit), sh, lod)


def plain_camera(width: int = 256, height: int = 256, f: float = 300.0) -> Camera:
    return Camera(R=_f32(np.eye(3)), t=_f32(np.zeros(3)), fx=f, fy=f,
                  cx=width / 2.0, cy=height / 2.0, width=width, height=height,
                  campos=_f32(np.zeros(3)))


def noise_target(width: int, height: int, seed: int = 2, channels: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _f32(rng.uniform(0.0, 1.0, size=(channels, height, width)))


def look_at_camera(pos, target, up, width, height, hfov_deg) -> Camera:
    """Camera at ``pos`` looking at ``target``; image y points along -up."""
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])  # rows: camera axes in world coordinates
    t = -R @ pos
    f = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    R32 = _f32(R)
    t32 = _f32(t)
    campos = _f32(-(R32.astype(np.float64).T @ t32.astype(np.float64)))
    return Camera(R=R32, t=t32, fx=float(np.float32(f)), fy=float(np.float32(f)),
                  cx=width / 2.0, cy=height / 2.0, width=width, height=height, campos=campos)


def city_scene(n: int, seed: int = 3, extent: float = 2000.0, n_boxes: int = 200,
               ground_frac: float = 0.6, n_levels: int = 6) -> GaussianSet:
    """City-shaped scene: ground plane plus building faces over extent x extent metres."""
    rng = np.random.default_rng(seed)
    half = extent / 2.0
    n_ground = int(round(n * ground_frac))
    n_box = n - n_ground
    mean = np.empty((3, n))
    mean[0, :n_ground] = rng.uniform(-half, half, n_ground)
    mean[1, :n_ground] = rng.uniform(-half, half, n_ground)
    mean[2, :n_ground] = rng.normal(0.0, 0.5, n_ground)

    # boxes: centre, footprint (sx, sy), height h; faces = 4 walls + roof, area-weighted
    bc = rng.uniform(-half * 0.9, half * 0.9, size=(n_boxes, 2))
    bs = rng.uniform(20.0, 120.0, size=(n_boxes, 2))
    bh = rng.uniform(10.0, 80.0, size=n_boxes)
    # face areas: 0:-x wall, 1:+x wall, 2:-y wall, 3:+y wall, 4:roof
    areas = np.stack([bs[:, 1] * bh, bs[:, 1] * bh, bs[:, 0] * bh, bs[:, 0] * bh,
                      bs[:, 0] * bs[:, 1]], axis=1)
    p = (areas / areas.sum()).ravel()
    pick = rng.choice(p.size, size=n_box, p=p)
    b, face = pick // 5, pick % 5
    u = rng.uniform(-0.5, 0.5, n_box)   # position along the face
    u2 = rng.uniform(-0.5, 0.5, n_box)  # second roof coordinate
    w = rng.uniform(0.0, 1.0, n_box)    # height fraction on walls
    # faces 0/1 are the -x/+x walls (y varies), 2/3 the -y/+y walls (x varies), 4 the roof
    fx = np.where(face == 0, -0.5, np.where(face == 1, 0.5, u))
    fy = np.where(face == 2, -0.5, np.where(face == 3, 0.5, np.where(face == 4, u2, u)))
    x = bc[b, 0] + fx * bs[b, 0]
    y = bc[b, 1] + fy * bs[b, 1]
    z = np.where(face == 4, bh[b], w * bh[b])
    mean[0, n_ground:] = x
    mean[1, n_ground:] = y
    mean[2, n_ground:] = z

    log_scale = math.log(0.3) + rng.standard_normal((3, n))
    quat = _random_quats(rng, n)
    opacity_logit = rng.standard_normal(n)
    sh = _sh(rng, n)
    mean_scale = np.exp(log_scale).mean(axis=0)
    lod = np.clip(np.round(np.log2(2.4 / mean_scale)), 0, n_levels - 1).astype(np.uint8)
    return GaussianSet(_f32(mean.T), _f32(log_scale.T), quat, _f32(opacity_logit), sh, lod)


def aerial_camera(seed: int, width: int = 1920, height: int = 1080, hfov_deg: float = 60.0,
                  extent: float = 2000.0, alt_range=(150.0, 400.0), pitch_deg: float = 45.0) -> Camera:
    rng = np.random.default_rng(seed)
    half = extent / 2.0
    alt = rng.uniform(*alt_range)
    yaw = rng.uniform(0.0, 2.0 * math.pi)
    target = np.array([rng.uniform(-0.8 * half, 0.8 * half), rng.uniform(-0.8 * half, 0.8 * half), 0.0])
    horiz = alt / math.tan(math.radians(pitch_deg))
    pos = target - horiz * np.array([math.cos(yaw), math.sin(yaw), 0.0]) + np.array([0.0, 0.0, alt])
    return look_at_camera(pos, target, up=(0.0, 0.0, 1.0), width=width, height=height, hfov_deg=hfov_deg)


def perturbed_copy(g: GaussianSet, seed: int, mean_sigma: float = 0.1, dc_sigma: float = 0.05) -> GaussianSet:
    """Target scene for the training loop: means + N(0, mean_sigma), SH DC + N(0, dc_sigma)."""
    rng = np.random.default_rng(seed)
    out = g.copy()
    out.mean = _f32(out.mean + rng.normal(0.0, mean_sigma, size=out.mean.shape))
    out.sh = out.sh.copy()
    out.sh[:, 0] = (out.sh[:, 0] + rng.normal(0.0, dc_sigma, size=out.sh[:, 0].shape)).astype(np.float32)
    return out


def random_cull_bits(n: int, frac: float, seed: int) -> np.ndarray:
    """Bit-packed cull column (bit i of word i//32 set = Gaussian i culled)."""
    rng = np.random.default_rng(seed)
    bits = rng.uniform(size=n) < frac
    return pack_bits(bits)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    bits = np.asarray(bits, bool)
    n = bits.size
    words = (n + 31) // 32
    padded = np.zeros(words * 32, bool)
    padded[:n] = bits
    w = padded.reshape(words, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)
    return np.ascontiguousarray(w.sum(axis=1).astype(np.uint32))


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, np.uint32)
    bits = (words[:, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.ravel()[:n].astype(bool)


def mixed_cameras(n_cams: int, seed: int, sizes=((640, 480), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)),
                  dist_range=(50.0, 2000.0), extent: float = 2000.0):
    """Cameras of mixed resolution at log-uniform distances from their ground target."""
    rng = np.random.default_rng(seed)
    cams = []
    half = extent / 2.0
    for i in range(n_cams):
        w, h = sizes[rng.integers(len(sizes))]
        d = math.exp(rng.uniform(math.log(dist_range[0]), math.log(dist_range[1])))
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        pitch = math.radians(rng.uniform(30.0, 60.0))
        target = np.array([rng.uniform(-0.8 * half, 0.8 * half), rng.uniform(-0.8 * half, 0.8 * half), 0.0])
        pos = target + d * np.array([-math.cos(yaw) * math.cos(pitch), -math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
        cams.append(look_at_camera(pos, target, (0.0, 0.0, 1.0), w, h, 60.0))
    return cams
