"""Seeded synthetic scenes and pinhole cameras for the quadric rasterizer.

This module only draws inputs. It holds none of the renderer's arithmetic, so
that the CUDA path and the FP64 oracle can be fed the same bytes without
sharing any computation.

The shapes follow the workloads the paper evaluates on (object-centric DTU-like
captures, unbounded Mip-NeRF 360-like scenes; Sec. 4 and the supplementary
speed/storage table): primitive counts, image sizes and the parameter set of a
quadric Gaussian (mean, unit quaternion, in-surface scales s_u, s_v,
curvatures a, b, opacity, degree-3 SH colour, Sec. 3.2).

Parameter layout (all host numpy arrays, C-contiguous):
  mean     float32 [N, 3]   world-space centre
  quat     float32 [N, 4]   (w, x, y, z), any norm
  scale    float32 [N, 2]   (s_u, s_v) > 0
  curv     float32 [N, 2]   (a, b): local surface z = a*x^2 + b*y^2
  opacity  float32 [N]      in (0, 1)
  sh       uint16  [N, 48]  bfloat16 bit patterns, index k*3 + c (coefficient k, channel c)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    mean: np.ndarray
    quat: np.ndarray
    scale: np.ndarray
    curv: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(*(np.ascontiguousarray(getattr(self, k)[idx]) for k in
                       ("mean", "quat", "scale", "curv", "opacity", "sh")))

    def copy(self) -> "Scene":
        return Scene(*(getattr(self, k).copy() for k in
                       ("mean", "quat", "scale", "curv", "opacity", "sh")))


@dataclass
class Camera:
    """Pinhole camera. x_cam = R_cw @ x_world + t_cw; pixel (u, v) = (fx*x/z + cx, fy*y/z + cy)."""
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    R_cw: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    t_cw: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))
    near: float = 0.2

    def __post_init__(self):
        self.R_cw = np.ascontiguousarray(self.R_cw, dtype=np.float32).reshape(3, 3)
        self.t_cw = np.ascontiguousarray(self.t_cw, dtype=np.float32).reshape(3)

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """The same rays restricted to a w x h window whose top-left pixel is (x0, y0)."""
        return Camera(w, h, self.fx, self.fy, self.cx - x0, self.cy - y0,
                      self.R_cw.copy(), self.t_cw.copy(), self.near)


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest even) and return the 16-bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def _unit_dirs(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _finish(rng, mean, scale, kappa, n):
    curv = kappa / scale
    opacity = 1.0 / (1.0 + np.exp(-rng.standard_normal(n)))
    sh = f32_to_bf16_bits(rng.normal(0.0, 0.2, (n, 48)).astype(np.float32))
    return Scene(np.ascontiguousarray(mean, np.float32), _unit_quats(rng, n),
                 np.ascontiguousarray(scale, np.float32), np.ascontiguousarray(curv, np.float32),
                 np.clip(opacity, 1e-4, 1 - 1e-4).astype(np.float32), sh)


def look_at(pos, target=(0.0, 0.0, 0.0), up=(0.0, -1.0, 0.0)):
    """World-to-camera rotation and translation for a camera at `pos` looking at `target`.
    Camera axes: +z forward, +x right, +y down in the image (so `up` maps to -y)."""
    pos = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - pos
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    x = np.cross(up, f)
    if np.linalg.norm(x) < 1e-8:
        x = np.cross(np.array([1.0, 0.0, 0.0]), f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ pos
    return R.astype(np.float32), t.astype(np.float32)


# --------------------------------------------------------------------------- workloads

def scene_small(seed: int = 0, n: int = 1000) -> tuple[Scene, Camera]:
    """1,000 quadrics in front of a 128x128 camera (fx = fy = 128) looking down +z.
    Centres: x, y uniform over a unit extent, z uniform in [3, 5]."""
    rng = np.random.default_rng([seed, 0])
    mean = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n),
                     rng.uniform(3.0, 5.0, n)], 1)
    scale = _log_uniform(rng, 0.005, 0.05, (n, 2))
    kappa = rng.uniform(-5.0, 5.0, (n, 2))
    sc = _finish(rng, mean, scale, kappa, n)
    cam = Camera(128, 128, 128.0, 128.0, 64.0, 64.0)
    return sc, cam


def scene_object(seed: int = 0, n: int = 300_000) -> tuple[Scene, Camera]:
    """DTU-shaped object: centres on a noisy unit sphere (radial sigma 0.02), scales
    log-uniform [0.002, 0.02], curvatures uniform [-20, 20]/s; a 1600x1200 camera at
    distance 3 looking at the origin (60 degree horizontal field of view)."""
    rng = np.random.default_rng([seed, 1])
    mean = _unit_dirs(rng, n) * (1.0 + rng.normal(0.0, 0.02, n))[:, None]
    scale = _log_uniform(rng, 0.002, 0.02, (n, 2))
    kappa = rng.uniform(-20.0, 20.0, (n, 2))
    sc = _finish(rng, mean, scale, kappa, n)
    W, H = 1600, 1200
    R, t = look_at((0.0, 0.0, -3.0))
    cam = Camera(W, H, 0.866 * W, 0.866 * W, W / 2, H / 2, R, t)
    return sc, cam


def _unbounded_scene(rng, n):
    n_in = int(round(0.7 * n))
    n_out = n - n_in
    r_in = rng.uniform(0.0, 1.0, n_in) ** (1.0 / 3.0)
    inv_r = rng.uniform(1.0 / 20.0, 1.0, n_out)
    r = np.concatenate([r_in, 1.0 / inv_r])
    mean = _unit_dirs(rng, n) * r[:, None]
    perm = rng.permutation(n)
    mean, r = mean[perm], r[perm]
    scale = _log_uniform(rng, 0.001, 0.1, (n, 2)) * np.maximum(r, 0.05)[:, None]
    planar = rng.uniform(0.0, 1.0, n) < 0.2
    kappa = np.where(planar[:, None], rng.uniform(-1e-6, 1e-6, (n, 2)),
                     rng.uniform(-10.0, 10.0, (n, 2)))
    return _finish(rng, mean, scale, kappa, n)


def scene_unbounded(seed: int = 0, n: int = 3_000_000) -> tuple[Scene, Camera]:
    """Mip-NeRF 360-shaped scene: 70% of centres uniform in the unit ball, 30% in a
    1..20 shell with inverse radius uniform; scales log-uniform [0.001, 0.1] times the
    radius (radius floored at 0.05); 20% near-planar (|kappa| < 1e-6), the rest with
    kappa uniform in [-10, 10]; curvature = kappa / scale. One 1297x840 camera at the
    origin looking down +z (60 degree horizontal field of view)."""
    rng = np.random.default_rng([seed, 2])
    sc = _unbounded_scene(rng, n)
    W, H = 1297, 840
    cam = Camera(W, H, 0.866 * W, 0.866 * W, W / 2, H / 2)
    return sc, cam


SERVE_RESOLUTIONS = ((256, 256), (512, 384), (1024, 768), (1920, 1080))


def serving_scene(seed: int = 0, n: int = 1_000_000) -> Scene:
    """Resident scene for the serving workloads (distribution as scene_unbounded)."""
    rng = np.random.default_rng([seed, 3, n])
    return _unbounded_scene(rng, n)


def orbit_camera(rng, radius: float = 2.0, res=None) -> Camera:
    """Camera uniformly distributed on a sphere of `radius`, looking at the origin."""
    if res is None:
        res = SERVE_RESOLUTIONS[rng.integers(len(SERVE_RESOLUTIONS))]
    W, H = res
    pos = _unit_dirs(rng, 1)[0] * radius
    R, t = look_at(pos)
    return Camera(W, H, 0.866 * W, 0.866 * W, W / 2, H / 2, R, t)


WORKLOADS = {
    "small_1k_128": scene_small,
    "object_300k_1600x1200": scene_object,
    "unbounded_3m_1297x840": scene_unbounded,
}
