"""Seeded synthetic scenes and cameras shaped like the paper's workloads.

This module holds none of the render method's arithmetic: it only draws
parameters from fixed distributions and builds pinhole cameras.  Both the
CUDA path and the FP64 oracle consume its plain FP32 arrays.

Parameter layout (one row per Gaussian, all float32, C-contiguous):
  mean          [N, 4]   (x, y, z, t)
  log_scale     [N, 4]   log of (s_x, s_y, s_z, s_t)
  q_l, q_r      [N, 4]   left / right quaternions (real part first)
  opacity_logit [N]      opacity = sigmoid(logit)
  sh            [N, K, 3] K = (L+1)^2 (n_max+1), index n*(L+1)^2 + l*l + l + m

Distributions (the paper's datasets are not available; these stand in for the
Plenoptic Video scenes at 2x downsampling, 1352x1014, and the Gaussian counts
the paper reports after training, 0.5M-3M):
  mean_xyz ~ U(box), mean_t ~ U[0, 1]
  spatial log-scales ~ U[ln lo, ln hi], temporal log-scale ~ U[ln 0.05, ln 0.3]
  quaternions ~ N(0, I4) normalised; logit ~ N(0, 1); sh ~ N(0, 0.2^2)

Cameras follow the OpenCV convention (x right, y down, z forward), with
fx = fy = (W/2) / tan(hfov/2), cx = W/2, cy = H/2 and a 3x4 row-major
world-to-camera matrix.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SCENE_SEED = 0
TARGET_SEED = 1
POSE_SEED = 2


@dataclass
class Scene:
    mean: np.ndarray
    log_scale: np.ndarray
    q_l: np.ndarray
    q_r: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int
    t_order: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def as_dict(self) -> dict:
        return {"mean": self.mean, "log_scale": self.log_scale, "q_l": self.q_l, "q_r": self.q_r,
                "opacity_logit": self.opacity_logit, "sh": self.sh}

    def subset(self, idx) -> "Scene":
        return Scene(self.mean[idx].copy(), self.log_scale[idx].copy(), self.q_l[idx].copy(),
                     self.q_r[idx].copy(), self.opacity_logit[idx].copy(), self.sh[idx].copy(),
                     self.sh_degree, self.t_order)


def make_scene(n: int, seed: int, box_lo, box_hi, spatial_log_scale=(math.log(0.01), math.log(0.1)),
               temporal_log_scale=(math.log(0.05), math.log(0.3)), sh_degree: int = 3, t_order: int = 2,
               sh_std: float = 0.2) -> Scene:
    rng = np.random.default_rng(seed)
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    mean = np.empty((n, 4), dtype=np.float64)
    mean[:, :3] = lo + (hi - lo) * rng.random((n, 3))
    mean[:, 3] = rng.random(n)
    ls = np.empty((n, 4), dtype=np.float64)
    ls[:, :3] = rng.uniform(spatial_log_scale[0], spatial_log_scale[1], (n, 3))
    ls[:, 3] = rng.uniform(temporal_log_scale[0], temporal_log_scale[1], n)
    ql = rng.standard_normal((n, 4))
    ql /= np.linalg.norm(ql, axis=1, keepdims=True)
    qr = rng.standard_normal((n, 4))
    qr /= np.linalg.norm(qr, axis=1, keepdims=True)
    logit = rng.standard_normal(n)
    K = (sh_degree + 1) ** 2 * (t_order + 1)
    sh = (sh_std * rng.standard_normal((n, K, 3))).astype(np.float32)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f32(mean), f32(ls), f32(ql), f32(qr), f32(logit), sh, sh_degree, t_order)


def look_at(center, target, up, width: int, height: int, t: float, hfov_deg: float = 60.0) -> dict:
    """Pinhole camera at ``center`` looking at ``target``; ``up`` is the world
    direction that appears upward in the image (camera -y)."""
    c = np.asarray(center, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    u = np.asarray(up, dtype=np.float64)
    x = np.cross(f, u)
    if np.linalg.norm(x) < 1e-9:  # looking along up: pick another up
        x = np.cross(f, np.array([1.0, 0.0, 0.0]) if abs(f[0]) < 0.9 else np.array([0.0, 0.0, 1.0]))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    Wr = np.stack([x, y, f])
    T = -Wr @ c
    vm = np.concatenate([Wr, T[:, None]], axis=1).astype(np.float32)
    focal = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return {"width": int(width), "height": int(height), "fx": np.float32(focal), "fy": np.float32(focal),
            "cx": np.float32(width / 2.0), "cy": np.float32(height / 2.0), "viewmat": vm,
            "campos": c.astype(np.float32), "t": np.float32(t)}


# ----------------------------------------------------------------- configs

def tiny_scene(seed: int = SCENE_SEED) -> Scene:
    """2,000 Gaussians in [-1,1]^3 x [0,1], SH degree 1, temporal order 1."""
    return make_scene(2000, seed, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)


def tiny_view(width: int = 128, height: int = 96, t: float = 0.5) -> dict:
    """Camera 3 units from the origin looking at it along +z."""
    return look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), width, height, t)


def orbit_scene(n: int = 300_000, seed: int = SCENE_SEED) -> Scene:
    """300k Gaussians in [-3,3]^3 x [0,1], SH degree 3 x temporal order 2."""
    return make_scene(n, seed, (-3, -3, -3), (3, 3, 3), sh_degree=3, t_order=2)


def orbit_view(k: int, count: int = 300, width: int = 1352, height: int = 1014) -> dict:
    """k-th view of the timestamp sweep: orbit of radius 6 at angle 2 pi k /
    count, timestamp k / (count - 1)."""
    th = 2.0 * math.pi * k / count
    t = k / (count - 1) if count > 1 else 0.0
    return look_at((6.0 * math.sin(th), 0.0, -6.0 * math.cos(th)), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0),
                   width, height, t)


def train_views(batch: int = 4, width: int = 1352, height: int = 1014, seed: int = POSE_SEED) -> list:
    """``batch`` seeded timestamps in [0,1] seen by the orbit camera at angle 0."""
    rng = np.random.default_rng(seed)
    ts = rng.random(batch)
    return [look_at((0.0, 0.0, -6.0), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), width, height, float(t)) for t in ts]


def sphere_scene(n: int = 1_000_000, seed: int = SCENE_SEED) -> Scene:
    """1M Gaussians in [-5,5]^3 x [0,1]."""
    return make_scene(n, seed, (-5, -5, -5), (5, 5, 5), sh_degree=3, t_order=2)


SPHERE_RESOLUTIONS = ((512, 512), (800, 800), (1014, 1352), (1352, 1014))


def sphere_views(count: int = 64, seed: int = POSE_SEED) -> list:
    """``count`` views of mixed resolution on a sphere of radius 8 looking at
    the origin, timestamps uniform in [0,1]."""
    rng = np.random.default_rng(seed)
    views = []
    for _ in range(count):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        w, h = SPHERE_RESOLUTIONS[int(rng.integers(len(SPHERE_RESOLUTIONS)))]
        views.append(look_at(8.0 * d, (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), w, h, float(rng.random())))
    return views


def urban_scene(n: int = 3_000_000, seed: int = SCENE_SEED) -> Scene:
    """3M Gaussians in [-30,30]^2 x [-3,3] x [0,1] (z vertical) with spatial
    log-scales U[ln 0.02, ln 1.0]."""
    return make_scene(n, seed, (-30, -30, -3), (30, 30, 3), spatial_log_scale=(math.log(0.02), math.log(1.0)),
                      sh_degree=3, t_order=2)


def urban_views(ts=(0.25, 0.75), width: int = 1920, height: int = 1080) -> list:
    """Six outward cameras (yaw 0, 60, ..., 300 degrees) on a ring of radius 2
    around a rig at (-20 + 40 t, 0, 1.5), for each timestamp in ``ts``."""
    views = []
    for t in ts:
        rig = np.array([-20.0 + 40.0 * t, 0.0, 1.5])
        for k in range(6):
            yaw = math.radians(60.0 * k)
            d = np.array([math.cos(yaw), math.sin(yaw), 0.0])
            views.append(look_at(rig + 2.0 * d, rig + 3.0 * d, (0.0, 0.0, 1.0), width, height, float(t)))
    return views
