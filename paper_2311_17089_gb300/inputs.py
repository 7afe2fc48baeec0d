"""Seeded synthetic scenes and pinhole cameras.

This module only draws random numbers and builds camera frames; it holds
none of the rendering method's arithmetic (no projection, coverage,
selection, sorting or blending).  Both the CUDA path and the FP64 oracle
take their inputs from here, so the two sides always see identical bytes.

Scene recipes stand in for the paper's datasets (Mip-NeRF 360, Tanks and
Temples, Deep Blending; Sec. 5), which are not available: they mimic
unbounded multi-level scenes whose coarse levels hold Gaussians about 4x
larger per level, the level structure of Sec. 4.1 ("4 levels of detail,
corresponding to the 1x, 4x, 16x and 64x downsampled resolution").

Arrays are float32, C-contiguous, structure-of-arrays:
    mean      [N, 3]      world position
    log_scale [N, 3]      log of the per-axis standard deviation
    quat      [N, 4]      rotation (w, x, y, z), not necessarily unit length
    opacity   [N]         activated opacity sigma in (0, 1)
    color     [N, K, 3]   SH coefficients, K = (deg+1)^2  (sh_degree >= 0)
              [N, 3]      plain RGB                       (sh_degree == -1)
    level     [N] uint8   1 (finest) .. n_levels (coarsest)
    s_max     [N]         maximum pixel coverage, initialised to 0
    s_min     [N]         minimum pixel coverage, initialised to +inf
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Scene", "Camera", "look_at", "pinhole", "downscale",
    "single_level_scene", "multiscale_scene", "near_far_scene",
    "tiny_scene", "config1_camera", "config2_camera", "orbit_cameras",
    "SCALES",
]

SCALES = (1, 2, 4, 8, 16, 32, 64, 128)


@dataclasses.dataclass
class Scene:
    mean: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity: np.ndarray
    color: np.ndarray
    level: np.ndarray
    n_levels: int
    sh_degree: int
    s_max: np.ndarray
    s_min: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.mean[idx].copy(), self.log_scale[idx].copy(),
                     self.quat[idx].copy(), self.opacity[idx].copy(),
                     self.color[idx].copy(), self.level[idx].copy(),
                     self.n_levels, self.sh_degree,
                     self.s_max[idx].copy(), self.s_min[idx].copy())

    def copy(self) -> "Scene":
        return self.subset(np.arange(self.n))


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    R (3x3, row-major) and t map world to camera: X_c = R X_w + t.
    Pixel (i, j) covers [i, i+1) x [j, j+1); its sample is the centre.
    """
    R: np.ndarray
    t: np.ndarray
    campos: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2
    bg: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros(3, np.float32))

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16


def _f32(x) -> float:
    return float(np.float32(x))


def look_at(eye, target, up) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """World->camera rotation and translation for a camera at `eye`.

    `up` is the world direction that appears upwards in the image.
    """
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    down = -np.asarray(up, np.float64)
    right = np.cross(down, fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float64)
    t = -R @ eye
    return R.astype(np.float32), t.astype(np.float32), eye.astype(np.float32)


def pinhole(eye, target, up, width: int, height: int, fovx_deg: float,
            near: float = 0.2, bg=(0.0, 0.0, 0.0)) -> Camera:
    R, t, c = look_at(eye, target, up)
    f = (0.5 * width) / math.tan(math.radians(fovx_deg) * 0.5)
    return Camera(R, t, c, _f32(f), _f32(f), _f32(0.5 * width),
                  _f32(0.5 * height), int(width), int(height), _f32(near),
                  np.asarray(bg, np.float32))


def downscale(cam: Camera, s: int) -> Camera:
    """The same view rendered s times smaller per side (Sec. 5: 1x .. 128x)."""
    w = max(1, cam.width // s)
    h = max(1, cam.height // s)
    return Camera(cam.R.copy(), cam.t.copy(), cam.campos.copy(),
                  _f32(cam.fx / s), _f32(cam.fy / s), _f32(0.5 * w),
                  _f32(0.5 * h), w, h, cam.near, cam.bg.copy())


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sigmoid_normal(rng, n):
    return (1.0 / (1.0 + np.exp(-rng.standard_normal(n)))).astype(np.float32)


def _sh_coeffs(rng, n, deg):
    k = (deg + 1) ** 2
    c = np.empty((n, k, 3), np.float32)
    c[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if k > 1:
        c[:, 1:, :] = rng.normal(0.0, 0.05, (n, k - 1, 3))
    return c


def _fresh_range(n):
    return np.zeros(n, np.float32), np.full(n, np.inf, np.float32)


def single_level_scene(n: int = 10_000, seed: int = 0) -> Scene:
    """Single-level scene: means U[-1,1]^3, log-scales N(-3.5, 0.5),
    random unit quaternions, opacity sigmoid(N(0,1)), plain RGB U(0,1)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scale = rng.normal(-3.5, 0.5, (n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid_normal(rng, n)
    color = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    level = np.ones(n, np.uint8)
    smax, smin = _fresh_range(n)
    return Scene(mean, log_scale, quat, opacity, color, level, 1, -1,
                 smax, smin)


def _level_counts(n, split):
    counts = [int(round(n * f)) for f in split]
    counts[0] += n - sum(counts)
    return counts


def multiscale_scene(n: int = 1_000_000, seed: int = 0,
                     split=(0.70, 0.20, 0.07, 0.03), sh_degree: int = 3,
                     n_clusters: int = 64, box: float = 10.0,
                     cluster_sigma: float = 1.0,
                     level_step: float = 1.4) -> Scene:
    """Four-level clustered scene.

    Means: `n_clusters` centres U[-box, box]^3, each point a centre plus
    N(0, cluster_sigma^2 I), clipped to the box.  Level l log-scales
    N(-3.5 + level_step (l-1), 0.5); exp(1.4) ~ 4, one level per 4x.
    SH of degree `sh_degree`: DC U(0,1), higher orders N(0, 0.05).
    """
    rng = np.random.default_rng(seed)
    counts = _level_counts(n, split)
    centres = rng.uniform(-box, box, (n_clusters, 3))
    which = rng.integers(0, n_clusters, n)
    mean = centres[which] + rng.normal(0.0, cluster_sigma, (n, 3))
    mean = np.clip(mean, -box, box).astype(np.float32)
    level = np.concatenate([np.full(c, l + 1, np.uint8)
                            for l, c in enumerate(counts)])
    level = level[rng.permutation(n)]
    log_scale = (rng.normal(0.0, 0.5, (n, 3))
                 + (-3.5 + level_step * (level.astype(np.float64) - 1.0))[:, None]
                 ).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid_normal(rng, n)
    color = _sh_coeffs(rng, n, sh_degree)
    smax, smin = _fresh_range(n)
    return Scene(mean, log_scale, quat, opacity, color, level, len(split),
                 sh_degree, smax, smin)


def near_far_scene(n: int = 3_000_000, seed: int = 0, n_fore: int | None = None,
                   split=(0.70, 0.20, 0.07, 0.03), sh_degree: int = 3) -> Scene:
    """Dense foreground ball of radius 1 plus a sparse shell of radius 50 +- 2.

    Two thirds of the Gaussians are foreground (the split is not given by
    the workload description; 2:1 is this recipe's choice).  Background
    Gaussians get log-scale base +2.0 so the shell reads as large splats.
    """
    rng = np.random.default_rng(seed)
    n_fore = (2 * n) // 3 if n_fore is None else n_fore
    n_back = n - n_fore
    d = rng.standard_normal((n_fore, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(0.0, 1.0, n_fore) ** (1.0 / 3.0)
    fore = d * r[:, None]
    d = rng.standard_normal((n_back, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    back = d * rng.uniform(48.0, 52.0, n_back)[:, None]
    mean = np.concatenate([fore, back]).astype(np.float32)
    counts = _level_counts(n, split)
    level = np.concatenate([np.full(c, l + 1, np.uint8)
                            for l, c in enumerate(counts)])
    level = level[rng.permutation(n)]
    base = np.concatenate([np.full(n_fore, -3.5), np.full(n_back, 2.0 - 3.5)])
    log_scale = (rng.normal(0.0, 0.5, (n, 3))
                 + (base + 1.4 * (level.astype(np.float64) - 1.0))[:, None]
                 ).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid_normal(rng, n)
    color = _sh_coeffs(rng, n, sh_degree)
    smax, smin = _fresh_range(n)
    return Scene(mean, log_scale, quat, opacity, color, level, len(split),
                 sh_degree, smax, smin)


def tiny_scene(n: int = 48, seed: int = 0, sh_degree: int = -1,
               n_levels: int = 1, extent: float = 0.6,
               log_scale_mean: float = -2.5) -> Scene:
    """A handful of Gaussians in front of config-1 style camera, for brute
    force checks on 64x64 images."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-extent, extent, (n, 3)).astype(np.float32)
    log_scale = rng.normal(log_scale_mean, 0.6, (n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid_normal(rng, n)
    if sh_degree < 0:
        color = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    else:
        color = _sh_coeffs(rng, n, sh_degree)
    level = rng.integers(1, n_levels + 1, n).astype(np.uint8)
    smax, smin = _fresh_range(n)
    return Scene(mean, log_scale, quat, opacity, color, level, n_levels,
                 sh_degree, smax, smin)


def config1_camera(width: int = 256, height: int = 256) -> Camera:
    """Camera at (0, 0, -3) looking at the origin, fov 60 deg, image up = -y."""
    return pinhole((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0),
                   width, height, 60.0)


def config2_camera(width: int = 1256, height: int = 832,
                   distance: float = 25.0) -> Camera:
    """Camera `distance` units out on -z looking at the origin, fovx 60 deg."""
    return pinhole((0.0, 0.0, -distance), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0),
                   width, height, 60.0)


def orbit_cameras(k: int, seed: int = 0, radius=25.0, width: int = 1256,
                  height: int = 832, elevation_deg: float = 15.0):
    """k cameras on a horizontal orbit around the origin at seeded azimuths
    and elevations within +-elevation_deg.  `radius` is a scalar or a
    length-k sequence (the near/far workload spaces radii 2 .. 60)."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 2.0 * math.pi, k)
    el = np.radians(rng.uniform(-elevation_deg, elevation_deg, k))
    radii = np.broadcast_to(np.asarray(radius, np.float64), (k,))
    cams = []
    for a, e, r in zip(az, el, radii):
        eye = (r * math.cos(e) * math.sin(a), r * math.sin(e),
               -r * math.cos(e) * math.cos(a))
        cams.append(pinhole(eye, (0.0, 0.0, 0.0), (0.0, -1.0, 0.0),
                            width, height, 60.0))
    return cams
