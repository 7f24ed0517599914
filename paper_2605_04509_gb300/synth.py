"""Seeded synthetic inputs: Gaussian scenes, arc camera rigs and lenticular panels.

This module draws random numbers and builds input arrays. It holds none of the
renderer's arithmetic (no projection, no view-index mapping, no blending), so
that both the CUDA path and the FP64 CPU oracle can be fed the very same
float32 inputs without sharing any code.

The trained Blender / Mip-NeRF 360 scenes the paper measures on (Sec. 5.1) are
not available; the distributions below stand in for them:

* tiny scene: means uniform in [-1, 1]^3 around the origin;
* mixture scene: 64 centres uniform in a ball of radius 10, means drawn
  around them with standard deviation 0.3;
* both: log-scales N(-3, 0.5) per axis, unit quaternions from normalised
  N(0, 1)^4 draws (w, x, y, z order), opacity sigmoid(N(0, 1.5)), degree-3
  SH with DC ~ N(0.5, 0.2) and higher bands ~ N(0, 0.1).

Cameras sit on a horizontal arc around the scene origin and look at it; view
0 is the leftmost camera, matching the view ordering of the panel's view
index (Sec. 3.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np

SH_COEFFS = 16  # degree 3


@dataclasses.dataclass(frozen=True)
class Panel:
    """Lenticular panel parameters (Sec. 3.1): resolution, view count, tan of
    the grating tilt angle alpha, grating pitch L_x in subpixels and the
    lens-to-panel offset K_offset."""

    width: int
    height: int
    num_views: int
    tan_slant: float
    pitch: float
    k_offset: float = 0.0

    @property
    def subpixels(self) -> int:
        return 3 * self.width * self.height


@dataclasses.dataclass(frozen=True)
class Rig:
    """Camera rig: the view cone of the display."""

    num_views: int
    cone_deg: float
    radius: float
    fov_x_deg: float


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    num_gaussians: int
    scene: str  # "uniform" or "mixture"
    seed: int
    panel: Panel
    rig: Rig


# Workloads with the sizes of the paper-scale evaluation (4K panel, 45 views)
# and the small case the oracle finishes in seconds.
WORKLOADS: Dict[str, Workload] = {
    "tiny": Workload(
        "tiny", 2000, "uniform", 1,
        Panel(256, 144, 8, 1.0 / 6.0, 4.5, 0.0),
        Rig(8, 40.0, 4.0, 50.0)),
    "paper4k": Workload(
        "paper4k", 1_000_000, "mixture", 2,
        Panel(3840, 2160, 45, math.tan(0.2), 5.3, 0.0),
        Rig(45, 40.0, 30.0, 50.0)),
    "precision8k": Workload(
        "precision8k", 3_000_000, "mixture", 3,
        Panel(7680, 4320, 100, math.tan(0.18), 6.1, 0.0),
        Rig(100, 50.0, 30.0, 50.0)),
    "diff1080": Workload(
        "diff1080", 500_000, "mixture", 5,
        Panel(1920, 1080, 24, math.tan(0.2), 4.8, 0.0),
        Rig(24, 40.0, 30.0, 50.0)),
}


def _sigmoid(x: np.ndarray) -> np.ndarray:
    return 1.0 / (1.0 + np.exp(-x))


def _attributes(rng: np.random.Generator, m: int) -> Dict[str, np.ndarray]:
    log_scales = rng.normal(-3.0, 0.5, size=(m, 3))
    quats = rng.normal(0.0, 1.0, size=(m, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    opac = _sigmoid(rng.normal(0.0, 1.5, size=m))
    sh = rng.normal(0.0, 0.1, size=(m, SH_COEFFS, 3))
    sh[:, 0, :] = rng.normal(0.5, 0.2, size=(m, 3))
    return {
        "scales": np.exp(log_scales).astype(np.float32),
        "quats": quats.astype(np.float32),
        "opacities": opac.astype(np.float32),
        "sh": sh.astype(np.float32),
    }


def uniform_scene(m: int, seed: int, half_extent: float = 1.0) -> Dict[str, np.ndarray]:
    """Means uniform in [-half_extent, half_extent]^3."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-half_extent, half_extent, size=(m, 3))
    out = {"means": means.astype(np.float32)}
    out.update(_attributes(rng, m))
    return out


def mixture_scene(m: int, seed: int, centres: int = 64, std: float = 0.3,
                  radius: float = 10.0) -> Dict[str, np.ndarray]:
    """Means from a Gaussian mixture whose centres are uniform in a ball."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(centres, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, size=(centres, 1)) ** (1.0 / 3.0)
    c = d * r
    pick = rng.integers(0, centres, size=m)
    means = c[pick] + rng.normal(0.0, std, size=(m, 3))
    out = {"means": means.astype(np.float32)}
    out.update(_attributes(rng, m))
    return out


def scene_for(w: Workload, num_gaussians: Optional[int] = None) -> Dict[str, np.ndarray]:
    m = w.num_gaussians if num_gaussians is None else num_gaussians
    if w.scene == "uniform":
        return uniform_scene(m, w.seed)
    return mixture_scene(m, w.seed)


def arc_cameras(rig: Rig, width: int, height: int) -> np.ndarray:
    """Pinhole cameras on a horizontal arc looking at the origin.

    Returns float32 [n, 16]: row-major world->camera rotation R (9), translation
    t (3), fx, fy, cx, cy. Camera axes follow the OpenCV convention (x right,
    y down, z forward); world y points down. Camera j sits at angle
    theta_j = -cone/2 + cone * j / (n - 1) (0 for a single view), at
    (radius sin theta, 0, -radius cos theta). fx = fy = (W/2) / tan(fov_x/2),
    principal point at the panel centre; every view renders at panel size.
    """
    n = rig.num_views
    out = np.zeros((n, 16), dtype=np.float64)
    f = (width / 2.0) / math.tan(math.radians(rig.fov_x_deg) / 2.0)
    for j in range(n):
        th = 0.0 if n == 1 else math.radians(-rig.cone_deg / 2.0 + rig.cone_deg * j / (n - 1))
        centre = np.array([rig.radius * math.sin(th), 0.0, -rig.radius * math.cos(th)])
        z = -centre / np.linalg.norm(centre)
        y = np.array([0.0, 1.0, 0.0])
        x = np.cross(y, z)
        x /= np.linalg.norm(x)
        y = np.cross(z, x)
        rot = np.stack([x, y, z])
        t = -rot @ centre
        out[j, 0:9] = rot.reshape(-1)
        out[j, 9:12] = t
        out[j, 12:16] = (f, f, width / 2.0, height / 2.0)
    return out.astype(np.float32)


def random_subpixels(panel: Panel, count: int, seed: int) -> np.ndarray:
    """Seeded sample of subpixel coordinates, int32 [count, 3] = (x, y, u)."""
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, panel.width, size=count)
    ys = rng.integers(0, panel.height, size=count)
    us = rng.integers(0, 3, size=count)
    return np.stack([xs, ys, us], axis=1).astype(np.int32)


def random_conics(count: int, seed: int, min_sigma: float = 0.6,
                  max_sigma: float = 40.0) -> np.ndarray:
    """Random symmetric positive-definite 2x2 inverse covariances (a, b, c).

    Built as R^T diag(1/s0^2, 1/s1^2) R from a random angle and random
    log-uniform standard deviations; float32 [count, 3].
    """
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, math.pi, size=count)
    s = np.exp(rng.uniform(math.log(min_sigma), math.log(max_sigma), size=(count, 2)))
    cth, sth = np.cos(th), np.sin(th)
    l0, l1 = 1.0 / s[:, 0] ** 2, 1.0 / s[:, 1] ** 2
    a = cth * cth * l0 + sth * sth * l1
    b = cth * sth * (l0 - l1)
    c = sth * sth * l0 + cth * cth * l1
    return np.stack([a, b, c], axis=1).astype(np.float32)
