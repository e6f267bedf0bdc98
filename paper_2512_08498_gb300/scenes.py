"""Seeded synthetic scenes and cameras for the rasterizer workloads.

This module only *constructs inputs*: Gaussian parameters (means, log-scales,
quaternions, opacity logits, SH coefficients), pinhole cameras (intrinsics and
world-to-camera matrices), per-view Gaussian subsets and L1 target images.  It
holds none of the rasterizer's arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.

Conventions (OpenCV camera axes): x right, y down, z forward.  The world frame
shares the y-down convention, so the ground plane of the street scenes is at
y = +1.6 m below a rig mounted at height 0.  ``viewmat`` is the row-major 4x4
world-to-camera transform [R | t].

Workloads (one function each, seed = workload number):

* ``small_box``      10k Gaussians in a 4x4x(2..10) m box, one 256x256 view.
* ``single_hd``      500k Gaussians, SH degree 3, one 1920x1080 view.
* ``rig6``           1M-Gaussian street corridor, 6-camera rig at 1600x900.
* ``window30``       3M-Gaussian corridor, 5 keyframes x 6 cameras, mixed
                     resolutions, per-keyframe Gaussian subsets.
* ``road300``        6M Gaussians on a 300 m corridor plus a sky shell,
                     10 keyframes x 6 cameras at 1920x1080.

These stand in for the road-scene captures used for the per-keyframe
optimisation timings (Table 3, 1920x1080 rig cameras of Sec. 4): the datasets
themselves are not available, so the scene statistics are synthetic.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class View:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray                  # (4, 4) float32, world -> camera, row-major
    subset: Optional[np.ndarray] = None  # ascending uint32 Gaussian indices, or None = all


@dataclasses.dataclass
class Scene:
    name: str
    means: np.ndarray           # (N, 3) float32
    log_scales: np.ndarray      # (N, 3) float32
    quats: np.ndarray           # (N, 4) float32, (w, x, y, z), not normalised
    opacity_logits: np.ndarray  # (N,) float32
    sh: np.ndarray              # (N, (D+1)^2, 3) float32
    sh_degree: int
    views: List[View]
    tile: tuple = (16, 16)
    bg: tuple = (0.0, 0.0, 0.0)
    target_seed: int = 0

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def targets(self) -> List[np.ndarray]:
        """Seeded U(0,1) target images, one (3, H, W) float32 array per view."""
        rng = np.random.default_rng(self.target_seed)
        return [rng.random((3, v.height, v.width), dtype=np.float32) for v in self.views]

    def view_counts(self) -> List[int]:
        return [self.n if v.subset is None else int(v.subset.shape[0]) for v in self.views]


# ----------------------------------------------------------------------------
# helpers (input construction only)
# ----------------------------------------------------------------------------

def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def world_to_camera(r_wc: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """4x4 world-to-camera matrix from a camera-to-world rotation and a centre."""
    m = np.eye(4, dtype=np.float64)
    r = r_wc.T
    m[:3, :3] = r
    m[:3, 3] = -r @ centre
    return m.astype(np.float32)


def _sh(rng, n, degree, dc_low=0.0, dc_high=1.0, rest_std=0.1):
    k = (degree + 1) ** 2
    sh = np.empty((n, k, 3), dtype=np.float32)
    sh[:, 0, :] = rng.uniform(dc_low, dc_high, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, k - 1, 3))
    return sh


def _corridor_means(rng, n, z_lo, z_hi):
    """Street corridor: 40% ground, 50% two facades at x = +-8 m, 10% uniform."""
    n_ground = int(round(0.4 * n))
    n_facade = int(round(0.5 * n))
    n_free = n - n_ground - n_facade
    g = np.empty((n_ground, 3))
    g[:, 0] = rng.uniform(-8.0, 8.0, n_ground)
    g[:, 1] = 1.6 + rng.uniform(-0.3, 0.3, n_ground)
    g[:, 2] = rng.uniform(z_lo, z_hi, n_ground)
    f = np.empty((n_facade, 3))
    side = np.where(rng.random(n_facade) < 0.5, -8.0, 8.0)
    f[:, 0] = side + rng.uniform(-0.1, 0.1, n_facade)
    f[:, 1] = rng.uniform(-10.0, 1.6, n_facade)
    f[:, 2] = rng.uniform(z_lo, z_hi, n_facade)
    u = np.empty((n_free, 3))
    u[:, 0] = rng.uniform(-8.0, 8.0, n_free)
    u[:, 1] = rng.uniform(-10.0, 1.6, n_free)
    u[:, 2] = rng.uniform(z_lo, z_hi, n_free)
    m = np.concatenate([g, f, u], axis=0)
    m = m[rng.permutation(n)]
    return m.astype(np.float32)


def _rig_views(rng, rig_centre, width, height, n_cams=6, jitter=True, size_choices=None):
    """A ring of ``n_cams`` cameras yawed 360/n_cams apart about the world y axis.

    Each camera gets a seeded extrinsic offset of +-2 cm and +-1 degree (Euler
    x, y, z) on top of its nominal mounting.  90 degree horizontal FOV:
    fx = fy = W / 2, principal point at the image centre.
    """
    views = []
    for k in range(n_cams):
        if size_choices is not None:
            width, height = size_choices[int(rng.integers(0, len(size_choices)))]
        yaw = 2.0 * math.pi * k / n_cams
        if jitter:
            off = rng.uniform(-0.02, 0.02, 3)
            eul = np.deg2rad(rng.uniform(-1.0, 1.0, 3))
        else:
            off = np.zeros(3)
            eul = np.zeros(3)
        r_wc = _rot_y(yaw) @ _rot_z(eul[2]) @ _rot_y(eul[1]) @ _rot_x(eul[0])
        centre = np.asarray(rig_centre, dtype=np.float64) + off
        f = width / 2.0
        views.append(View(width, height, f, f, width / 2.0, height / 2.0,
                          world_to_camera(r_wc, centre)))
    return views


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def small_box(seed: int = 1, n: int = 10_000) -> Scene:
    """10k Gaussians uniform in [-2,2]x[-2,2]x[2,10] m, one 256x256 identity camera.

    log-scales U(-4,-1), unit quaternions from normalised N(0,1)^4, opacity
    logits N(0,1), SH degree 0 with the RGB DC coefficients drawn U(0,1).
    """
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3), dtype=np.float32)
    means[:, 0] = rng.uniform(-2.0, 2.0, n)
    means[:, 1] = rng.uniform(-2.0, 2.0, n)
    means[:, 2] = rng.uniform(2.0, 10.0, n)
    log_scales = rng.uniform(-4.0, -1.0, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    sh = _sh(rng, n, 0)
    view = View(256, 256, 256.0, 256.0, 128.0, 128.0, np.eye(4, dtype=np.float32))
    return Scene("small_box_10k_256", means, log_scales, quats, opac, sh, 0, [view],
                 tile=(16, 16), target_seed=100 + seed)


def single_hd(seed: int = 2, n: int = 500_000) -> Scene:
    """500k Gaussians in the frustum of one 1920x1080 camera (fx=fy=1100), SH degree 3.

    Depth log-uniform in [1, 80] m, image position uniform, log-scales
    U(-5,-1), DC coefficients U(0,1), higher bands N(0, 0.1).
    """
    rng = np.random.default_rng(seed)
    w, h, f, cx, cy = 1920, 1080, 1100.0, 960.0, 540.0
    z = np.exp(rng.uniform(math.log(1.0), math.log(80.0), n))
    u = rng.uniform(0.0, w, n)
    v = rng.uniform(0.0, h, n)
    means = np.stack([(u - cx) * z / f, (v - cy) * z / f, z], axis=1).astype(np.float32)
    log_scales = rng.uniform(-5.0, -1.0, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    sh = _sh(rng, n, 3)
    view = View(w, h, f, f, cx, cy, np.eye(4, dtype=np.float32))
    return Scene("single_hd_500k_1080p", means, log_scales, quats, opac, sh, 3, [view],
                 tile=(16, 16), target_seed=100 + seed)


def rig6(seed: int = 3, n: int = 1_000_000) -> Scene:
    """1M-Gaussian street corridor (z in [-30, 30] m) seen by a 6-camera rig at 1600x900."""
    rng = np.random.default_rng(seed)
    means = _corridor_means(rng, n, -30.0, 30.0)
    log_scales = rng.uniform(-5.0, -1.0, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    sh = _sh(rng, n, 3)
    views = _rig_views(rng, (0.0, 0.0, 0.0), 1600, 900)
    return Scene("rig6_1M_1600x900", means, log_scales, quats, opac, sh, 3, views,
                 tile=(16, 16), target_seed=100 + seed)


def window30(seed: int = 4, n: int = 3_000_000) -> Scene:
    """5 keyframes x 6 cameras over a 3M-Gaussian corridor, uneven resolutions and subsets.

    Keyframe rig centres at z = -4, -2, 0, 2, 4 m.  Keyframe k renders the
    n_k Gaussians nearest to its rig centre, with n = {200k, 3M, three
    log-uniform draws in [200k, 3M]} in shuffled order; each view's resolution
    is drawn from {1920x1080, 1600x900, 960x540}.
    """
    rng = np.random.default_rng(seed)
    means = _corridor_means(rng, n, -30.0, 30.0)
    log_scales = rng.uniform(-5.0, -1.0, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    sh = _sh(rng, n, 3)
    lo, hi = 200_000, n
    counts = [lo, hi] + [int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3)]
    counts = [counts[i] for i in rng.permutation(5)]
    sizes = [(1920, 1080), (1600, 900), (960, 540)]
    views = []
    m64 = means.astype(np.float64)
    for k, zk in enumerate((-4.0, -2.0, 0.0, 2.0, 4.0)):
        centre = np.array([0.0, 0.0, zk])
        d2 = np.sum((m64 - centre) ** 2, axis=1)
        nk = counts[k]
        if nk >= n:
            subset = np.arange(n, dtype=np.uint32)
        else:
            subset = np.sort(np.argpartition(d2, nk - 1)[:nk]).astype(np.uint32)
        for v in _rig_views(rng, centre, 0, 0, size_choices=sizes):
            v.subset = subset
            views.append(v)
    return Scene("window30_3M_mixed", means, log_scales, quats, opac, sh, 3, views,
                 tile=(16, 16), target_seed=100 + seed)


def road300(seed: int = 5, n: int = 6_000_000) -> Scene:
    """6M Gaussians: 95% corridor over z in [-150, 150] m, 5% sky shell at 500 m.

    Sky Gaussians lie on the upper (y < 0) hemisphere of radius 500 m with
    log-scales U(1, 3).  10 keyframes every 10 m along z (z = -45 ... 45) x
    6 cameras at 1920x1080; every view renders all Gaussians.
    """
    rng = np.random.default_rng(seed)
    n_sky = int(round(0.05 * n))
    n_road = n - n_sky
    road = _corridor_means(rng, n_road, -150.0, 150.0)
    d = rng.standard_normal((n_sky, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:, 1] = -np.abs(d[:, 1])
    sky = (500.0 * d).astype(np.float32)
    means = np.concatenate([road, sky], axis=0)
    log_scales = np.concatenate([
        rng.uniform(-5.0, -1.0, (n_road, 3)),
        rng.uniform(1.0, 3.0, (n_sky, 3))], axis=0).astype(np.float32)
    perm = rng.permutation(n)
    means, log_scales = means[perm], log_scales[perm]
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    sh = _sh(rng, n, 3)
    views = []
    for k in range(10):
        views += _rig_views(rng, (0.0, 0.0, -45.0 + 10.0 * k), 1920, 1080)
    return Scene("road300_6M_60x1080p", means, log_scales, quats, opac, sh, 3, views,
                 tile=(16, 16), target_seed=100 + seed)


WORKLOADS = {
    "small_box": small_box,
    "single_hd": single_hd,
    "rig6": rig6,
    "window30": window30,
    "road300": road300,
}


def scaled(fn, scale: float, seed: Optional[int] = None) -> Scene:
    """A workload with its Gaussian count multiplied by ``scale`` (views unchanged)."""
    import inspect
    n_default = inspect.signature(fn).parameters["n"].default
    kw = {"n": max(1, int(round(n_default * scale)))}
    if seed is not None:
        kw["seed"] = seed
    return fn(**kw)


def random_scene(seed: int, n: int, views: List[View], sh_degree: int,
                 z_range=(1.0, 6.0), xy_half=1.5, log_scale_range=(-3.5, -1.0),
                 tile=(16, 16), bg=(0.0, 0.0, 0.0)) -> Scene:
    """Small generic scene for tests: Gaussians in a box in front of the origin."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3), dtype=np.float32)
    means[:, 0] = rng.uniform(-xy_half, xy_half, n)
    means[:, 1] = rng.uniform(-xy_half, xy_half, n)
    means[:, 2] = rng.uniform(z_range[0], z_range[1], n)
    log_scales = rng.uniform(log_scale_range[0], log_scale_range[1], (n, 3)).astype(np.float32)
    quats = rng.standard_normal((n, 4)).astype(np.float32)  # unnormalised on purpose
    opac = rng.standard_normal(n).astype(np.float32)
    sh = _sh(rng, n, sh_degree, dc_low=-0.5, dc_high=1.0, rest_std=0.2)
    return Scene(f"random_{seed}_{n}", means, log_scales, quats, opac, sh, sh_degree, views,
                 tile=tile, bg=bg, target_seed=1000 + seed)


def pinhole(width, height, f=None, cx=None, cy=None, viewmat=None, subset=None) -> View:
    f = float(width) if f is None else float(f)
    cx = width / 2.0 if cx is None else float(cx)
    cy = height / 2.0 if cy is None else float(cy)
    vm = np.eye(4, dtype=np.float32) if viewmat is None else np.asarray(viewmat, dtype=np.float32)
    return View(width, height, f, f, cx, cy, vm, subset)


def look_from(centre, yaw_deg=0.0, pitch_deg=0.0, roll_deg=0.0) -> np.ndarray:
    """World-to-camera matrix of a camera at ``centre`` rotated by yaw (y), pitch (x), roll (z)."""
    r_wc = _rot_y(math.radians(yaw_deg)) @ _rot_x(math.radians(pitch_deg)) @ _rot_z(math.radians(roll_deg))
    return world_to_camera(r_wc, np.asarray(centre, dtype=np.float64))
