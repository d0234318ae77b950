"""Seeded synthetic scenes and camera rigs for the Gaussian-splatting renderer.

This module only draws random numbers and lays out cameras; it contains none
of the rendering arithmetic, so both the CUDA path and the FP64 oracle can be
fed from it without sharing any of the method's code.

The scenes stand in for the outdoor driving and handheld sequences the paper
evaluates on (Waymo, KITTI, DL3DV; Sec. 4.1). Those datasets are not used:
every scene here is drawn from a fixed-seed ``numpy.random.default_rng`` and
converted to float32, with the shapes and value distributions of the five
workloads described below.

Parameter layout (all float32, structure of arrays, row-major):
  means          (n, 3)             world-space centres mu (Eq. 1)
  log_scales     (n, 3)             log of the diagonal of S (Eq. 1)
  quats          (n, 4)             unnormalised rotation quaternion (w, x, y, z)
  opacity_logits (n,)               logit of the opacity
  colors         (n, (d+1)^2, 3)    per-Gaussian colour / SH coefficients
Camera (one dict per view): width, height, fx, fy, cx, cy and T_cw, a 3x4
row-major world-to-camera transform (the convention of Eq. 9).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "camera", "look_at_pose", "random_gaussians", "config_scene",
    "tiny_scene", "perturb_scene", "CONFIG_NAMES",
]

CONFIG_NAMES = {
    1: "plain single view, 4096 Gaussians, 160x120",
    2: "outdoor single frame, 500k Gaussians, 1241x376, SH degree 3",
    3: "mapping window, 1M Gaussians, 12 x 1241x376",
    4: "uneven-resolution batch, 2M Gaussians, 16 mixed views, pose-only backward",
    5: "long trajectory, 5M Gaussians, SH degree 3, 24 mixed views",
}


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    colors: np.ndarray
    sh_degree: int
    cameras: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def params(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.colors)

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity_logits[idx].copy(), self.colors[idx].copy(), self.sh_degree,
                     [dict(c) for c in self.cameras])


def camera(width, height, fx, fy, cx, cy, T_cw=None) -> dict:
    """One pinhole view. ``T_cw`` is a 3x4 world-to-camera matrix (default identity)."""
    if T_cw is None:
        T_cw = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    T = np.asarray(T_cw, dtype=np.float64).reshape(3, 4)
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fy),
                cx=float(cx), cy=float(cy), T_cw=T.astype(np.float32))


def look_at_pose(position, yaw, pitch=0.0) -> np.ndarray:
    """World-to-camera 3x4 for a camera at ``position`` looking along yaw (about -y).

    Camera frame: x right, y down, z forward. World frame is y-down as well, so a
    level camera with yaw 0 looks along world +z.
    """
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    # camera-to-world rotation: columns are the camera axes in world coordinates
    fwd = np.array([sy_ * cp, sp, cy_ * cp])
    right = np.array([cy_, 0.0, -sy_])
    down = np.cross(fwd, right)
    R_wc = np.stack([right, down, fwd], axis=1)
    R_cw = R_wc.T
    t_cw = -R_cw @ np.asarray(position, dtype=np.float64)
    return np.concatenate([R_cw, t_cw[:, None]], axis=1)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _colors(rng, n, sh_degree, rgb_low=0.0, rgb_high=1.0):
    nc = (sh_degree + 1) ** 2
    c = np.zeros((n, nc, 3))
    c[:, 0, :] = rng.uniform(rgb_low, rgb_high, (n, 3))
    if nc > 1:
        c[:, 1:, :] = rng.normal(0.0, 0.2, (n, nc - 1, 3))
    return c


def random_gaussians(rng, means, sh_degree=0, log_scale_mean=math.log(0.05), log_scale_std=0.5):
    """Attributes for Gaussians at the given world-space means (the config-1 recipe)."""
    n = means.shape[0]
    log_s = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _unit_quats(rng, n)
    opac_logit = rng.standard_normal(n)
    cols = _colors(rng, n, sh_degree)
    return Scene(means.astype(np.float32), log_s.astype(np.float32), quats.astype(np.float32),
                 opac_logit.astype(np.float32), cols.astype(np.float32), sh_degree, [])


def _box_points(rng, n, T_wc_R=None, T_wc_t=None):
    """Camera-relative box x,y in [-4,4], z in [2,20], mapped to world by (R_wc, t_wc)."""
    p = np.stack([rng.uniform(-4, 4, n), rng.uniform(-4, 4, n), rng.uniform(2, 20, n)], axis=1)
    if T_wc_R is not None:
        p = p @ T_wc_R.T + T_wc_t
    return p


def _arc_trajectory(rng, n_keyframes, n_past, length=100.0, radius=60.0):
    """Poses along a circular arc of the given length; yaw follows the tangent.

    Keyframes are evenly spaced; ``n_past`` extra views sit at random earlier arc
    positions. Each position gets +-0.2 m jitter.
    """
    s_kf = np.linspace(length / n_keyframes, length, n_keyframes)
    s_past = rng.uniform(0.0, s_kf[-1] * 0.9, n_past)
    poses = []
    for s in list(s_kf) + list(s_past):
        theta = s / radius
        pos = np.array([radius * (1.0 - math.cos(theta)), 0.0, radius * math.sin(theta)])
        pos += rng.uniform(-0.2, 0.2, 3)
        poses.append(look_at_pose(pos, yaw=theta))
    return poses


def _trajectory_scene(rng, n_total, poses, sh_degree, log_scale_mean, log_scale_std):
    """One camera-relative config-1 box of n_total/len(poses) Gaussians per pose."""
    counts = np.full(len(poses), n_total // len(poses))
    counts[: n_total - counts.sum()] += 1
    pts = []
    for T, c in zip(poses, counts):
        R_cw, t_cw = T[:, :3], T[:, 3]
        R_wc = R_cw.T
        pts.append(_box_points(rng, int(c), R_wc, -R_wc @ t_cw))
    means = np.concatenate(pts, axis=0)
    return random_gaussians(rng, means, sh_degree, log_scale_mean, log_scale_std)


def config_scene(cid: int, n_override: int | None = None) -> Scene:
    """The five seeded workloads (seed = 1000 + config id)."""
    rng = np.random.default_rng(1000 + cid)
    if cid == 1:
        n = n_override or 4096
        means = _box_points(rng, n)
        sc = random_gaussians(rng, means, 0)
        sc.cameras = [camera(160, 120, 150.0, 150.0, 80.0, 60.0)]
        return sc
    if cid == 2:
        n = n_override or 500_000
        n_ground = int(0.6 * n)
        n_blob = n - n_ground
        ground = np.stack([rng.uniform(-15, 15, n_ground), 1.65 + rng.normal(0, 0.05, n_ground),
                           rng.uniform(1, 80, n_ground)], axis=1)
        n_clusters = 400
        side = rng.choice([-1.0, 1.0], n_clusters)
        centres = np.stack([side * rng.uniform(4, 12, n_clusters), rng.uniform(-3, 1.5, n_clusters),
                            rng.uniform(1, 80, n_clusters)], axis=1)
        which = rng.integers(0, n_clusters, n_blob)
        blobs = centres[which] + rng.normal(0.0, 1.0, (n_blob, 3))
        means = np.concatenate([ground, blobs], axis=0)
        sc = random_gaussians(rng, means, 3)
        sc.cameras = [camera(1241, 376, 718.0, 718.0, 620.5, 187.5)]
        return sc
    if cid == 3:
        n = n_override or 1_000_000
        poses = _arc_trajectory(rng, 10, 2)
        sc = _trajectory_scene(rng, n, poses, 0, math.log(0.05), 0.5)
        sc.cameras = [camera(1241, 376, 718.0, 718.0, 620.5, 187.5, T) for T in poses]
        return sc
    if cid == 4:
        n = n_override or 2_000_000
        n_dense = int(0.2 * n)
        n_sparse = n - n_dense
        # scene volume x in [-20,20], y in [-4,4], z in [0,80]; the dense sub-box
        # x in [-5,5] (1/4), z in [20,36] (1/5) holds 20% of Gaussians in 5% of it
        sparse = np.stack([rng.uniform(-20, 20, n_sparse), rng.uniform(-4, 4, n_sparse),
                           rng.uniform(0, 80, n_sparse)], axis=1)
        dense = np.stack([rng.uniform(-5, 5, n_dense), rng.uniform(-4, 4, n_dense),
                          rng.uniform(20, 36, n_dense)], axis=1)
        means = np.concatenate([sparse, dense], axis=0)
        sc = random_gaussians(rng, means, 0)
        sizes = [(1920, 1280)] * 6 + [(960, 540)] * 5 + [(640, 480)] * 5
        cams = []
        for k, (w, h) in enumerate(sizes):
            pos = np.array([rng.uniform(-6, 6), rng.uniform(-0.5, 0.5), rng.uniform(-4, 0)])
            T = look_at_pose(pos, yaw=rng.uniform(-0.17, 0.17), pitch=rng.uniform(-0.05, 0.05))
            f = 0.9 * w
            cams.append(camera(w, h, f, f, w / 2.0, h / 2.0, T))
        sc.cameras = cams
        return sc
    if cid == 5:
        n = n_override or 5_000_000
        poses = _arc_trajectory(rng, 18, 6, length=200.0, radius=90.0)
        sc = _trajectory_scene(rng, n, poses, 3, math.log(0.1), 0.8)
        cams = []
        for k, T in enumerate(poses):
            if k % 2 == 0:
                cams.append(camera(1241, 376, 718.0, 718.0, 620.5, 187.5, T))
            else:
                cams.append(camera(1920, 1280, 1728.0, 1728.0, 960.0, 640.0, T))
        sc.cameras = cams
        return sc
    raise ValueError(f"unknown config {cid}")


def tiny_scene(seed: int, n: int = 6, width: int = 24, height: int = 20, sh_degree: int = 0,
               max_opacity: float = 0.9, n_views: int = 1, scale: float = 0.35) -> Scene:
    """A handful of Gaussians in front of small cameras (finite-difference scale)."""
    rng = np.random.default_rng(seed)
    f = 1.1 * width
    means = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n),
                      rng.uniform(3.0, 6.0, n)], axis=1)
    log_s = np.log(scale) + rng.normal(0.0, 0.25, (n, 3))
    quats = _unit_quats(rng, n) * rng.uniform(0.7, 1.4, (n, 1))
    op = rng.uniform(0.2, max_opacity, n)
    logit = np.log(op / (1.0 - op))
    cols = _colors(rng, n, sh_degree, 0.1, 0.9)
    sc = Scene(means.astype(np.float32), log_s.astype(np.float32), quats.astype(np.float32),
               logit.astype(np.float32), cols.astype(np.float32), sh_degree, [])
    cams = []
    for v in range(n_views):
        if v == 0:
            T = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
        else:
            pos = rng.uniform(-0.3, 0.3, 3)
            T = look_at_pose(pos, yaw=rng.uniform(-0.08, 0.08), pitch=rng.uniform(-0.05, 0.05))
        cams.append(camera(width, height, f, f, width / 2.0 - 0.5 + rng.uniform(-1, 1),
                           height / 2.0 - 0.5 + rng.uniform(-1, 1), T))
    sc.cameras = cams
    return sc


def perturb_scene(sc: Scene, seed: int, sigma_pos=0.02, sigma_col=0.05) -> Scene:
    """A nearby scene whose renders serve as synthetic mapping-loss targets."""
    rng = np.random.default_rng(seed)
    out = sc.subset(slice(None))
    out.means = (sc.means + rng.normal(0, sigma_pos, sc.means.shape)).astype(np.float32)
    out.colors = (sc.colors + rng.normal(0, sigma_col, sc.colors.shape)).astype(np.float32)
    return out


def pointmap_pair(width: int, height: int, seed: int, scale: float = 1.1, fx: float = 718.0, fy: float = 718.0,
                  hole_frac: float = 0.05, bad_frac: float = 0.15, noise: float = 0.02):
    """A seeded (rendered, pre-trained) pair of camera-frame pointmaps, float32 (3, H, W).

    Stands in for the 3DGS pointmap X^r and a learned pointmap prior X^p of a
    driving frame (Sec. 3.3): a ground plane 1.65 m below the camera, a far
    background at 60-80 m and a dozen box obstacles at 5-40 m, seen through a
    pinhole camera. X^p is the same geometry at 1/scale of the scene's size with
    per-pixel multiplicative depth noise and, over ``bad_frac`` of the image in
    random blocks, depths distorted by a factor in [0.5, 2] (poorly predicted
    regions). X^r has holes (all-zero points, as where a render has no
    Gaussians) over ``hole_frac`` of the image in random blocks.
    """
    rng = np.random.default_rng(seed)
    cx, cy = width / 2.0 - 0.5, height / 2.0 - 0.5
    jj, ii = np.meshgrid(np.arange(height, dtype=np.float64), np.arange(width, dtype=np.float64), indexing="ij")
    z = rng.uniform(60.0, 80.0) + rng.normal(0.0, 0.5, (height, width))
    below = jj > cy + 1.0
    ground = np.where(below, 1.65 * fy / np.maximum(jj - cy, 1e-6), np.inf)
    z = np.where(below, np.minimum(z, np.clip(ground, 2.0, 80.0)), z)

    def blocks(frac, lo, hi):
        m = np.zeros((height, width), dtype=bool)
        target = frac * width * height
        while m.sum() < target:
            bw = int(rng.integers(lo, hi + 1)); bh = int(rng.integers(lo, hi + 1))
            x0 = int(rng.integers(0, max(width - bw, 0) + 1)); y0 = int(rng.integers(0, max(height - bh, 0) + 1))
            m[y0:y0 + bh, x0:x0 + bw] = True
        return m

    for _ in range(12):
        bw = int(rng.integers(max(width // 40, 2), max(width // 8, 3)))
        bh = int(rng.integers(max(height // 20, 2), max(height // 3, 3)))
        x0 = int(rng.integers(0, max(width - bw, 0) + 1)); y0 = int(rng.integers(0, max(height - bh, 0) + 1))
        z[y0:y0 + bh, x0:x0 + bw] = np.minimum(z[y0:y0 + bh, x0:x0 + bw], rng.uniform(5.0, 40.0))
    ray = np.stack([(ii - cx) / fx, (jj - cy) / fy, np.ones_like(ii)])
    X_true = ray * z[None]
    X_r = X_true * (1.0 + rng.normal(0.0, 0.5 * noise, (1, height, width)))
    X_r[:, blocks(hole_frac, 4, max(min(width, height) // 6, 5))] = 0.0
    depth_factor = 1.0 + rng.normal(0.0, noise, (height, width))
    bad = blocks(bad_frac, 6, max(min(width, height) // 4, 7))
    depth_factor[bad] *= rng.uniform(0.5, 2.0, int(bad.sum()))
    X_p = X_true / scale * depth_factor[None]
    return X_r.astype(np.float32), X_p.astype(np.float32)
