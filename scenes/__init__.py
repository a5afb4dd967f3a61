"""Seeded synthetic inputs for the moment-based Gaussian rasterizer.

This module only draws random Gaussian scenes and builds pinhole cameras.
It holds none of the rendering method's arithmetic, so both the FP64 CPU
oracle (``oracle/``) and the CUDA path (``paper_2512_11800_gb300``) may
consume it without sharing any computation.

Conventions (shared *input* conventions, not method arithmetic):

* Gaussians are float32 structure-of-arrays: ``means[P,3]``, ``scales[P,3]``
  (positive, already exponentiated), ``quats[P,4]`` (w, x, y, z; not
  necessarily normalised), ``weights[P]`` (peak density w >= 0, already
  through softplus), ``sh[P,K,3]`` with K = (degree+1)^2.
* Cameras are OpenCV pinholes: x right, y down, z forward.  ``viewmat`` is
  the 4x4 row-major world->camera transform.  Intrinsics use a vertical
  field of view, fx = fy = (H/2)/tan(fov/2), principal point at the image
  centre.  Pixel (x, y) has its centre at (x + 0.5, y + 0.5).

The scene recipes mirror the paper's workload sizes (0.95M-3.8M Gaussians
per scene, Sec. 4 per-scene table) with synthetic, seeded content; the
paper's datasets are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Real spherical-harmonic band-0 constant 1/(2 sqrt(pi)); used only to encode
# a target RGB as a degree-0 coefficient (input preparation).
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    weights: np.ndarray
    sh: np.ndarray
    sh_degree: int
    name: str = ""

    @property
    def P(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.weights[idx].copy(), self.sh[idx].copy(), self.sh_degree,
                     self.name + "[subset]")


@dataclass
class Camera:
    viewmat: np.ndarray          # (4,4) float32, world -> camera, row-major
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    eye: np.ndarray = field(default_factory=lambda: np.zeros(3))

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """Camera whose image is the sub-rectangle [x0,x0+w) x [y0,y0+h)."""
        return Camera(self.viewmat.copy(), self.fx, self.fy, self.cx - x0, self.cy - y0, w, h,
                      self.eye.copy())


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_deg=60.0,
            width=128, height=128) -> Camera:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])                      # rows: camera axes in world coords
    t = -R @ eye
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = t
    fy = (height / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    f32 = lambda x: float(np.float32(x))     # the C ABI takes float32 intrinsics
    return Camera(V.astype(np.float32), f32(fy), f32(fy), f32(width / 2.0), f32(height / 2.0),
                  int(width), int(height), eye.copy())


def _rand_quats(rng, P):
    q = rng.standard_normal((P, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _log_uniform(rng, lo, hi, P):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), P))


def _random_rotations(rng, n):
    """Random proper rotations via QR of Gaussian matrices (input drawing only)."""
    A = rng.standard_normal((n, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    det = np.linalg.det(Q)
    Q[:, :, 0] *= det[:, None]
    return Q


def _pack(means, scales, quats, weights, sh, deg, name) -> Scene:
    return Scene(np.ascontiguousarray(means, np.float32), np.ascontiguousarray(scales, np.float32),
                 np.ascontiguousarray(quats, np.float32), np.ascontiguousarray(weights, np.float32),
                 np.ascontiguousarray(sh, np.float32), int(deg), name)


def scene_uniform(P=2000, seed=0, name="uniform2k") -> Scene:
    """Small scene: means U[-1,1]^3, log-scales N(-3,0.5), unit random
    rotations, densities U[0.5,5], SH degree 0 with RGB U[0,1]."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (P, 3))
    scales = np.exp(rng.normal(-3.0, 0.5, (P, 3)))
    quats = _rand_quats(rng, P)
    weights = rng.uniform(0.5, 5.0, P)
    rgb = rng.uniform(0.0, 1.0, (P, 3))
    sh = ((rgb - 0.5) / _Y00)[:, None, :]
    return _pack(means, scales, quats, weights, sh, 0, name)


def scene_clusters(P=200_000, seed=1, name="clusters200k") -> Scene:
    """16 isotropic clusters (sigma 0.3) with centres U[-2,2]^3, log-scales
    N(-4,0.7), densities log-uniform [0.1,20], SH degree 3 ~ N(0,0.2)."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-2.0, 2.0, (16, 3))
    which = rng.integers(0, 16, P)
    means = centers[which] + rng.normal(0.0, 0.3, (P, 3))
    scales = np.exp(rng.normal(-4.0, 0.7, (P, 3)))
    quats = _rand_quats(rng, P)
    weights = _log_uniform(rng, 0.1, 20.0, P)
    sh = rng.normal(0.0, 0.2, (P, 16, 3))
    return _pack(means, scales, quats, weights, sh, 3, name)


def scene_shells(P=1_000_000, seed=2, name="shells1M") -> Scene:
    """70% of Gaussians in 64 anisotropic clusters, 30% on 8 interpenetrating
    low-density spherical shells; log-scales N(-4.5,0.8), SH degree 3."""
    rng = np.random.default_rng(seed)
    n_cl = int(round(P * 0.7))
    n_sh = P - n_cl
    centers = rng.uniform(-1.5, 1.5, (64, 3))
    Rc = _random_rotations(rng, 64)
    sc = rng.uniform(0.05, 0.4, (64, 3))
    which = rng.integers(0, 64, n_cl)
    z = rng.standard_normal((n_cl, 3)) * sc[which]
    cl_means = centers[which] + np.einsum("nij,nj->ni", Rc[which], z)
    cl_w = _log_uniform(rng, 0.1, 20.0, n_cl)
    s_centers = rng.uniform(-1.0, 1.0, (8, 3))
    s_radius = rng.uniform(0.4, 1.0, 8)
    s_which = rng.integers(0, 8, n_sh)
    u = rng.standard_normal((n_sh, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = s_radius[s_which] + rng.normal(0.0, 0.01, n_sh)
    sh_means = s_centers[s_which] + r[:, None] * u
    sh_w = rng.uniform(0.05, 0.5, n_sh)
    means = np.concatenate([cl_means, sh_means])
    weights = np.concatenate([cl_w, sh_w])
    scales = np.exp(rng.normal(-4.5, 0.8, (P, 3)))
    quats = _rand_quats(rng, P)
    sh = rng.normal(0.0, 0.2, (P, 16, 3))
    return _pack(means, scales, quats, weights, sh, 3, name)


def target_image(height, width, seed=12) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (height, width, 3)).astype(np.float32)


def multiview_cameras(n_views=16, seed=4, radius=3.0, fov_deg=60.0):
    """Random poses on a sphere of the given radius looking at the origin,
    resolutions drawn from {640x360, 1280x720, 1920x1080}."""
    rng = np.random.default_rng(seed)
    res = [(640, 360), (1280, 720), (1920, 1080)]
    cams = []
    up = np.array([0.0, 1.0, 0.0])
    for _ in range(n_views):
        W, H = res[int(rng.integers(0, 3))]
        while True:
            e = rng.standard_normal(3)
            e = radius * e / np.linalg.norm(e)
            f = -e / np.linalg.norm(e)
            if abs(float(f @ up)) <= 0.99:
                break
        cams.append(look_at(e, (0, 0, 0), up, fov_deg, W, H))
    return cams


# The five workloads: (scene factory, camera factory).
WORKLOADS = {
    "uniform2k_128": (lambda: scene_uniform(2000, 0), lambda: look_at((0, 0, -3), fov_deg=60, width=128, height=128)),
    "clusters200k_720p": (lambda: scene_clusters(200_000, 1), lambda: look_at((0, 0, -5), fov_deg=50, width=1280, height=720)),
    "shells1M_1080p": (lambda: scene_shells(1_000_000, 2), lambda: look_at((0, 0, -3), fov_deg=60, width=1920, height=1080)),
    "shells3M_1080p": (lambda: scene_shells(3_000_000, 3, "shells3M"), lambda: look_at((0, 0, -3), fov_deg=60, width=1920, height=1080)),
}


def workload(name):
    s, c = WORKLOADS[name]
    return s(), c()


def tiny_scene(P=8, seed=100, spread=0.4, log_scale=(-1.8, 0.3), w_range=(0.5, 4.0), deg=0) -> Scene:
    """Handful of Gaussians near the origin for brute-force checks."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, (P, 3))
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (P, 3)))
    quats = _rand_quats(rng, P)
    weights = rng.uniform(w_range[0], w_range[1], P)
    K = (deg + 1) ** 2
    if deg == 0:
        rgb = rng.uniform(0.0, 1.0, (P, 3))
        sh = ((rgb - 0.5) / _Y00)[:, None, :]
    else:
        sh = rng.normal(0.0, 0.3, (P, K, 3))
    return _pack(means, scales, quats, weights, sh, deg, "tiny")
