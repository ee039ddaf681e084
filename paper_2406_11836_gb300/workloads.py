"""Seeded synthetic inputs shaped like the paper's workloads.

The paper trains on MipNeRF-360, ScanNet++, Mega-NeRF and MatrixCity (Sec. 4,
"Datasets"). None of those are available here, so every scene, camera, target
image and pixel sample is drawn from a seeded generator in this module.  The
scenes keep the structure of those workloads: compact object-centred clusters
(the MipNeRF-360 stand-in) and city-like layouts of many anisotropic clusters
on a ground plane (the MatrixCity stand-in).

This module holds no rendering arithmetic at all: no projection, no blending,
no partitioning.  It only produces random parameters, camera poses and sample
positions.  Both the FP64 oracle tests and the CUDA tests take their inputs
from here, and nothing else is shared between the two sides.

Conventions (they define the *inputs*, both sides read them the same way):
  * splat parameters are float32 structure-of-arrays:
      means [N,3], log_scales [N,3], quats [N,4] as (w,x,y,z), opacity_logits [N],
      sh [N,(deg+1)^2,3] (coefficient-major, RGB innermost);
  * a camera is a world->camera 4x4 matrix (row-major, OpenCV axes: x right,
    y down, z forward) plus pinhole intrinsics fx, fy, cx, cy and the image size;
  * the horizontal field of view is 60 degrees for every workload, so
    fx = fy = (W/2)/tan(30 deg), cx = W/2, cy = H/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


# --------------------------------------------------------------------------- data types
@dataclass
class Scene:
    means: torch.Tensor           # [N,3] float32
    log_scales: torch.Tensor      # [N,3] float32
    quats: torch.Tensor           # [N,4] float32, (w,x,y,z), not normalised
    opacity_logits: torch.Tensor  # [N]   float32
    sh: torch.Tensor              # [N,(deg+1)^2,3] float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def to(self, device) -> "Scene":
        return Scene(self.means.to(device), self.log_scales.to(device), self.quats.to(device),
                     self.opacity_logits.to(device), self.sh.to(device), self.sh_degree)

    def tensors(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)


@dataclass
class Camera:
    viewmat: np.ndarray           # [4,4] float64, world->camera, row-major
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near_z: float = 0.2

    @property
    def center(self) -> np.ndarray:
        """Camera centre o in world coordinates (input bookkeeping, not rendering)."""
        R = self.viewmat[:3, :3]
        t = self.viewmat[:3, 3]
        return -R.T @ t


@dataclass
class Workload:
    name: str
    scene: Scene
    cameras: list
    depth_L: int
    tile: int = 16
    notes: dict = field(default_factory=dict)


# --------------------------------------------------------------------------- cameras
def intrinsics(width: int, height: int, fov_x_deg: float = 60.0):
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return fx, fx, width / 2.0, height / 2.0


def look_at(eye, target, width, height, up=(0.0, 0.0, 1.0), fov_x_deg=60.0, near_z=0.2) -> Camera:
    """Pinhole camera at `eye` whose optical axis points at `target` (OpenCV axes)."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    if abs(float(f @ up)) > 0.999:          # looking straight along `up`: pick another up
        up = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])               # rows: camera axes in world coordinates
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = -R @ eye
    fx, fy, cx, cy = intrinsics(width, height, fov_x_deg)
    return Camera(V, fx, fy, cx, cy, width, height, near_z)


def axis_camera(eye, width, height, fov_x_deg=60.0, near_z=0.2) -> Camera:
    """Identity-rotation camera at `eye` (looks along world +z, image x = world x)."""
    V = np.eye(4)
    V[:3, 3] = -np.asarray(eye, np.float64)
    fx, fy, cx, cy = intrinsics(width, height, fov_x_deg)
    return Camera(V, fx, fy, cx, cy, width, height, near_z)


# --------------------------------------------------------------------------- scenes
def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _common_attrs(n: int, g: torch.Generator, device, sh_degree: int, dc_uniform: bool):
    quats = torch.randn(n, 4, generator=g, device=device)
    quats = quats / quats.norm(dim=1, keepdim=True)
    logits = torch.randn(n, generator=g, device=device)
    nsh = (sh_degree + 1) ** 2
    if dc_uniform:
        sh = torch.rand(n, nsh, 3, generator=g, device=device)
    else:
        sh = torch.randn(n, nsh, 3, generator=g, device=device) * 0.2
    return quats.float().contiguous(), logits.float().contiguous(), sh.float().contiguous()


def uniform_cube_scene(n: int, seed: int = 0, device="cpu", log_scale_mean=-4.0, log_scale_std=0.5,
                       extent=1.0, sh_degree=0) -> Scene:
    """Means uniform in [-extent, extent]^3, log-scales N(mean, std), unit quaternions,
    opacity logits N(0,1), SH coefficients U[0,1] (degree 0) or N(0,0.2) (degree > 0)."""
    g = _gen(seed, device)
    means = (torch.rand(n, 3, generator=g, device=device) * 2 - 1) * extent
    log_scales = torch.randn(n, 3, generator=g, device=device) * log_scale_std + log_scale_mean
    quats, logits, sh = _common_attrs(n, g, device, sh_degree, dc_uniform=(sh_degree == 0))
    return Scene(means.float().contiguous(), log_scales.float().contiguous(), quats, logits, sh, sh_degree)


def cluster_scene(n: int, n_clusters: int, seed: int, device="cpu", sh_degree=3, *,
                  centre_lo, centre_hi, std_lo, std_hi, log_scale_cluster=None,
                  log_scale_mean=-4.0, log_scale_std=0.5, chunk=1 << 24) -> Scene:
    """Mixture of anisotropic Gaussian clusters.

    centre_lo/hi: per-axis bounds of the uniform cluster centres.
    std_lo/hi:    per-axis bounds of the uniform per-cluster standard deviations.
    log_scale_cluster: (mean, std) of a per-cluster log-scale offset; when given, each
                  splat's log-scale is cluster_offset + N(0, log_scale_std); otherwise
                  N(log_scale_mean, log_scale_std).
    Generated in chunks so that 100M-splat scenes fit the host or device memory.
    """
    g = _gen(seed, device)
    lo = torch.tensor(centre_lo, dtype=torch.float32, device=device)
    hi = torch.tensor(centre_hi, dtype=torch.float32, device=device)
    slo = torch.tensor(std_lo, dtype=torch.float32, device=device)
    shi = torch.tensor(std_hi, dtype=torch.float32, device=device)
    centres = lo + (hi - lo) * torch.rand(n_clusters, 3, generator=g, device=device)
    stds = slo + (shi - slo) * torch.rand(n_clusters, 3, generator=g, device=device)
    if log_scale_cluster is not None:
        ls_c = torch.randn(n_clusters, generator=g, device=device) * log_scale_cluster[1] + log_scale_cluster[0]
    nsh = (sh_degree + 1) ** 2
    means = torch.empty(n, 3, dtype=torch.float32, device=device)
    log_scales = torch.empty(n, 3, dtype=torch.float32, device=device)
    quats = torch.empty(n, 4, dtype=torch.float32, device=device)
    logits = torch.empty(n, dtype=torch.float32, device=device)
    sh = torch.empty(n, nsh, 3, dtype=torch.float32, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        m = e - s
        cid = torch.randint(0, n_clusters, (m,), generator=g, device=device)
        means[s:e] = centres[cid] + stds[cid] * torch.randn(m, 3, generator=g, device=device)
        base = ls_c[cid, None] if log_scale_cluster is not None else log_scale_mean
        log_scales[s:e] = base + torch.randn(m, 3, generator=g, device=device) * log_scale_std
        q, lg, c = _common_attrs(m, g, device, sh_degree, dc_uniform=False)
        quats[s:e] = q
        logits[s:e] = lg
        sh[s:e] = c
    return Scene(means, log_scales, quats, logits, sh, sh_degree)


# --------------------------------------------------------------------------- the five workloads
def _sphere_dirs(seeds, upper_only=False):
    out = []
    for s in seeds:
        r = np.random.default_rng(s)
        while True:
            v = r.normal(size=3)
            nv = np.linalg.norm(v)
            if nv < 1e-6:
                continue
            v /= nv
            if upper_only and v[2] < 0.05:
                continue
            out.append(v)
            break
    return out


def _ground_cams(n, seed, half_extent, width, height):
    r = np.random.default_rng(seed)
    cams = []
    while len(cams) < n:
        eye = np.array([r.uniform(-half_extent, half_extent), r.uniform(-half_extent, half_extent),
                        r.uniform(2.0, 20.0)])
        tgt = np.array([r.uniform(-half_extent, half_extent), r.uniform(-half_extent, half_extent), 0.0])
        if np.linalg.norm(tgt - eye) < 10.0:
            continue
        cams.append(look_at(eye, tgt, width, height))
    return cams


def tiny(device="cpu") -> Workload:
    """4,096 splats, means U[-1,1]^3, log-scales N(-4,0.5), SH degree 0 with U[0,1]
    coefficients; one 128x128 camera at (0,0,-3) looking along +z; KD depth 1 (K=2)."""
    scene = uniform_cube_scene(4096, seed=0, device=device)
    cam = axis_camera((0.0, 0.0, -3.0), 128, 128)
    return Workload("tiny-4k-128px-K2", scene, [cam], depth_L=1)


def object_1m(device="cpu", n=1_000_000, width=1600, height=1060, n_views=20) -> Workload:
    """1M splats in 200 isotropic clusters (centres U[-5,5]^3, std 0.5), SH degree 3 with
    N(0,0.2) coefficients; 20 views on a radius-8 sphere looking at the origin; K=8."""
    scene = cluster_scene(n, 200, seed=1, device=device, sh_degree=3,
                          centre_lo=(-5, -5, -5), centre_hi=(5, 5, 5), std_lo=(0.5,) * 3, std_hi=(0.5,) * 3)
    cams = [look_at(8.0 * d, (0, 0, 0), width, height) for d in _sphere_dirs(range(100, 100 + n_views))]
    return Workload("object-1M-1600x1060-K8", scene, cams, depth_L=3)


def city_10m(device="cpu", n=10_000_000, width=3840, height=2160, n_views=10) -> Workload:
    """10M splats in 1,000 anisotropic clusters on a ground plane (spread 50x50x5), per-cluster
    log-scale mean N(-3,1) plus per-splat N(0,0.5); SH degree 3; 10 cameras at heights 2-20
    looking at ground points at least 10 units away; 3840x2160; K=16."""
    scene = cluster_scene(n, 1000, seed=2, device=device, sh_degree=3,
                          centre_lo=(-25, -25, 0), centre_hi=(25, 25, 5),
                          std_lo=(0.5, 0.5, 0.1), std_hi=(3.0, 3.0, 1.0), log_scale_cluster=(-3.0, 1.0))
    cams = _ground_cams(n_views, 200, 25.0, width, height)
    return Workload("city-10M-3840x2160-K16", scene, cams, depth_L=4)


def serving_5m(device="cpu", n=5_000_000) -> Workload:
    """5M splats in the city layout, SH degree 3, K=8; cameras are drawn per request."""
    scene = cluster_scene(n, 1000, seed=3, device=device, sh_degree=3,
                          centre_lo=(-25, -25, 0), centre_hi=(25, 25, 5),
                          std_lo=(0.5, 0.5, 0.1), std_hi=(3.0, 3.0, 1.0), log_scale_cluster=(-3.0, 1.0))
    return Workload("serve-5M-K8", scene, [], depth_L=3)


def city_100m(device="cpu", n=100_000_000, width=3840, height=2160, n_views=5) -> Workload:
    """100M splats in 10,000 clusters spread 500x500x20; SH degree 3; 5 ground cameras; K=64."""
    scene = cluster_scene(n, 10_000, seed=4, device=device, sh_degree=3,
                          centre_lo=(-250, -250, 0), centre_hi=(250, 250, 20),
                          std_lo=(0.5, 0.5, 0.1), std_hi=(3.0, 3.0, 1.0), log_scale_cluster=(-3.0, 1.0))
    cams = _ground_cams(n_views, 400, 250.0, width, height)
    return Workload("city-100M-3840x2160-K64", scene, cams, depth_L=6)


RESOLUTIONS = ((800, 600), (1600, 1200), (3840, 2160))


def request_stream(n_requests: int, rate_hz: float = 200.0, seed: int = 7, radius: float = 10.0):
    """Poisson arrivals (mean `rate_hz`), resolution uniform over RESOLUTIONS, pose uniform on
    the upper hemisphere of the given radius looking at the origin.  Returns a list of
    (arrival_time_s, Camera)."""
    r = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += r.exponential(1.0 / rate_hz)
        w, h = RESOLUTIONS[r.integers(len(RESOLUTIONS))]
        while True:
            v = r.normal(size=3)
            v /= np.linalg.norm(v)
            if v[2] > 0.05:
                break
        out.append((t, look_at(radius * v, (0, 0, 0), int(w), int(h))))
    return out


# --------------------------------------------------------------------------- targets and samples
def target_image(width: int, height: int, seed: int = 1, device="cpu") -> torch.Tensor:
    """Uniform-random [3,H,W] float32 target for the L1 loss."""
    g = _gen(seed, device)
    return torch.rand(3, height, width, generator=g, device=device)


def sample_pixels(width: int, height: int, count: int = 4096, seed: int = 11) -> np.ndarray:
    """`count` distinct seeded pixel indices (py*W + px), sorted ascending."""
    r = np.random.default_rng(seed)
    count = min(count, width * height)
    return np.sort(r.choice(width * height, size=count, replace=False)).astype(np.int64)


def loss_weights(width: int, height: int, seed: int = 5) -> np.ndarray:
    """Seeded smooth-loss weights w [3,H,W] (float64) for L = <w, C>, used by the
    finite-difference checks (a linear loss has no kinks)."""
    r = np.random.default_rng(seed)
    return r.uniform(-1.0, 1.0, size=(3, height, width))
