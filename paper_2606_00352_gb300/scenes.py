"""Seeded synthetic scenes and cameras (input generation only).

This module draws the random inputs that both the CUDA render path and the
FP64 oracle consume.  It holds none of the render method's arithmetic: it only
samples gaussian parameters and builds pinhole cameras.  It depends on numpy
alone so that the oracle side and the GPU side can both import it without
importing each other.

Scene layout (structure of arrays, float32, what the renderer takes as input):
    means          [N, 3]   world-space centres
    log_scales     [N, 3]   per-axis log standard deviations
    quats          [N, 4]   rotation quaternions (w, x, y, z), not normalised
    opacity_logits [N]      opacity = sigmoid(logit)
    sh             [N, K, 3] real spherical-harmonic coefficients,
                            K = (degree + 1)^2, coefficient k = l*l + l + m

Camera: world->camera 4x4 row-major matrix (x right, y down, z forward),
focal lengths fx, fy and principal point cx, cy in pixels, image size.

Workload recipes (readings of the paper's evaluation scenes, which are
trained Mip-NeRF 360 models that are not available; sizes follow Sec. 5.1):
  * uniform scene: means ~ U[-1,1]^3, log-scales ~ N(-4, 0.5), random unit
    quaternions, opacity logits ~ N(0, 1.5), SH degree 0 with rgb ~ U[0,1]
    stored as the DC coefficient (rgb - 0.5) / Y_00.
  * cluster scene: means from a Zipf-weighted mixture of anisotropic gaussian
    clusters, log-scales ~ N(-4.5, 0.7), opacity logits ~ N(0, 1.5), SH
    degree 3 with DC ~ N(0.5, 0.2) and the other 45 coefficients ~ N(0, 0.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Y_00 of the real SH basis, 1 / (2 sqrt(pi)); used only to store an RGB
# colour as a DC coefficient when a scene is generated.
_Y00 = 0.5 / math.sqrt(math.pi)


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox generator used for every synthetic input."""
    return np.random.Generator(np.random.Philox(seed))


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.sh_degree, dict(self.meta))

    def copy(self) -> "Scene":
        return self.subset(slice(None))

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.means, self.log_scales, self.quats,
                                      self.opacity_logits, self.sh))


@dataclass
class Camera:
    viewmat: np.ndarray  # [4, 4] float32, world -> camera, row-major
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def pixels(self) -> int:
        return self.width * self.height


def _check(scene: Scene) -> Scene:
    n = scene.n
    k = (scene.sh_degree + 1) ** 2
    assert scene.means.shape == (n, 3) and scene.means.dtype == np.float32
    assert scene.log_scales.shape == (n, 3) and scene.log_scales.dtype == np.float32
    assert scene.quats.shape == (n, 4) and scene.quats.dtype == np.float32
    assert scene.opacity_logits.shape == (n,) and scene.opacity_logits.dtype == np.float32
    assert scene.sh.shape == (n, k, 3) and scene.sh.dtype == np.float32
    for a in (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh):
        assert a.flags.c_contiguous
    return scene


def _unit_quats(g: np.random.Generator, n: int) -> np.ndarray:
    q = g.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def uniform_scene(n: int = 10_000, seed: int = 0) -> Scene:
    """Uniform cube scene with SH degree 0 (the tiny plain-path workload)."""
    g = rng(seed)
    means = g.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = g.normal(-4.0, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(g, n)
    logits = g.normal(0.0, 1.5, n).astype(np.float32)
    rgb = g.uniform(0.0, 1.0, (n, 3))
    sh = ((rgb - 0.5) / _Y00).astype(np.float32).reshape(n, 1, 3)
    return _check(Scene(means, log_scales, quats, logits, sh, 0,
                        {"kind": "uniform", "n": n, "seed": seed}))


def cluster_scene(n: int, n_clusters: int, zipf: float, seed: int = 0,
                  sigma_range=(0.02, 0.3), sh_degree: int = 3, extent: float = 1.0,
                  chunk: int = 1 << 21) -> Scene:
    """Zipf-weighted mixture of anisotropic gaussian clusters.

    Cluster k has weight proportional to k^-zipf (k = 1..n_clusters), a centre
    ~ U[-E,E]^3 (E = `extent`), per-axis standard deviations
    E exp(U[ln lo, ln hi]) and a random rotation.  The gaussians' own
    log-scales do not depend on E, so E sets how large they look on screen
    from an orbit of radius 3E.  Large scenes are drawn in chunks to bound
    host memory.
    """
    g = rng(seed)
    centres = g.uniform(-extent, extent, (n_clusters, 3))
    lo, hi = sigma_range
    sig = extent * np.exp(g.uniform(math.log(lo), math.log(hi), (n_clusters, 3)))
    rot = _quat_to_rot_np(_unit_quats(g, n_clusters).astype(np.float64))
    w = np.arange(1, n_clusters + 1, dtype=np.float64) ** (-zipf)
    w /= w.sum()
    k_sh = (sh_degree + 1) ** 2
    means = np.empty((n, 3), np.float32)
    log_scales = np.empty((n, 3), np.float32)
    quats = np.empty((n, 4), np.float32)
    logits = np.empty(n, np.float32)
    sh = np.empty((n, k_sh, 3), np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        m = e - s
        cid = g.choice(n_clusters, size=m, p=w)
        z = g.standard_normal((m, 3)) * sig[cid]
        means[s:e] = (centres[cid] + np.einsum("nij,nj->ni", rot[cid], z)).astype(np.float32)
        log_scales[s:e] = g.normal(-4.5, 0.7, (m, 3)).astype(np.float32)
        quats[s:e] = _unit_quats(g, m)
        logits[s:e] = g.normal(0.0, 1.5, m).astype(np.float32)
        c = g.normal(0.0, 0.2, (m, k_sh, 3))
        c[:, 0, :] = g.normal(0.5, 0.2, (m, 3))
        sh[s:e] = c.astype(np.float32)
    return _check(Scene(means, log_scales, quats, logits, sh, sh_degree,
                        {"kind": "cluster", "n": n, "clusters": n_clusters,
                         "zipf": zipf, "seed": seed, "sigma_range": tuple(sigma_range),
                         "extent": extent}))


# Higher-order SH whose energy falls with the degree: band l >= 1 drawn from
# N(0, 0.2 * DECAY^l).  A stand-in for trained scenes, whose view-dependent
# colour is a small correction of the base colour (the i.i.d. N(0, 0.2) of
# the configs gives every band the DC band's spread).
SH_DECAY = 0.25


def decaying_sh(scene: Scene, seed: int = 5, decay: float = SH_DECAY) -> Scene:
    """Copy of a degree-3 scene with its bands 1-3 redrawn from N(0, 0.2
    decay^l) (the DC band kept)."""
    g = rng(seed)
    out = scene.copy()
    sh = out.sh.copy()
    for l in range(1, scene.sh_degree + 1):
        sh[:, l * l:(l + 1) * (l + 1)] = g.normal(0.0, 0.2 * decay ** l, sh[:, l * l:(l + 1) * (l + 1)].shape)
    out.sh = sh.astype(np.float32)
    return out


def perturbed(scene: Scene, seed: int = 1, mean_sigma: float = 1e-3,
              logit_sigma: float = 0.1) -> Scene:
    """Copy with means + N(0, mean_sigma) and opacity logits + N(0, logit_sigma)."""
    g = rng(seed)
    out = scene.copy()
    out.means += g.normal(0.0, mean_sigma, out.means.shape).astype(np.float32)
    out.opacity_logits += g.normal(0.0, logit_sigma, out.opacity_logits.shape).astype(np.float32)
    return out


def _quat_to_rot_np(q: np.ndarray) -> np.ndarray:
    # Used only to orient the synthetic clusters (input sampling).
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), fov_x_deg: float = 60.0,
            width: int = 256, height: int = 256) -> Camera:
    """Pinhole camera at `eye` looking at `target`; fov is horizontal."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    rot = np.stack([r, d, f])
    vm = np.eye(4)
    vm[:3, :3] = rot
    vm[:3, 3] = -rot @ eye
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(vm.astype(np.float32), float(np.float32(fx)), float(np.float32(fx)),
                  0.5 * width, 0.5 * height, int(width), int(height))


def orbit(n_poses: int, radius: float = 3.0, width: int = 1920, height: int = 1080,
          fov_x_deg: float = 60.0, elevation: float = 0.0, phase: float = 0.0):
    """`n_poses` cameras evenly spaced on a horizontal circle around the origin."""
    cams = []
    for k in range(n_poses):
        th = phase + 2.0 * math.pi * k / n_poses
        eye = (radius * math.cos(th), radius * math.sin(th), elevation)
        cams.append(look_at(eye, width=width, height=height, fov_x_deg=fov_x_deg))
    return cams


# Named workloads --------------------------------------------------------

RES = {"720p": (1280, 720), "1080p": (1920, 1080), "4k": (3840, 2160), "256": (256, 256)}


def tiny_workload(seed: int = 0):
    """10k gaussians, SH0, one camera at distance 3, 256x256."""
    scene = uniform_scene(10_000, seed)
    cam = look_at((3.0, 0.0, 0.0), width=256, height=256)
    return scene, [cam]


# World extent and cluster spread of the cluster scenes.  With the
# per-gaussian log-scales fixed at N(-4.5, 0.7), an extent of 10 seen from an
# orbit of radius 30 (fov 60 deg) puts the densest 8x8 tile of the
# 5.8M-gaussian scene at about 2,300 gaussians at 1080p (the paper reports a
# peak of 2,485 for its 5.8M-gaussian scene) with ~20M rect tile pairs.
EXTENT = 10.0
CLUSTER_SIGMA = (0.15, 1.0)
ORBIT_RADIUS = 3.0 * EXTENT


def scene_1m(seed: int = 0, n: int = 1_000_000) -> Scene:
    """1M gaussians, 64 clusters, Zipf(1.2), SH degree 3."""
    return cluster_scene(n, 64, 1.2, seed, sigma_range=CLUSTER_SIGMA, extent=EXTENT)


def scene_5m8(seed: int = 0, n: int = 5_800_000) -> Scene:
    """5.8M gaussians, 256 clusters, Zipf(1.4), SH degree 3."""
    return cluster_scene(n, 256, 1.4, seed, sigma_range=CLUSTER_SIGMA, extent=EXTENT)


def scene_orbit(n_poses: int, width: int = 1920, height: int = 1080, phase: float = 0.0):
    """Orbit cameras for the cluster scenes."""
    return orbit(n_poses, ORBIT_RADIUS, width, height, phase=phase)
