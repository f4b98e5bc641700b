"""Seeded synthetic inputs for the 3DGS Levenberg-Marquardt hot path.

This module only draws random numbers and builds posed pinhole cameras. It holds
none of the method's arithmetic: no projection, no compositing, no derivatives.
Both the FP64 CPU oracle (``oracle/``) and the CUDA path consume what it returns,
so the two sides always see bit-identical float32 inputs.

Parameter layout (one row per Gaussian, 59 float32 values), following the
parameter count stated in the paper's supplement (Sec. A, "Design of applyJ and
diagJTJ": 11 geometric parameters plus 48 SH coefficients of degree 3):

    0..2   position (x, y, z)
    3..5   log-scale
    6..9   rotation quaternion (w, x, y, z), not normalised
    10     opacity logit
    11..58 SH coefficients, index 11 + 3*coeff + channel, coeff l-major (0..15)

Cameras use OpenCV axes (x right, y down, z forward): a world point X maps to
camera coordinates R @ X + t, then to pixels (fx*x/z + cx, fy*y/z + cy).

Seeds: every named workload has a base seed; independent sub-streams are drawn
with ``np.random.default_rng([seed, stream])`` for the scene, the perturbed
copy, the pixel noise, the cameras and the subset permutations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_PARAMS = 59
P_POS, P_LOGSCALE, P_QUAT, P_OPACITY, P_SH = 0, 3, 6, 10, 11
SH_COEFFS = 16

STREAM_SCENE, STREAM_PERTURB, STREAM_NOISE, STREAM_CAMERAS, STREAM_SUBSETS, STREAM_TARGETS = 1, 2, 3, 4, 5, 6


@dataclass
class Camera:
    R: np.ndarray          # (3, 3) float32, world -> camera rotation
    t: np.ndarray          # (3,) float32, world -> camera translation
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Workload:
    """A named synthetic workload: its sizes and the recipe of its inputs."""
    name: str
    seed: int
    n_gaussians: int
    n_cameras: int
    resolutions: list          # list of (W, H); cycled over the cameras
    cam_radius: float
    subset_sizes: list         # views per image subset (n_b = len)
    lm_steps: int
    pcg_iters: int = 8
    lambda0: float = 1e-3
    lambda_min: float = 1e-4
    lambda_max: float = 1e4
    pos_extent: float = 1.0          # uniform positions in [-e, e]^3 when n_clusters == 0
    n_clusters: int = 0              # > 0: mixture of anisotropic normal clusters
    cluster_box: float = 3.0         # cluster centres uniform in [-b, b]^3
    jitter_deg: float = 0.0          # camera direction jitter (std, degrees)
    jitter_radius: float = 0.0       # relative camera radius jitter (std)
    hfov_deg: float = 60.0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    # 1,000 Gaussians, 8 views of 64x64, one subset.
    "tiny": Workload("tiny", 1001, 1000, 8, [(64, 64)], 4.0, [8], 5),
    # 100k Gaussians, 32 views of 400x300, four subsets of eight views.
    "medium": Workload("medium", 1002, 100_000, 32, [(400, 300)], 6.0, [8, 8, 8, 8], 10, pos_extent=2.0),
    # 1.5M Gaussians in 20 clusters, 200 jittered views of 1264x832, four subsets of 25.
    "paper": Workload("paper", 1003, 1_500_000, 200, [(1264, 832)], 8.0, [25, 25, 25, 25], 5,
                      n_clusters=20, jitter_deg=2.0, jitter_radius=0.02),
    # 3M Gaussians in 40 clusters, 300 views at mixed resolutions, eight uneven subsets.
    "uneven": Workload("uneven", 1005, 3_000_000, 300,
                       [(960, 540), (1280, 720), (1264, 832), (1600, 1066)], 8.0,
                       [10, 17, 24, 31, 38, 45, 52, 60], 5, n_clusters=40,
                       jitter_deg=2.0, jitter_radius=0.02),
}


def small_workload(name: str, seed: int, n_gaussians: int, n_cameras: int, width: int, height: int,
                   cam_radius: float = 4.0, subset_sizes=None, pos_extent: float = 1.0,
                   log_scale_mean: float = -3.5) -> Workload:
    """A test-sized workload with the 'tiny' distributions and free sizes (ragged tiles allowed)."""
    wl = Workload(name, seed, n_gaussians, n_cameras, [(width, height)], cam_radius,
                  subset_sizes or [n_cameras], 3, pos_extent=pos_extent)
    wl.extra["log_scale_mean"] = log_scale_mean
    return wl


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([seed, stream])


def _random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _quat_matrix(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion (w, x, y, z); used only to orient cluster shapes."""
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def make_gaussians(wl: Workload) -> np.ndarray:
    """Scene parameters, shape (N, 59) float32 (layout in the module docstring)."""
    rng = _rng(wl.seed, STREAM_SCENE)
    n = wl.n_gaussians
    out = np.zeros((n, N_PARAMS), np.float64)
    if wl.n_clusters > 0:
        k = wl.n_clusters
        centres = rng.uniform(-wl.cluster_box, wl.cluster_box, (k, 3))
        rots = [_quat_matrix(q) for q in _random_unit_quats(rng, k)]
        sig = rng.uniform(0.15, 0.8, (k, 3))
        label = np.arange(n) % k                      # equal weights
        z = rng.standard_normal((n, 3))
        pos = np.empty((n, 3))
        for c in range(k):
            m = label == c
            pos[m] = centres[c] + (z[m] * sig[c]) @ rots[c].T
        out[:, 0:3] = pos
    else:
        out[:, 0:3] = rng.uniform(-wl.pos_extent, wl.pos_extent, (n, 3))
    out[:, 3:6] = rng.normal(wl.extra.get("log_scale_mean", -3.5), 0.3, (n, 3))
    out[:, 6:10] = _random_unit_quats(rng, n)
    out[:, 10] = rng.normal(0.0, 1.0, n)
    sh = np.empty((n, SH_COEFFS, 3))
    sh[:, 0, :] = rng.normal(0.0, 0.5, (n, 3))
    sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, SH_COEFFS - 1, 3))
    out[:, 11:] = sh.reshape(n, 48)
    return out.astype(np.float32)


def cluster_labels(wl: Workload) -> np.ndarray:
    """Cluster index of every Gaussian (equal-weight assignment used by make_gaussians)."""
    return np.arange(wl.n_gaussians) % max(wl.n_clusters, 1)


def perturbed_copy(wl: Workload, params: np.ndarray) -> np.ndarray:
    """Target scene: positions + N(0, 0.02), every SH coefficient + N(0, 0.1)."""
    rng = _rng(wl.seed, STREAM_PERTURB)
    p = params.astype(np.float64).copy()
    p[:, 0:3] += rng.normal(0.0, 0.02, (p.shape[0], 3))
    p[:, 11:] += rng.normal(0.0, 0.1, (p.shape[0], 48))
    return p.astype(np.float32)


def pixel_noise(wl: Workload, n_values: int) -> np.ndarray:
    """N(0, 0.01) noise added to rendered targets (flat float32 array)."""
    return _rng(wl.seed, STREAM_NOISE).normal(0.0, 0.01, n_values).astype(np.float32)


def look_at(position: np.ndarray, target=(0.0, 0.0, 0.0)):
    """World->camera (R, t) for a camera at `position` looking at `target`, OpenCV axes.

    World up is +z; when the viewing direction is within ~8 degrees of it, +y is used.
    """
    f = np.asarray(target, np.float64) - position
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(f @ up) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ position
    return R, t


def fibonacci_sphere(n: int, radius: float) -> np.ndarray:
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def make_cameras(wl: Workload) -> list:
    rng = _rng(wl.seed, STREAM_CAMERAS)
    pos = fibonacci_sphere(wl.n_cameras, wl.cam_radius)
    cams = []
    for i in range(wl.n_cameras):
        p = pos[i]
        if wl.jitter_deg > 0 or wl.jitter_radius > 0:
            axis = rng.standard_normal(3)
            axis /= np.linalg.norm(axis)
            ang = math.radians(wl.jitter_deg) * rng.standard_normal()
            # Rodrigues rotation of the camera position about a random axis.
            p = (p * math.cos(ang) + np.cross(axis, p) * math.sin(ang)
                 + axis * (axis @ p) * (1 - math.cos(ang)))
            p = p * (1.0 + wl.jitter_radius * rng.standard_normal())
        W, H = wl.resolutions[i % len(wl.resolutions)]
        R, t = look_at(p)
        f = (W / 2.0) / math.tan(math.radians(wl.hfov_deg) / 2.0)   # horizontal field of view
        cams.append(Camera(R.astype(np.float32), t.astype(np.float32), np.float32(f), np.float32(f),
                           np.float32(W / 2.0), np.float32(H / 2.0), W, H))
    return cams


def subset_views(wl: Workload, step: int) -> list:
    """Image subsets of one LM step: a seeded permutation of the cameras cut into slices."""
    rng = np.random.default_rng([wl.seed, STREAM_SUBSETS, step])
    total = sum(wl.subset_sizes)
    if total == wl.n_cameras:
        perm = rng.permutation(wl.n_cameras) if len(wl.subset_sizes) > 1 else np.arange(wl.n_cameras)
    else:
        perm = rng.permutation(wl.n_cameras)[:total]
    out, o = [], 0
    for s in wl.subset_sizes:
        out.append(sorted(int(v) for v in perm[o:o + s]))
        o += s
    return out


def smooth_images(seed: int, cams: list, n_waves: int = 6) -> list:
    """Low-frequency random colour images in [0, 1] (H, W, 3) float32, one per camera.

    A non-rendered stand-in for target images where only the residual's shape matters.
    """
    rng = _rng(seed, STREAM_TARGETS)
    out = []
    for c in cams:
        yy, xx = np.mgrid[0:c.height, 0:c.width].astype(np.float64)
        img = np.full((c.height, c.width, 3), 0.5)
        for _ in range(n_waves):
            kx, ky = rng.normal(0, 2 * math.pi / max(c.width, 1) * 3, 2)
            ph = rng.uniform(0, 2 * math.pi)
            amp = rng.uniform(0.02, 0.12, 3)
            img += amp * np.sin(kx * xx + ky * yy + ph)[..., None]
        out.append(np.clip(img, 0, 1).astype(np.float32))
    return out


def random_vector(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Standard-normal float32 test vector (for J*p, J^T*u and adjoint checks)."""
    return (scale * _rng(seed, 7).standard_normal(shape)).astype(np.float32)


def crop_2k(wl: Workload, params: np.ndarray, n_keep: int = 2000) -> np.ndarray:
    """Indices of the n_keep Gaussians of cluster 0 nearest that cluster's mean position."""
    lab = cluster_labels(wl)
    idx = np.nonzero(lab == 0)[0]
    pos = params[idx, 0:3].astype(np.float64)
    c = pos.mean(axis=0)
    order = np.argsort(np.linalg.norm(pos - c, axis=1), kind="stable")
    return np.sort(idx[order[:n_keep]])
