"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module only draws random numbers and lays them out; it holds none of the
optimiser's or the rasteriser's arithmetic.  Every generator is a pure function
of its seed.

Parameter layout (one float32 array of shape [rows, n_pad], row pitch n_pad):

    rows 0..2    means mu (x, y, z)
    rows 3..5    log-scales (x, y, z)              s = exp(log_scale)
    rows 6..9    quaternion (x, y, z, w), unnormalised
    row  10      opacity logit                     alpha = sigmoid(logit)
    rows 11..    SH coefficients, row 11 + 3*k + c for coefficient k, channel c
                 (K = (deg+1)^2 coefficients)

Columns n..n_pad-1 are padding and are ignored by every consumer.  The paper
groups the parameter vector by type (Sec. 3.1, "x = (x_position, x_scaling,
x_rotation, x_opacity, x_color)"); this layout is that grouping.

Distributions (stand-ins for the SfM-initialised scenes of the paper's
datasets, which are not available here):
    means       uniform in a cube, or a mixture of isotropic clusters
    log-scales  N(-3, 0.5) + shift
    quaternion  N(0, 1)^4, normalised at generation
    opacity     logits N(0, 1)
    SH DC       N(0, 0.709)  (a colour N(0.5, 0.2) under the degree-0 basis)
    SH rest     N(0, 0.1)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ROW_MEAN = 0
ROW_LOG_SCALE = 3
ROW_QUAT = 6
ROW_OPACITY = 10
ROW_SH = 11


def n_sh_coeffs(sh_degree: int) -> int:
    return (sh_degree + 1) ** 2


def n_rows(sh_degree: int) -> int:
    return ROW_SH + 3 * n_sh_coeffs(sh_degree)


def pad_count(n: int, multiple: int = 32) -> int:
    return max(multiple, ((n + multiple - 1) // multiple) * multiple)


@dataclass
class Scene:
    params: np.ndarray  # float32 [rows, n_pad]
    n: int
    sh_degree: int

    @property
    def n_pad(self) -> int:
        return self.params.shape[1]


def make_scene(n: int, sh_degree: int = 0, *, seed: int = 1000, kind: str = "cube",
               extent: float = 1.0, n_clusters: int = 20, cluster_sigma: float = 0.3,
               log_scale_shift: float | None = None) -> Scene:
    """Draw a seeded Gaussian scene.

    kind="cube":     means uniform in [-extent, extent]^3; log-scales shifted by
                     ln(extent) unless ``log_scale_shift`` is given.
    kind="clusters": ``n_clusters`` equal-weight isotropic clusters (std
                     ``cluster_sigma``) with centres uniform in the ball of radius
                     ``extent``; log-scales unshifted unless given.
    """
    rng = np.random.default_rng(seed)
    K = n_sh_coeffs(sh_degree)
    n_pad = pad_count(n)
    p = np.zeros((n_rows(sh_degree), n_pad), np.float32)
    if kind == "cube":
        mu = rng.uniform(-extent, extent, size=(3, n))
        shift = math.log(extent) if log_scale_shift is None else log_scale_shift
    elif kind == "clusters":
        # centres uniform in the ball: direction uniform, radius ~ extent * U^(1/3)
        d = rng.normal(size=(3, n_clusters))
        d /= np.linalg.norm(d, axis=0, keepdims=True)
        rad = extent * rng.uniform(0, 1, size=n_clusters) ** (1.0 / 3.0)
        centres = d * rad
        lab = rng.integers(0, n_clusters, size=n)
        mu = centres[:, lab] + rng.normal(0.0, cluster_sigma, size=(3, n))
        shift = 0.0 if log_scale_shift is None else log_scale_shift
    else:
        raise ValueError(f"unknown scene kind {kind!r}")
    p[0:3, :n] = mu
    p[3:6, :n] = rng.normal(-3.0, 0.5, size=(3, n)) + shift
    q = rng.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    p[6:10, :n] = q
    p[10, :n] = rng.normal(0.0, 1.0, size=n)
    sh = np.zeros((K, 3, n))
    sh[0] = rng.normal(0.0, 0.709, size=(3, n))
    if K > 1:
        sh[1:] = rng.normal(0.0, 0.1, size=(K - 1, 3, n))
    p[ROW_SH:, :n] = sh.reshape(K * 3, n)
    return Scene(p, n, sh_degree)


@dataclass
class Camera:
    viewmat: np.ndarray  # float64 [4, 4], world -> camera, row-major (x right, y down, z forward)
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    width: int
    height: int


def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera matrix for a camera at ``position`` looking at ``target``."""
    p = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    Rc = np.stack([r, d, f])
    m = np.eye(4)
    m[:3, :3] = Rc
    m[:3, 3] = -Rc @ p
    return m


def pinhole(width: int, height: int, hfov_deg: float = 60.0, near: float = 0.2):
    fx = 0.5 * width / math.tan(math.radians(hfov_deg) / 2)
    return dict(fx=fx, fy=fx, cx=0.5 * width, cy=0.5 * height, near=near, width=width, height=height)


def single_camera(width: int, height: int, distance: float = 4.0) -> Camera:
    return Camera(look_at((distance, 0.0, 0.0)), **pinhole(width, height))


def camera_ring(n: int, width: int, height: int, scene_radius: float, *, seed: int = 7,
                ring_factor: float = 2.4, elev_deg: float = 15.0, jitter: float = 0.02) -> list[Camera]:
    """``n`` cameras on a jittered ring of radius ring_factor*scene_radius, looking at the origin."""
    rng = np.random.default_rng(seed)
    cams = []
    R = ring_factor * scene_radius
    for k in range(n):
        az = 2 * math.pi * k / n
        el = math.radians(rng.uniform(-elev_deg, elev_deg))
        pos = R * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        pos = pos + rng.normal(0.0, jitter * scene_radius, size=3)
        cams.append(Camera(look_at(pos), **pinhole(width, height)))
    return cams


def noise_target(n_views: int, height: int, width: int, *, seed: int = 2000) -> np.ndarray:
    """Seeded target images, float32 [V, 3, H, W], values in [0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n_views, 3, height, width)).astype(np.float32)


def smooth_target(n_views: int, height: int, width: int, *, seed: int = 2000) -> np.ndarray:
    """Seeded low-frequency target images (sum of random sinusoids), float32 [V, 3, H, W] in [0, 1]."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    out = np.empty((n_views, 3, height, width), np.float32)
    for v in range(n_views):
        for c in range(3):
            img = np.full((height, width), 0.5)
            for _ in range(4):
                kx, ky = rng.uniform(0.5, 4.0, size=2) * 2 * math.pi
                ph = rng.uniform(0, 2 * math.pi)
                img += 0.12 * np.sin(kx * xx / width + ky * yy / height + ph)
            out[v, c] = np.clip(img, 0.0, 1.0)
    return out


def projected_records(n: int, width: int, height: int, *, seed: int = 11,
                      zero_radius_frac: float = 0.1, dup_depth_frac: float = 0.1,
                      max_radius: int = 120):
    """Seeded stand-ins for projected splats, as the binning step receives them.

    Returns float32 means (x, y), int32 radii, float32 depths, the footprint
    half-extents (x, y) as packed halves (uint32, x in the low 16 bits) and the
    conics (A, B, C) as a float32 [3, n] array.  Some radii are 0 (culled), some
    centres lie off-screen, a fraction of depths are exact duplicates of others
    so that ties are exercised, the half-extents range from 0 to beyond the
    radius, with some -inf (no pixel reached) and some +inf (unbounded), and the
    conics are positive definite with correlations up to +-0.999 (and a few with
    A = 0, not positive definite).
    """
    rng = np.random.default_rng(seed)
    mx = rng.uniform(-60.0, width + 60.0, size=n).astype(np.float32)
    my = rng.uniform(-60.0, height + 60.0, size=n).astype(np.float32)
    r = np.minimum(np.ceil(np.exp(rng.normal(1.8, 0.9, size=n))), max_radius).astype(np.int32)
    r[rng.uniform(size=n) < zero_radius_frac] = 0
    depth = rng.uniform(0.25, 50.0, size=n).astype(np.float32)
    dup = rng.uniform(size=n) < dup_depth_frac
    if n > 1 and dup.any():
        depth[dup] = depth[rng.integers(0, n, size=int(dup.sum()))]
    h = (np.maximum(r, 1)[None, :] * rng.uniform(0.1, 1.4, size=(2, n))).astype(np.float16)
    kind = rng.uniform(size=n)
    h[:, kind < 0.04] = -np.inf
    h[:, (kind >= 0.04) & (kind < 0.08)] = np.inf
    h[:, (kind >= 0.08) & (kind < 0.11)] = 0.0
    bits = h.view(np.uint16).astype(np.uint32)
    ext = bits[0] | (bits[1] << np.uint32(16))
    A = np.exp(rng.uniform(np.log(2e-3), np.log(3.3), size=n))
    C = np.exp(rng.uniform(np.log(2e-3), np.log(3.3), size=n))
    rho = rng.uniform(-0.999, 0.999, size=n)
    B = -rho * np.sqrt(A * C)
    A[rng.uniform(size=n) < 0.01] = 0.0
    conic = np.stack([A, B, C]).astype(np.float32)
    return mx, my, r, depth, ext, conic


# --------------------------------------------------------------- serving
SERVED_SIZES = ((256, 256), (800, 600), (1297, 840), (1920, 1080))


def served_scene_specs(n_scenes: int = 16, *, seed: int = 5000, n_min: int = 50_000,
                       n_max: int = 2_000_000) -> list[tuple[int, int, int]]:
    """(Gaussians, width, height) of each resident scene of the served workload:
    counts log-uniform in [n_min, n_max], image size uniform over SERVED_SIZES."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_scenes)).astype(np.int64)
    sizes = rng.integers(0, len(SERVED_SIZES), n_scenes)
    return [(int(n), *SERVED_SIZES[s]) for n, s in zip(ns, sizes)]


def request_stream(n_requests: int, rate: float, n_scenes: int, n_views: int, *, seed: int = 99,
                   train_fraction: float = 0.7) -> list[tuple[float, str, int, int]]:
    """Seeded Poisson arrivals at `rate` per second: (arrival time s, kind
    'train' or 'render', scene, view), scenes and views uniform."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_requests)
    kinds = np.where(rng.uniform(size=n_requests) < train_fraction, "train", "render")
    scenes = rng.integers(0, n_scenes, n_requests)
    views = rng.integers(0, n_views, n_requests)
    t = np.cumsum(gaps)
    return [(float(a), str(k), int(s), int(v)) for a, k, s, v in zip(t, kinds, scenes, views)]
