"""Seeded synthetic scenes, cameras and loss inputs.

This module only draws inputs: splat parameters, pinhole cameras, target
images and image-gradient fields.  It holds none of the renderer's arithmetic
(no projection, blending or gradient), so the CPU oracle and the CUDA path can
both consume the same arrays without sharing any of the method's code.

All arrays are float32 (the dtype the CUDA path reads); the oracle upcasts the
same float32 values to float64, so both sides see bit-identical inputs.

Scene recipes follow the workloads of the paper's evaluation (pretrained
MipNeRF360 scenes at native resolution, Sec. 4), which are not available here;
seeded distributions of matching shape stand in for them.  Parameters are the
*activated* values: scales > 0, opacities in [0, 1], quaternions (w, x, y, z)
unnormalised, SH coefficients laid out [N, K, 3] with K = (deg + 1)^2.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Y_0^0 = 1 / (2 sqrt(pi)): used only to turn a drawn base colour into the DC
# coefficient so that SH-degree-0 splats have exactly that colour.
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclass
class Scene:
    means: np.ndarray      # [N, 3]
    scales: np.ndarray     # [N, 3]  (> 0)
    quats: np.ndarray      # [N, 4]  (w, x, y, z), unnormalised
    opacities: np.ndarray  # [N]     in [0, 1]
    sh: np.ndarray         # [N, K, 3]
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return self.means, self.scales, self.quats, self.opacities, self.sh

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacities[idx].copy(), self.sh[idx].copy(), self.sh_degree)


@dataclass
class Camera:
    viewmat: np.ndarray    # [3, 4] world -> camera [R | t]; OpenCV axes (x right, y down, z fwd)
    campos: np.ndarray     # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2
    extra: dict = field(default_factory=dict)

    def as_f64_array(self) -> np.ndarray:
        """Flat float64 view of the float32 camera values (oracle layout)."""
        v = np.zeros(22, dtype=np.float64)
        v[0:12] = self.viewmat.astype(np.float32).astype(np.float64).reshape(-1)
        v[12:15] = self.campos.astype(np.float32).astype(np.float64)
        v[15] = np.float32(self.fx)
        v[16] = np.float32(self.fy)
        v[17] = np.float32(self.cx)
        v[18] = np.float32(self.cy)
        v[19] = self.width
        v[20] = self.height
        v[21] = np.float32(self.znear)
        return v


def _normalize(v):
    return v / np.linalg.norm(v)


def look_at(eye, target, fovy_deg: float, width: int, height: int, up=(0.0, 1.0, 0.0),
            cx: float | None = None, cy: float | None = None, znear: float = 0.2) -> Camera:
    """Pinhole camera at `eye` looking at `target`; vertical field of view `fovy_deg`.

    Built in float64 and stored as float32.  Rows of R are the camera axes in
    world coordinates: z forward, x = normalize(z x up), y = z x x (y down).
    """
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    up = np.asarray(up, dtype=np.float64)
    z = _normalize(target - eye)
    x = _normalize(np.cross(z, up))
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    fy = height / (2.0 * math.tan(math.radians(fovy_deg) / 2.0))
    view = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    return Camera(viewmat=view, campos=eye.astype(np.float32), fx=float(np.float32(fy)),
                  fy=float(np.float32(fy)),
                  cx=float(np.float32(width / 2.0 if cx is None else cx)),
                  cy=float(np.float32(height / 2.0 if cy is None else cy)),
                  width=int(width), height=int(height), znear=float(np.float32(znear)))


def orbit_camera(angle: float, radius: float, fovy_deg: float, width: int, height: int,
                 **kw) -> Camera:
    """Camera on a circle of `radius` around the world y axis, looking at the origin."""
    eye = (radius * math.cos(angle), 0.0, radius * math.sin(angle))
    return look_at(eye, (0.0, 0.0, 0.0), fovy_deg, width, height, **kw)


def _random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh_from_rgb(rng, rgb, deg, hi_sigma):
    k = (deg + 1) ** 2
    sh = np.zeros((rgb.shape[0], k, 3), dtype=np.float64)
    sh[:, 0, :] = (rgb - 0.5) / _Y00
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, hi_sigma, size=(rgb.shape[0], k - 1, 3))
    return sh


def _pack(means, scales, quats, opac, sh, deg) -> Scene:
    f = np.float32
    return Scene(np.ascontiguousarray(means, dtype=f), np.ascontiguousarray(scales, dtype=f),
                 np.ascontiguousarray(quats, dtype=f), np.ascontiguousarray(opac, dtype=f),
                 np.ascontiguousarray(sh, dtype=f), int(deg))


def cube_scene(n: int, seed: int, sh_degree: int = 0, hi_sigma: float = 0.05,
               log_scale_mean: float = -3.0, log_scale_std: float = 0.5,
               extent: float = 1.0) -> Scene:
    """Tiny-scene distribution: means U[-extent, extent]^3, log-scales N(-3, 0.5),
    uniform unit quaternions, opacity sigmoid(N(0, 1)), base colour U[0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-extent, extent, size=(n, 3))
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(n, 3)))
    quats = _random_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    sh = _sh_from_rgb(rng, rgb, sh_degree, hi_sigma)
    return _pack(means, scales, quats, opac, sh, sh_degree)


def mipnerf360_like_scene(n: int, seed: int, sh_degree: int = 3, n_clusters: int = 64,
                          shell_frac: float = 0.10) -> Scene:
    """Large-scene distribution: (1 - shell_frac) of the means from a 64-cluster
    isotropic mixture (centres uniform in the radius-10 ball, cluster sigma
    U[0.05, 0.5], equal weights), the rest on a background shell of radius
    U[20, 50]; log-scales N(-4.5, 1); opacity sigmoid(N(-1, 1.5)); SH degree 3
    with DC from a U[0, 1] base colour and higher bands N(0, 0.05)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_shell = int(round(n * shell_frac))
    n_cl = n - n_shell
    # cluster centres: uniform in the ball (direction uniform, radius ~ R * u^(1/3))
    d = rng.standard_normal((n_clusters, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centres = d * (10.0 * rng.uniform(0.0, 1.0, size=(n_clusters, 1)) ** (1.0 / 3.0))
    sig = rng.uniform(0.05, 0.5, size=n_clusters)
    which = rng.integers(0, n_clusters, size=n_cl)
    cl = centres[which] + rng.standard_normal((n_cl, 3)) * sig[which, None]
    ds = rng.standard_normal((n_shell, 3))
    ds /= np.linalg.norm(ds, axis=1, keepdims=True)
    shell = ds * rng.uniform(20.0, 50.0, size=(n_shell, 1))
    means = np.concatenate([cl, shell], axis=0)
    scales = np.exp(rng.normal(-4.5, 1.0, size=(n, 3)))
    quats = _random_quats(rng, n)
    opac = _sigmoid(rng.normal(-1.0, 1.5, size=n))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    sh = _sh_from_rgb(rng, rgb, sh_degree, 0.05)
    return _pack(means, scales, quats, opac, sh, sh_degree)


def uniform_image(height: int, width: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """[H, W, 3] float32 field U[lo, hi] (targets, or dL/dC ~ U[-1, 1] as in Sec. 4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(height, width, 3)).astype(np.float32)


# ---------------------------------------------------------------------------
# Named workloads (sizes and distributions of the five benchmark settings)
# ---------------------------------------------------------------------------

def tiny_scene_1k():
    """1,024 splats, SH0, camera (0,0,-4) -> origin, 60 deg vertical FOV, 128x128."""
    scene = cube_scene(1024, seed=1, sh_degree=0)
    cam = look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 60.0, 128, 128)
    target = uniform_image(128, 128, seed=101)
    return scene, cam, target


def mipnerf_scene_3m(n: int = 3_000_000):
    """3.0M splats (cluster mixture + shell, SH3), radius-4 orbit camera, 50 deg FOV, 1256x828."""
    scene = mipnerf360_like_scene(n, seed=2)
    cam = orbit_camera(0.0, 4.0, 50.0, 1256, 828)
    target = uniform_image(828, 1256, seed=102)
    return scene, cam, target


def precision_sweep_views(n_views: int = 8):
    """Tiny scene seen from eight radius-4 orbit angles (seeded), 60 deg FOV, 128x128."""
    scene = cube_scene(1024, seed=1, sh_degree=0)
    rng = np.random.Generator(np.random.PCG64(3))
    angles = rng.uniform(0.0, 2.0 * math.pi, size=n_views)
    cams = [orbit_camera(float(a), 4.0, 60.0, 128, 128) for a in angles]
    return scene, cams


def training_scene_1m(n: int = 1_000_000, width: int = 1600, height: int = 1060, n_views: int = 8):
    """1.0M splats (tiny-scene distributions, SH3), 8 orbit cameras at 2*pi*k/8, 60 deg FOV."""
    scene = cube_scene(n, seed=4, sh_degree=3)
    cams = [orbit_camera(2.0 * math.pi * k / n_views, 4.0, 60.0, width, height)
            for k in range(n_views)]
    targets = [uniform_image(height, width, seed=400 + k) for k in range(n_views)]
    return scene, cams, targets


def gradcheck_subscene(seed: int = 44, n: int = 64, size: int = 32, sh_degree: int = 3):
    """64 splats seen at 32x32 (finite-difference sub-scene)."""
    scene = cube_scene(n, seed=seed, sh_degree=sh_degree, log_scale_mean=-2.0)
    cam = look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 40.0, size, size)
    return scene, cam


SERVING_SCENE_SIZES = (500_000, 1_500_000, 3_000_000, 6_000_000)
SERVING_RESOLUTIONS = ((640, 360), (1256, 828), (1920, 1080), (3840, 2160))


def serving_requests(n_requests: int = 2000, rate_hz: float = 200.0, seed: int = 5,
                     bwd_frac: float = 0.2):
    """Poisson arrivals over the four resident scenes, resolutions drawn uniformly,
    `bwd_frac` of the requests being fwd+bwd fine-tune steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps)
    scene_idx = rng.integers(0, len(SERVING_SCENE_SIZES), size=n_requests)
    res_idx = rng.integers(0, len(SERVING_RESOLUTIONS), size=n_requests)
    is_bwd = rng.uniform(0.0, 1.0, size=n_requests) < bwd_frac
    angles = rng.uniform(0.0, 2.0 * math.pi, size=n_requests)
    out = []
    for i in range(n_requests):
        w, h = SERVING_RESOLUTIONS[res_idx[i]]
        out.append(dict(arrival=float(arrivals[i]), scene=int(scene_idx[i]), width=w, height=h,
                        backward=bool(is_bwd[i]), angle=float(angles[i])))
    return out
