"""Seeded synthetic 3DGS scenes and camera rigs.

This module only builds inputs.  It holds none of the importance-score
arithmetic, so both the CUDA path and the FP64 oracle can consume what it
produces without sharing any of the method's code.

Primitive layout (Eq. 1 of the paper: G_i = (mu, s, q, c, alpha), 59 numbers)
is structure-of-arrays, one row per parameter:

  rows 0-2    mean xyz                      (``pos``, always float32)
  rows 3-5    log-scale                     (``attr`` rows 0-2)
  rows 6-9    rotation quaternion (w,x,y,z) (``attr`` rows 3-6)
  row  10     opacity logit                 (``attr`` row 7)
  rows 11-13  SH DC (r,g,b)                 (``attr`` rows 8-10)
  rows 14-58  SH degree 1..3, 15 coefficients x 3 channels, channel-major
                                            (``attr`` rows 11-55)

``attr`` is float32, or bfloat16 bit patterns (uint16) for the BF16 storage
form.  Cameras are a numpy structured array whose records are byte-identical
to ``refine_camera`` in ``include/refine.h`` (80 bytes each, OpenCV axes:
x right, y down, z forward; R and t map world to camera).

The recipes follow the synthetic stand-ins for MipNeRF360 / Tanks&Temples /
Deep Blending scenes: random draws happen in the order
means -> log-scales -> quaternions -> opacity logits -> SH DC -> SH rest ->
cameras, all from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_PARAMS = 59
N_ATTR = 56  # rows 3..58

CAMERA_DTYPE = np.dtype(
    [
        ("R", "<f4", (9,)),
        ("t", "<f4", (3,)),
        ("fx", "<f4"),
        ("fy", "<f4"),
        ("cx", "<f4"),
        ("cy", "<f4"),
        ("width", "<i4"),
        ("height", "<i4"),
        ("znear", "<f4"),
        ("zfar", "<f4"),
    ]
)
assert CAMERA_DTYPE.itemsize == 80

RESOLUTIONS = ((960, 540), (1297, 840), (1600, 1063))


@dataclasses.dataclass
class Scene:
    """A scene in SoA form. ``pos`` is float32 [3, n]; ``attr`` is float32
    [56, n] (``dtype == 'f32'``), uint16 bfloat16 bits [56, n]
    (``dtype == 'bf16'``), or float32 [56, n] whose rows 3..55 hold
    bfloat16-rounded values and rows 0..2 (log-scales) float32 values
    (``dtype == 'bf16s'``, the storage form with float32 log-scales)."""

    pos: np.ndarray
    attr: np.ndarray
    dtype: str = "f32"

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])

    def attr_f32(self) -> np.ndarray:
        """Attributes widened to float32 (exact for both storage forms)."""
        if self.dtype in ("f32", "bf16s"):
            return self.attr
        return bf16_bits_to_f32(self.attr)

    def params_f64(self) -> np.ndarray:
        """All 59 rows as float64 [59, n] -- an exact widening of what is
        stored, used to feed the oracle the very same numbers."""
        out = np.empty((N_PARAMS, self.n), dtype=np.float64)
        out[:3] = self.pos
        out[3:] = self.attr_f32()
        return out

    def subset(self, idx: np.ndarray) -> "Scene":
        return Scene(np.ascontiguousarray(self.pos[:, idx]),
                     np.ascontiguousarray(self.attr[:, idx]), self.dtype)

    def to_bf16(self) -> "Scene":
        if self.dtype == "bf16":
            return self
        return Scene(self.pos.copy(), f32_to_bf16_bits(self.attr_f32()), "bf16")

    def to_bf16s(self) -> "Scene":
        """Log-scale rows kept float32, the other 53 rows rounded to bfloat16."""
        if self.dtype == "bf16s":
            return self
        a = np.array(self.attr_f32(), dtype=np.float32, copy=True)
        a[3:] = bf16_bits_to_f32(f32_to_bf16_bits(a[3:]))
        return Scene(self.pos.copy(), a, "bf16s")


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round-to-nearest-even), returning the bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    rounding = ((b >> 16) & 1) + np.uint32(0x7FFF)
    return ((b + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


# ---------------------------------------------------------------- Gaussians

def _draw_gaussians(rng: np.random.Generator, n: int, means: str) -> Scene:
    if means == "normal2":
        # per axis N(0, 2^2), clipped to +-6
        mu = np.clip(rng.normal(0.0, 2.0, size=(3, n)), -6.0, 6.0)
    elif means == "core_shell":
        # 70% N(0, 1.5^2) core, 30% shell of radius U(6, 10), uniform direction
        is_core = rng.random(n) < 0.7
        core = rng.normal(0.0, 1.5, size=(3, n))
        d = rng.normal(size=(3, n))
        d /= np.maximum(np.linalg.norm(d, axis=0, keepdims=True), 1e-12)
        rad = rng.uniform(6.0, 10.0, size=n)
        mu = np.where(is_core[None, :], core, d * rad[None, :])
    else:
        raise ValueError(means)
    logscale = rng.normal(-4.5, 1.0, size=(3, n))
    q = rng.normal(size=(4, n))
    q /= np.maximum(np.linalg.norm(q, axis=0, keepdims=True), 1e-12)
    logit = rng.normal(0.0, 2.0, size=(1, n))
    dc = rng.normal(0.0, 0.5, size=(3, n))
    rest = rng.standard_normal(size=(45, n), dtype=np.float32) * np.float32(0.1)
    attr = np.empty((N_ATTR, n), dtype=np.float32)
    attr[0:3] = logscale
    attr[3:7] = q
    attr[7:8] = logit
    attr[8:11] = dc
    attr[11:56] = rest
    return Scene(np.ascontiguousarray(mu, dtype=np.float32), attr, "f32")


# ------------------------------------------------------------------ cameras

def look_at(center, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World-to-camera (R, t) for a camera at ``center`` looking at
    ``target`` with OpenCV axes (x right, y down, z forward) in a z-up world.
    Falls back to up = +y when the view direction is parallel to ``up``."""
    c = np.asarray(center, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    up = np.asarray(up, dtype=np.float64)
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])  # rows: x (right), y (down), z (forward)
    t = -R @ c
    return R, t


def make_cameras(centers, width, height, focal, znear=0.01, zfar=100.0):
    cams = np.zeros(len(centers), dtype=CAMERA_DTYPE)
    for k, c in enumerate(centers):
        R, t = look_at(c)
        cams[k]["R"] = R.reshape(-1)
        cams[k]["t"] = t
    cams["fx"] = focal
    cams["fy"] = focal
    cams["cx"] = width / 2.0
    cams["cy"] = height / 2.0
    cams["width"] = width
    cams["height"] = height
    cams["znear"] = znear
    cams["zfar"] = zfar
    return cams


def ring_centers(v, radius=4.0, height=1.0):
    th = 2.0 * math.pi * np.arange(v) / v
    return np.stack([radius * np.cos(th), radius * np.sin(th), np.full(v, height)], axis=1)


def hemisphere_centers(rng, v, rmin=3.5, rmax=4.5):
    d = rng.normal(size=(v, 3))
    d[:, 2] = np.abs(d[:, 2])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(rmin, rmax, size=v)
    return d * r[:, None]


# ------------------------------------------------------------------ recipes

@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cams: np.ndarray
    ratios: tuple

    @property
    def pairs(self) -> int:
        return self.scene.n * len(self.cams)


def config0(seed: int = 0, n: int = 10_000, v: int = 16) -> Workload:
    """Small plain-FP32 scene: N=10k, 16 views on a ring of radius 4 at
    height 1, 640x480, f=512."""
    rng = np.random.default_rng(seed)
    sc = _draw_gaussians(rng, n, "normal2")
    cams = make_cameras(ring_centers(v), 640, 480, 512.0)
    return Workload(f"small N={n} V={v} 640x480", sc, cams, (0.5,))


def config_core_shell(seed: int, n: int, v: int, width: int, height: int,
                      focal: float = 1100.0) -> Workload:
    rng = np.random.default_rng(seed)
    sc = _draw_gaussians(rng, n, "core_shell")
    cams = make_cameras(hemisphere_centers(rng, v), width, height, focal)
    return Workload(f"core-shell N={n} V={v} {width}x{height}", sc, cams, ())


def config1(seed: int = 1, n: int = 1_000_000, v: int = 150) -> Workload:
    w = config_core_shell(seed, n, v, 1297, 840)
    w.ratios = (0.5, 0.66, 0.9)
    return w


def config2(seed: int = 2, n: int = 3_500_000, v: int = 250, dtype: str = "f32") -> Workload:
    w = config_core_shell(seed, n, v, 1600, 1063)
    w.ratios = (0.5,)
    if dtype == "bf16":
        w.scene = w.scene.to_bf16()
    elif dtype == "bf16s":
        w.scene = w.scene.to_bf16s()
    return w


def batch_scene(seed: int, nmin: int = 50_000, nmax: int = 2_000_000,
                dtype: str = "bf16") -> Workload:
    """One scene of the 64-scene batching workload (seeds 100..163): N
    log-uniform in [nmin, nmax], V uniform in 50..300, resolution drawn from
    RESOLUTIONS, core-shell distributions, BF16 storage."""
    rng = np.random.default_rng(seed)
    n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
    v = int(rng.integers(50, 301))
    wh = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
    sc = _draw_gaussians(rng, n, "core_shell")
    cams = make_cameras(hemisphere_centers(rng, v), wh[0], wh[1], 1100.0)
    if dtype == "bf16":
        sc = sc.to_bf16()
    elif dtype == "bf16s":
        sc = sc.to_bf16s()
    return Workload(f"batch seed={seed} N={n} V={v} {wh[0]}x{wh[1]}", sc, cams, (0.66,))


def job_arrivals(n_jobs: int = 2000, rate: float = 20.0, seed: int = 999) -> np.ndarray:
    """Poisson arrival times (seconds) of the serving workload."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))


def job_spec(seed: int):
    """(N, V, (w, h), ratio) of serving job ``seed`` (seeds 1000..2999)
    without drawing the Gaussians."""
    rng = np.random.default_rng(seed)
    n = int(round(math.exp(rng.uniform(math.log(50_000), math.log(3_500_000)))))
    v = int(rng.integers(50, 301))
    wh = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
    ratio = (0.5, 0.66, 0.9)[int(rng.integers(0, 3))]
    return n, v, wh, ratio


def job_scene(seed: int, dtype: str = "bf16", n_override: int | None = None) -> Workload:
    n, v, wh, ratio = job_spec(seed)
    if n_override is not None:
        n = n_override
    rng = np.random.default_rng(seed + 1_000_000)
    sc = _draw_gaussians(rng, n, "core_shell")
    cams = make_cameras(hemisphere_centers(rng, v), wh[0], wh[1], 1100.0)
    if dtype == "bf16":
        sc = sc.to_bf16()
    elif dtype == "bf16s":
        sc = sc.to_bf16s()
    return Workload(f"job seed={seed} N={n} V={v}", sc, cams, (ratio,))


def random_scene(seed: int, n: int, v: int, width: int = 640, height: int = 480,
                 focal: float = 512.0, means: str = "normal2") -> Workload:
    """Small scene with ``v`` cameras on the z>=0 hemisphere (for ragged-size
    tests)."""
    rng = np.random.default_rng(seed)
    sc = _draw_gaussians(rng, n, means)
    cams = make_cameras(hemisphere_centers(rng, v), width, height, focal)
    return Workload(f"random seed={seed} N={n} V={v}", sc, cams, (0.5,))
