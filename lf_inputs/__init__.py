"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

This module holds no arithmetic of the light-field sampling method. It only
draws the random parameters of the synthetic scenes and builds camera views:

* ``View``: a pinhole camera as the library and the oracle both consume it
  (eye, orthonormal right/up/forward basis and the tangents of the half field
  of view, all rounded once from FP64 to FP32; image size; output offset).
* ``draw_lobes``: the parameters of the smooth random lobe radiance field that
  stands in for the paper's path-traced light field (axes, sharpness, colours,
  and the seed of the per-texel noise). Each side evaluates the field with its
  own code.
* ``config_*``: the five workloads (small, precision, batching,
  differentiation, large) with their tables' shapes and their views.

Every draw comes from ``numpy.random.default_rng(seed)`` in a fixed order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

FOV_Y_DEG = 45.0          # vertical field of view of every camera
STEREO_HALF_IPD = 0.032   # eye offset along `right`, in units of R


@dataclass(frozen=True)
class View:
    eye: Tuple[float, float, float]
    right: Tuple[float, float, float]
    up: Tuple[float, float, float]
    forward: Tuple[float, float, float]
    tan_half_x: float
    tan_half_y: float
    width: int
    height: int
    out_offset: int = 0

    @property
    def pixels(self) -> int:
        return self.width * self.height

    def floats14(self) -> np.ndarray:
        """eye, right, up, forward, tan_half_x, tan_half_y as 14 float32."""
        return np.array(list(self.eye) + list(self.right) + list(self.up) + list(self.forward)
                        + [self.tan_half_x, self.tan_half_y], dtype=np.float32)

    def with_offset(self, off: int) -> "View":
        return View(self.eye, self.right, self.up, self.forward, self.tan_half_x,
                    self.tan_half_y, self.width, self.height, off)


def _f32(v) -> Tuple[float, ...]:
    return tuple(float(np.float32(x)) for x in v)


def _unit(v: np.ndarray) -> np.ndarray:
    return v / math.sqrt(float(v @ v))


def look_at(eye, target, width: int, height: int, fov_y_deg: float = FOV_Y_DEG,
            out_offset: int = 0) -> View:
    """Pinhole camera at `eye` looking at `target` (FP64 basis, rounded to FP32).

    forward = normalise(target - eye); right = normalise(forward x world_up) with
    world_up = +z (or +y when |forward.z| > 0.999); up = right x forward.
    """
    eye = np.asarray(eye, dtype=np.float64)
    fwd = _unit(np.asarray(target, dtype=np.float64) - eye)
    wup = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) <= 0.999 else np.array([0.0, 1.0, 0.0])
    right = _unit(np.cross(fwd, wup))
    up = np.cross(right, fwd)
    ty = math.tan(math.radians(fov_y_deg) * 0.5)
    tx = ty * width / height
    return View(_f32(eye), _f32(right), _f32(up), _f32(fwd), float(np.float32(tx)),
                float(np.float32(ty)), int(width), int(height), int(out_offset))


def stereo_pair(center, target, width: int, height: int, R: float,
                fov_y_deg: float = FOV_Y_DEG) -> Tuple[View, View]:
    """Two eyes offset by -+STEREO_HALF_IPD*R along the centre camera's `right`,
    with parallel optical axes (both keep the centre camera's basis)."""
    c = look_at(center, target, width, height, fov_y_deg)
    r = np.array(c.right, dtype=np.float64)
    ctr = np.asarray(center, dtype=np.float64)
    views = []
    for s in (-1.0, 1.0):
        e = ctr + s * STEREO_HALF_IPD * R * r
        views.append(View(_f32(e), c.right, c.up, c.forward, c.tan_half_x, c.tan_half_y,
                          width, height, 0))
    return views[0], views[1]


def pack_offsets(views: Sequence[View]) -> List[View]:
    """Assign consecutive output offsets (in pixels) in list order."""
    out, off = [], 0
    for v in views:
        out.append(v.with_offset(off))
        off += v.pixels
    return out


def total_pixels(views: Sequence[View]) -> int:
    return max((v.out_offset + v.pixels for v in views), default=0)


# --------------------------------------------------------------------------
# Lobe radiance field parameters
# --------------------------------------------------------------------------
@dataclass
class Lobes:
    seed: int
    L: int
    C: int
    ap: np.ndarray    # [L,3] unit position axes
    ad: np.ndarray    # [L,3] unit direction axes
    kp: np.ndarray    # [L] position sharpness, U[2,20]
    kd: np.ndarray    # [L] direction sharpness, U[2,20]
    col: np.ndarray   # [L,C] colours, U[0,1]
    noise_seed: int = 0


def draw_lobes(seed: int, L: int, C: int) -> Lobes:
    rng = np.random.default_rng(seed)
    ap = rng.standard_normal((L, 3))
    ad = rng.standard_normal((L, 3))
    ap /= np.linalg.norm(ap, axis=1, keepdims=True)
    ad /= np.linalg.norm(ad, axis=1, keepdims=True)
    kp = rng.uniform(2.0, 20.0, L)
    kd = rng.uniform(2.0, 20.0, L)
    col = rng.uniform(0.0, 1.0, (L, C))
    return Lobes(seed, L, C, np.ascontiguousarray(ap), np.ascontiguousarray(ad),
                 np.ascontiguousarray(kp), np.ascontiguousarray(kd),
                 np.ascontiguousarray(col), noise_seed=int(seed))


@dataclass
class Volume:
    """An analytic emission-absorption scene inside S for the light-field
    precompute: Gaussian blobs (centre, width, peak density per unit length,
    emitted RGB colour), a direction-only background bg0 + bg1 (1 + d_z) / 2,
    and the sampling controls (jittered samples per texel, midpoint steps per
    sample, generator seed)."""
    mu: np.ndarray      # [B,3] centres
    width: np.ndarray   # [B]
    dens: np.ndarray    # [B]
    emit: np.ndarray    # [B,3]
    bg0: Tuple[float, float, float] = (0.125, 0.125, 0.1875)
    bg1: Tuple[float, float, float] = (0.25, 0.375, 0.5)
    spp: int = 4
    steps: int = 64
    jitter: int = 1
    seed: int = 0
    R: float = 1.0
    O: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    @property
    def B(self) -> int:
        return len(self.width)


def draw_volume(seed: int, B: int = 8, R: float = 1.0, O=(0.0, 0.0, 0.0), spp: int = 4,
                steps: int = 64, jitter: int = 1) -> Volume:
    """B blobs: centres uniform in the ball of radius 0.6R around O, widths
    U[0.08, 0.25]R, peak densities U[2, 12]/R, colours U[0, 1]^3."""
    rng = np.random.default_rng(seed + 7000)
    u = rng.standard_normal((B, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    rad = 0.6 * R * rng.uniform(0.0, 1.0, B) ** (1.0 / 3.0)
    mu = np.asarray(O, np.float64)[None, :] + u * rad[:, None]
    width = rng.uniform(0.08, 0.25, B) * R
    dens = rng.uniform(2.0, 12.0, B) / R
    emit = rng.uniform(0.0, 1.0, (B, 3))

    def f32(a):     # parameters exactly representable in FP32 (the library's input type)
        return np.ascontiguousarray(np.asarray(a, np.float32).astype(np.float64))
    return Volume(f32(mu), f32(width), f32(dens), f32(emit), spp=spp, steps=steps, jitter=jitter,
                  seed=int(seed), R=float(R), O=tuple(float(x) for x in O))


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
@dataclass
class Config:
    name: str
    M: int
    N: int
    C: int
    L: int
    seed: int
    dtypes: Tuple[str, ...]
    views: List[View]
    R: float = 1.0
    O: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)

    @property
    def rays(self) -> int:
        return total_pixels(self.views)

    def lobes(self) -> Lobes:
        return draw_lobes(self.seed, self.L, self.C)


def _random_dir(rng) -> np.ndarray:
    return _unit(rng.standard_normal(3))


def config_small(seed: int = 0) -> Config:
    """1,024 x 256 RGB FP32, 8 lobes; one 256x256 camera at 3R on +x."""
    v = look_at((3.0, 0.0, 0.0), (0.0, 0.0, 0.0), 256, 256)
    return Config("small", 1024, 256, 3, 8, seed, ("f32",), [v])


def config_precision(seed: int = 0) -> Config:
    """65,536 x 1,024 RGBA, 16 lobes, FP32/FP16/E4M3; one 1920x1080 view at 2.5R."""
    rng = np.random.default_rng(seed + 1000)
    v = look_at(2.5 * _random_dir(rng), (0.0, 0.0, 0.0), 1920, 1080)
    return Config("precision", 65536, 1024, 4, 16, seed, ("f32", "f16", "e4m3"), [v])


def config_batching(seed: int = 0) -> Config:
    """16,384 x 512 RGBA FP16; 64 views of uneven size at distances U[1.5R, 4R]:
    16 stereo pairs 1440x1600, one 256x256, one 2048x1080, 30 random sizes."""
    rng = np.random.default_rng(seed + 2000)
    views: List[View] = []
    for _ in range(16):
        c = rng.uniform(1.5, 4.0) * _random_dir(rng)
        views.extend(stereo_pair(c, (0.0, 0.0, 0.0), 1440, 1600, 1.0))
    views.append(look_at(rng.uniform(1.5, 4.0) * _random_dir(rng), (0, 0, 0), 256, 256))
    views.append(look_at(rng.uniform(1.5, 4.0) * _random_dir(rng), (0, 0, 0), 2048, 1080))
    for _ in range(30):
        w = 8 * int(rng.integers(32, 257))
        h = 8 * int(rng.integers(32, 136))
        views.append(look_at(rng.uniform(1.5, 4.0) * _random_dir(rng), (0, 0, 0), w, h))
    return Config("batching", 16384, 512, 4, 16, seed, ("f16",), pack_offsets(views))


def config_differentiation(seed: int = 0, n_train: int = 32, n_held: int = 8) -> Config:
    """Ground truth 16,384 x 512 RGB FP32; 32 target views 512x512 plus 8 held out."""
    rng = np.random.default_rng(seed + 3000)
    views = [look_at(rng.uniform(2.0, 4.0) * _random_dir(rng), (0, 0, 0), 512, 512)
             for _ in range(n_train + n_held)]
    views = pack_offsets(views)
    return Config("differentiation", 16384, 512, 3, 8, seed, ("f32",), views,
                  extra={"n_train": n_train, "n_held": n_held, "lr": 1e-2, "steps": 500,
                         "fd_M": 256, "fd_N": 64})


def config_precompute(seed: int = 0) -> Config:
    """Light-field precompute of an analytic volume scene (8 Gaussian blobs,
    4 jittered samples per texel, 64 midpoint steps) into a 16,384 x 512 RGBA
    FP32 table (the size of the differentiation table), rendered from the
    differentiation workload's 8 held-out views."""
    d = config_differentiation(seed)
    views = pack_offsets(d.views[-8:])
    return Config("precompute", 16384, 512, 4, 8, seed, ("f32",), views,
                  extra={"volume": draw_volume(seed, B=8)})


def config_post_filter(seed: int = 0, n_train: int = 40, n_test: int = 8) -> Config:
    """Learned post-filter: n_train training and n_test held-out volume scenes
    (draw_volume with 8 blobs, 2 jittered samples per texel, 32 midpoint steps;
    seeds 100 + k and 500 + k), each with views aimed at a point within 0.2R of
    the centre from distances U[2, 4]R: 8 views of 128x128 per training scene,
    4 of 256x256 per held-out scene. The light field of each scene is a
    1,024 x 256 RGBA FP32 table; its ground truth the direct render. extra:
    "train" and "test", lists of (volume, views)."""
    rng = np.random.default_rng(seed + 9000)

    def views_of(n, size):
        vs = [look_at(rng.uniform(2.0, 4.0) * _random_dir(rng), 0.2 * rng.uniform(0, 1) * _random_dir(rng),
                      size, size) for _ in range(n)]
        return pack_offsets(vs)
    train = [(draw_volume(seed + 100 + k, B=8, spp=2, steps=32), views_of(8, 128)) for k in range(n_train)]
    test = [(draw_volume(seed + 500 + k, B=8, spp=2, steps=32), views_of(4, 256)) for k in range(n_test)]
    return Config("post_filter", 1024, 256, 4, 8, seed, ("f32",), test[0][1],
                  extra={"train": train, "test": test})


def orbit_frame(f: int, frames: int = 240, dist: float = 3.0, elev_deg: float = 20.0,
                width: int = 3840, height: int = 2160, R: float = 1.0) -> List[View]:
    """Frame f of the orbit: centre at distance `dist`, elevation 20 degrees,
    azimuth 2*pi*f/frames, as a stereo pair (left then right)."""
    az = 2.0 * math.pi * f / frames
    el = math.radians(elev_deg)
    c = dist * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return pack_offsets(list(stereo_pair(c, (0.0, 0.0, 0.0), width, height, R)))


def config_large(seed: int = 0, frame: int = 0) -> Config:
    """262,144 x 4,096 RGBA in E4M3 (4 GiB), FP16 (8 GiB), FP32 (16 GiB); one
    frame of the 240-frame orbit, a 3840x2160 stereo pair (16,588,800 rays)."""
    return Config("large", 262144, 4096, 4, 16, seed, ("e4m3", "f16", "f32"),
                  orbit_frame(frame), extra={"frames": 240, "frame": frame})


def config_paper(seed: int = 0, width: int = 1280, height: int = 720) -> Config:
    """The paper's own table shape: M = 12,288 origins of which only the upper
    hemisphere (6,144 rows) is stored, N = 23,576 directions, 4-byte texels
    (E4M3 RGBA): 0.5 x 12,288 x 23,576 x 4 B = 579,403,776 B. A stereo pair of
    1280x720 views at 2.5R, 35 degrees above the equator, looking at the centre."""
    el, az = math.radians(35.0), math.radians(30.0)
    c = 2.5 * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    views = pack_offsets(list(stereo_pair(c, (0.0, 0.0, 0.0), width, height, 1.0)))
    return Config("paper", 12288, 23576, 4, 16, seed, ("e4m3",), views, extra={"upper": True})


CONFIGS = {
    "small": config_small,
    "precision": config_precision,
    "batching": config_batching,
    "differentiation": config_differentiation,
    "large": config_large,
    "paper": config_paper,
    "precompute": config_precompute,
}


def pixel_list(views: Sequence[View], stride: int = 1) -> np.ndarray:
    """All (view, x, y) of the views, every `stride`-th in raster order: [n,3] uint32."""
    parts = []
    for vi, v in enumerate(views):
        ys, xs = np.meshgrid(np.arange(v.height, dtype=np.uint32),
                             np.arange(v.width, dtype=np.uint32), indexing="ij")
        p = np.stack([np.full(v.pixels, vi, np.uint32), xs.ravel(), ys.ravel()], axis=1)
        parts.append(p)
    allp = np.concatenate(parts) if parts else np.zeros((0, 3), np.uint32)
    return np.ascontiguousarray(allp[::stride])


def sample_pixels(views: Sequence[View], n: int, seed: int = 0) -> np.ndarray:
    """n distinct random pixels (view, x, y) drawn uniformly over all views' pixels."""
    tot = total_pixels(views)
    rng = np.random.default_rng(seed)
    flat = np.sort(rng.choice(tot, size=min(n, tot), replace=False))
    out = np.zeros((len(flat), 3), np.uint32)
    for vi, v in enumerate(views):
        m = (flat >= v.out_offset) & (flat < v.out_offset + v.pixels)
        loc = flat[m] - v.out_offset
        out[m, 0] = vi
        out[m, 1] = loc % v.width
        out[m, 2] = loc // v.width
    return out


def pixel_offsets(views: Sequence[View], pix: np.ndarray) -> np.ndarray:
    """Output-buffer pixel offset of each (view, x, y)."""
    offs = np.array([v.out_offset for v in views], np.int64)
    ws = np.array([v.width for v in views], np.int64)
    return offs[pix[:, 0]] + pix[:, 2].astype(np.int64) * ws[pix[:, 0]] + pix[:, 1]
