"""Seeded synthetic rectified stereo scenes.

The paper evaluates on its own INDEMIND captures and on Middlebury 2014
(Sect. 4.4, Sect. 7.1); neither is available here, so every input is a
synthetic plane scene shaped like those workloads: textured planes at
integer or slanted disparities over a background plane, the right view
made by forward-warping the left view along the epipolar line (rows), with
holes in the right view filled by fresh texture.

This module is the only code shared by the oracle tests, the GPU tests and
the benchmark.  It draws random numbers and builds images; it holds none of
the matcher's arithmetic (no census, arm, cost, aggregation or WTA step).

Two albedo recipes: "fine" (uniform noise blurred with sigma 1: busy
texture, arms of one or two pixels) and "mixed" (per surface a base colour,
smooth shading and fine texture of a contrast from nearly flat to busy, as
on the walls, floors and objects of indoor frames: at 640x480 the arms
average 4 pixels, median 2, 90th percentile 17, longest 33).  Config 1 uses
"fine", configs 2-5 "mixed".

Workload recipes (seed = 2203_02300 + 1000*config + item):
  1  320x240, D=32, 4-8 fronto-parallel planes, d in [2,30], no noise.
  2  640x480, D=64, 12 slanted planes (|dd/dx|,|dd/dy| <= 0.2), d in [2,60],
     Gaussian noise sigma=2 per channel, right view gain 1.03 offset +5.
  3  32 pairs, size from {320x240, 640x480, 960x540, 1280x720},
     D = 32/64/128/128 by size, 4-16 fronto-parallel planes, sigma=2.
  4  4 camera streams (640x480 D=64, 960x540 D=96, 1280x720 D=128 x2),
     planes translating 0-3 px/frame, Poisson arrivals at 30 Hz.
  5  8 pairs 1920x1080, D=256, 32 planes + 200 discs at d in [160,250],
     sigma=3.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage

SEED_BASE = 2203_02300


@dataclasses.dataclass
class Scene:
    left: np.ndarray      # (H, W, 3) uint8, rectified left view
    right: np.ndarray     # (H, W, 3) uint8, rectified right view
    disp: np.ndarray      # (H, W) float32 ground-truth left disparity
    occluded: np.ndarray  # (H, W) bool: left pixel has no visible match
    D: int                # number of disparities searched, d in [0, D-1]

    @property
    def W(self) -> int:
        return self.left.shape[1]

    @property
    def H(self) -> int:
        return self.left.shape[0]


def seed_for(config: int, item: int = 0) -> int:
    return SEED_BASE + 1000 * config + item


def _texture(rng: np.random.Generator, h: int, w: int) -> np.ndarray:
    """Uniform u8 noise per channel, Gaussian-blurred with sigma=1 (radius 3)."""
    noise = rng.integers(0, 256, size=(h, w, 3), dtype=np.uint8).astype(np.float32)
    blurred = ndimage.gaussian_filter(noise, sigma=(1.0, 1.0, 0.0), truncate=3.0,
                                      mode="reflect")
    return blurred


# standard deviation (grey levels) of a surface's fine texture in the mixed
# recipe: from nearly flat (walls, floors: long arms) to busy
MIXED_CONTRAST = (2.0, 5.0, 12.0, 30.0)


def _mixed_texture(rng: np.random.Generator, h: int, w: int) -> np.ndarray:
    """Indoor-like albedo of one surface: a base colour (uniform in [40, 215]
    per channel), smooth shading (standard-normal noise on a grid of one node
    per 32 pixels, cubic-interpolated, scaled to a standard deviation of 10
    levels) and fine texture (standard-normal noise blurred with sigma 1,
    scaled to a contrast drawn from MIXED_CONTRAST)."""
    base = rng.uniform(40.0, 215.0, size=3).astype(np.float32)
    contrast = float(MIXED_CONTRAST[int(rng.integers(0, len(MIXED_CONTRAST)))])
    gh, gw = h // 32 + 2, w // 32 + 2
    coarse = rng.standard_normal((gh, gw, 3)).astype(np.float32)
    # per channel: the same cubic spline as one 3-D zoom with factor 1 on the
    # channel axis (identical values), without its 64-tap evaluation
    low = np.stack([ndimage.zoom(coarse[:, :, c], (h / gh, w / gw), order=3, mode="reflect", grid_mode=True)
                    for c in range(3)], axis=2)[:h, :w]
    low = low * (10.0 / (float(low.std()) + 1e-6))
    fine = ndimage.gaussian_filter(rng.standard_normal((h, w, 3)).astype(np.float32), sigma=(1.0, 1.0, 0.0),
                                   truncate=3.0, mode="reflect")
    fine = fine * (contrast / (float(fine.std()) + 1e-6))
    return base + low + fine


def _albedo(kind: str):
    return _mixed_texture if kind == "mixed" else _texture


@dataclasses.dataclass
class _Surface:
    x0: int
    y0: int
    tex: np.ndarray          # (h, w, 3) float32 plane-local albedo
    mask: np.ndarray         # (h, w) bool support inside the bounding box
    a: float = 0.0           # disparity slope along x
    b: float = 0.0           # disparity slope along y
    c: float = 0.0           # disparity at the box centre


def _rect(rng, W, H, dlo, dhi, slanted, slope, texture="fine"):
    w = int(rng.integers(max(2, W // 8), max(3, W // 2) + 1))
    h = int(rng.integers(max(2, H // 8), max(3, H // 2) + 1))
    x0 = int(rng.integers(-w // 4, W - (3 * w) // 4 + 1))
    y0 = int(rng.integers(-h // 4, H - (3 * h) // 4 + 1))
    c = float(rng.integers(dlo, dhi + 1)) if not slanted else float(rng.uniform(dlo, dhi))
    a = float(rng.uniform(-slope, slope)) if slanted else 0.0
    b = float(rng.uniform(-slope, slope)) if slanted else 0.0
    return _Surface(x0, y0, _albedo(texture)(rng, h, w), np.ones((h, w), bool), a, b, c)


def _disc(rng, W, H, dlo, dhi, texture="fine"):
    r = int(rng.integers(3, 13))
    cx = int(rng.integers(0, W))
    cy = int(rng.integers(0, H))
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    mask = (xx * xx + yy * yy) <= r * r
    c = float(rng.integers(dlo, dhi + 1))
    return _Surface(cx - r, cy - r, _albedo(texture)(rng, 2 * r + 1, 2 * r + 1), mask, 0.0, 0.0, c)


def _render(W, H, surfaces, dclip, rng, noise_sigma, gain, offset, texture="fine", fill=None):
    """Z-buffer the surfaces into the left view, forward-warp to the right view."""
    disp = np.full((H, W), -1.0, np.float32)
    left = np.zeros((H, W, 3), np.float32)
    for s in surfaces:
        h, w = s.mask.shape
        gx0, gy0 = max(s.x0, 0), max(s.y0, 0)
        gx1, gy1 = min(s.x0 + w, W), min(s.y0 + h, H)
        if gx0 >= gx1 or gy0 >= gy1:
            continue
        ly, lx = np.mgrid[gy0 - s.y0:gy1 - s.y0, gx0 - s.x0:gx1 - s.x0]
        d = s.c + s.a * (lx - (w - 1) / 2.0) + s.b * (ly - (h - 1) / 2.0)
        d = np.clip(d, dclip[0], dclip[1]).astype(np.float32)
        m = s.mask[ly, lx]
        tgt = disp[gy0:gy1, gx0:gx1]
        win = m & (d > tgt)
        tgt[win] = d[win]
        left[gy0:gy1, gx0:gx1][win] = s.tex[ly[win], lx[win]]
    assert (disp >= 0).all(), "background must cover the frame"

    # Forward warp R(x - d, y) = L(x, y); the larger disparity wins a collision.
    di = np.rint(disp).astype(np.int64)
    ys, xs = np.mgrid[0:H, 0:W]
    xr = xs - di
    inb = xr >= 0
    key = np.full((H, W), -1, np.int64)
    k_src = di * W + xs
    np.maximum.at(key, (ys[inb], xr[inb]), k_src[inb])
    right = _albedo(texture)(rng, H, W) if fill is None else fill.copy()   # fresh texture fills the holes
    filled = key >= 0
    src_x = key[filled] % W
    right[filled] = left[ys[filled], src_x]
    occluded = np.ones((H, W), bool)
    vis = inb.copy()
    vis[inb] = key[ys[inb], xr[inb]] == k_src[inb]
    occluded[vis] = False

    if noise_sigma > 0:
        left = left + rng.normal(0.0, noise_sigma, left.shape).astype(np.float32)
        right = right + rng.normal(0.0, noise_sigma, right.shape).astype(np.float32)
    left_u8 = np.clip(np.rint(left), 0, 255).astype(np.uint8)
    right_u8 = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    if gain != 1.0 or offset != 0.0:
        right_u8 = np.clip(np.rint(gain * right_u8.astype(np.float32) + offset),
                           0, 255).astype(np.uint8)
    return left_u8, right_u8, disp, occluded


def plane_scene(W: int, H: int, D: int, n_planes: int, seed: int, *,
                slanted: bool = False, slope: float = 0.2, noise_sigma: float = 0.0,
                gain: float = 1.0, offset: float = 0.0, n_discs: int = 0,
                disc_range=(160, 250), drange=None, texture: str = "fine") -> Scene:
    """A background plane plus `n_planes` rectangles (and optional discs);
    texture "fine" (blurred uniform noise) or "mixed" (indoor-like)."""
    rng = np.random.default_rng(seed)
    dlo, dhi = drange if drange is not None else (2, max(2, min(D - 2, 60 if D <= 64 else D - 2)))
    bg = _Surface(0, 0, _albedo(texture)(rng, H, W), np.ones((H, W), bool),
                  0.0, 0.0, float(dlo))
    surfaces = [bg]
    for _ in range(n_planes):
        surfaces.append(_rect(rng, W, H, dlo, dhi, slanted, slope, texture))
    for _ in range(n_discs):
        surfaces.append(_disc(rng, W, H, *disc_range, texture=texture))
    left, right, disp, occ = _render(W, H, surfaces, (dlo, dhi if not n_discs else max(dhi, disc_range[1])),
                                     rng, noise_sigma, gain, offset, texture)
    return Scene(left, right, disp, occ, D)


def config_scene(config: int, item: int = 0) -> Scene:
    """Scene `item` of workload `config` (1-5), recipe in the module docstring."""
    seed = seed_for(config, item)
    rng = np.random.default_rng(seed)
    if config == 1:
        n = int(rng.integers(4, 9))
        return plane_scene(320, 240, 32, n, seed + 7, drange=(2, 30))
    if config == 2:
        return plane_scene(640, 480, 64, 12, seed + 7, slanted=True, slope=0.2,
                           noise_sigma=2.0, gain=1.03, offset=5.0, drange=(2, 60), texture="mixed")
    if config == 3:
        sizes = [(320, 240, 32), (640, 480, 64), (960, 540, 128), (1280, 720, 128)]
        W, H, D = sizes[int(rng.integers(0, 4))]
        n = int(rng.integers(4, 17))
        return plane_scene(W, H, D, n, seed + 7, noise_sigma=2.0, drange=(2, D - 2), texture="mixed")
    if config == 5:
        return plane_scene(1920, 1080, 256, 32, seed + 7, noise_sigma=3.0,
                           n_discs=200, disc_range=(160, 250), drange=(2, 150), texture="mixed")
    raise ValueError(f"config {config} has no single-scene recipe")


def batch_config3(n: int = 32):
    return [config_scene(3, i) for i in range(n)]


STREAMS_CONFIG4 = [(640, 480, 64), (960, 540, 96), (1280, 720, 128), (1280, 720, 128)]


class StreamScene:
    """A camera stream whose planes translate 0-3 px per frame (config 4)."""

    def __init__(self, stream: int, W: int, H: int, D: int, n_planes: int = 8):
        self.W, self.H, self.D = W, H, D
        self.seed = seed_for(4, stream)
        rng = np.random.default_rng(self.seed)
        self.dlo, self.dhi = 2, D - 2
        self.bg = _mixed_texture(rng, H, W)
        self.planes = [_rect(rng, W, H, self.dlo, self.dhi, False, 0.0, "mixed") for _ in range(n_planes)]
        self.vel = []
        for _ in range(n_planes):
            speed = rng.uniform(0.0, 3.0)
            ang = rng.uniform(0.0, 2.0 * math.pi)
            self.vel.append((speed * math.cos(ang), speed * math.sin(ang)))
        self.rng = rng
        self.fill = _mixed_texture(np.random.default_rng(self.seed * 31 + 1), H, W)   # the right view's holes

    def frame(self, t: int) -> Scene:
        surfaces = [_Surface(0, 0, self.bg, np.ones((self.H, self.W), bool), 0, 0, float(self.dlo))]
        for p, (vx, vy) in zip(self.planes, self.vel):
            surfaces.append(dataclasses.replace(p, x0=p.x0 + int(round(vx * t)),
                                                y0=p.y0 + int(round(vy * t))))
        rng = np.random.default_rng(self.seed * 7919 + t)
        left, right, disp, occ = _render(self.W, self.H, surfaces, (self.dlo, self.dhi),
                                         rng, 2.0, 1.0, 0.0, "mixed", fill=self.fill)
        return Scene(left, right, disp, occ, self.D)


def poisson_arrivals(n_frames: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps of mean 1/rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n_frames))


def random_pair(W: int, H: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Two independent uniform-noise images (edge-case and ragged-size tests)."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)
    b = rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)
    return a, b
