"""Seeded synthetic stereo pairs shaped like the paper's workloads.

This module only draws inputs; it holds none of the matching arithmetic and
serves the CUDA path and the CPU oracle alike.  The paper evaluates on KITTI
Stereo 2015 crops and live camera streams (Sec. 4); neither is available, so
rectified pairs are synthesised with a known ground-truth disparity:

* random numbers come from SplitMix64 (Steele, Lea, Flood 2014) used as a
  counter-based generator, ``u_i = mix(seed + i * 0x9E3779B97F4A7C15)``, so
  every machine draws the same bytes;
* Gaussian noise is the Irwin-Hall sum of twelve uniforms minus six (only
  additions and multiplications, hence bit-identical everywhere);
* the right image is the left image forward-warped by the ground-truth
  disparity (x_r = x - d) with a z-buffer (larger disparity wins); right
  pixels nothing maps to get fresh texture.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """SplitMix64 stream; ``draw(n)`` returns the next n 64-bit outputs."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def draw(self, n: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + n + 1, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            return _mix(self.seed + idx * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits."""
        return (self.draw(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform in [lo, hi] (inclusive)."""
        return (lo + np.floor(self.uniform(n) * (hi - lo + 1))).astype(np.int64)

    def integer(self, lo: int, hi: int) -> int:
        return int(self.integers(lo, hi, 1)[0])

    def normal(self, n: int) -> np.ndarray:
        u = self.uniform(12 * n).reshape(n, 12)
        acc = np.zeros(n)
        for j in range(12):
            acc = acc + u[:, j]
        return acc - 6.0


def blur_texture(rng: Rng, W: int, H: int) -> np.ndarray:
    """Uniform [0,255] noise smoothed by a 3x3 box, floor((sum + 4) / 9), clamped borders."""
    t = rng.integers(0, 255, W * H).reshape(H, W)
    p = np.pad(t, 1, mode="edge")
    s = sum(p[1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    return ((s + 4) // 9).astype(np.uint8)


def value_noise(rng: Rng, W: int, H: int, cell: int = 8) -> np.ndarray:
    """Integer value noise: random lattice values every ``cell`` pixels,
    bilinear weights in 1/cell^2 steps; a fine octave (cell/4) adds detail."""
    def octave(c: int) -> np.ndarray:
        gw, gh = W // c + 2, H // c + 2
        g = rng.integers(0, 255, gw * gh).reshape(gh, gw)
        y, x = np.mgrid[0:H, 0:W]
        i, fx = x // c, x % c
        j, fy = y // c, y % c
        v = ((c - fx) * (c - fy) * g[j, i] + fx * (c - fy) * g[j, i + 1]
             + (c - fx) * fy * g[j + 1, i] + fx * fy * g[j + 1, i + 1])
        return (v + c * c // 2) // (c * c)
    coarse = octave(cell)
    fine = octave(max(cell // 4, 1))
    return ((3 * coarse + fine + 2) // 4).astype(np.uint8)


def warp_right(left: np.ndarray, gt: np.ndarray, fresh: np.ndarray) -> np.ndarray:
    """Forward-warp the left image to the right view: right(x - d, y) = left(x, y);
    where several left pixels land on one right pixel the largest d wins."""
    H, W = left.shape
    y, x = np.mgrid[0:H, 0:W]
    d = gt.astype(np.int64)
    xr = x - d
    ok = xr >= 0
    zbuf = np.full((H, W), -1, np.int64)
    np.maximum.at(zbuf, (y[ok], xr[ok]), d[ok])
    win = ok.copy()
    win[ok] = zbuf[y[ok], xr[ok]] == d[ok]
    right = fresh.copy()
    right[y[win], xr[win]] = left[win]
    return right


def add_noise(rng: Rng, img: np.ndarray, sigma: float) -> np.ndarray:
    if sigma <= 0:
        return img.copy()
    n = np.rint(sigma * rng.normal(img.size)).astype(np.int64).reshape(img.shape)
    return np.clip(img.astype(np.int64) + n, 0, 255).astype(np.uint8)


@dataclass
class Scene:
    left: np.ndarray
    right: np.ndarray
    # ground-truth disparity of the left image, int16; -1 where ground_scene's
    # occlusion mask replaced the match.  Pixels hidden in the right view by a
    # nearer surface keep their own disparity.
    gt: np.ndarray
    meta: dict = field(default_factory=dict)


def _texture(rng: Rng, W: int, H: int, kind: str) -> np.ndarray:
    return blur_texture(rng, W, H) if kind == "blur" else value_noise(rng, W, H)


def boxes_scene(W: int, H: int, D: int, seed: int, n_boxes: int = 4, background: int = 4,
                dlo: int = 4, dhi: int = 60, texture: str = "blur", sigma: float = 1.0) -> Scene:
    """Fronto-parallel rectangles of constant disparity over a constant background."""
    rng = Rng(seed)
    gt = np.full((H, W), background, np.int64)
    for _ in range(n_boxes):
        d = rng.integer(dlo, min(dhi, D - 1))
        bw, bh = rng.integer(W // 8, W // 3), rng.integer(H // 8, H // 3)
        x0, y0 = rng.integer(0, W - bw), rng.integer(0, H - bh)
        region = gt[y0:y0 + bh, x0:x0 + bw]
        np.maximum(region, d, out=region)
    left = _texture(rng, W, H, texture)
    right = warp_right(left, gt, _texture(rng, W, H, texture))
    right = add_noise(rng, right, sigma)
    return Scene(left, right, gt.astype(np.int16), {"kind": "boxes", "seed": seed})


def ground_scene(W: int, H: int, D: int, seed: int, n_obstacles: int, bands=None,
                 dlo: int = 20, dhi: int = 110, texture: str = "value", sigma: float = 2.0,
                 occlusion: float = 0.0, horizon_frac: float = 0.4, bottom_frac: float = 0.7) -> Scene:
    """Ground plane (disparity 0 at the horizon row, bottom_frac*D at the last row,
    linear in between; 0 above the horizon) with box obstacles of constant
    disparity standing on it.  ``bands`` lists (lo, hi) ranges the obstacle
    disparities are drawn from in turn; otherwise they are uniform in [dlo, dhi].
    A Bernoulli(``occlusion``) subset of left pixels has its right-image match
    overwritten with fresh texture."""
    rng = Rng(seed)
    hz = int(round(horizon_frac * H))
    dbot = int(round(bottom_frac * D))
    y = np.arange(H)
    ground = np.where(y <= hz, 0, np.rint(dbot * (y - hz) / max(H - 1 - hz, 1))).astype(np.int64)
    gt = np.repeat(ground[:, None], W, axis=1)
    for k in range(n_obstacles):
        if bands:
            lo, hi = bands[k % len(bands)]
        else:
            lo, hi = dlo, dhi
        d = rng.integer(lo, min(hi, D - 1))
        foot = hz + int(round(d / max(dbot, 1) * (H - 1 - hz)))
        foot = min(max(foot, hz + 1), H - 1)
        bh = max(4, int(round(d * rng.integer(60, 140) / 100.0 * H / 375.0)))
        bw = max(4, int(round(d * rng.integer(40, 120) / 100.0 * W / 1242.0 * 2)))
        bw = min(bw, W // 2)
        x0 = rng.integer(0, W - bw)
        y0 = max(0, foot - bh)
        region = gt[y0:foot + 1, x0:x0 + bw]
        np.maximum(region, d, out=region)
    left = _texture(rng, W, H, texture)
    right = warp_right(left, gt, _texture(rng, W, H, texture))
    gt_out = gt.copy()
    if occlusion > 0:
        mask = rng.uniform(W * H).reshape(H, W) < occlusion
        yy, xx = np.nonzero(mask)
        xr = xx - gt[yy, xx]
        ok = xr >= 0
        fresh = _texture(rng, W, H, texture)
        right[yy[ok], xr[ok]] = fresh[yy[ok], xr[ok]]
        gt_out[yy, xx] = -1
    right = add_noise(rng, right, sigma)
    return Scene(left, right, gt_out.astype(np.int16), {"kind": "ground", "seed": seed})


def shifted_pair(W: int, H: int, d: int, seed: int, texture: str = "blur") -> Scene:
    """Right image = left image shifted by a constant d (no noise): right(x) = left(x + d)."""
    rng = Rng(seed)
    left = _texture(rng, W, H, texture)
    right = _texture(rng, W, H, texture)
    right[:, : W - d] = left[:, d:]
    gt = np.full((H, W), d, np.int16)
    return Scene(left, right, gt, {"kind": "shift", "d": d, "seed": seed})


# ---------------------------------------------------------------------------
# Workload presets.  Seeds are 1807 + workload index + pair index.
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    W: int
    H: int
    D: int
    census_w: int
    census_h: int
    path_mask: int
    P1: int
    P2: int
    lr_tol: int
    median_k: int
    uv: bool
    cost: int = 0  # 0: census Hamming distance, 1: SAD over the same window

    @property
    def de_per_frame(self) -> int:
        return self.W * self.H * self.D


PATHS_4 = 0x0F
PATHS_8 = 0xFF
PATHS_STREAM4 = 0x55

# 320x240, D=64, 5x5 census, 4 paths (L->R, R->L, T->B, B->T), P1=4, P2=24.
SMALL_320 = Workload("pair-320x240-d64-census5x5-4path", 320, 240, 64, 5, 5, PATHS_4, 4, 24, 1, 5, True)
# KITTI-shaped 1242x375, D=128, 9x7 census (62 bits), 8 paths, P1=8, P2=96, LR tol 1, 3x3 median.
KITTI_1242 = Workload("kitti-1242x375-d128-census9x7-8path", 1242, 375, 128, 9, 7, PATHS_8, 8, 96, 1, 3, True)
# 1280x720, D=128, the 320x240 parameter set plus U/V maps.
HD_1280 = Workload("hd-1280x720-d128-census5x5-4path-uv", 1280, 720, 128, 5, 5, PATHS_4, 4, 24, 1, 5, True)
# The paper's own setting (Sec. 4.1): 640x360, d in [0,60), 5x5 census, the four
# streaming paths, P1=8, P2=32, 5x5 median.
PAPER_640 = Workload("paper-640x360-d60-census5x5-stream4", 640, 360, 60, 5, 5, PATHS_STREAM4, 8, 32, 1, 5, True)
# The same setting with the paper's other matching cost (Sec. 4.1): 5x5 SAD,
# P1=200, P2=800.
PAPER_640_SAD = Workload("paper-640x360-d60-sad5x5-stream4", 640, 360, 60, 5, 5, PATHS_STREAM4, 200, 800,
                         1, 5, True, cost=1)

WORKLOADS = {w.name: w for w in (SMALL_320, KITTI_1242, HD_1280, PAPER_640, PAPER_640_SAD)}


def scene_for(w: Workload, seed: int) -> Scene:
    """The synthetic scene recipe that goes with each workload."""
    if w is SMALL_320 or (w.W, w.H) == (320, 240):
        return boxes_scene(w.W, w.H, w.D, seed, n_boxes=4, background=4, dlo=4, dhi=60,
                           texture="blur", sigma=1.0)
    if w is KITTI_1242:
        return ground_scene(w.W, w.H, w.D, seed, n_obstacles=6, dlo=20, dhi=110,
                            texture="value", sigma=2.0, occlusion=0.05)
    if w is HD_1280:
        return ground_scene(w.W, w.H, w.D, seed, n_obstacles=10,
                            bands=[(20, 30), (50, 60), (90, 100)], texture="blur", sigma=1.0)
    if w is PAPER_640 or w is PAPER_640_SAD:
        return boxes_scene(w.W, w.H, w.D, seed, n_boxes=4, background=4, dlo=4, dhi=55,
                           texture="blur", sigma=1.0)
    return ground_scene(w.W, w.H, w.D, seed, n_obstacles=6, dlo=max(1, w.D // 6),
                        dhi=max(2, (w.D * 6) // 7), texture="value", sigma=2.0, occlusion=0.05)


def workload_seed(index: int, pair: int = 0) -> int:
    return 1807 + index + pair
