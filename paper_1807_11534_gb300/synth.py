"""Seeded synthetic inputs shaped like the paper's test problems.

The paper (Section 4) segments three 128x128 images with the piecewise-constant
term (Eq. CV) and the distance-selective term (Eq. DS); the images themselves
are not published, so every workload here is drawn from a seeded generator:
piecewise-constant shapes on a background plus Gaussian noise.

This module only draws inputs (image z, label mask, marker pixels, per-image
parameters).  It contains none of the method's arithmetic: no fitting term,
no domain, no iteration.  It is the one module shared by the CUDA path's
tests/benchmark and the FP64 oracle's tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One synthetic image and the parameters it is solved with."""

    z: np.ndarray                     # float32 [H, W] image
    label: np.ndarray                 # uint8 [H, W]: 1 where a dark (foreground) shape was painted
    c1: float = 0.3                   # foreground intensity constant
    c2: float = 0.7                   # background intensity constant
    markers: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))  # int32 [M, 2] (row, col)
    gamma: float = 0.0                # weight of the distance-selective term
    lam: float = 1.0
    theta: float = 0.2
    tau: float = 0.125
    iters: int = 500
    delta: float = float("inf")       # domain threshold q-hat
    q: float = -1.0                   # target restricted fraction (quantile mode when >= 0)
    name: str = ""

    @property
    def shape(self):
        return self.z.shape


def _disk(mask, cy, cx, r):
    H, W = mask.shape
    y0, y1 = max(0, int(math.floor(cy - r)) - 1), min(H, int(math.ceil(cy + r)) + 2)
    x0, x1 = max(0, int(math.floor(cx - r)) - 1), min(W, int(math.ceil(cx + r)) + 2)
    if y0 >= y1 or x0 >= x1:
        return mask
    yy, xx = np.mgrid[y0:y1, x0:x1]
    # pixel centres at integer coordinates
    inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
    mask[y0:y1, x0:x1] |= inside
    return mask


def _rect(mask, y0, x0, h, w):
    H, W = mask.shape
    a, b = max(0, int(y0)), min(H, int(y0 + h))
    c, d = max(0, int(x0)), min(W, int(x0 + w))
    if a < b and c < d:
        mask[a:b, c:d] = True
    return mask


def _ellipse(H, W, cy, cx, ay, ax, ang):
    r = max(ay, ax)
    y0, y1 = max(0, int(cy - r) - 1), min(H, int(cy + r) + 2)
    x0, x1 = max(0, int(cx - r) - 1), min(W, int(cx + r) + 2)
    if y0 >= y1 or x0 >= x1:
        return None
    yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    dy, dx = yy - cy, xx - cx
    c, s = math.cos(ang), math.sin(ang)
    u = c * dx + s * dy
    w = -s * dx + c * dy
    inside = (u / ax) ** 2 + (w / ay) ** 2 <= 1.0
    return (slice(y0, y1), slice(x0, x1), inside)


def _convex_polygon(H, W, cy, cx, radius, nv, rng):
    ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, size=nv))
    rad = radius * rng.uniform(0.6, 1.0, size=nv)
    vy = cy + rad * np.sin(ang)
    vx = cx + rad * np.cos(ang)
    y0, y1 = max(0, int(vy.min()) - 1), min(H, int(vy.max()) + 2)
    x0, x1 = max(0, int(vx.min()) - 1), min(W, int(vx.max()) + 2)
    if y0 >= y1 or x0 >= x1:
        return None
    yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    inside = np.ones(yy.shape, bool)
    # vertices sorted by angle are counter-clockwise in (x, y); keep the left side of each edge
    for k in range(nv):
        ax_, ay_ = vx[k], vy[k]
        bx_, by_ = vx[(k + 1) % nv], vy[(k + 1) % nv]
        cross = (bx_ - ax_) * (yy - ay_) - (by_ - ay_) * (xx - ax_)
        inside &= cross >= 0.0
    return (slice(y0, y1), slice(x0, x1), inside)


def shapes_image(H, W, n_shapes, size_lo, size_hi, fg=0.3, bg=0.7, sigma=0.05, seed=0):
    """Disks and rectangles (probability 1/2 each) of size U[size_lo, size_hi]
    at intensity `fg` on a background `bg`, plus N(0, sigma) noise."""
    rng = np.random.default_rng(seed)
    mask = np.zeros((H, W), bool)
    for _ in range(n_shapes):
        size = rng.uniform(size_lo, size_hi)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        if rng.random() < 0.5:
            _disk(mask, cy, cx, size / 2.0)
        else:
            h = size
            w = rng.uniform(size_lo, size_hi)
            _rect(mask, cy - h / 2, cx - w / 2, h, w)
    z = np.where(mask, fg, bg) + rng.normal(0.0, sigma, size=(H, W))
    return z.astype(np.float32), mask.astype(np.uint8)


def small_example(seed=0, H=256, W=256, iters=500, delta=float("inf")) -> Problem:
    """Single 256x256 image: 3 random disks/rectangles of size 16-64 px at
    0.3 on a 0.7 background + N(0, 0.05); c1 = 0.3, c2 = 0.7, lambda = 1."""
    z, lab = shapes_image(H, W, 3, 16, 64, 0.3, 0.7, 0.05, seed)
    return Problem(z=z, label=lab, c1=0.3, c2=0.7, lam=1.0, iters=iters, delta=delta,
                   name=f"shapes{H}x{W}_s{seed}")


def noisy_example(seed=0, H=96, W=96, sigma=0.25, iters=600) -> Problem:
    """Strong-noise case for the robust restriction: 3 disks/rectangles of
    size H/6..H/2 at 0.3 on 0.7 + N(0, sigma) (sigma = 0.25 flips the sign of
    the Chan-Vese term on about a fifth of the pixels); c1 = 0.3, c2 = 0.7,
    lambda = 2."""
    z, lab = shapes_image(H, W, 3, max(H // 6, 2), max(H // 2, 3), 0.3, 0.7, sigma, seed)
    return Problem(z=z, label=lab, c1=0.3, c2=0.7, lam=2.0, iters=iters, delta=float("inf"),
                   name=f"noisy{H}x{W}_s{seed}")


def spheres_volume(seed=0, D=64, H=64, W=64, n_spheres=12, sigma=0.1, lam=2.0, iters=200):
    """Volume [D, H, W]: `n_spheres` balls of radius U[4, 24] (scaled with the
    smallest side) at 0.3 on a 0.7 background, + N(0, sigma); label = the
    balls; c1 = 0.3, c2 = 0.7."""
    rng = np.random.default_rng(seed)
    scale = min(D, H, W) / 64.0
    zz, yy, xx = np.mgrid[:D, :H, :W]
    lab = np.zeros((D, H, W), bool)
    for _ in range(n_spheres):
        r = rng.uniform(4, 24) * max(scale, 0.1)
        cz, cy, cx = rng.uniform(0, D), rng.uniform(0, H), rng.uniform(0, W)
        lab |= (zz - cz) ** 2 + (yy - cy) ** 2 + (xx - cx) ** 2 < r * r
    z = np.where(lab, 0.3, 0.7) + rng.normal(0.0, sigma, size=(D, H, W))
    return Problem(z=z.astype(np.float32), label=lab.astype(np.uint8), c1=0.3, c2=0.7, lam=lam,
                   iters=iters, delta=float("inf"), name=f"spheres{D}x{H}x{W}_s{seed}")


def ellipses_ds(seed=0, H=2048, W=2048, n_ell=40, n_markers=20, lam=2.0, gamma=0.5,
                iters=1000, delta=float("inf")) -> Problem:
    """2048x2048 image: `n_ell` ellipses with semi-axes U[10, 120] (scaled with
    the image side) and random angle, each dark U(0.2, 0.4) or bright
    U(0.6, 0.8), painted in order on 0.7, + N(0, 0.1); `n_markers` marker
    pixels drawn uniformly inside the dark ellipses for the distance-selective
    term (Eq. DS).  c1, c2 are left to the class means of the label mask."""
    rng = np.random.default_rng(seed)
    scale = min(H, W) / 2048.0
    z = np.full((H, W), 0.7, np.float64)
    lab = np.zeros((H, W), np.uint8)
    for _ in range(n_ell):
        ay = rng.uniform(10, 120) * max(scale, 0.05)
        ax = rng.uniform(10, 120) * max(scale, 0.05)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        ang = rng.uniform(0, math.pi)
        dark = rng.random() < 0.5
        val = rng.uniform(0.2, 0.4) if dark else rng.uniform(0.6, 0.8)
        e = _ellipse(H, W, cy, cx, ay, ax, ang)
        if e is None:
            continue
        sy, sx, inside = e
        z[sy, sx] = np.where(inside, val, z[sy, sx])
        lab[sy, sx] = np.where(inside, 1 if dark else 0, lab[sy, sx])
    z = z + rng.normal(0.0, 0.1, size=(H, W))
    cand = np.flatnonzero(lab.ravel())
    if cand.size == 0:
        cand = np.arange(H * W)
    pick = rng.choice(cand, size=min(n_markers, cand.size), replace=False)
    markers = np.stack([pick // W, pick % W], axis=1).astype(np.int32)
    return Problem(z=z.astype(np.float32), label=lab, c1=float("nan"), c2=float("nan"),
                   markers=markers, gamma=gamma, lam=lam, iters=iters, delta=delta,
                   name=f"ellipsesDS{H}x{W}_s{seed}")


def polygons(seed=0, H=4096, W=4096, n_poly=200, sigma=0.08, iters=2000,
             delta=float("inf")) -> Problem:
    """4096x4096 image of `n_poly` random convex polygons (3-8 vertices,
    radius U[8, 200] scaled with the image side) at 0.3 on 0.7, + N(0, sigma);
    CV term with c1 = 0.3, c2 = 0.7."""
    rng = np.random.default_rng(seed)
    scale = min(H, W) / 4096.0
    mask = np.zeros((H, W), bool)
    for _ in range(n_poly):
        nv = int(rng.integers(3, 9))
        radius = rng.uniform(8, 200) * max(scale, 0.05)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        pg = _convex_polygon(H, W, cy, cx, radius, nv, rng)
        if pg is None:
            continue
        sy, sx, inside = pg
        mask[sy, sx] |= inside
    z = np.where(mask, 0.3, 0.7) + rng.normal(0.0, sigma, size=(H, W))
    return Problem(z=z.astype(np.float32), label=mask.astype(np.uint8), c1=0.3, c2=0.7,
                   lam=1.0, iters=iters, delta=delta, name=f"polygons{H}x{W}_s{seed}")


def batch(seed=0, n_images=64, side_lo=128, side_hi=1024, sigma=0.05, iters=500,
          q_lo=0.02, q_hi=0.40):
    """Batch of `n_images` random-shape piecewise-constant images with H and W
    drawn independently from U{side_lo..side_hi}, + N(0, sigma); each image
    gets a target restricted fraction q ~ U[q_lo, q_hi] (quantile mode)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_images):
        H = int(rng.integers(side_lo, side_hi + 1))
        W = int(rng.integers(side_lo, side_hi + 1))
        n_sh = max(2, int(H * W / 40000))
        sub = int(rng.integers(0, 2**31 - 1))
        z, lab = shapes_image(H, W, n_sh, max(8, min(H, W) // 16), max(16, min(H, W) // 4),
                              0.3, 0.7, sigma, sub)
        q = float(rng.uniform(q_lo, q_hi))
        out.append(Problem(z=z, label=lab, c1=0.3, c2=0.7, lam=1.0, iters=iters, q=q,
                           name=f"batch{k}_{H}x{W}"))
    return out


def training_batch(seed=0, n_images=8, side=1024, iters=200):
    """Batch of `n_images` side x side random-shape images with their
    generator masks as targets (differentiation workload)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_images):
        sub = int(rng.integers(0, 2**31 - 1))
        z, lab = shapes_image(side, side, max(3, side * side // 40000), side // 32, side // 4,
                              0.3, 0.7, 0.05, sub)
        out.append(Problem(z=z, label=lab, c1=0.3, c2=0.7, lam=1.0, iters=iters, delta=0.2,
                           name=f"train{k}_{side}"))
    return out


def random_state(H, W, seed=0, pmax=1.0):
    """Random dual field p with |p| <= pmax pointwise and random v in [0, 1]
    (used to test operators and warm starts)."""
    rng = np.random.default_rng(seed)
    p1 = rng.uniform(-1, 1, (H, W))
    p2 = rng.uniform(-1, 1, (H, W))
    n = np.maximum(1.0, np.sqrt(p1 * p1 + p2 * p2)) / pmax
    v = rng.uniform(0, 1, (H, W))
    return p1 / n, p2 / n, v


def disk_fitting(H, W, r, cy=None, cx=None):
    """The fitting term of the disk closed form: -1 inside radius r, +1 outside
    (this is an input f, not a fitting-term computation)."""
    cy = (H - 1) / 2.0 if cy is None else cy
    cx = (W - 1) / 2.0 if cx is None else cx
    yy, xx = np.mgrid[0:H, 0:W]
    inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
    return np.where(inside, -1.0, 1.0).astype(np.float32), inside
