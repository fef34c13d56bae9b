"""Seeded synthetic inputs: cartoon images, textures, noise and masks.

This module holds no shearlet arithmetic.  Both the CUDA path's tests and
the FP64 oracle consume the arrays it returns, so it stays numpy-only and
imports nothing else from this package.

The images stand in for the paper's test images (the flower image of
Sec. 4.1 and the unnamed 512 x 512 images of Sec. 4.2-4.3), which are not
available: piecewise-constant "cartoons" whose edges are curves, the image
class shearlets are designed for.

Recipes (``numpy.random.default_rng(seed)``, PCG64):

* ``ellipses``: ``n`` filled ellipses, centres U[0, N)^2, semi-axes
  U[N/16, N/4], angle U[0, pi), intensity U[0, 1], painted in order (later
  ones overwrite), background 0.
* ``cartoon``: U{12..20} shapes, each an ellipse or (probability 1/2) a
  convex polygon of U{3..7} vertices on a circle of radius U[N/16, N/4]
  around a centre U[0, N)^2, intensity U[0, 1].
* ``texture``: ``0.1 sum_{q=1..3} sin(2 pi (u_q . x) / N + phi_q)`` with
  integer frequency vectors of norm in [8, 32] and phi_q ~ U[0, 2 pi).
* ``cartoon_texture``: ``clip(cartoon + texture, 0, 1)``.
* ``bernoulli_mask``: i.i.d. keep-probability p (1 = observed pixel).
* ``square_mask``: the "squared" occlusion pattern of the inpainting
  experiments (whose exact layout the paper does not give): U{count}
  axis-aligned squares of side U{N/32..N/8}, top-left corners U[0, N-side]^2,
  set to 0 (missing); about 16 % of the pixels at the defaults.
* ``gaussian_noise``: i.i.d. N(0, sigma^2).
* ``shepp_logan``: the modified Shepp-Logan head phantom (Toft's published
  table of ten ellipses, values in [0, 1]), the test object of Sec. 4.4,
  on the square [-1, 1]^2 (row index = y).
* ``random_ellipses``: the training objects of Sec. 4.4 ("randomly
  generated ellipses"; the recipe is a reading): U{3..10} ellipses with
  centre radius U[0, 0.6] at angle U[0, 2 pi), semi-axes U[0.05, 0.45],
  rotation U[0, pi), value U[0.1, 0.6] and negative with probability 0.3,
  summed and clipped to [0, 1].
* ``ellipse_phantom``: pixel averages (``supersample``^2 point samples per
  pixel) of a table of (value, a, b, x0, y0, alpha) ellipses on the
  N x N grid of pixel side 2/N covering [-1, 1]^2.
"""

from __future__ import annotations

import numpy as np


def _coords(n: int, m: int):
    y, x = np.mgrid[0:n, 0:m]
    return y.astype(np.float64), x.astype(np.float64)


def _box(n, m, cy, cx, r):
    """Index ranges of the grid points within distance r of (cy, cx)."""
    y0, y1 = max(0, int(np.floor(cy - r)) - 1), min(n, int(np.ceil(cy + r)) + 2)
    x0, x1 = max(0, int(np.floor(cx - r)) - 1), min(m, int(np.ceil(cx + r)) + 2)
    return slice(y0, y1), slice(x0, x1)


def _paint_ellipse(img, rng, y, x):
    n, m = img.shape
    s = min(n, m)
    cy, cx = rng.uniform(0, n), rng.uniform(0, m)
    a, b = rng.uniform(s / 16, s / 4), rng.uniform(s / 16, s / 4)
    th = rng.uniform(0, np.pi)
    val = rng.uniform(0, 1)
    sy, sx = _box(n, m, cy, cx, max(a, b))      # only points that can be inside
    dy, dx = y[sy, sx] - cy, x[sy, sx] - cx
    u = dx * np.cos(th) + dy * np.sin(th)
    v = -dx * np.sin(th) + dy * np.cos(th)
    sub = img[sy, sx]
    sub[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = val


def _paint_polygon(img, rng, y, x):
    n, m = img.shape
    s = min(n, m)
    cy, cx = rng.uniform(0, n), rng.uniform(0, m)
    r = rng.uniform(s / 16, s / 4)
    nv = int(rng.integers(3, 8))
    ang = np.sort(rng.uniform(0, 2 * np.pi, size=nv))
    val = rng.uniform(0, 1)
    vy, vx = cy + r * np.sin(ang), cx + r * np.cos(ang)
    sy, sx = _box(n, m, cy, cx, r)              # the polygon lies in its circle
    yy, xx = y[sy, sx], x[sy, sx]
    inside = np.ones(yy.shape, dtype=bool)
    for k in range(nv):
        y0, x0 = vy[k], vx[k]
        y1, x1 = vy[(k + 1) % nv], vx[(k + 1) % nv]
        # counter-clockwise vertices: interior on the left of each edge
        cross = (x1 - x0) * (yy - y0) - (y1 - y0) * (xx - x0)
        inside &= cross >= 0
    sub = img[sy, sx]
    sub[inside] = val


def ellipses(n: int, m: int | None = None, count: int = 8, seed: int = 1):
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    y, x = _coords(n, m)
    img = np.zeros((n, m))
    for _ in range(count):
        _paint_ellipse(img, rng, y, x)
    return img


def cartoon(n: int, m: int | None = None, seed: int = 0):
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    y, x = _coords(n, m)
    img = np.zeros((n, m))
    for _ in range(int(rng.integers(12, 21))):
        if rng.uniform() < 0.5:
            _paint_ellipse(img, rng, y, x)
        else:
            _paint_polygon(img, rng, y, x)
    return img


def texture(n: int, m: int | None = None, seed: int = 0):
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    y, x = _coords(n, m)
    out = np.zeros((n, m))
    for _ in range(3):
        while True:
            u = rng.integers(-32, 33, size=2)
            if 8 <= np.hypot(u[0], u[1]) <= 32:
                break
        phi = rng.uniform(0, 2 * np.pi)
        out += 0.1 * np.sin(2 * np.pi * (u[0] * y / n + u[1] * x / m) + phi)
    return out


def cartoon_texture(n: int, m: int | None = None, seed: int = 0):
    m = n if m is None else m
    return np.clip(cartoon(n, m, seed) + texture(n, m, seed + 7919), 0.0, 1.0)


def bernoulli_mask(n: int, m: int | None = None, p: float = 0.5, seed: int = 0):
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    return (rng.uniform(size=(n, m)) < p).astype(np.float64)


def square_mask(n: int, m: int | None = None, count: int = 24, seed: int = 0):
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    mask = np.ones((n, m), np.float64)
    for _ in range(count):
        side = int(rng.integers(max(1, min(n, m) // 32), max(2, min(n, m) // 8) + 1))
        y = int(rng.integers(0, n - side + 1))
        x = int(rng.integers(0, m - side + 1))
        mask[y:y + side, x:x + side] = 0.0
    return mask


def gaussian_noise(shape, sigma: float, seed: int = 0):
    rng = np.random.default_rng(seed)
    return sigma * rng.standard_normal(shape)


def uniform_field(shape, seed: int = 0, lo=-1.0, hi=1.0):
    """Plain i.i.d. uniform array (for transform parity inputs)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


# ------------------------------------------------------------- workloads
def plain_transform_image(n: int = 256, seed: int = 1):
    """8 filled ellipses plus N(0, 0.05^2) noise (plain-transform workload)."""
    return ellipses(n, n, 8, seed) + gaussian_noise((n, n), 0.05, seed + 1)


def denoise_batch(b: int = 16, n: int = 512, sigma: float = 30 / 255,
                  seed0: int = 100):
    """Clean cartoons and their noisy copies, seeds seed0 .. seed0+b-1."""
    clean = np.stack([cartoon(n, n, seed0 + i) for i in range(b)])
    noisy = clean + np.stack([gaussian_noise((n, n), sigma, 10_000 + seed0 + i)
                              for i in range(b)])
    return clean, noisy


def inpaint_batch(b: int = 8, n: int = 512, p: float = 0.5, seed0: int = 2000,
                  kind: str = "random"):
    """Cartoon+texture images, masks (``random``: Bernoulli(p) keep; ``squared``:
    square holes) and masked images."""
    clean = np.stack([cartoon_texture(n, n, seed0 + i) for i in range(b)])
    if kind == "squared":
        mask = np.stack([square_mask(n, n, seed=60_000 + seed0 + i) for i in range(b)])
    else:
        mask = np.stack([bernoulli_mask(n, n, p, 50_000 + seed0 + i) for i in range(b)])
    return clean, mask, clean * mask


# ------------------------------------------------------------ phantoms
def shepp_logan():
    """Rows (value, a, b, x0, y0, alpha [rad]) of the modified Shepp-Logan
    phantom (Toft's table: the original's contrasts raised for display)."""
    deg = np.pi / 180.0
    return np.array([
        [1.0, 0.69, 0.92, 0.0, 0.0, 0.0],
        [-0.8, 0.6624, 0.874, 0.0, -0.0184, 0.0],
        [-0.2, 0.11, 0.31, 0.22, 0.0, -18 * deg],
        [-0.2, 0.16, 0.41, -0.22, 0.0, 18 * deg],
        [0.1, 0.21, 0.25, 0.0, 0.35, 0.0],
        [0.1, 0.046, 0.046, 0.0, 0.1, 0.0],
        [0.1, 0.046, 0.046, 0.0, -0.1, 0.0],
        [0.1, 0.046, 0.023, -0.08, -0.605, 0.0],
        [0.1, 0.023, 0.023, 0.0, -0.606, 0.0],
        [0.1, 0.023, 0.046, 0.06, -0.605, 0.0],
    ])


def random_ellipses(seed: int = 0):
    """Ellipse table of one random training object (recipe in the module
    docstring)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 11))
    rad, ang = rng.uniform(0.0, 0.6, n), rng.uniform(0.0, 2 * np.pi, n)
    val = rng.uniform(0.1, 0.6, n) * np.where(rng.random(n) < 0.3, -1.0, 1.0)
    return np.stack([val, rng.uniform(0.05, 0.45, n), rng.uniform(0.05, 0.45, n),
                     rad * np.cos(ang), rad * np.sin(ang), rng.uniform(0.0, np.pi, n)], axis=1)


def ellipse_phantom(table, n: int, supersample: int = 2, clip: bool = True):
    """Pixel averages of the ellipses of ``table`` on the n x n grid."""
    h = 2.0 / n
    q = (np.arange(n * supersample) + 0.5) * (h / supersample) - 1.0
    Y, X = np.meshgrid(q, q, indexing="ij")
    img = np.zeros_like(X)
    for val, a, b, x0, y0, al in np.asarray(table, np.float64):
        u = (X - x0) * np.cos(al) + (Y - y0) * np.sin(al)
        v = -(X - x0) * np.sin(al) + (Y - y0) * np.cos(al)
        img += val * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    img = img.reshape(n, supersample, n, supersample).mean(axis=(1, 3))
    return np.clip(img, 0.0, 1.0) if clip else img
