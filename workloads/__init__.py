"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module draws images only. It holds none of the transform's arithmetic:
no dyadic offsets, no sums along patterns, no quadrant or fhtshift logic. Both
the CUDA path and the CPU oracle receive the arrays built here, so the two never
share anything else.

The paper measures nothing on a public dataset; its applications are document
images with text lines and tomography phantoms (Section 1). The generators below
stand in for those with the shapes, sizes and value mixes of the five workloads
the library is benchmarked on:

* ``edges_and_lines``  binary edge maps (Bernoulli edge pixels plus a few
  rasterised straight lines), uint8, 0/1;
* ``text_stripes``     a page-like grayscale image: light background, dark skewed
  stripes standing in for text lines, then salt-and-pepper noise, uint8;
* ``ellipse_phantom``  additive random ellipses plus Gaussian noise, float32;
* ``batch_shapes`` / ``edge_batch``  many edge maps of log-uniform sizes.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "edges_and_lines",
    "text_stripes",
    "ellipse_phantom",
    "batch_shapes",
    "edge_batch",
    "random_image",
]


def _draw_line(img: np.ndarray, x0: float, y0: float, theta: float, value: int) -> None:
    """Rasterise the straight line through (x0, y0) at angle theta across img.

    One pixel per step along the major axis, rounded to the nearest pixel
    (a plain DDA/Bresenham-style digital line)."""
    h, w = img.shape
    dx, dy = math.cos(theta), math.sin(theta)
    if abs(dy) >= abs(dx):  # mostly vertical: one pixel per row
        ys = np.arange(h, dtype=np.float64)
        xs = x0 + (ys - y0) * dx / dy
    else:  # mostly horizontal: one pixel per column
        xs = np.arange(w, dtype=np.float64)
        ys = y0 + (xs - x0) * dy / dx
    xi = np.floor(xs + 0.5).astype(np.int64)
    yi = np.floor(ys + 0.5).astype(np.int64)
    keep = (xi >= 0) & (xi < w) & (yi >= 0) & (yi < h)
    img[yi[keep], xi[keep]] = value


def edges_and_lines(h: int, w: int, p_edge: float = 0.05, n_lines: int = 4,
                    seed: int = 0) -> np.ndarray:
    """Binary edge map: Bernoulli(p_edge) pixels set to 1, plus n_lines digital
    lines (value 1) through random points at random angles. uint8, h x w."""
    rng = np.random.default_rng(seed)
    img = (rng.random((h, w)) < p_edge).astype(np.uint8)
    for _ in range(n_lines):
        x0 = rng.uniform(0, w)
        y0 = rng.uniform(0, h)
        theta = rng.uniform(0.0, math.pi)
        _draw_line(img, x0, y0, theta, 1)
    return img


def text_stripes(h: int, w: int, n_stripes: int = 40, seed: int = 1,
                 background: int = 200, ink: int = 30, noise_frac: float = 0.10,
                 max_skew_deg: float = 15.0) -> np.ndarray:
    """Page-like uint8 image.

    Background ``background``; ``n_stripes`` dark rectangles of value ``ink``
    (thickness U[4,16] px, length U[0.3,0.9]*w, centre uniform, skew uniform in
    [-max_skew_deg, max_skew_deg] from horizontal); then a ``noise_frac``
    Bernoulli fraction of pixels replaced by uniform values 0..255."""
    rng = np.random.default_rng(seed)
    img = np.full((h, w), background, dtype=np.uint8)
    for _ in range(n_stripes):
        thick = rng.uniform(4.0, 16.0)
        length = rng.uniform(0.3, 0.9) * w
        cx = rng.uniform(0, w)
        cy = rng.uniform(0, h)
        skew = math.radians(rng.uniform(-max_skew_deg, max_skew_deg))
        ux, uy = math.cos(skew), math.sin(skew)          # along the stripe
        half_l, half_t = length / 2.0, thick / 2.0
        ext_x = abs(ux) * half_l + abs(uy) * half_t
        ext_y = abs(uy) * half_l + abs(ux) * half_t
        xa, xb = max(0, int(cx - ext_x)), min(w, int(cx + ext_x) + 2)
        ya, yb = max(0, int(cy - ext_y)), min(h, int(cy + ext_y) + 2)
        if xa >= xb or ya >= yb:
            continue
        yy, xx = np.mgrid[ya:yb, xa:xb]
        rx = xx + 0.5 - cx
        ry = yy + 0.5 - cy
        along = rx * ux + ry * uy
        across = -rx * uy + ry * ux
        inside = (np.abs(along) <= half_l) & (np.abs(across) <= half_t)
        img[ya:yb, xa:xb][inside] = ink
    noisy = rng.random((h, w)) < noise_frac
    img[noisy] = rng.integers(0, 256, size=int(noisy.sum()), dtype=np.uint8)
    return img


def ellipse_phantom(n: int, n_ellipses: int = 20, noise_sigma: float = 0.05,
                    seed: int = 2, m: int | None = None) -> np.ndarray:
    """float32 n x m phantom: sum of n_ellipses filled ellipses (centre uniform,
    semi-axes U[0.02,0.3]*n, orientation U[0,pi), intensity U[0,1]) plus
    N(0, noise_sigma^2) noise on every pixel."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    img = np.zeros((n, m), dtype=np.float32)
    side = min(n, m)
    for _ in range(n_ellipses):
        cx = rng.uniform(0, m)
        cy = rng.uniform(0, n)
        a = rng.uniform(0.02, 0.3) * side
        b = rng.uniform(0.02, 0.3) * side
        ang = rng.uniform(0.0, math.pi)
        val = np.float32(rng.uniform(0.0, 1.0))
        ca, sa = math.cos(ang), math.sin(ang)
        ext = max(a, b)
        xa, xb = max(0, int(cx - ext)), min(m, int(cx + ext) + 2)
        ya, yb = max(0, int(cy - ext)), min(n, int(cy + ext) + 2)
        if xa >= xb or ya >= yb:
            continue
        xs = (np.arange(xa, xb, dtype=np.float32) + np.float32(0.5 - cx))[None, :]
        ys = (np.arange(ya, yb, dtype=np.float32) + np.float32(0.5 - cy))[:, None]
        u = xs * np.float32(ca) + ys * np.float32(sa)
        v = -xs * np.float32(sa) + ys * np.float32(ca)
        inside = (u / np.float32(a)) ** 2 + (v / np.float32(b)) ** 2 <= 1.0
        img[ya:yb, xa:xb] += inside * val
    img += rng.normal(0.0, noise_sigma, size=(n, m)).astype(np.float32)
    return img


def batch_shapes(count: int = 512, lo: int = 64, hi: int = 1024,
                 seed: int = 3) -> list[tuple[int, int]]:
    """count (h, w) pairs, h and w independently log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    hs = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    ws = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return [(int(round(a)), int(round(b))) for a, b in zip(hs, ws)]


def edge_batch(shapes: list[tuple[int, int]], p_edge: float = 0.08,
               seed: int = 3) -> list[np.ndarray]:
    """One binary uint8 edge map per shape, Bernoulli(p_edge)."""
    rng = np.random.default_rng(seed + 1000)
    return [(rng.random(s) < p_edge).astype(np.uint8) for s in shapes]


def random_image(h: int, w: int, dtype: str = "u8", seed: int = 0,
                 hi: int = 256) -> np.ndarray:
    """Plain i.i.d. random image for edge-case tests: uint8 in [0, hi),
    int32 in [-hi, hi), or float32 standard normal."""
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, hi, size=(h, w), dtype=np.uint8)
    if dtype == "i32":
        return rng.integers(-hi, hi, size=(h, w), dtype=np.int32)
    if dtype == "f32":
        return rng.standard_normal(size=(h, w)).astype(np.float32)
    raise ValueError(dtype)
