"""CPU oracle for the Brady dyadic fast Hough transform (FHT).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
library's product path never does, and this package imports nothing from the
library: the two share only the seeded input generators in ``workloads``.

What is computed (Aliev, Ershov, Nikolaev, arXiv:1811.06378):

* ``quadrant``     one quadrant of the Hough image on the zero-padded image
                   (Section 3.1: padding by an h x h zero block, result (w+h) x h;
                   the four angle quadrants; mostly-horizontal lines handled by
                   transposing the image).
* ``full``         the four quadrants concatenated on their common edge rows,
                   flipping Q0 and Q2 (Section 3.3, Eq. 1-2, 2(w+h)-3 rows and
                   the per-quadrant row ranges at the end of Section 3.3).
* ``range_slice``  the slopes of an inclination range only (Section 4; the
                   slope-pruning reading returns exactly that slice).
* ``fhtshift``     per-row cyclic regrouping around the accumulator centre
                   (Section 5).
* ``point_segment`` the image pixels one Hough point sums (Section 3.2).
* ``quadrant_op``  maximum or minimum along the patterns instead of the sum.
* ``sheared_quadrant`` the quadrant of the sheared image (Section 4).
* ``scaled_quadrant`` the quadrant of the image scaled along its rows, then
                   sheared (Section 4, both operations).
* ``adjoint_*``    the transpose of each map (not in the paper; defined by the
                   transform being linear), computed as the opposite-sign
                   transform of the gradient because the dyadic offsets are
                   symmetric in (t, y).

The butterfly itself lives in ``fht_oracle.c`` (plain C, compiled on demand
with gcc, no fast-math). Readings of points the paper leaves open:

1. The butterfly is the standard Brady recursion: both halves of a merged strip
   use slope floor(t/2); the bottom half is shifted by ceil(t/2).
2. Slopes t = 0..n-1, n = next power of two >= h; t = n-1 is 45 degrees.
3. Padding is on the right (cyclic width W = w + n) and at the bottom.
4. Q2 is the negative-sign transform of the transposed image and Q3 the
   positive-sign one, fixed by continuity of the shared rows.
5. Full-image rows: see ``full_row_map``.
6. fhtshift rotates row t of a quadrant right by floor(b/2) (+ t for the
   positive-sign quadrants), b = W - w_in - t the black-zone width.
7. Angle ranges map to slopes by t = (n-1)*tan(theta); see ``angle_to_slopes``.
8. The shear of Section 4 (``sheared_quadrant``): row y of the (transposed)
   image is shifted cyclically right by s(y) = floor(y*spl + 1/2) columns
   (spl, the shift per line; the paper gives no rounding), evaluated exactly
   with spl in fixed point (32 fractional bits, rounded half up), then the plain
   quadrant transform runs on the cyclic width W = w + n, which the paper
   keeps (Section 4: the black zone only moves, nothing wraps into the
   meaningful zone).
9. The scale of Section 4 (``scaled_quadrant``): the paper fixes no discrete
   resampling. Column x' of the row scaled by alpha is column
   floor(x' * D / 2^32) of the original, D = ceil(2^32 / alpha) (nearest
   neighbour on the integer grid, in fixed point so that both sides take the
   same integer decision), for the w_alpha = ceil(w * 2^32 / D) columns whose
   source lies inside the row. The scale comes first, then the shear, on the
   cyclic width w_alpha + n.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfht_oracle.so")
_lock = threading.Lock()
_lib = None

Q0, Q1, Q2, Q3 = 0, 1, 2, 3
SIGMA = {Q0: +1, Q1: -1, Q2: -1, Q3: +1}
TRANSPOSED = {Q0: False, Q1: False, Q2: True, Q3: True}

_CT = {"i64": (np.int64, ctypes.c_int64), "f32": (np.float32, ctypes.c_float),
       "f64": (np.float64, ctypes.c_double)}


def build(force: bool = False) -> str:
    """Compile fht_oracle.c into a shared library (gcc -O2, IEEE arithmetic)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i = ctypes.c_int
            i64 = ctypes.c_int64
            lib.fo_offset.restype = i64
            lib.fo_offset.argtypes = [i64, i64, i64]
            for name in ("fo_brute_i64", "fo_brute_f64", "fo_brute_adjoint_i64",
                         "fo_brute_adjoint_f64"):
                getattr(lib, name).restype = None
                getattr(lib, name).argtypes = [p, i, i, i, p]
            for name in ("fo_butterfly_i64", "fo_butterfly_f32", "fo_butterfly_f64",
                         "fo_adjoint_i64", "fo_adjoint_f32", "fo_adjoint_f64"):
                getattr(lib, name).restype = i
                getattr(lib, name).argtypes = [p, i, i, i]
            for name in ("fo_butterfly_op_i64", "fo_butterfly_op_f32"):
                getattr(lib, name).restype = i
                getattr(lib, name).argtypes = [p, i, i, i, i]
            lib.fo_points.restype = None
            lib.fo_points.argtypes = [p, i, i, i, i64, i, i, i, i, i, p, p, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def next_pow2(v: int) -> int:
    n = 1
    while n < v:
        n *= 2
    return n


# ---------------------------------------------------------------- definitions

def offset(n: int, t: int, y: int) -> int:
    """off_n(t, y): column offset of row y on the slope-t dyadic pattern."""
    return int(_load().fo_offset(n, t, y))


def pattern_table(n: int) -> np.ndarray:
    """n x n table T[t, y] = off_n(t, y)."""
    lib = _load()
    return np.array([[lib.fo_offset(n, t, y) for y in range(n)] for t in range(n)],
                    dtype=np.int64)


def butterfly(P: np.ndarray, sigma: int, kind: str = "i64") -> np.ndarray:
    """Level-by-level butterfly of the n x W array P (n a power of two)."""
    dt, _ = _CT[kind]
    A = np.ascontiguousarray(P, dtype=dt).copy()
    n, W = A.shape
    if getattr(_load(), f"fo_butterfly_{kind}")(_ptr(A), n, W, sigma) != 0:
        raise MemoryError("oracle butterfly scratch allocation failed")
    return A


OP_SUM, OP_MAX, OP_MIN = 0, 1, 2


def butterfly_op(P: np.ndarray, sigma: int, op: int, kind: str = "i64") -> np.ndarray:
    """The butterfly with maximum (op 1) or minimum (op 2) in place of the
    sum; op 0 is the sum."""
    if op == OP_SUM:
        return butterfly(P, sigma, kind)
    dt, _ = _CT[kind]
    A = np.ascontiguousarray(P, dtype=dt).copy()
    n, W = A.shape
    if getattr(_load(), f"fo_butterfly_op_{kind}")(_ptr(A), n, W, sigma, op) != 0:
        raise MemoryError("oracle butterfly scratch allocation failed")
    return A


def adjoint_butterfly(G: np.ndarray, sigma: int, kind: str = "i64") -> np.ndarray:
    """Transposed butterfly of the n x W array G."""
    dt, _ = _CT[kind]
    A = np.ascontiguousarray(G, dtype=dt).copy()
    n, W = A.shape
    if getattr(_load(), f"fo_adjoint_{kind}")(_ptr(A), n, W, sigma) != 0:
        raise MemoryError("oracle adjoint scratch allocation failed")
    return A


def brute(P: np.ndarray, sigma: int, kind: str = "i64") -> np.ndarray:
    """Sums along explicitly enumerated patterns (tiny sizes only)."""
    kind = "f64" if kind != "i64" else "i64"
    dt, _ = _CT[kind]
    A = np.ascontiguousarray(P, dtype=dt)
    n, W = A.shape
    H = np.zeros_like(A)
    getattr(_load(), f"fo_brute_{kind}")(_ptr(A), n, W, sigma, _ptr(H))
    return H


def brute_adjoint(G: np.ndarray, sigma: int, kind: str = "i64") -> np.ndarray:
    """Back-projection sum, the transpose of ``brute`` (tiny sizes only)."""
    kind = "f64" if kind != "i64" else "i64"
    dt, _ = _CT[kind]
    A = np.ascontiguousarray(G, dtype=dt)
    n, W = A.shape
    out = np.zeros_like(A)
    getattr(_load(), f"fo_brute_adjoint_{kind}")(_ptr(A), n, W, sigma, _ptr(out))
    return out


# ---------------------------------------------------------------- geometry

def quadrant_geometry(h: int, w: int, q: int) -> tuple[int, int]:
    """(rows n, cols W) of quadrant q of an h x w image (Section 3.1): the
    vertical quadrants pad to n = next_pow2(h) rows and W = w + n columns; the
    horizontal ones do the same on the transposed image."""
    if TRANSPOSED[q]:
        h, w = w, h
    n = next_pow2(h)
    return n, w + n


def full_geometry(h: int, w: int) -> tuple[int, int]:
    """(rows, cols) of the full Hough image: the image is padded to
    h_p x w_p (powers of two), every quadrant is then (w_p + h_p) wide and the
    concatenation drops one shared row per seam: 2*(h_p + w_p) - 3 rows
    (Section 3.3)."""
    hp, wp = next_pow2(h), next_pow2(w)
    return 2 * hp + 2 * wp - 3, hp + wp


def full_row_map(h: int, w: int) -> list[tuple[int, int]]:
    """For every full-image row r, the (quadrant, slope) it holds.

    Order (Section 3.3): Q0 flipped, Q1, Q2 flipped, Q3; each seam's shared row
    is kept once (Q1's t=0 equals Q0's t=0, Q2's t=n_w-1 equals Q1's t=n_h-1,
    Q3's t=0 equals Q2's t=0)."""
    hp, wp = next_pow2(h), next_pow2(w)
    rows = []
    for t in range(hp - 1, -1, -1):
        rows.append((Q0, t))
    for t in range(1, hp):
        rows.append((Q1, t))
    for t in range(wp - 2, -1, -1):
        rows.append((Q2, t))
    for t in range(1, wp):
        rows.append((Q3, t))
    return rows


def padded(img: np.ndarray, rows: int, cols: int, kind: str) -> np.ndarray:
    """img zero-padded at the bottom and right to rows x cols."""
    dt, _ = _CT[kind]
    P = np.zeros((rows, cols), dtype=dt)
    P[: img.shape[0], : img.shape[1]] = img
    return P


# ---------------------------------------------------------------- transforms

def quadrant(img: np.ndarray, q: int, kind: str = "i64") -> np.ndarray:
    """Quadrant q of the Hough image of img (h x w), shape (n, W)."""
    src = img.T if TRANSPOSED[q] else img
    n, W = quadrant_geometry(img.shape[0], img.shape[1], q)
    return butterfly(padded(src, n, W, kind), SIGMA[q], kind)


def quadrant_op(img: np.ndarray, q: int, op: int, kind: str = "i64") -> np.ndarray:
    """Quadrant q with the maximum (op 1) or minimum (op 2) along every
    pattern instead of the sum (the generalisation to associative-commutative
    operations of the introduction); the padding stays zero (Section 3.1),
    so a pattern that leaves the image takes zeros into its maximum or
    minimum."""
    src = img.T if TRANSPOSED[q] else img
    n, W = quadrant_geometry(img.shape[0], img.shape[1], q)
    return butterfly_op(padded(src, n, W, kind), SIGMA[q], op, kind)


def _full_quadrants(img: np.ndarray, kind: str) -> dict[int, np.ndarray]:
    h, w = img.shape
    hp, wp = next_pow2(h), next_pow2(w)
    W = hp + wp
    out = {}
    for q in (Q0, Q1, Q2, Q3):
        if TRANSPOSED[q]:
            out[q] = butterfly(padded(img.T, wp, W, kind), SIGMA[q], kind)
        else:
            out[q] = butterfly(padded(img, hp, W, kind), SIGMA[q], kind)
    return out


def full(img: np.ndarray, kind: str = "i64") -> np.ndarray:
    """Full Hough image (all four quadrants concatenated), shape full_geometry."""
    quads = _full_quadrants(img, kind)
    return np.stack([quads[q][t] for q, t in full_row_map(*img.shape)])


def range_slice(img: np.ndarray, q: int, t_lo: int, t_hi: int,
                kind: str = "i64") -> np.ndarray:
    """Rows t_lo..t_hi of quadrant q (the range variant's exact result)."""
    return quadrant(img, q, kind)[t_lo: t_hi + 1]


def fhtshift_amount(t: int, W: int, w_in: int, sigma: int) -> int:
    """Right rotation of slope row t: the meaningful zone (w_in + t columns)
    starts at floor(b/2), b = W - w_in - t the black-zone width (Section 5)."""
    b = W - w_in - t
    return b // 2 + (t if sigma > 0 else 0)


def fhtshift_quadrant(H: np.ndarray, h: int, w: int, q: int,
                      inverse: bool = False) -> np.ndarray:
    """fhtshift of a single quadrant of an h x w image."""
    w_in = h if TRANSPOSED[q] else w
    n, W = H.shape
    out = np.empty_like(H)
    for t in range(n):
        s = fhtshift_amount(t, W, w_in, SIGMA[q])
        out[t] = np.roll(H[t], -s if inverse else s)
    return out


def fhtshift_full(F: np.ndarray, h: int, w: int, inverse: bool = False) -> np.ndarray:
    """fhtshift of a full Hough image of an h x w image."""
    hp, wp = next_pow2(h), next_pow2(w)
    W = F.shape[1]
    out = np.empty_like(F)
    for r, (q, t) in enumerate(full_row_map(h, w)):
        w_in = hp if TRANSPOSED[q] else wp
        s = fhtshift_amount(t, W, w_in, SIGMA[q])
        out[r] = np.roll(F[r], -s if inverse else s)
    return out


def angle_to_slopes(phi_lo: float, phi_hi: float, h: int, w: int
                    ) -> tuple[list[int], list[int]]:
    """Slope ranges per quadrant for line angles phi in [phi_lo, phi_hi] degrees.

    Quadrant spans: Q0 [-45, 0], Q1 [0, 45], Q2 [45, 90], Q3 [90, 135]. Within a
    quadrant with n slopes, slope t sits at theta(t) = atan(t / (n-1)) from the
    quadrant's t = 0 edge (0 deg for Q0/Q1, 90 deg for Q2/Q3); t is kept iff
    theta(t) lies in the requested interval. A row shared by two quadrants is
    kept in the first one (order Q0, Q1, Q2, Q3). Unused quadrants get -1."""
    spans = {Q0: (-45.0, 0.0), Q1: (0.0, 45.0), Q2: (45.0, 90.0), Q3: (90.0, 135.0)}
    lo = [-1] * 4
    hi = [-1] * 4
    for q in (Q0, Q1, Q2, Q3):
        a, b = max(phi_lo, spans[q][0]), min(phi_hi, spans[q][1])
        if a > b:
            continue
        # theta measured away from the quadrant's t = 0 edge
        if q == Q0:
            th_a, th_b = -b, -a
        elif q == Q1:
            th_a, th_b = a, b
        elif q == Q2:
            th_a, th_b = 90.0 - b, 90.0 - a
        else:
            th_a, th_b = a - 90.0, b - 90.0
        n, _ = quadrant_geometry(h, w, q)
        if n == 1:
            t_lo = t_hi = 0
        else:
            t_lo = math.ceil((n - 1) * math.tan(math.radians(th_a)) - 1e-9)
            t_hi = math.floor((n - 1) * math.tan(math.radians(th_b)) + 1e-9)
            t_lo, t_hi = max(t_lo, 0), min(t_hi, n - 1)
        if t_lo <= t_hi:
            lo[q], hi[q] = t_lo, t_hi
    # shared seam rows, kept once
    n_h, _ = quadrant_geometry(h, w, Q0)
    n_w, _ = quadrant_geometry(h, w, Q2)
    if lo[Q0] == 0 and lo[Q1] == 0:
        lo[Q1] = 1
    if hi[Q1] == n_h - 1 and hi[Q2] == n_w - 1:
        hi[Q2] = n_w - 2
    if lo[Q2] == 0 and lo[Q3] == 0:
        lo[Q3] = 1
    for q in (Q0, Q1, Q2, Q3):
        if lo[q] > hi[q]:
            lo[q] = hi[q] = -1
    return lo, hi


# ---------------------------------------------------------------- Hough point -> segment (Section 3.2)

def point_segment(h: int, w: int, q: int, t: int, x: int):
    """The part of the image that Hough point (t, x) of quadrant q sums
    (Section 3.2): the slope-t pattern from column x, taken modulo the
    extended width W = w + n (case b: a pattern leaving the extended image on
    the right re-enters the original image on the left), cut to the image
    (case a); None when no pixel of it lies in the image (case c).

    Returns (count, (r0, c0), (r1, c1)): the number of its pixels inside the
    image and its first and last one as image (row, column), ordered by the
    pattern's row y (an image column for Q2/Q3)."""
    n, W = quadrant_geometry(h, w, q)
    hc, wc = (w, h) if TRANSPOSED[q] else (h, w)
    inside = []
    for y in range(min(n, hc)):
        c = (x + SIGMA[q] * offset(n, t, y)) % W
        if c < wc:
            inside.append((y, c))
    if not inside:
        return None
    (ya, ca), (yb, cb) = inside[0], inside[-1]
    if TRANSPOSED[q]:
        return len(inside), (ca, ya), (cb, yb)
    return len(inside), (ya, ca), (yb, cb)


# ---------------------------------------------------------------- shear (Section 4)

def shear_fixed(spl: float) -> int:
    """spl in fixed point with 32 fractional bits, rounded half up:
    P = floor(spl * 2^32 + 1/2) (exact in float64 for |spl| <= 1)."""
    return int(math.floor(float(spl) * 2.0**32 + 0.5))


def shear_shifts(rows: int, spl: float) -> np.ndarray:
    """s(y) = floor(y*spl + 1/2) for y < rows, the shift per line of Section 4
    rounded half up, evaluated exactly on the 32-bit fixed-point spl:
    s(y) = floor((y*P + 2^31) / 2^32), P = shear_fixed(spl)."""
    P = shear_fixed(spl)
    return np.array([(y * P + 2**31) >> 32 for y in range(rows)], dtype=np.int64)


def sheared_quadrant(img: np.ndarray, q: int, spl: float, kind: str = "i64",
                     t_lo: int = 0, t_hi: int | None = None) -> np.ndarray:
    """Quadrant q of the sheared image (Section 4): row y of the image (of the
    transposed image for Q2/Q3) is zero-padded to the cyclic width W = w + n
    and rotated right by s(y) columns; the plain butterfly of that n x W array
    with the quadrant's sign, rows t_lo..t_hi. A line with dx/dy = k in the
    image (columns per row of the transposed image for Q2/Q3) lies on the
    sheared image's slope k + spl: with spl = tan(beta) the quadrant's slopes
    t/(n-1) in [0, 1] cover k in [-spl, 1 - spl]."""
    src = img.T if TRANSPOSED[q] else img
    n, W = quadrant_geometry(img.shape[0], img.shape[1], q)
    P = padded(src, n, W, kind)
    s = shear_shifts(src.shape[0], spl)
    for y in range(src.shape[0]):
        P[y] = np.roll(P[y], int(s[y]))
    H = butterfly(P, SIGMA[q], kind)
    t_hi = n - 1 if t_hi is None else t_hi
    return H[t_lo:t_hi + 1].copy()


def shear_range(phi_lo: float, phi_hi: float, h: int, w: int
                ) -> tuple[int, float, int, int]:
    """One sheared quadrant for the line angles [phi_lo, phi_hi] (degrees,
    the quadrant spans of ``angle_to_slopes``): (q, spl, t_lo, t_hi), or
    None when the range does not fit one quadrant.

    Mostly vertical ranges (inside [-45, 45]) use Q0 with spl = tan(phi_hi):
    its row t then holds the lines at phi(t) = atan(spl - t/(n-1)), from phi_hi
    at t = 0 down to phi_lo. Mostly horizontal ranges (inside [45, 135]) use Q3
    with spl = -tan(phi_lo - 90): phi(t) = 90 + atan(t/(n-1) - spl), from phi_lo
    up. t runs from 0 to floor((n-1) * (tan(b) - tan(a))), a and b the range's
    ends measured from the quadrant's axis, which must differ by at most 1 in
    tangent (45 degrees around the axis)."""
    if phi_lo > phi_hi:
        return None
    if -45.0 <= phi_lo and phi_hi <= 45.0:
        q, a, b = Q0, phi_lo, phi_hi
        spl = math.tan(math.radians(b))
    elif 45.0 <= phi_lo and phi_hi <= 135.0:
        q, a, b = Q3, phi_lo - 90.0, phi_hi - 90.0
        spl = -math.tan(math.radians(a))
    else:
        return None
    span = math.tan(math.radians(b)) - math.tan(math.radians(a))
    if span > 1.0 + 1e-12:
        return None
    n, _ = quadrant_geometry(h, w, q)
    t_hi = 0 if n == 1 else min(n - 1, math.floor((n - 1) * span + 1e-9))
    return q, spl, 0, t_hi


# ---------------------------------------------------------------- scale (Section 4)

def scale_step(alpha: float) -> int:
    """Source-column step of the image scaled along OX by alpha, in fixed
    point with 32 fractional bits, rounded up: D = ceil(2^32 / alpha), the
    quotient taken in float64 (the library computes the same double)."""
    return int(math.ceil(2.0**32 / float(alpha)))


def scaled_width(w: int, alpha: float) -> int:
    """Columns x' of the scaled row whose source column src(x') = floor(x' *
    D / 2^32) lies inside the w image columns: ceil(w * 2^32 / D)."""
    D = scale_step(alpha)
    return (w * 2**32 + D - 1) // D


def scale_columns(w: int, alpha: float) -> np.ndarray:
    """src(x') = floor(x' * D / 2^32) for every column x' of the scaled row:
    nearest-neighbour resampling on the integer grid (the paper fixes no
    rule); exactly floor(x'/k) for an integer factor k (each column repeated
    k times) and k*x' for alpha = 1/k (every k-th column)."""
    D = scale_step(alpha)
    return np.array([(x * D) >> 32 for x in range(scaled_width(w, alpha))], dtype=np.int64)


def scaled_image(img: np.ndarray, alpha: float) -> np.ndarray:
    """The image scaled along OX by alpha > 0 (Section 4, first operation):
    column x' of the result is column src(x') of img. A line with dx/dy = k
    becomes one with dx/dy = alpha * k, the paper's tg(beta) -> alpha*tg(beta)."""
    return img[:, scale_columns(img.shape[1], alpha)]


def scaled_quadrant(img: np.ndarray, q: int, alpha: float, spl: float = 0.0,
                    kind: str = "i64", t_lo: int = 0, t_hi: int | None = None) -> np.ndarray:
    """Quadrant q after both operations of Section 4: the image (the
    transposed image for Q2/Q3, i.e. the original scaled along OY) scaled
    along its rows by alpha, then sheared by spl; the butterfly of that n x W
    array with W = w_alpha + n (w_alpha = scaled_width of the row length) and
    the quadrant's sign, rows t_lo..t_hi. A line with dx/dy = k (columns per
    row of the transposed image for Q2/Q3) lies on slope alpha*k + spl."""
    src = img.T if TRANSPOSED[q] else img
    scaled = scaled_image(src, alpha)
    n = next_pow2(src.shape[0])
    W = scaled.shape[1] + n
    P = padded(scaled, n, W, kind)
    s = shear_shifts(src.shape[0], spl)
    for y in range(src.shape[0]):
        P[y] = np.roll(P[y], int(s[y]))
    H = butterfly(P, SIGMA[q], kind)
    t_hi = n - 1 if t_hi is None else t_hi
    return H[t_lo:t_hi + 1].copy()


def scale_range(phi_lo: float, phi_hi: float, h: int, w: int, alpha_max: float = 16.0):
    """One scaled and sheared quadrant for the line angles [phi_lo, phi_hi]
    (degrees, the quadrant spans of ``angle_to_slopes``): (q, alpha, spl,
    t_lo, t_hi), or None. The two operations of Section 4 map the range onto
    as many of the quadrant's slope rows as the shear's |spl| <= 1 allows,
    so that its angles are resolved alpha times finer than in the plain
    quadrant.

    Mostly vertical ranges (midpoint within [-45, 45], ends inside (-90, 90))
    use Q0: row t holds phi(t) = atan((spl - t/(n-1)) / alpha), phi_hi at
    t = 0, with alpha = min(1/(tan(b) - tan(a)), 1/|tan(b)|, alpha_max) and
    spl = alpha*tan(b). Mostly horizontal ranges (midpoint within [45, 135],
    ends inside (0, 180)) use Q3 with the angles a, b measured from 90
    degrees: row t holds 90 + atan((t/(n-1) - spl) / alpha), phi_lo at t = 0,
    alpha = min(1/(tan(b) - tan(a)), 1/|tan(a)|, alpha_max), spl =
    -alpha*tan(a). t runs from 0 to floor((n-1) * alpha * (tan(b) - tan(a)))."""
    if not phi_lo <= phi_hi:
        return None
    mid = 0.5 * (phi_lo + phi_hi)
    if -45.0 <= mid <= 45.0 and -90.0 < phi_lo and phi_hi < 90.0:
        q, a, b = Q0, phi_lo, phi_hi
        edge = math.tan(math.radians(b))
    elif 45.0 < mid <= 135.0 and 0.0 < phi_lo and phi_hi < 180.0:
        q, a, b = Q3, phi_lo - 90.0, phi_hi - 90.0
        edge = math.tan(math.radians(a))
    else:
        return None
    span = math.tan(math.radians(b)) - math.tan(math.radians(a))
    alpha = alpha_max
    if span > 0:
        alpha = min(alpha, 1.0 / span)
    if edge != 0:
        alpha = min(alpha, 1.0 / abs(edge))
    spl = alpha * edge if q == Q0 else -alpha * edge
    n, _ = quadrant_geometry(h, w, q)
    t_hi = 0 if n == 1 else min(n - 1, math.floor((n - 1) * alpha * span + 1e-9))
    return q, alpha, spl, 0, t_hi


# ---------------------------------------------------------------- adjoints

def adjoint_quadrant(G: np.ndarray, h: int, w: int, q: int,
                     kind: str = "f64") -> np.ndarray:
    """Transpose of ``quadrant``: (n, W) gradient -> (h, w) image gradient.

    The dyadic offsets are symmetric, off_n(t, y) = off_n(y, t) (pinned by the
    tests), so the transpose sum_t G[t][(c - sigma*off(t, y)) mod W] is the
    opposite-sign transform of G read as an n-row image:
    sum_t G[t][(c + (-sigma)*off(y, t)) mod W]. Floating-point kinds add along
    that recursion's tree; ``adjoint_butterfly`` (the transposed network) and
    ``explicit_matrix`` are independent checks of the same map."""
    A = butterfly(G, -SIGMA[q], kind)
    if TRANSPOSED[q]:
        return A[:w, :h].T.copy()
    return A[:h, :w].copy()


def adjoint_full(G: np.ndarray, h: int, w: int, kind: str = "f64") -> np.ndarray:
    """Transpose of ``full``: each full-image row's gradient goes back to the
    quadrant row it came from (rows dropped at the seams get zero); the
    quadrant adjoints are summed in the order Q0, Q1, Q2, Q3."""
    hp, wp = next_pow2(h), next_pow2(w)
    W = hp + wp
    dt, _ = _CT[kind]
    per_q = {q: np.zeros(((wp if TRANSPOSED[q] else hp), W), dtype=dt)
             for q in (Q0, Q1, Q2, Q3)}
    for r, (q, t) in enumerate(full_row_map(h, w)):
        per_q[q][t] = G[r]
    acc = None
    for q in (Q0, Q1, Q2, Q3):
        A = butterfly(per_q[q], -SIGMA[q], kind)
        part = A[:w, :h].T if TRANSPOSED[q] else A[:h, :w]
        acc = part.copy() if acc is None else (acc + part).astype(dt)
    return acc


def adjoint_quadrant_transposed_network(G: np.ndarray, h: int, w: int, q: int,
                                        kind: str = "f64") -> np.ndarray:
    """The same transpose computed by the transposed butterfly network (levels
    in reverse, each merge turned into a split): an independent check."""
    A = adjoint_butterfly(G, SIGMA[q], kind)
    if TRANSPOSED[q]:
        return A[:w, :h].T.copy()
    return A[:h, :w].copy()


def explicit_matrix(h: int, w: int, q: int) -> np.ndarray:
    """The quadrant map as an explicit (n*W) x (h*w) integer matrix, column j
    being the brute-force transform of the j-th unit image (tiny sizes only)."""
    n, W = quadrant_geometry(h, w, q)
    M = np.zeros((n * W, h * w), dtype=np.int64)
    for j in range(h * w):
        e = np.zeros((h, w), dtype=np.int64)
        e.flat[j] = 1
        src = e.T if TRANSPOSED[q] else e
        M[:, j] = brute(padded(src, n, W, "i64"), SIGMA[q], "i64").ravel()
    return M


# ---------------------------------------------------------------- sampled

_DT_CODE = {np.dtype(np.uint8): 0, np.dtype(np.int32): 1, np.dtype(np.float32): 2}


def points(img: np.ndarray, q: int, ts, xs, full_layout: bool = False) -> np.ndarray:
    """Brute-force values of single Hough points (t, x) of quadrant q, straight
    from the unpadded image. With full_layout the geometry is that of the full
    image (image padded to powers of two). Returns float64 (exact for
    integer images below 2^53)."""
    img = np.ascontiguousarray(img)
    h, w = img.shape
    if full_layout:
        hp, wp = next_pow2(h), next_pow2(w)
        n, W = (wp, hp + wp) if TRANSPOSED[q] else (hp, hp + wp)
    else:
        n, W = quadrant_geometry(h, w, q)
    th, tw = (w, h) if TRANSPOSED[q] else (h, w)
    ts = np.ascontiguousarray(ts, dtype=np.int64)
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    out = np.zeros(len(ts), dtype=np.float64)
    _load().fo_points(_ptr(img), _DT_CODE[img.dtype], th, tw, img.shape[1],
                      int(TRANSPOSED[q]), n, W, SIGMA[q], len(ts), _ptr(ts),
                      _ptr(xs), _ptr(out))
    return out
