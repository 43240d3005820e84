"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own formulas. CPU only."""

import math

import numpy as np
import pytest

import oracle as O
from workloads import edges_and_lines, random_image



# --------------------------------------------------------------- patterns

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128])
def test_patterns_are_digital_segments(n):
    """Each dyadic pattern is a connected digital segment from (x0, 0) to
    (x0 + t, n-1) (Section 3.2, step 1: a slope-t pattern joins the two
    horizontal sides), with 0/1 steps in y and in t, and it stays within
    log2(n)/6 of the ideal straight segment (the known approximation bound of
    the dyadic recursion)."""
    T = O.pattern_table(n)
    K = int(math.log2(n))
    assert (T[:, 0] == 0).all()
    assert (T[:, n - 1] == np.arange(n)).all()
    if n > 1:
        assert set(np.unique(np.diff(T, axis=1))) <= {0, 1}
        assert set(np.unique(np.diff(T, axis=0))) <= {0, 1}
        ideal = np.arange(n)[:, None] * np.arange(n)[None, :] / (n - 1)
        assert np.abs(T - ideal).max() <= K / 6 + 1e-12


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024, 4096])
def test_pattern_table_is_symmetric(n):
    """off_n(t, y) = off_n(y, t): the slope-t pattern's offset at row y equals
    the slope-y pattern's offset at row t. Checked on the oracle's table for
    small n and on an independent vectorised evaluation of the closed form
    (the sum of bit_{K-j}(y) * ceil(floor(t/2^(j-1))/2)) up to n = 4096. The
    adjoint relies on it."""
    K = n.bit_length() - 1
    t = np.arange(n)[:, None]
    y = np.arange(n)[None, :]
    T = np.zeros((n, n), np.int64)
    for j in range(1, K + 1):
        T += ((y >> (K - j)) & 1) * (((t >> (j - 1)) + 1) // 2)
    assert (T == T.T).all()
    if n <= 64:
        assert (O.pattern_table(n) == T).all()


@pytest.mark.parametrize("n", [2, 4, 8])
def test_small_patterns_equal_rounded_lines(n):
    """For n <= 8 every pattern is exactly the nearest-pixel digitisation of the
    straight segment (x0,0)->(x0+t,n-1): round(t*y/(n-1)), halves rounded up."""
    T = O.pattern_table(n)
    t = np.arange(n)[:, None]
    y = np.arange(n)[None, :]
    expect = (2 * t * y + (n - 1)) // (2 * (n - 1))
    assert (T == expect).all()


# --------------------------------------------------------------- butterfly

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("sigma", [1, -1])
def test_butterfly_equals_pattern_sums(n, sigma):
    """The level-by-level recursion equals the sum along explicitly enumerated
    patterns, for integer and float arithmetic."""
    rng = np.random.default_rng(n * 10 + (sigma > 0))
    for w in (1, 3, n, n + 5):
        W = w + n
        P = np.zeros((n, W), np.int64)
        P[:, :w] = rng.integers(-50, 50, size=(n, w))
        assert (O.butterfly(P, sigma, "i64") == O.brute(P, sigma, "i64")).all()
        Pf = np.zeros((n, W))
        Pf[:, :w] = rng.standard_normal((n, w))
        np.testing.assert_allclose(O.butterfly(Pf, sigma, "f64"),
                                   O.brute(Pf, sigma, "f64"), rtol=0, atol=1e-12)


def _quads(img):
    return {q: O.quadrant(img, q) for q in (O.Q0, O.Q1, O.Q2, O.Q3)}


@pytest.mark.parametrize("h,w", [(1, 1), (3, 7), (8, 8), (13, 5), (32, 20)])
def test_every_row_sums_to_image_mass(h, w):
    """Each pattern takes exactly one pixel per row of the padded image, so every
    slope row of every quadrant sums to the image mass."""
    img = random_image(h, w, "u8", seed=h * 31 + w)
    mass = int(img.astype(np.int64).sum())
    for q, H in _quads(img).items():
        assert (H.sum(axis=1) == mass).all(), q


@pytest.mark.parametrize("h,w", [(4, 4), (5, 9), (16, 3), (31, 31)])
def test_black_zone_is_zero(h, w):
    """The padded transform always has a zero triangle (Section 3.2, case c):
    positive-sign rows are zero on [w_in, W - t), negative-sign rows on
    [w_in + t, W); w_in is the (transposed) image width. When the image fills
    all n rows, everything outside that triangle is reached by some pixel."""
    img = random_image(h, w, "u8", seed=7, hi=5) + 1   # strictly positive image
    for q, H in _quads(img).items():
        n, W = H.shape
        w_in = h if O.TRANSPOSED[q] else w
        h_in = w if O.TRANSPOSED[q] else h
        for t in range(n):
            if O.SIGMA[q] > 0:
                zero, live = np.arange(w_in, W - t), np.r_[0:w_in, W - t:W]
            else:
                zero, live = np.arange(w_in + t, W), np.arange(0, w_in + t)
            assert (H[t, zero] == 0).all()
            if h_in == n:
                assert (H[t, live] > 0).all()


@pytest.mark.parametrize("h,w", [(8, 8), (6, 11), (16, 9)])
def test_vertical_and_diagonal_rows(h, w):
    """Slope 0 is the vertical pattern (column sums); slope n-1 is the exact
    45-degree diagonal."""
    img = random_image(h, w, "u8", seed=3)
    n, W = O.quadrant_geometry(h, w, O.Q0)
    P = O.padded(img, n, W, "i64")
    H0, H1 = O.quadrant(img, O.Q0), O.quadrant(img, O.Q1)
    assert (H0[0] == P.sum(axis=0)).all()
    assert (H1[0] == P.sum(axis=0)).all()
    diag_pos = np.array([sum(P[y, (x + y) % W] for y in range(n)) for x in range(W)])
    diag_neg = np.array([sum(P[y, (x - y) % W] for y in range(n)) for x in range(W)])
    assert (H0[n - 1] == diag_pos).all()
    assert (H1[n - 1] == diag_neg).all()


def test_line_on_pattern_gives_exact_peak():
    """A digital line drawn by rounding (which equals the dyadic pattern for
    n = 8) is summed completely by exactly one Hough point, which is the
    maximum of the whole quadrant."""
    n, w = 8, 12
    for t in range(n):
        for x0 in (0, 3, 5):
            img = np.zeros((n, w), np.uint8)
            for y in range(n):
                c = x0 + (2 * t * y + (n - 1)) // (2 * (n - 1))
                if c < w:
                    img[y, c] = 1
            H = O.quadrant(img, O.Q0)
            assert H[t, x0] == img.sum()
            assert H.max() == img.sum()


def test_drawn_line_peaks_at_its_parameters():
    """A rasterised straight line crossing the whole image from (x0, 0) to
    (x0 + t, n-1) gives the quadrant maximum at (t, x0) (within one cell for
    ties), collecting most of its pixels: the dyadic pattern and the rounded
    line differ by at most log2(n)/6 + 1/2 columns per row."""
    rng = np.random.default_rng(5)
    for n in (32, 64, 128):
        for _ in range(8):
            t_true = int(rng.integers(1, n - 1))
            x0 = int(rng.integers(0, n - t_true))
            img = np.zeros((n, n), np.uint8)
            for y in range(n):
                img[y, int(math.floor(x0 + t_true * y / (n - 1) + 0.5))] = 1
            H = O.quadrant(img, O.Q0)
            t_pk, x_pk = np.unravel_index(np.argmax(H), H.shape)
            assert abs(int(t_pk) - t_true) <= 1 and abs(int(x_pk) - x0) <= 1
            assert H[t_true, x0] >= 0.6 * n


# --------------------------------------------------------------- full image

def test_full_geometry_matches_paper_counts():
    """Quadrant size (w+h) x h (Section 3.1) and full size 2(w+h)-3 rows
    (Section 3.3) on power-of-two images."""
    for h, w in [(4, 4), (8, 16), (32, 8), (2048, 2048)]:
        assert O.quadrant_geometry(h, w, O.Q0) == (h, w + h)
        assert O.quadrant_geometry(h, w, O.Q2) == (w, h + w)
        assert O.full_geometry(h, w) == (2 * (w + h) - 3, w + h)
    assert O.full_geometry(2048, 2048) == (8189, 4096)


@pytest.mark.parametrize("h,w", [(4, 4), (8, 4), (4, 16), (16, 16)])
def test_full_row_ranges_follow_paper_thresholds(h, w):
    """End of Section 3.3: row r is in Q0 if r < h, Q1 if h <= r < 2h-1, Q2 if
    2h-1 <= r < 2h+w-2, Q3 otherwise; Q0 and Q2 are flipped."""
    rows = O.full_row_map(h, w)
    for r, (q, t) in enumerate(rows):
        if r < h:
            assert q == O.Q0 and t == h - 1 - r
        elif r < 2 * h - 1:
            assert q == O.Q1
        elif r < 2 * h + w - 2:
            assert q == O.Q2
        else:
            assert q == O.Q3
    # within each quadrant block, the slope is monotone: flipped blocks descend
    q2 = [t for q, t in rows if q == O.Q2]
    q3 = [t for q, t in rows if q == O.Q3]
    assert q2 == sorted(q2, reverse=True) and q3 == sorted(q3)


@pytest.mark.parametrize("h,w", [(8, 8), (5, 12), (16, 4), (3, 3)])
def test_full_seams_are_shared_rows(h, w):
    """The rows dropped at each seam equal the row kept (Section 3.3: quadrants
    are concatenated by their common edge rows)."""
    img = random_image(h, w, "u8", seed=11)
    quads = O._full_quadrants(img, "i64")
    hp, wp = O.next_pow2(h), O.next_pow2(w)
    assert (quads[O.Q0][0] == quads[O.Q1][0]).all()
    assert (quads[O.Q1][hp - 1] == quads[O.Q2][wp - 1]).all()
    assert (quads[O.Q2][0] == quads[O.Q3][0]).all()
    F = O.full(img)
    assert F.shape == O.full_geometry(h, w)


@pytest.mark.parametrize("py,px", [(0, 0), (3, 5), (7, 2), (6, 6)])
def test_point_maps_to_angle(py, px):
    """A single pixel maps to one nonzero per full-image row; along the
    mostly-vertical block the column runs monotonically from px-py to px+py and
    along the mostly-horizontal block back from py+px to py-px, each a digital
    straight segment (Eq. 1-2), the two meeting on the 45-degree seam row -- the
    "angle" figure of Section 6."""
    n = 8
    img = np.zeros((n, n), np.uint8)
    img[py, px] = 1
    F = O.full(img)
    R, W = F.shape
    assert (F.sum(axis=1) == 1).all()
    pos = np.argmax(F, axis=1)
    v = 2 * n - 1                       # rows of the mostly-vertical block
    unwrap = lambda a, ref: ((a - ref + W // 2) % W) - W // 2 + ref
    pv = unwrap(pos[:v], px)
    ph = unwrap(pos[v - 1:], py)        # shares the 45-degree row
    assert pv[0] == px - py and pv[-1] == px + py
    assert ph[0] == py + px and ph[-1] == py - px
    assert (np.diff(pv) >= 0).all() and (np.diff(ph) <= 0).all()
    K = 3
    for seg, a, b in ((pv[: n], px - py, px), (pv[n - 1:], px, px + py),
                      (ph[: n], py + px, py), (ph[n - 1:], py, py - px)):
        ideal = a + (b - a) * np.arange(n) / (n - 1)
        assert np.abs(seg - ideal).max() <= K / 6 + 1e-12


# --------------------------------------------------------------- range

def test_angle_to_slopes_at_2048():
    """[-15, 15] degrees at n = 2048: t <= floor(2047 tan 15deg) = 548 in Q0 and
    Q1, the 0-degree row once: 1097 rows."""
    lo, hi = O.angle_to_slopes(-15.0, 15.0, 2048, 2048)
    assert lo == [0, 1, -1, -1] and hi == [548, 548, -1, -1]
    assert math.floor(2047 * math.tan(math.radians(15))) == 548
    lo, hi = O.angle_to_slopes(75.0, 105.0, 2048, 2048)
    assert lo == [-1, -1, 0, 1] and hi == [-1, -1, 548, 548]
    lo, hi = O.angle_to_slopes(-45.0, 135.0, 64, 32)
    assert lo == [0, 1, 0, 1] and hi == [63, 63, 30, 31]


@pytest.mark.parametrize("a,b", [(-30.0, -10.0), (5.0, 44.0), (50.0, 80.0),
                                 (100.0, 130.0), (-45.0, 45.0)])
def test_angle_to_slopes_selects_exactly_the_range(a, b):
    n = 256
    lo, hi = O.angle_to_slopes(a, b, n, n)
    for q in range(4):
        for t in range(n):
            th = math.degrees(math.atan(t / (n - 1)))
            phi = {0: -th, 1: th, 2: 90 - th, 3: 90 + th}[q]
            inside = a - 1e-9 <= phi <= b + 1e-9
            chosen = lo[q] != -1 and lo[q] <= t <= hi[q]
            shared = ((q == 1 and t == 0 and lo[0] == 0) or
                      (q == 2 and t == n - 1 and hi[1] == n - 1) or
                      (q == 3 and t == 0 and lo[2] == 0))
            assert chosen == (inside and not shared), (q, t, phi)


def test_range_slice_is_quadrant_slice():
    img = edges_and_lines(64, 48, seed=4)
    H = O.quadrant(img, O.Q1)
    assert (O.range_slice(img, O.Q1, 5, 40) == H[5:41]).all()


# --------------------------------------------------------------- fhtshift

@pytest.mark.parametrize("h,w", [(8, 8), (16, 5), (7, 12)])
def test_fhtshift_centres_meaningful_zone(h, w):
    """After fhtshift each row holds its w_in + t meaningful pixels as one
    contiguous run starting at floor(b/2), the black zone split around it
    (Section 5); fhtshift is a permutation and its inverse undoes it."""
    img = random_image(h, w, "u8", seed=2, hi=4) + 1
    for q in range(4):
        H = O.quadrant(img, q)
        S = O.fhtshift_quadrant(H, h, w, q)
        n, W = H.shape
        w_in = h if O.TRANSPOSED[q] else w
        h_in = w if O.TRANSPOSED[q] else h
        for t in range(n):
            b = W - w_in - t
            start = b // 2
            if h_in == n:
                assert (S[t, start: start + w_in + t] > 0).all()
            assert S[t, :start].sum() == 0 and S[t, start + w_in + t:].sum() == 0
            assert sorted(S[t]) == sorted(H[t])
        assert (O.fhtshift_quadrant(S, h, w, q, inverse=True) == H).all()


def test_fhtshift_amounts_follow_paper():
    """Section 5, quadrant [315, 0] after flipping: the row on the 45-degree
    edge moves by about h and the vertical-lines row by h/2, rows in between by
    h - i/2 (i counted from the 45-degree row)."""
    n = w = 64
    W = w + n
    for t in range(n):
        s = O.fhtshift_amount(t, W, w, +1)
        i = n - 1 - t
        assert abs(s - (n - i / 2)) <= 1


def test_fhtshift_full_image_roundtrip():
    img = random_image(6, 10, "u8", seed=9, hi=3) + 1
    F = O.full(img)
    S = O.fhtshift_full(F, 6, 10)
    assert (O.fhtshift_full(S, 6, 10, inverse=True) == F).all()
    assert (np.sort(S, axis=1) == np.sort(F, axis=1)).all()


# --------------------------------------------------------------- adjoint

@pytest.mark.parametrize("h,w", [(4, 4), (3, 5), (8, 6)])
def test_adjoint_is_matrix_transpose(h, w):
    """The transposed butterfly equals the explicit matrix transpose and the
    back-projection sum, exactly in integers, for all four quadrants."""
    rng = np.random.default_rng(h + w)
    for q in range(4):
        M = O.explicit_matrix(h, w, q)
        n, W = O.quadrant_geometry(h, w, q)
        G = rng.integers(-9, 9, size=(n, W)).astype(np.int64)
        got = O.adjoint_quadrant(G, h, w, q, "i64")
        assert (got.ravel() == M.T @ G.ravel()).all()
        x = rng.integers(-9, 9, size=(h, w)).astype(np.int64)
        assert (O.quadrant(x, q).ravel() == M @ x.ravel()).all()
        sig = O.SIGMA[q]
        assert (O.adjoint_butterfly(G, sig, "i64") == O.brute_adjoint(G, sig, "i64")).all()
        assert (O.adjoint_quadrant_transposed_network(G, h, w, q, "i64") == got).all()


@pytest.mark.parametrize("h,w", [(64, 64), (100, 37), (33, 130)])
def test_adjoint_float_agrees_with_transposed_network(h, w):
    """The FP32 adjoint (opposite-sign recursion) and the FP32 transposed
    network round differently but both stay within the FP32 bound of FP64."""
    rng = np.random.default_rng(h)
    for q in range(4):
        n, W = O.quadrant_geometry(h, w, q)
        G = rng.standard_normal((n, W)).astype(np.float32)
        mass = float(np.abs(G.astype(np.float64)).sum())
        ref = O.adjoint_quadrant(G.astype(np.float64), h, w, q, "f64")
        for got in (O.adjoint_quadrant(G, h, w, q, "f32"),
                    O.adjoint_quadrant_transposed_network(G, h, w, q, "f32")):
            assert np.abs(got - ref).max() <= 1e-5 * mass
        assert np.abs(ref - O.adjoint_quadrant_transposed_network(
            G.astype(np.float64), h, w, q, "f64")).max() <= 1e-9 * mass


@pytest.mark.parametrize("h,w", [(32, 32), (20, 13)])
def test_full_adjoint_dot_product(h, w):
    """<F x, y> = <x, F^T y> for the full-image map (float64)."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((h, w))
    R, W = O.full_geometry(h, w)
    y = rng.standard_normal((R, W))
    lhs = float((O.full(x, "f64") * y).sum())
    rhs = float((x * O.adjoint_full(y, h, w, "f64")).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))


def test_finite_differences_of_fit_loss():
    """Gradient of L(x) = ||F x - b||^2 is 2 F^T (F x - b); check it against
    central differences at 32 x 32 (exact up to rounding: L is quadratic)."""
    h = w = 32
    rng = np.random.default_rng(2)
    x = rng.standard_normal((h, w))
    b = O.full(rng.standard_normal((h, w)), "f64")
    grad = 2.0 * O.adjoint_full(O.full(x, "f64") - b, h, w, "f64")
    L = lambda z: float(((O.full(z, "f64") - b) ** 2).sum())
    for k in range(6):
        i, j = rng.integers(0, h), rng.integers(0, w)
        e = np.zeros_like(x)
        e[i, j] = 1e-3
        fd = (L(x + e) - L(x - e)) / 2e-3
        assert abs(fd - grad[i, j]) <= 1e-6 * max(1.0, abs(fd))


# --------------------------------------------------------------- precision

def test_fp32_tree_within_tolerance_of_fp64():
    """The FP32 recursion stays within 1e-5 * sum|I| of FP64 (each output is a
    depth-log2(n) pairwise sum, error <= log2(n) * 2^-24 * sum|terms|)."""
    img = random_image(128, 96, "f32", seed=5)
    mass = float(np.abs(img.astype(np.float64)).sum())
    for q in range(4):
        a = O.quadrant(img, q, "f32").astype(np.float64)
        b = O.quadrant(img.astype(np.float64), q, "f64")
        assert np.abs(a - b).max() <= 1e-5 * mass
        K = int(math.log2(a.shape[0]))
        assert np.abs(a - b).max() <= K * 2.0 ** -24 * mass


def test_sampled_points_match_full_transform():
    img = edges_and_lines(37, 53, seed=8)
    rng = np.random.default_rng(0)
    for q in range(4):
        H = O.quadrant(img, q)
        n, W = H.shape
        ts = rng.integers(0, n, 50)
        xs = rng.integers(0, W, 50)
        assert (O.points(img, q, ts, xs) == H[ts, xs]).all()
        F = O._full_quadrants(img, "i64")[q]
        n2, W2 = F.shape
        ts = rng.integers(0, n2, 50)
        xs = rng.integers(0, W2, 50)
        assert (O.points(img, q, ts, xs, full_layout=True) == F[ts, xs]).all()


# --------------------------------------------------------------- shear (Section 4)

def test_shear_shifts_round_half_up():
    """s(y) = floor(y*spl + 1/2): exact halves round up, negative shifts round
    towards +infinity at halves, spl = 0 gives no shift; with spl in 32-bit
    fixed point the result equals the real-number formula away from halves."""
    rng = np.random.default_rng(0)
    for spl in rng.uniform(-1, 1, 20):
        ys = np.arange(4096)
        exact = np.floor(ys * spl + 0.5)
        near_half = np.abs((ys * spl + 0.5) - np.round(ys * spl + 0.5)) < 1e-6
        assert (O.shear_shifts(4096, spl)[~near_half] == exact[~near_half]).all()
    assert list(O.shear_shifts(5, 0.5)) == [0, 1, 1, 2, 2]
    assert list(O.shear_shifts(5, -0.5)) == [0, 0, -1, -1, -2]
    assert list(O.shear_shifts(4, 0.0)) == [0, 0, 0, 0]
    assert list(O.shear_shifts(4, 1.0)) == [0, 1, 2, 3]
    assert list(O.shear_shifts(4, -1.0)) == [0, -1, -2, -3]


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_shear_zero_is_the_plain_quadrant(q):
    img = random_image(37, 21, "u8", seed=q)
    assert (O.sheared_quadrant(img, q, 0.0) == O.quadrant(img, q)).all()


@pytest.mark.parametrize("q,spl", [(0, 0.37), (1, -0.6), (2, 1.0), (3, -1.0), (0, -0.25),
                                   (3, 0.8)])
def test_shear_equals_brute_force_sums(q, spl):
    """Every point is the sum of the image along the pattern minus the per-row
    shift, H[t][x] = sum_y P[y][(x + sigma*off(t, y) - s(y)) mod W], written
    out with the closed-form offsets (no butterfly, no array rotation)."""
    img = random_image(11, 6, "u8", seed=7)
    h, w = img.shape
    src = img.T if O.TRANSPOSED[q] else img
    n, W = O.quadrant_geometry(h, w, q)
    sg = O.SIGMA[q]
    s = [math.floor(y * spl + 0.5) for y in range(src.shape[0])]
    H = np.zeros((n, W), np.int64)
    for t in range(n):
        for x in range(W):
            acc = 0
            for y in range(src.shape[0]):
                c = (x + sg * O.offset(n, t, y) - s[y]) % W
                if c < src.shape[1]:
                    acc += int(src[y, c])
            H[t, x] = acc
    assert (O.sheared_quadrant(img, q, spl) == H).all()


def test_unit_shear_turns_45_degree_row_into_column_sums():
    """off_n(n-1, y) = y, so the 45-degree row after a unit shear against it
    sums straight down the columns: Q0 with spl = 1 and Q1 with spl = -1 give
    the image's column sums at their row n - 1 (and Q3 with spl = 1 the row
    sums, through the transpose)."""
    img = random_image(29, 40, "u8", seed=3)
    h, w = img.shape
    n, W = O.quadrant_geometry(h, w, 0)
    col = np.zeros(W, np.int64)
    col[:w] = img.astype(np.int64).sum(axis=0)
    assert (O.sheared_quadrant(img, 0, 1.0)[n - 1] == col).all()
    assert (O.sheared_quadrant(img, 1, -1.0)[n - 1] == col).all()
    n3, W3 = O.quadrant_geometry(h, w, 3)
    row = np.zeros(W3, np.int64)
    row[:h] = img.astype(np.int64).sum(axis=1)
    assert (O.sheared_quadrant(img, 3, 1.0)[n3 - 1] == row).all()


@pytest.mark.parametrize("phi", [-14.0, -6.5, 0.0, 3.0, 11.0, 15.0])
def test_sheared_range_finds_lines_at_their_angle(phi):
    """A straight line at angle phi (dx/dy = -tan(phi), the angle convention
    of the quadrants: Q0 holds [-45, 0]) rasterised into a 256 x 256 image
    peaks, in the one sheared quadrant that shear_range picks for
    [-15, 15] degrees, at the row whose angle is phi within one slope step, and
    the range's rows stop exactly at its ends."""
    n = 256
    q, spl, t_lo, t_hi = O.shear_range(-15.0, 15.0, n, n)
    assert q == 0 and t_lo == 0
    assert spl == pytest.approx(math.tan(math.radians(15.0)))
    # row angles: phi(t) = atan(spl - t/(n-1)) within [-15, 15], the next outside
    ang = lambda t: math.degrees(math.atan(spl - t / (n - 1)))  # noqa: E731
    assert ang(0) == pytest.approx(15.0)
    assert ang(t_hi) >= -15.0 - 1e-9 and ang(t_hi + 1) < -15.0
    img = np.zeros((n, n), np.uint8)
    k = -math.tan(math.radians(phi))
    x0 = n / 2 - k * n / 2
    for y in range(n):
        img[y, int(math.floor(x0 + k * y + 0.5))] = 1
    H = O.sheared_quadrant(img, q, spl, t_lo=t_lo, t_hi=t_hi)
    t_pk = int(np.unravel_index(np.argmax(H), H.shape)[0])
    step = math.degrees(math.atan(1 / (n - 1)))
    assert abs(ang(t_pk) - phi) <= 1.5 * step
    # the pattern (within log2(n)/6 columns of straight), the shear's and the
    # line's roundings (half a column each) leave at most about 2.3 columns
    # between the peak's pattern and the line: most of its pixels are summed
    assert H.max() >= 0.5 * n


def test_shear_range_horizontal_and_rejections():
    """Mostly horizontal ranges go to Q3 (angles from phi_lo up); ranges that
    cross 45 degrees or span more than 45 degrees around an axis do not fit
    one quadrant."""
    q, spl, t_lo, t_hi = O.shear_range(75.0, 105.0, 300, 2048)
    n, _ = O.quadrant_geometry(300, 2048, 3)
    assert q == 3 and t_lo == 0
    assert spl == pytest.approx(math.tan(math.radians(15.0)))
    assert t_hi == math.floor((n - 1) * 2 * math.tan(math.radians(15.0)) + 1e-9)
    assert O.shear_range(30.0, 60.0, 64, 64) is None
    assert O.shear_range(-30.0, 30.0, 64, 64) is None
    assert O.shear_range(-45.0, 0.0, 64, 64)[3] == 63


# --------------------------------------------------------------- point -> segment (Section 3.2)

@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_point_segment_is_what_the_point_sums(q):
    """An image that is 1 exactly on the returned pixels' run (the pattern
    between the two ends, rows in between included) and 0 elsewhere makes
    the Hough point's value the returned count; a random image's value at
    the point is the sum over those pixels. Covers every point of a small
    quadrant, cases a, b and c included."""
    h, w = 9, 14
    img = random_image(h, w, "u8", seed=q)
    H = O.quadrant(img, q)
    n, W = O.quadrant_geometry(h, w, q)
    ones = O.quadrant(np.ones((h, w), np.uint8), q)
    for t in range(n):
        for x in range(W):
            seg = O.point_segment(h, w, q, t, x)
            if seg is None:
                assert H[t, x] == 0 and ones[t, x] == 0
                continue
            count, a, b = seg
            assert ones[t, x] == count
            # the pixels: the pattern's rows between the two ends
            tot = 0
            ya, yb = (a[1], b[1]) if O.TRANSPOSED[q] else (a[0], b[0])
            for y in range(ya, yb + 1):
                c = (x + O.SIGMA[q] * O.offset(n, t, y)) % W
                r, cc = (c, y) if O.TRANSPOSED[q] else (y, c)
                assert 0 <= r < h and 0 <= cc < w
                tot += int(img[r, cc])
            assert tot == H[t, x]


def test_point_segment_paper_cases():
    """Section 3.2 for Q0 of a 6 x 10 image (n = 8, W = 18): (case a) a
    pattern that leaves the image through its right side keeps the part
    inside; (case b) one that leaves the extended image re-enters on the left
    (columns modulo w + n); (case c) one wholly in the extension sums
    nothing."""
    h, w = 6, 10
    # vertical pattern from column 3: all six image rows
    assert O.point_segment(h, w, 0, 0, 3) == (6, (0, 3), (5, 3))
    # 45-degree pattern from column 7: rows 0..2 at columns 7..9, then leaves (a)
    assert O.point_segment(h, w, 0, 7, 7) == (3, (0, 7), (2, 9))
    # 45-degree pattern from column 15: columns 15, 16, 17 in the extension,
    # then 18 = 0 (mod 18): rows 3..5 at columns 0..2 (b)
    assert O.point_segment(h, w, 0, 7, 15) == (3, (3, 0), (5, 2))
    # vertical pattern in the extension (c)
    assert O.point_segment(h, w, 0, 0, 12) is None


# --------------------------------------------------------------- other operations (max, min)

@pytest.mark.parametrize("q", [0, 1, 2, 3])
@pytest.mark.parametrize("op", [1, 2])
def test_max_min_equal_brute_force(q, op):
    """Every point is the maximum (minimum) of the zero-padded image along the
    pattern, written out with the closed-form offsets."""
    img = random_image(7, 11, "u8", seed=q + 10 * op)
    h, w = img.shape
    src = img.T if O.TRANSPOSED[q] else img
    n, W = O.quadrant_geometry(h, w, q)
    P = np.zeros((n, W), np.int64)
    P[:src.shape[0], :src.shape[1]] = src
    f = max if op == 1 else min
    H = np.array([[f(int(P[y, (x + O.SIGMA[q] * O.offset(n, t, y)) % W]) for y in range(n))
                   for x in range(W)] for t in range(n)])
    assert (O.quadrant_op(img, q, op) == H).all()


@pytest.mark.parametrize("hw", [(16, 16), (13, 40), (64, 9)])
def test_max_min_of_binary_images_follow_the_sum(hw):
    """On a 0/1 image the maximum along a pattern is 1 exactly where the sum
    is positive; on an all-ones image the minimum is 1 exactly where the
    pattern never leaves the image (sum = n)."""
    h, w = hw
    img = (random_image(h, w, "u8", seed=h) > 200).astype(np.uint8)
    for q in range(4):
        assert (O.quadrant_op(img, q, 1) == (O.quadrant(img, q) > 0)).all()
        ones = np.ones((h, w), np.uint8)
        n, _ = O.quadrant_geometry(h, w, q)
        assert (O.quadrant_op(ones, q, 2) == (O.quadrant(ones, q) == n)).all()


def test_min_is_negated_max_of_negated_image():
    """min along a pattern = -max of the negated values (zero padding is its
    own negation), in int64 and in float32."""
    img = random_image(20, 33, "i32", seed=4, hi=100)
    for q in range(4):
        assert (O.quadrant_op(img, q, 2) == -O.quadrant_op(-img, q, 1)).all()
        f = img.astype(np.float32) / 7
        assert (O.quadrant_op(f, q, 2, "f32") == -O.quadrant_op(-f, q, 1, "f32")).all()


# --------------------------------------------------------------- scale (Section 4)

def test_scale_columns_replicate_and_subsample():
    """Column x' of the row scaled by alpha is column floor(x'/alpha): an
    integer factor k repeats every column k times (np.repeat), 1/k keeps
    every k-th column, 1 is the identity; the scaled width counts the
    columns whose source lies inside the row."""
    img = random_image(9, 13, "u8", seed=5)
    for k in (2, 3, 5, 7):
        assert np.array_equal(O.scaled_image(img, float(k)), np.repeat(img, k, axis=1))
        assert O.scaled_width(13, float(k)) == 13 * k
    for k in (2, 4, 8):
        assert np.array_equal(O.scaled_image(img, 1.0 / k), img[:, ::k])
        assert O.scaled_width(13, 1.0 / k) == -(-13 // k)
    assert np.array_equal(O.scaled_image(img, 1.0), img)
    # any factor: monotone, steps of floor(1/alpha) or ceil(1/alpha) source
    # columns, within one column of x'/alpha, and every source column < w
    for alpha in (0.3, 0.7, 1.37, 2.5, 5.9):
        src = O.scale_columns(101, alpha)
        assert src[0] == 0 and src[-1] < 101
        assert abs(src - np.floor(np.arange(len(src)) / alpha)).max() <= 1
        assert set(np.unique(np.diff(src))) <= {math.floor(1 / alpha), math.ceil(1 / alpha)}
        assert O.scale_columns(101, alpha).size == O.scaled_width(101, alpha)
        assert (O.scaled_width(101, alpha) * O.scale_step(alpha)) >> 32 >= 101


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_scale_one_is_the_plain_quadrant(q):
    img = random_image(37, 21, "u8", seed=q)
    assert (O.scaled_quadrant(img, q, 1.0) == O.quadrant(img, q)).all()
    assert (O.scaled_quadrant(img, q, 1.0, 0.4) == O.sheared_quadrant(img, q, 0.4)).all()


@pytest.mark.parametrize("q,alpha,spl", [(0, 2.0, 0.0), (1, 3.0, -0.3), (2, 0.5, 0.6),
                                         (3, 0.25, -1.0), (0, 0.5, 1.0), (3, 2.0, 0.45)])
def test_scaled_quadrant_equals_brute_force_sums(q, alpha, spl):
    """Every point is the sum along the pattern over the scaled, sheared
    image, written out with the closed-form offsets and the real-number
    source column floor(c/alpha) (exact for these factors): H[t][x] =
    sum_y I[y][floor(c/alpha)] at c = (x + sigma*off(t, y) - s(y)) mod W when
    c < w_alpha, with W = w_alpha + n. No butterfly, no resampled array."""
    img = random_image(10, 7, "u8", seed=11)
    h, w = img.shape
    src = img.T if O.TRANSPOSED[q] else img
    rows, cols = src.shape
    n = O.next_pow2(rows)
    wa = math.ceil(cols * alpha - 1e-12)   # columns x' with floor(x'/alpha) < cols
    W = wa + n
    sg = O.SIGMA[q]
    # the per-row shifts as pinned by test_shear_shifts_round_half_up (exact
    # halves such as 5 * -0.3 + 1/2 follow the fixed-point spl)
    s = [int(v) for v in O.shear_shifts(rows, spl)]
    H = np.zeros((n, W), np.int64)
    for t in range(n):
        for x in range(W):
            acc = 0
            for y in range(rows):
                c = (x + sg * O.offset(n, t, y) - s[y]) % W
                if c < wa:
                    acc += int(src[y, int(math.floor(c / alpha + 1e-12))])
            H[t, x] = acc
    got = O.scaled_quadrant(img, q, alpha, spl)
    assert got.shape == (n, W)
    assert (got == H).all()


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_scaled_rows_sum_to_the_scaled_mass(q):
    """Every slope row of the scaled quadrant (no shear) sums to the mass of
    the scaled image: each of its pixels lies on exactly one pattern per row
    (the mass invariant of the plain quadrant, on the resampled image)."""
    img = random_image(45, 30, "u8", seed=20 + q)
    src = img.T if O.TRANSPOSED[q] else img
    for alpha in (0.6, 1.8, 3.0):
        H = O.scaled_quadrant(img, q, alpha)
        mass = int(O.scaled_image(src, alpha).astype(np.int64).sum())
        assert (H.sum(axis=1) == mass).all()


def test_scaled_line_lands_on_the_45_degree_row():
    """Section 4: scaling by alpha turns a line at tg(beta) = 1/alpha into one
    at 45 degrees. A line with dx/dy = 1/2 (one column every second row),
    scaled by 2, is a two-pixel-wide staircase whose left edge is the exact
    diagonal, which the slope n-1 pattern (off(n-1, y) = y) follows: that
    Hough point sums one pixel of every row."""
    n, x0 = 64, 5
    img = np.zeros((n, n), np.uint8)
    for y in range(n):
        img[y, x0 + y // 2] = 1
    H = O.scaled_quadrant(img, 0, 2.0)
    assert H[n - 1, 2 * x0] == n
    assert H.max() == n
    assert np.unravel_index(np.argmax(H[:, 2 * x0]), (n,))[0] == n - 1


@pytest.mark.parametrize("phi", [-14.0, -6.5, 0.0, 3.0, 11.0, 15.0])
def test_scale_range_finds_lines_at_their_angle(phi):
    """The [-15, 15] degree range as one scaled and sheared quadrant: alpha
    = 1/(2 tan 15) stretches it over every slope row (spl = 1/2), so its
    angles are resolved 1.87 times finer than with the shear alone; a
    rasterised line at phi peaks at the row whose angle is phi within about
    one of those finer steps, and the last row is the range's lower end."""
    n = 256
    q, alpha, spl, t_lo, t_hi = O.scale_range(-15.0, 15.0, n, n)
    assert q == 0 and t_lo == 0 and t_hi == n - 1
    assert alpha == pytest.approx(1 / (2 * math.tan(math.radians(15.0))))
    assert spl == pytest.approx(0.5)
    ang = lambda t: math.degrees(math.atan((spl - t / (n - 1)) / alpha))  # noqa: E731
    assert ang(0) == pytest.approx(15.0) and ang(n - 1) == pytest.approx(-15.0)
    img = np.zeros((n, n), np.uint8)
    k = -math.tan(math.radians(phi))
    x0 = n / 2 - k * n / 2
    for y in range(n):
        img[y, int(math.floor(x0 + k * y + 0.5))] = 1
    H = O.scaled_quadrant(img, q, alpha, spl, t_lo=t_lo, t_hi=t_hi)
    t_pk = int(np.unravel_index(np.argmax(H), H.shape)[0])
    step = math.degrees(math.atan(1 / ((n - 1) * alpha)))
    assert abs(ang(t_pk) - phi) <= 2.5 * step
    assert H.max() >= 0.5 * n


def test_scale_range_choices():
    """Symmetric ranges fill the quadrant with spl = 1/2; an off-axis narrow
    range is stretched until its far end reaches the unit shear; mostly
    horizontal ranges go to Q3; the paper's arctg(1/2) neighbourhood of zero
    needs no scale (alpha = 1, spl = 1/2)."""
    for g in (5.0, 20.0, 40.0, 60.0):
        q, alpha, spl, t_lo, t_hi = O.scale_range(-g, g, 512, 512)
        assert q == 0 and spl == pytest.approx(0.5) and t_hi == 511
        assert alpha == pytest.approx(min(16.0, 1 / (2 * math.tan(math.radians(g)))))
    g = math.degrees(math.atan(0.5))
    q, alpha, spl, _, t_hi = O.scale_range(-g, g, 512, 512)
    assert alpha == pytest.approx(1.0) and spl == pytest.approx(0.5) and t_hi == 511
    q, alpha, spl, _, t_hi = O.scale_range(10.0, 20.0, 512, 512)
    assert q == 0 and spl == pytest.approx(1.0)
    assert alpha == pytest.approx(1 / math.tan(math.radians(20.0)))
    assert t_hi == math.floor(511 * alpha * (math.tan(math.radians(20.0)) -
                                             math.tan(math.radians(10.0))) + 1e-9)
    q, alpha, spl, _, t_hi = O.scale_range(80.0, 100.0, 300, 600)
    assert q == 3 and spl == pytest.approx(0.5) and t_hi == O.quadrant_geometry(300, 600, 3)[0] - 1
    assert O.scale_range(20.0, 10.0, 64, 64) is None
    assert O.scale_range(-95.0, 0.0, 64, 64) is None
