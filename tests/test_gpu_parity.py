"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results are compared bit for bit. FP32 results are compared bit for
bit with the oracle's FP32 run of the same addition tree, and within
1e-5 * sum|I| of the FP64 oracle (the bound the recursion's depth-log2(n)
pairwise sums guarantee with a wide margin: log2(n) * 2^-24 < 1e-6)."""

import math

import numpy as np
import pytest
import torch

import oracle as O
from workloads import (edges_and_lines, ellipse_phantom, random_image, text_stripes,
                       batch_shapes, edge_batch)

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def as_i32(a: np.ndarray) -> np.ndarray:
    """int64 oracle values reduced modulo 2^32, as the int32 kernels wrap."""
    return a.astype(np.int64).astype(np.int32)


SIZES = [(1, 1), (1, 7), (2, 3), (5, 1), (3, 40), (37, 53), (64, 64), (100, 300),
         (256, 256), (300, 129), (513, 200), (1000, 77)]


@pytest.mark.parametrize("h,w", SIZES)
def test_quadrants_u8_i32_bit_exact(fht, h, w):
    img = edges_and_lines(h, w, seed=h * 7 + w) if h > 2 and w > 2 else \
        random_image(h, w, "u8", seed=h + w)
    x = dev(img)
    for q in range(4):
        got = host(fht.forward(x, q))
        assert got.dtype == np.int32
        assert (got == as_i32(O.quadrant(img, q))).all(), q


@pytest.mark.parametrize("h,w", [(37, 53), (129, 300), (700, 90)])
def test_quadrants_i32_signed_bit_exact(fht, h, w):
    img = random_image(h, w, "i32", seed=5, hi=1 << 20)
    x = dev(img)
    for q in range(4):
        assert (host(fht.forward(x, q)) == as_i32(O.quadrant(img, q))).all(), q


@pytest.mark.parametrize("h,w", [(37, 53), (256, 300), (700, 513)])
def test_quadrants_f32(fht, h, w):
    img = random_image(h, w, "f32", seed=h)
    x = dev(img)
    mass = float(np.abs(img.astype(np.float64)).sum())
    for q in range(4):
        got = host(fht.forward(x, q, acc=torch.float32))
        assert (got == O.quadrant(img, q, "f32")).all(), q
        ref = O.quadrant(img.astype(np.float64), q, "f64")
        assert np.abs(got - ref).max() <= FP32_TOL * mass


def test_u8_into_f32(fht):
    img = text_stripes(200, 330, n_stripes=5, seed=3)
    x = dev(img)
    for q in range(4):
        got = host(fht.forward(x, q, acc=torch.float32))
        assert (got == O.quadrant(img, q, "f32")).all(), q


@pytest.mark.parametrize("h,w", [(256, 256), (300, 257), (77, 1000)])
def test_range_is_bit_exact_slice(fht, h, w):
    img = edges_and_lines(h, w, seed=9)
    x = dev(img)
    for q in range(4):
        H = O.quadrant(img, q)
        n = H.shape[0]
        for lo, hi in [(0, 0), (0, n - 1), (n - 1, n - 1), (1, n // 3), (n // 5, n // 2 + 3),
                       (n // 2, n - 2)]:
            if not 0 <= lo <= hi < n:
                continue
            got = host(fht.forward_range(x, q, lo, hi))
            assert (got == as_i32(H[lo: hi + 1])).all(), (q, lo, hi)


def test_range_f32(fht):
    img = random_image(190, 260, "f32", seed=1)
    x = dev(img)
    H = O.quadrant(img, 1, "f32")
    got = host(fht.forward_range(x, 1, 17, 100, acc=torch.float32))
    assert (got == H[17:101]).all()


@pytest.mark.parametrize("h,w", [(1, 1), (5, 12), (37, 53), (256, 256), (300, 129),
                                 (64, 1000)])
def test_full_image_bit_exact(fht, h, w):
    img = edges_and_lines(h, w, seed=2) if min(h, w) > 2 else random_image(h, w, "u8")
    x = dev(img)
    F = O.full(img)
    assert (host(fht.full_quadrants(x)) == as_i32(F)).all()
    S = O.fhtshift_full(F, h, w)
    assert (host(fht.full_quadrants(x, apply_fhtshift=True)) == as_i32(S)).all()


def test_full_image_f32(fht):
    img = ellipse_phantom(150, n_ellipses=6, seed=4, m=211)
    x = dev(img)
    assert (host(fht.full_quadrants(x, acc=torch.float32)) == O.full(img, "f32")).all()


@pytest.mark.parametrize("h,w", [(8, 8), (37, 53), (256, 100)])
def test_fhtshift_standalone(fht, h, w):
    img = edges_and_lines(h, w, seed=6)
    x = dev(img)
    F = fht.full_quadrants(x)
    S = host(fht.fhtshift(F, h, w, fht.LAYOUT_FULL))
    assert (S == as_i32(O.fhtshift_full(O.full(img), h, w))).all()
    back = host(fht.fhtshift(dev(S), h, w, fht.LAYOUT_FULL, inverse=True))
    assert (back == host(F)).all()
    for q in range(4):
        H = fht.forward(x, q)
        S = host(fht.fhtshift(H, h, w, fht.LAYOUT_QUADRANT, q))
        assert (S == as_i32(O.fhtshift_quadrant(O.quadrant(img, q), h, w, q))).all()
        Hf = H.float()
        Sf = host(fht.fhtshift(Hf, h, w, fht.LAYOUT_QUADRANT, q))
        assert (Sf == S.astype(np.float32)).all()


def test_fhtshift_pitches_and_alignment(fht):
    """Rows move as 16-byte vectors when the row width, both pitches and both
    base addresses allow it, else word by word: every combination gives the
    oracle's rows."""
    h, w = 300, 500
    img = edges_and_lines(h, w, seed=8)
    want = as_i32(O.fhtshift_full(O.full(img), h, w))
    F = fht.full_quadrants(dev(img))
    R, W = F.shape
    assert W % 4 == 0
    for in_extra, in_off, out_extra, out_off in [(0, 0, 4, 0), (3, 0, 0, 0), (4, 1, 0, 0),
                                                 (0, 0, 8, 3), (5, 2, 7, 1)]:
        src_buf = torch.zeros((R, W + in_extra + in_off), dtype=torch.int32, device="cuda")
        src = src_buf[:, in_off:in_off + W]
        src.copy_(F)
        dst_buf = torch.full((R, W + out_extra + out_off), -5, dtype=torch.int32, device="cuda")
        dst = dst_buf[:, out_off:out_off + W]
        fht.fhtshift(src, h, w, fht.LAYOUT_FULL, out=dst)
        got = host(dst_buf)
        assert (got[:, out_off:out_off + W] == want).all(), (in_extra, in_off, out_extra, out_off)
        assert (got[:, :out_off] == -5).all() and (got[:, out_off + W:] == -5).all()


@pytest.mark.parametrize("h,w", [(1, 1), (3, 5), (32, 32), (37, 53), (200, 129)])
def test_adjoint_quadrant(fht, h, w):
    rng = np.random.default_rng(h * w)
    for q in range(4):
        n, W = O.quadrant_geometry(h, w, q)
        g = rng.standard_normal((n, W)).astype(np.float32)
        got = host(fht.adjoint(dev(g), h, w, fht.LAYOUT_QUADRANT, q))
        assert (got == O.adjoint_quadrant(g, h, w, q, "f32")).all(), q
        gi = rng.integers(-1000, 1000, size=(n, W)).astype(np.int32)
        got = host(fht.adjoint(dev(gi), h, w, fht.LAYOUT_QUADRANT, q))
        assert (got == as_i32(O.adjoint_quadrant(gi.astype(np.int64), h, w, q, "i64"))).all()


@pytest.mark.parametrize("h,w", [(1, 1), (5, 12), (32, 32), (100, 70)])
def test_adjoint_full(fht, h, w):
    rng = np.random.default_rng(7)
    R, W = O.full_geometry(h, w)
    g = rng.standard_normal((R, W)).astype(np.float32)
    got = host(fht.adjoint(dev(g), h, w, fht.LAYOUT_FULL))
    assert (got == O.adjoint_full(g, h, w, "f32")).all()


@pytest.mark.parametrize("h,w,q", [(1500, 300, 0), (300, 1500, 3), (1000, 77, 1),
                                   (8192, 200, 1), (200, 8192, 2)])
def test_adjoint_quadrant_multi_pass_exact(fht, h, w, q):
    """Two-pass (K = 10, 11) and three-pass (K = 13) quadrant adjoints, whose
    last intermediate level keeps only the columns its final pass reads,
    every element bit-exact against the oracle's FP32 recursion."""
    n, W = O.quadrant_geometry(h, w, q)
    g = np.random.default_rng(h + 3 * w + q).standard_normal((n, W)).astype(np.float32)
    got = host(fht.adjoint(dev(g), h, w, fht.LAYOUT_QUADRANT, q))
    assert (got == O.adjoint_quadrant(g, h, w, q, "f32")).all()


def test_adjoint_full_4096_complete(fht):
    """The benchmark's adjoint: a 16381 x 8192 FP32 gradient back-projected
    onto the 4096 x 4096 image (four quadrants, two passes each), every
    element bit-exact against the oracle's FP32 recursion."""
    R, W = O.full_geometry(4096, 4096)
    g = np.random.default_rng(4096).standard_normal((R, W), dtype=np.float32)
    got = host(fht.adjoint(dev(g), 4096, 4096, fht.LAYOUT_FULL))
    assert (got == O.adjoint_full(g, 4096, 4096, "f32")).all()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("h,w", [(32, 32), (50, 77)])
def test_dot_product_on_gpu(fht, h, w):
    """<F x, y> = <x, F^T y>, both sides computed by the CUDA kernels."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((h, w)).astype(np.float32)
    R, W = O.full_geometry(h, w)
    y = rng.standard_normal((R, W)).astype(np.float32)
    Fx = host(fht.full_quadrants(dev(x), acc=torch.float32)).astype(np.float64)
    Fty = host(fht.adjoint(dev(y), h, w, fht.LAYOUT_FULL)).astype(np.float64)
    lhs, rhs = float((Fx * y).sum()), float((x * Fty).sum())
    assert abs(lhs - rhs) <= 1e-4 * (np.abs(Fx * y).sum())


def test_autograd_matches_adjoint_and_descends(fht):
    h = w = 32
    xt = ellipse_phantom(h, n_ellipses=4, seed=9, noise_sigma=0.0)
    b = fht.full_quadrants(dev(xt), acc=torch.float32)
    x = torch.zeros((h, w), device="cuda", requires_grad=True)
    y = fht.FHTFunction.apply(x)
    loss = ((y - b) ** 2).sum()
    loss.backward()
    # d loss / d y = 2 (y - b), and scaling by 2 commutes with every FP32 add
    r = (y - b).detach().cpu().numpy()
    expect = 2.0 * O.adjoint_full(r, h, w, "f32")
    assert np.array_equal(x.grad.cpu().numpy(), expect)
    # finite difference of the loss along one coordinate (float64 on the host)
    xh = np.zeros((h, w))
    bh = O.full(xt.astype(np.float64), "f64")
    i, j = 10, 17
    e = np.zeros((h, w))
    e[i, j] = 1e-2
    L = lambda z: float(((O.full(z, "f64") - bh) ** 2).sum())
    fd = (L(xh + e) - L(xh - e)) / 2e-2
    assert abs(fd - float(x.grad[i, j])) <= 1e-3 * max(1.0, abs(fd))
    # a few gradient steps reduce the loss
    lr = 1.0 / (2.0 * 4 * (2 * 32) * 32)   # safe bound: lambda_max(F^T F) <= 4 * rows * n
    losses = []
    with torch.no_grad():
        z = torch.zeros((h, w), device="cuda")
        for _ in range(5):
            r = fht.full_quadrants(z, acc=torch.float32) - b
            losses.append(float((r * r).sum()))
            z -= lr * 2.0 * fht.adjoint(r, h, w)
    assert all(b2 <= a2 for a2, b2 in zip(losses, losses[1:])) and losses[-1] < losses[0]


# ----------------------------------------------------------- workload sizes

def test_config_256_u8_q0(fht):
    """256 x 256 binary edges + 4 lines, Q0 -> 256 x 512 int32."""
    img = edges_and_lines(256, 256, p_edge=0.05, n_lines=4, seed=0)
    got = host(fht.forward(dev(img), 0))
    assert got.shape == (256, 512)
    assert (got == O.quadrant(img, 0)).all()


def test_config_2048_full_range_fhtshift(fht):
    """2048 x 2048 text-stripe page: full image (8189 x 4096), the [-15, 15]
    and [75, 105] degree ranges, and fhtshift of the full image."""
    img = text_stripes(2048, 2048, seed=1)
    x = dev(img)
    F = O.full(img)
    assert F.shape == (8189, 4096)
    Fg = fht.full_quadrants(x)
    assert (host(Fg) == F).all()
    S = host(fht.fhtshift(Fg, 2048, 2048, fht.LAYOUT_FULL))
    assert (S == O.fhtshift_full(F, 2048, 2048)).all()
    for a, b in [(-15.0, 15.0), (75.0, 105.0)]:
        lo, hi = fht.angle_to_slopes(a, b, 2048, 2048)
        assert (lo, hi) == tuple(O.angle_to_slopes(a, b, 2048, 2048))
        rows = 0
        for q in range(4):
            if lo[q] < 0:
                continue
            got = host(fht.forward_range(x, q, lo[q], hi[q]))
            H = O.quadrant(img, q)
            assert (got == H[lo[q]: hi[q] + 1]).all(), q
            rows += got.shape[0]
        assert rows == 1097


def test_config_4096_u8_q0_complete(fht):
    """4096 x 4096 edge map, Q0 -> 4096 x 8192 int32, every element."""
    img = edges_and_lines(4096, 4096, p_edge=0.05, n_lines=4, seed=4096)
    got = host(fht.forward(dev(img), 0))
    assert (got == O.quadrant(img, 0)).all()


def test_config_4096_all_quadrants_sampled(fht):
    img = edges_and_lines(4096, 4096, p_edge=0.05, n_lines=4, seed=4097)
    x = dev(img)
    rng = np.random.default_rng(0)
    F = host(fht.full_quadrants(x))
    R, W = F.shape
    for q in range(4):
        H = host(fht.forward(x, q))
        n, Wq = H.shape
        ts, xs = rng.integers(0, n, 400), rng.integers(0, Wq, 400)
        ts[:4] = [0, n - 1, 0, n - 1]
        xs[:4] = [0, 0, Wq - 1, Wq - 1]
        assert (H[ts, xs] == O.points(img, q, ts, xs)).all(), q
    rows = rng.integers(0, R, 400)
    cols = rng.integers(0, W, 400)
    rowmap = O.full_row_map(4096, 4096)
    for q in range(4):
        sel = [k for k in range(400) if rowmap[rows[k]][0] == q]
        ts = np.array([rowmap[rows[k]][1] for k in sel])
        vals = O.points(img, q, ts, cols[sel], full_layout=True)
        assert (F[rows[sel], cols[sel]] == vals).all(), q


def test_bench_step_4096_complete(fht):
    """The benchmark's step on its own image and in its own calls (one shared
    workspace, the fused-range calls of the step): the 16381 x 8192 full Hough
    image, its fhtshift and the [-15, 15] degree slope rows of Q0 and Q1, every
    element against the oracle (the step's FP32 adjoint is checked complete by
    test_adjoint_full_4096_complete)."""
    S = 4096
    img = edges_and_lines(S, S, p_edge=0.05, n_lines=4, seed=4096)
    x = dev(img)
    ws = torch.empty(max(fht.workspace_size(S, S, fht.LAYOUT_FULL, 0, torch.uint8, torch.int32),
                         fht.workspace_size(S, S, fht.LAYOUT_QUADRANT, 1, torch.uint8,
                                            torch.int32)), dtype=torch.uint8, device="cuda")
    F = fht.full_quadrants(x, workspace=ws)
    Fs = fht.fhtshift(F, S, S, fht.LAYOUT_FULL)
    lo, hi = fht.angle_to_slopes(-15.0, 15.0, S, S)
    assert (lo[0], hi[0], lo[1], hi[1]) == (0, 1097, 1, 1097)
    rng_rows = {q: host(fht.forward_range(x, q, lo[q], hi[q], workspace=ws)) for q in (0, 1)}
    want_F = O.full(img)
    assert (host(F) == want_F).all()
    assert (host(Fs) == O.fhtshift_full(want_F, S, S)).all()
    for q in (0, 1):
        assert (rng_rows[q] == O.range_slice(img, q, lo[q], hi[q])).all(), q
    del F, Fs, ws
    torch.cuda.empty_cache()


def test_config_8192_f32_sampled_and_tree(fht):
    """8192 x 8192 FP32 ellipse phantom: Q0 bit-exact against the FP32 tree,
    all four quadrants within 1e-5 * sum|I| of FP64 brute force at sampled
    points (slopes, columns and the corners of the index space)."""
    img = ellipse_phantom(8192, seed=2)
    x = dev(img)
    mass = float(np.abs(img.astype(np.float64)).sum())
    rng = np.random.default_rng(1)
    for q in range(4):
        H = fht.forward(x, q, acc=torch.float32)
        n, W = H.shape
        ts, xs = rng.integers(0, n, 300), rng.integers(0, W, 300)
        ts[:4] = [0, n - 1, 0, n - 1]
        xs[:4] = [0, 0, W - 1, W - 1]
        got = H[torch.from_numpy(ts).cuda(), torch.from_numpy(xs).cuda()].cpu().numpy()
        ref = O.points(img, q, ts, xs)
        assert np.abs(got - ref).max() <= FP32_TOL * mass, q
        if q == 0:
            assert (host(H) == O.quadrant(img, 0, "f32")).all()
        del H


def test_config_batch_shapes_per_image(fht):
    """A slice of the mixed-size batch (log-uniform sides 64..1024, 8% edges),
    each image padded to its own power of two."""
    shapes = batch_shapes(512, seed=3)[:24]
    imgs = edge_batch(shapes, seed=3)
    for img in imgs:
        assert (host(fht.forward(dev(img), 0)) == O.quadrant(img, 0)).all()


@pytest.mark.parametrize("h,w,q", [(2048, 300, 0), (1500, 2000, 2), (8192, 700, 1), (700, 8192, 3)])
def test_range_pruning_matches_full_rows(fht, h, w, q):
    """forward_range skips butterfly items whose slopes no later pass uses;
    ranges that start and end inside items, groups and passes (two-pass
    K = 11, three-pass K = 13) give exactly the rows of the oracle's full
    quadrant."""
    img = edges_and_lines(h, w, seed=h + w + q)
    x = dev(img)
    full = O.quadrant(img, q)
    n = full.shape[0]
    rng = np.random.default_rng(q)
    cases = [(0, 0), (n - 1, n - 1), (5, 9), (63, 64), (100, 131), (n // 2 - 3, n // 2 + 70)]
    cases += [tuple(sorted(rng.integers(0, n, size=2))) for _ in range(4)]
    for t_lo, t_hi in cases:
        got = host(fht.forward_range(x, q, int(t_lo), int(t_hi)))
        assert (got == full[t_lo:t_hi + 1]).all(), (t_lo, t_hi)



@pytest.mark.parametrize("h,w", [(3000, 37), (37, 3000), (2049, 1001), (4096, 5)])
def test_two_pass_4096_rows_ragged(fht, h, w):
    """Quadrants with 4096 padded rows (two passes of six levels, the final
    one from a uint16 level) on images of ragged sizes: fewer column tiles
    than resident CTAs, a height that is not a power of two, single-digit
    widths; every element of all four quadrants."""
    img = edges_and_lines(h, w, seed=h + 3 * w)
    x = dev(img)
    for q in range(4):
        got = host(fht.forward(x, q))
        assert (got == as_i32(O.quadrant(img, q))).all(), q


def test_two_pass_4096_rows_full_shift_range(fht):
    """A 2500 x 2100 page (4096 padded rows and columns): full image with the
    fused fhtshift and the [-15, 15] and [75, 105] degree ranges, every
    element."""
    h, w = 2500, 2100
    img = text_stripes(h, w, seed=5)
    x = dev(img)
    F = O.full(img)
    assert (host(fht.full_quadrants(x, apply_fhtshift=True)) ==
            as_i32(O.fhtshift_full(F, h, w))).all()
    for a, b in ((-15.0, 15.0), (75.0, 105.0)):
        lo, hi = fht.angle_to_slopes(a, b, h, w)
        for q in range(4):
            if lo[q] < 0:
                continue
            got = host(fht.forward_range(x, q, lo[q], hi[q]))
            assert (got == as_i32(O.range_slice(img, q, lo[q], hi[q]))).all(), (a, q)


@pytest.mark.parametrize("h,w,q,kind", [(32768, 300, 0, "u8"), (300, 32768, 2, "u8"),
                                        (32768, 200, 1, "f32")])
def test_max_size_32768_sampled(fht, h, w, q, kind):
    """The largest supported quadrant (n = 32768 = 2^15: three passes of five
    levels, a uint16 level and then an int32 level for uint8 images): sampled
    outputs, the corners included, against the oracle's single-point sums
    (exact for integers, within 1e-5 * sum|I| for FP32)."""
    img = edges_and_lines(h, w, seed=15) if kind == "u8" else random_image(h, w, "f32", seed=15)
    acc = torch.int32 if kind == "u8" else torch.float32
    H = fht.forward(dev(img), q, acc=acc)
    n, Wq = H.shape
    assert n == 32768
    rng = np.random.default_rng(q)
    ts, xs = rng.integers(0, n, 300), rng.integers(0, Wq, 300)
    ts[:4] = [0, n - 1, 0, n - 1]
    xs[:4] = [0, 0, Wq - 1, Wq - 1]
    got = H[torch.from_numpy(ts).cuda(), torch.from_numpy(xs).cuda()].cpu().numpy()
    want = O.points(img, q, ts, xs)
    if kind == "u8":
        assert (got == want).all()
    else:
        mass = float(np.abs(img.astype(np.float64)).sum())
        assert np.abs(got.astype(np.float64) - want).max() <= FP32_TOL * mass
    del H
    torch.cuda.empty_cache()

def test_zz_no_device_error_recorded(fht):
    """No kernel run by this module recorded a device-side error (runs last
    in the module: the count covers all the launches above)."""
    assert fht.device_status() == fht.FHT_OK
