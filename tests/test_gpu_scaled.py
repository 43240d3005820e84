"""The scale of Section 4 on the GPU (fht_forward_scaled): the image scaled
along its rows by alpha (nearest neighbour on the fixed-point grid), then
sheared, then one quadrant, against the oracle's explicit resampling and
plain butterfly, bit for bit."""

import numpy as np
import pytest
import torch

import oracle as O
from workloads import edges_and_lines, random_image, text_stripes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def as_i32(a):
    return a.astype(np.int64).astype(np.int32)


@pytest.mark.parametrize("q", [0, 1, 2, 3])
@pytest.mark.parametrize("alpha,spl", [(1.0, 0.0), (2.0, 0.0), (3.0, 0.35), (0.5, -0.6),
                                       (0.7, 0.0), (1.8660254037844386, 0.5), (1.37, -1.0),
                                       (0.25, 1.0)])
def test_scaled_u8_bit_exact(fht, q, alpha, spl):
    img = edges_and_lines(300, 257, seed=q)
    got = host(fht.forward_scaled(dev(img), q, alpha, spl))
    want = O.scaled_quadrant(img, q, alpha, spl)
    assert got.shape == want.shape
    assert (got == as_i32(want)).all(), (q, alpha, spl)


@pytest.mark.parametrize("q", [0, 2])
def test_scaled_alpha_one_is_the_sheared_transform(fht, q):
    img = edges_and_lines(200, 130, seed=7 + q)
    x = dev(img)
    got = host(fht.forward_scaled(x, q, 1.0, 0.3))
    assert (got == host(fht.forward_sheared(x, q, 0.3))).all()
    assert (got == as_i32(O.sheared_quadrant(img, q, 0.3))).all()


@pytest.mark.parametrize("q,alpha,spl", [(0, 2.5, 0.2), (3, 0.6, -0.4)])
def test_scaled_f32_and_ranges(fht, q, alpha, spl):
    """FP32 images (same addition tree as the oracle's FP32 recursion) and
    slope ranges that start and end inside groups and passes."""
    img = random_image(257, 190, "f32", seed=3)
    full = O.scaled_quadrant(img, q, alpha, spl, kind="f32")
    got = host(fht.forward_scaled(dev(img), q, alpha, spl, acc=torch.float32))
    assert np.array_equal(got, full)
    n = full.shape[0]
    u8 = edges_and_lines(257, 190, seed=4)
    want = O.scaled_quadrant(u8, q, alpha, spl)
    for t_lo, t_hi in [(0, 0), (n - 1, n - 1), (5, 9), (63, 64), (100, n - 1), (17, 200)]:
        got = host(fht.forward_scaled(dev(u8), q, alpha, spl, t_lo, t_hi))
        assert (got == as_i32(want[t_lo:t_hi + 1])).all(), (t_lo, t_hi)


def test_scaled_three_passes_and_ragged(fht):
    """K = 13 (three passes) and ragged sizes with the scaled width crossing
    tile borders."""
    img = edges_and_lines(5000, 180, seed=9)
    got = host(fht.forward_scaled(dev(img), 0, 0.6, 0.25))
    assert (got == as_i32(O.scaled_quadrant(img, 0, 0.6, 0.25))).all()
    img = random_image(333, 77, "u8", seed=10)
    for q, alpha in ((1, 4.3), (2, 1.9)):
        got = host(fht.forward_scaled(dev(img), q, alpha, -0.15))
        assert (got == as_i32(O.scaled_quadrant(img, q, alpha, -0.15))).all(), q


def test_scale_range_2048_page_complete(fht):
    """The 2048 x 2048 text-stripe page: its [-15, 15] degree range as one
    scaled and sheared quadrant (alpha = 1/(2 tan 15), every slope row), and
    the [75, 105] range through Q3, each compared complete with the oracle."""
    img = text_stripes(2048, 2048, seed=2)
    x = dev(img)
    for rng_ in ((-15.0, 15.0), (75.0, 105.0)):
        q, alpha, spl, t_lo, t_hi = fht.scale_range(*rng_, 2048, 2048)
        got = host(fht.forward_scaled(x, q, alpha, spl, t_lo, t_hi))
        want = O.scaled_quadrant(img, q, alpha, spl, t_lo=t_lo, t_hi=t_hi)
        assert (got == as_i32(want)).all(), rng_


def test_scaled_view_with_pitch(fht):
    """An image view with a row pitch wider than its width and an odd
    starting column."""
    base = edges_and_lines(160, 300, seed=12)
    view = dev(base)[5:150, 3:203]
    img = base[5:150, 3:203]
    got = host(fht.forward_scaled(view, 1, 1.5, 0.1))
    assert (got == as_i32(O.scaled_quadrant(img, 1, 1.5, 0.1))).all()


@pytest.mark.parametrize("h,w,q,alpha", [(1, 1, 0, 0.5), (1, 1, 2, 3.0), (1, 7, 1, 1 / 256),
                                         (7, 1, 3, 1 / 256), (3, 300, 0, 100.0),
                                         (300, 3, 2, 100.0), (5, 300, 1, 1 / 256),
                                         (2, 2, 0, 256.0)])
def test_scaled_extreme_factors_and_degenerate_shapes(fht, h, w, q, alpha):
    """The ends of the factor range (1/256 leaves one or two scaled columns,
    100 and 256 widen a row to 30000 and 512 columns) on one-pixel, one-row
    and one-column images, through all four quadrants; the scaled copy and
    the transform against the oracle, bit for bit."""
    img = edges_and_lines(h, w, seed=h * 31 + w)
    got = host(fht.forward_scaled(dev(img), q, alpha, 0.3))
    want = O.scaled_quadrant(img, q, alpha, 0.3)
    assert got.shape == want.shape
    assert (got == as_i32(want)).all(), (h, w, q, alpha)
