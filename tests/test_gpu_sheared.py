"""The sheared forward transform of Section 4 (the image sheared by spl per
row inside the first butterfly iteration, then one quadrant) against the
oracle's explicitly sheared image: integers bit-exact, FP32 bit-exact against
the oracle's FP32 recursion."""

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
    return t.cpu().numpy()


def as_i32(a):
    return ((a.astype(np.int64) + 2**31) % 2**32 - 2**31).astype(np.int32)


SPLS = [0.0, 0.37, -0.6, 1.0, -1.0, 0.5]


@pytest.mark.parametrize("h,w", [(1, 1), (5, 12), (37, 53), (200, 129), (130, 700)])
def test_sheared_u8_all_quadrants(fht, h, w):
    """One- and two-pass sizes, all quadrants, positive, negative, unit and
    half-integer shears (exact halves exercise the rounding)."""
    img = edges_and_lines(h, w, seed=h * 7 + w)
    x = dev(img)
    for q in range(4):
        for spl in SPLS:
            got = host(fht.forward_sheared(x, q, spl))
            want = O.sheared_quadrant(img, q, spl)
            assert (got == as_i32(want)).all(), (q, spl)


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_sheared_zero_equals_plain_transform(fht, q):
    """spl = 0 takes the cyclic full-width path but returns exactly what the
    compact forward transform returns."""
    img = edges_and_lines(300, 257, seed=q)
    x = dev(img)
    assert (host(fht.forward_sheared(x, q, 0.0)) == O.quadrant(img, q)).all()


@pytest.mark.parametrize("q,spl", [(0, 0.3), (1, -0.45), (2, 0.9), (3, -0.2)])
def test_sheared_ranges_and_types(fht, q, spl):
    """Slope ranges inside and across groups; int32 and float32 images; uint8
    into float32."""
    h, w = 260, 190
    img = edges_and_lines(h, w, seed=11 + q)
    n, _ = O.quadrant_geometry(h, w, q)
    full = O.sheared_quadrant(img, q, spl)
    x = dev(img)
    for t_lo, t_hi in [(0, 0), (n - 1, n - 1), (5, 9), (63, 64), (100, 200)]:
        got = host(fht.forward_sheared(x, q, spl, t_lo, t_hi))
        assert (got == as_i32(full[t_lo:t_hi + 1])).all(), (t_lo, t_hi)
    xi = random_image(h, w, "i32", seed=q, hi=1000)
    got = host(fht.forward_sheared(dev(xi), q, spl))
    assert (got == as_i32(O.sheared_quadrant(xi, q, spl))).all()
    xf = random_image(h, w, "f32", seed=q)
    got = host(fht.forward_sheared(dev(xf), q, spl, acc=torch.float32))
    assert (got == O.sheared_quadrant(xf, q, spl, "f32")).all()
    got = host(fht.forward_sheared(x, q, spl, acc=torch.float32))
    assert (got == O.sheared_quadrant(img, q, spl, "f32")).all()


@pytest.mark.parametrize("rng_", [(-15.0, 15.0), (75.0, 105.0)])
def test_config_2048_page_one_sheared_quadrant(fht, rng_):
    """The 2048 x 2048 text-stripe page: the [-15, 15] and [75, 105] degree
    ranges as one sheared quadrant each (the paper's use of the shear), every
    element of the slope rows against the oracle."""
    img = text_stripes(2048, 2048, seed=1)
    q, spl, t_lo, t_hi = fht.shear_range(*rng_, 2048, 2048)
    assert (q, t_lo) == ((0 if rng_[0] < 45 else 3), 0)
    got = host(fht.forward_sheared(dev(img), q, spl, t_lo, t_hi))
    assert got.shape == (t_hi + 1, 4096)
    want = O.sheared_quadrant(img, q, spl, t_lo=t_lo, t_hi=t_hi)
    assert (got == as_i32(want)).all()


def test_sheared_three_passes(fht):
    """K = 13 (three passes of five, four and four levels), both signs."""
    img = edges_and_lines(8192, 160, seed=13)
    x = dev(img)
    for q, spl in ((0, 0.21), (1, -0.73)):
        got = host(fht.forward_sheared(x, q, spl, 1000, 2999))
        want = O.sheared_quadrant(img, q, spl, t_lo=1000, t_hi=2999)
        assert (got == as_i32(want)).all(), q


def test_sheared_and_ops_on_unaligned_views(fht):
    """Images that start at odd element offsets inside a wider buffer (odd
    pitch, unaligned rows): the sheared transform and the maximum still match
    the oracle exactly, so the vector fast paths and the edge paths agree."""
    h, w = 150, 203
    rng = np.random.default_rng(17)
    big = rng.integers(0, 256, size=(h + 3, w + 37)).astype(np.uint8)
    view = torch.from_numpy(big).cuda()[1:1 + h, 5:5 + w]      # pitch w + 37, offset 1 row + 5
    img = big[1:1 + h, 5:5 + w]
    for q, spl in ((0, 0.3), (2, -0.7)):
        got = fht.forward_sheared(view, q, spl).cpu().numpy()
        assert (got == as_i32(O.sheared_quadrant(img, q, spl))).all(), q
    got = fht.forward_op(view, 1, 1).cpu().numpy()
    assert (got == O.quadrant_op(img, 1, 1)).all()
    bigf = rng.standard_normal((h + 2, w + 9)).astype(np.float32)
    vf = torch.from_numpy(bigf).cuda()[2:2 + h, 3:3 + w]
    got = fht.forward_op(vf, 3, 2).cpu().numpy()
    assert (got == O.quadrant_op(bigf[2:2 + h, 3:3 + w], 3, 2, "f32")).all()
