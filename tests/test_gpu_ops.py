"""Maximum and minimum along the patterns (fht_forward_op) against the
oracle's max / min recursion, bit for bit; the sum through the same entry
point equals fht_forward_range."""

import numpy as np
import pytest
import torch

import oracle as O
from workloads import edges_and_lines, random_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("h,w", [(1, 1), (5, 12), (37, 53), (200, 129), (130, 700)])
@pytest.mark.parametrize("op", [1, 2])
def test_max_min_u8_all_quadrants(fht, h, w, op):
    """One- and two-pass sizes: uint8 images into int32 (uint16 levels)."""
    img = random_image(h, w, "u8", seed=h + w + op)
    x = dev(img)
    for q in range(4):
        got = fht.forward_op(x, q, op).cpu().numpy()
        assert (got == O.quadrant_op(img, q, op)).all(), q


@pytest.mark.parametrize("op", [1, 2])
def test_max_min_f32_ranges(fht, op):
    """float32 images with negative values, slope ranges inside and across
    groups and passes."""
    h, w = 300, 170
    img = random_image(h, w, "f32", seed=5 + op)
    x = dev(img)
    for q in range(4):
        full = O.quadrant_op(img, q, op, "f32")
        n = full.shape[0]
        for t_lo, t_hi in [(0, n - 1), (0, 0), (n - 1, n - 1), (63, 64), (100, 230)]:
            got = fht.forward_op(x, q, op, t_lo, t_hi).cpu().numpy()
            assert (got == full[t_lo:t_hi + 1]).all(), (q, t_lo, t_hi)


@pytest.mark.parametrize("op", [1, 2])
def test_max_min_three_passes(fht, op):
    """K = 13: three passes, uint16 at every intermediate level."""
    img = random_image(8192, 90, "u8", seed=op)
    got = fht.forward_op(dev(img), 1, op, 2000, 4100).cpu().numpy()
    assert (got == O.quadrant_op(img, 1, op)[2000:4101]).all()


def test_sum_through_forward_op_is_forward_range(fht):
    img = edges_and_lines(257, 300, seed=3)
    x = dev(img)
    for q in range(4):
        got = fht.forward_op(x, q, 0, 5, 90).cpu().numpy().astype(np.int64)
        assert (got == O.range_slice(img, q, 5, 90)).all(), q


def test_max_of_edge_map_marks_the_sum_support(fht):
    """On a 0/1 edge map the maximum along a pattern is 1 exactly where the
    sum is positive (4096 x 4096, the benchmark's image)."""
    img = edges_and_lines(4096, 4096, p_edge=0.05, n_lines=4, seed=4096)
    x = dev(img)
    mx = fht.forward_op(x, 0, 1).cpu().numpy()
    assert (mx == (O.quadrant(img, 0) > 0)).all()
