"""From Hough points back to lines: per-row maxima on the GPU against
numpy (first maximum on ties), and a drawn line found again through the full
Hough image, its peak and the point's image segment (Section 3.2)."""

import math

import numpy as np
import pytest
import torch

import oracle as O
from workloads import edges_and_lines

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


@pytest.mark.parametrize("rows,cols,extra", [(1, 1, 0), (7, 5, 3), (300, 1000, 0),
                                             (64, 4099, 13), (5000, 257, 0)])
@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_row_argmax_matches_numpy(fht, rows, cols, extra, dtype):
    """Values drawn from a small set, so most rows hold ties: the first
    column of the maximum wins, as numpy's argmax; padded pitches."""
    rng = np.random.default_rng(rows + cols)
    a = rng.integers(-20, 20, size=(rows, cols + extra)).astype(dtype)
    t = torch.from_numpy(a).cuda()[:, :cols]
    vals, idx = fht.row_argmax(t)
    b = a[:, :cols]
    assert (vals.cpu().numpy() == b.max(axis=1)).all()
    assert (idx.cpu().numpy() == b.argmax(axis=1)).all()


def test_row_argmax_full_image_4096(fht):
    """The benchmark's 16381 x 8192 full Hough image."""
    img = edges_and_lines(4096, 4096, p_edge=0.05, n_lines=4, seed=4096)
    F = fht.full_quadrants(torch.from_numpy(img).cuda())
    vals, idx = fht.row_argmax(F)
    Fh = F.cpu().numpy()
    assert (vals.cpu().numpy() == Fh.max(axis=1)).all()
    assert (idx.cpu().numpy() == Fh.argmax(axis=1)).all()


@pytest.mark.parametrize("phi", [-30.0, -3.0, 20.0, 60.0, 95.0, 128.0])
def test_drawn_line_is_found_again(fht, phi):
    """A straight line through a 512 x 512 image at angle phi (the quadrant
    convention: dx/dy = -tan(phi) for mostly vertical lines, dy/dx for the
    others through the transpose) plus 1% noise: the full Hough image's
    largest entry maps back (fht_segment) to a segment whose end points lie
    within 3 pixels of the drawn line, and it covers most of the line."""
    n = 512
    rng = np.random.default_rng(int(phi * 10) + 1000)
    img = (rng.random((n, n)) < 0.01).astype(np.uint8)
    pts = []
    if -45 <= phi <= 45:
        k = -math.tan(math.radians(phi))
        x0 = n / 2 - k * n / 2
        for y in range(n):
            x = int(math.floor(x0 + k * y + 0.5))
            if 0 <= x < n:
                img[y, x] = 1
                pts.append((y, x))
    else:
        k = math.tan(math.radians(phi - 90.0))   # rows per column of the image
        y0 = n / 2 - k * n / 2
        for x in range(n):
            y = int(math.floor(y0 + k * x + 0.5))
            if 0 <= y < n:
                img[y, x] = 1
                pts.append((y, x))
    F = fht.full_quadrants(torch.from_numpy(img).cuda())
    vals, idx = fht.row_argmax(F)
    r = int(torch.argmax(vals).item())
    c = int(idx[r].item())
    seg = fht.segment(n, n, r, c)
    assert seg is not None
    count, a, b = seg
    assert count >= 0.8 * len(pts)

    def dist(p):
        return min(math.hypot(p[0] - y, p[1] - x) for y, x in pts)

    assert dist(a) <= 3.0 and dist(b) <= 3.0
    # the point's value is what its segment sums (the oracle on the same image)
    assert int(F[r, c].item()) == int(O.full(img)[r, c])
