"""The oracle and the library's host-side geometry against values the
paper's text fixes (tests/golden/, one section cited per line): quadrant and
full-image sizes (Section 3.1, 3.3), the full image's quadrant thresholds
(Section 3.3), the end points of a Hough point's image segment in the cases
of Section 3.2, the meaningful zone of a row before and after fhtshift
(Section 5) and the shear ranges of Section 4. No GPU needed."""

import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _cases(name):
    """(args, expected, citation) per fixture line."""
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            body, _, cite = line.partition("#")
            lhs, _, rhs = body.partition("->")
            assert cite.strip().startswith("Section"), line
            out.append((lhs.split(), rhs.split(), cite.strip()))
    assert out, name
    return out


@pytest.fixture(scope="module")
def fht():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1811_06378_gb300 as m
    return m


def test_quadrant_sizes(fht):
    for args, want, cite in _cases("sizes.txt"):
        h, w, q = map(int, args)
        want = tuple(map(int, want))
        assert O.quadrant_geometry(h, w, q) == want, cite
        assert fht.query_shape(h, w, q) == want, cite


def test_full_sizes(fht):
    for args, want, cite in _cases("full_sizes.txt"):
        h, w = map(int, args)
        want = tuple(map(int, want))
        assert O.full_geometry(h, w) == want, cite
        assert fht.full_shape(h, w) == want, cite


def test_full_row_quadrants(fht):
    for args, want, cite in _cases("full_rows.txt"):
        h, w, r = map(int, args)
        q = int(want[0])
        assert O.full_row_map(h, w)[r][0] == q, (args, cite)
        assert fht.full_row_to_quadrant(h, w, r)[0] == q, (args, cite)
        if q == O.Q0:   # the first block is [315, 0] flipped: row r holds slope h-1-r
            assert O.full_row_map(h, w)[r][1] == h - 1 - r


def test_segments(fht):
    for args, want, cite in _cases("segments.txt"):
        h, w, q, t, x = map(int, args)
        if want == ["none"]:
            expect = None
        else:
            c, r0, c0, r1, c1 = map(int, want)
            expect = (c, (r0, c0), (r1, c1))
        assert O.point_segment(h, w, q, t, x) == expect, (args, cite)
        assert fht.segment(h, w, t, x, layout=fht.LAYOUT_QUADRANT, q=q) == expect, (args, cite)
        if expect is not None:   # the count is what the point sums on an all-ones image
            H = O.quadrant(np.ones((h, w), np.uint8), q)
            assert H[t, x] == expect[0], (args, cite)


def test_meaningful_zone():
    for args, want, cite in _cases("meaningful_zone.txt"):
        h, w, q, t = map(int, args)
        count, start, end = map(int, want)
        H = O.quadrant(np.ones((h, w), np.uint8), q)
        assert int((H[t] != 0).sum()) == count, (args, cite)
        S = O.fhtshift_quadrant(H, h, w, q)
        nz = np.flatnonzero(S[t])
        assert nz[0] == start and nz[-1] + 1 == end and len(nz) == end - start, (args, cite)


def test_shear_ranges(fht):
    for args, want, cite in _cases("shear_ranges.txt"):
        tan_lo, tan_hi, n = float(args[0]), float(args[1]), int(args[2])
        lo, hi = math.degrees(math.atan(tan_lo)), math.degrees(math.atan(tan_hi))
        q, spl, t_lo, t_hi = int(want[0]), float(want[1]), int(want[2]), int(want[3])
        for got in (O.shear_range(lo, hi, n, n), fht.shear_range(lo, hi, n, n)):
            assert got[0] == q and got[2:] == (t_lo, t_hi), (args, got, cite)
            assert abs(got[1] - spl) < 1e-12, (args, got, cite)
