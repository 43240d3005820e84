"""The C ABI without a GPU: the library loads, exports every declared symbol,
its host-side geometry agrees with the oracle, and bad arguments are rejected
before anything touches the device."""

import ctypes
import os
import re

import pytest
import torch

import numpy as np

import oracle as O
from workloads import random_image

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fht():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1811_06378_gb300 as m
    return m


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(fht\w*)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(fht):
    syms = _declared_symbols()
    assert "fht_forward" in syms and "fhtshift" in syms and len(syms) >= 12
    for s in syms:
        assert hasattr(fht.lib, s), s


def test_shapes_match_oracle(fht):
    for h, w in [(1, 1), (3, 7), (256, 256), (300, 129), (2048, 2048), (5, 1000)]:
        for q in range(4):
            assert fht.query_shape(h, w, q) == O.quadrant_geometry(h, w, q)
        assert fht.full_shape(h, w) == O.full_geometry(h, w)


def test_full_row_map_matches_oracle(fht):
    for h, w in [(1, 1), (4, 4), (5, 12), (16, 3), (64, 32)]:
        for r, (q, t) in enumerate(O.full_row_map(h, w)):
            assert fht.full_row_to_quadrant(h, w, r) == (q, t)


@pytest.mark.parametrize("rng_", [(-15, 15), (75, 105), (-45, 135), (-30, -10), (5, 44),
                                  (50, 80), (100, 130), (0, 0), (45, 45), (90, 90),
                                  (-45, -45), (135, 135), (10, 70)])
@pytest.mark.parametrize("hw", [(2048, 2048), (256, 100), (1, 1), (7, 300)])
def test_angle_to_slopes_matches_oracle(fht, rng_, hw):
    assert fht.angle_to_slopes(float(rng_[0]), float(rng_[1]), *hw) == \
        tuple(O.angle_to_slopes(float(rng_[0]), float(rng_[1]), *hw))


def test_workspace_sizes(fht):
    import torch
    # a single pass needs no intermediate
    assert fht.workspace_size(64, 64, fht.LAYOUT_QUADRANT, 0, torch.uint8, torch.int32) == 0
    a = fht.workspace_size(4096, 4096, fht.LAYOUT_QUADRANT, 0, torch.uint8, torch.int32)
    b = fht.workspace_size(4096, 4096, fht.LAYOUT_QUADRANT, 0, torch.int32, torch.int32)
    # 2 passes: one level-6 intermediate, uint16 for uint8 images
    assert 0 < a < b
    assert a >= 4096 * (4096 + 64) * 2
    full = fht.workspace_size(4096, 4096, fht.LAYOUT_FULL, 0, torch.float32, torch.float32)
    assert full >= b


EINVAL = 1


def test_bad_arguments_rejected_on_host(fht):
    L = fht.lib
    fake = ctypes.c_void_p(0x10000)   # never dereferenced: checks fail first
    null = ctypes.c_void_p(0)
    st = ctypes.c_void_p(0)
    U8, I32, F32 = 0, 1, 2
    # null pointers
    assert L.fht_forward(null, U8, 8, 8, 8, 0, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, U8, 8, 8, 8, 0, null, I32, 16, null, 0, st) == EINVAL
    # sizes and quadrant
    assert L.fht_forward(fake, U8, 0, 8, 8, 0, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, U8, 8, -1, 8, 0, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, U8, 8, 8, 8, 4, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, U8, 1 << 20, 8, 8, 0, fake, I32, 16, null, 0, st) == EINVAL
    # the largest padded side is 2^15: 32769 rows pad to 2^16
    big = 8 + (1 << 16)
    assert L.fht_forward(fake, U8, 32769, 8, 8, 0, fake, I32, big, fake, 1 << 40, st) == EINVAL
    assert L.fht_forward(fake, U8, 8, 32769, 32769, 2, fake, I32, big, fake, 1 << 40, st) == EINVAL
    # pitches
    assert L.fht_forward(fake, U8, 8, 8, 7, 0, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, U8, 8, 8, 8, 0, fake, I32, 15, null, 0, st) == EINVAL
    # dtype pairs: float images cannot accumulate in int32
    assert L.fht_forward(fake, F32, 8, 8, 8, 0, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, I32, 8, 8, 8, 0, fake, F32, 16, null, 0, st) == EINVAL
    assert L.fht_forward(fake, 7, 8, 8, 8, 0, fake, I32, 16, null, 0, st) == EINVAL
    # workspace required at 4096 x 4096 (two passes) but missing / too small
    assert L.fht_forward(fake, U8, 4096, 4096, 4096, 0, fake, I32, 8192, null, 0, st) == EINVAL
    assert L.fht_forward(fake, U8, 4096, 4096, 4096, 0, fake, I32, 8192, fake, 100, st) == EINVAL
    # slope ranges
    assert L.fht_forward_range(fake, U8, 8, 8, 8, 0, 3, 2, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward_range(fake, U8, 8, 8, 8, 0, -1, 2, fake, I32, 16, null, 0, st) == EINVAL
    assert L.fht_forward_range(fake, U8, 8, 8, 8, 0, 0, 8, fake, I32, 16, null, 0, st) == EINVAL
    # full image: output pitch below h_p + w_p
    assert L.fht_full_quadrants(fake, U8, 5, 9, 9, fake, I32, 23, 0, null, 0, st) == EINVAL
    # fhtshift: in place and bad dtype
    assert L.fhtshift(fake, fake, I32, 8, 8, 1, 0, 0, 16, 16, st) == EINVAL
    assert L.fhtshift(fake, ctypes.c_void_p(0x20000), U8, 8, 8, 1, 0, 0, 16, 16, st) == EINVAL
    assert L.fhtshift(fake, ctypes.c_void_p(0x20000), I32, 8, 8, 2, 0, 0, 16, 16, st) == EINVAL
    # adjoint: u8 gradients are not a thing; pitch too small
    assert L.fht_adjoint(fake, U8, 8, 8, 0, 0, 16, fake, 8, null, 0, st) == EINVAL
    assert L.fht_adjoint(fake, F32, 8, 8, 0, 0, 15, fake, 8, null, 0, st) == EINVAL
    assert L.fht_adjoint(fake, F32, 8, 8, 0, 0, 16, fake, 7, null, 0, st) == EINVAL
    # uniform batches: batch count, overlapping items, FP32 only (no other types exist here)
    assert L.fht_forward_many(fake, 0, 64, 8, 8, 8, 1, 0, fake, 512, 16, null, 0, st) == EINVAL
    assert L.fht_forward_many(fake, 65536, 64, 8, 8, 8, 1, 0, fake, 512, 16, null, 0, st) == EINVAL
    assert L.fht_forward_many(fake, 2, 63, 8, 8, 8, 1, 0, fake, 512, 16, null, 0, st) == EINVAL
    assert L.fht_forward_many(fake, 2, 64, 8, 8, 8, 1, 0, fake, 16 * 29 - 1, 16, null, 0,
                              st) == EINVAL
    assert L.fht_adjoint_many(fake, 2, 16 * 29, 8, 8, 1, 0, 16, fake, 63, 8, null, 0,
                              st) == EINVAL
    n = ctypes.c_size_t()
    assert L.fht_workspace_size_many(0, 8, 8, 1, 0, ctypes.byref(n)) == EINVAL
    assert L.fht_workspace_size_many(3, 100, 100, 1, 0, ctypes.byref(n)) == 0
    one = fht.workspace_size(100, 100, fht.LAYOUT_FULL, 0, torch.float32, torch.float32)
    assert n.value == 3 * ((one + 255) // 256 * 256)
    # geometry queries
    r = ctypes.c_int()
    assert L.fht_query_shape(0, 4, 0, ctypes.byref(r), ctypes.byref(r)) == EINVAL
    assert L.fht_full_row_to_quadrant(4, 4, 13, ctypes.byref(r), ctypes.byref(r)) == EINVAL
    lo = (ctypes.c_int * 4)()
    assert L.fht_angle_to_slopes(10.0, 5.0, 8, 8, lo, lo) == EINVAL
    assert fht.lib.fht_status_string(EINVAL) == b"invalid argument"


@pytest.mark.parametrize("rng_", [(-15, 15), (75, 105), (-45, 0), (0, 45), (-45, 45),
                                  (-20, -5), (60, 100), (45, 90), (90, 135), (30, 60),
                                  (-30, 30), (10, 10), (-50, 0)])
@pytest.mark.parametrize("hw", [(2048, 2048), (256, 100), (1, 1), (7, 300)])
def test_shear_range_matches_oracle(fht, rng_, hw):
    want = O.shear_range(float(rng_[0]), float(rng_[1]), *hw)
    if want is None:
        with pytest.raises(fht.FHTError):
            fht.shear_range(float(rng_[0]), float(rng_[1]), *hw)
        return
    got = fht.shear_range(float(rng_[0]), float(rng_[1]), *hw)
    assert got[0] == want[0] and got[2:] == want[2:]
    assert got[1] == want[1]   # the same double arithmetic on both sides


def test_sheared_bad_arguments_rejected_on_host(fht):
    L = fht.lib
    fake, null, st = ctypes.c_void_p(0x10000), ctypes.c_void_p(0), ctypes.c_void_p(0)
    U8, I32 = 0, 1
    ok = dict(spl=0.5, lo=0, hi=7)
    args = lambda spl, lo, hi, pitch=16: (fake, U8, 8, 8, 8, 0, spl, lo, hi, fake, I32,  # noqa
                                          pitch, null, 0, st)
    assert L.fht_forward_sheared(*args(1.5, 0, 7)) == EINVAL
    assert L.fht_forward_sheared(*args(-1.0001, 0, 7)) == EINVAL
    assert L.fht_forward_sheared(*args(float("nan"), 0, 7)) == EINVAL
    assert L.fht_forward_sheared(*args(ok["spl"], 3, 2)) == EINVAL
    assert L.fht_forward_sheared(*args(ok["spl"], 0, 8)) == EINVAL
    assert L.fht_forward_sheared(*args(ok["spl"], 0, 7, 15)) == EINVAL
    n = ctypes.c_size_t()
    assert L.fht_workspace_size_sheared(4096, 4096, 0, U8, I32, ctypes.byref(n)) == 0
    # two passes: one full-width level of n x W (pitch rounded to 64), uint16
    # for a uint8 image (sums of 2^6 bytes), int32 otherwise
    assert n.value == 4096 * 8192 * 2
    assert L.fht_workspace_size_sheared(4096, 4096, 0, I32, I32, ctypes.byref(n)) == 0
    assert n.value == 4096 * 8192 * 4
    assert L.fht_workspace_size_sheared(4096, 4096, 4, U8, I32, ctypes.byref(n)) == EINVAL


@pytest.mark.parametrize("alpha", [1.0, 2.0, 3.0, 0.5, 0.25, 0.7, 1.37, 1.8660254037844386,
                                   5.9, 1 / 3, 16.0])
def test_scaled_geometry_matches_oracle(fht, alpha):
    """The scaled width and shape (host) take the oracle's integer decisions:
    the same double quotient, the same fixed-point step."""
    for w in (1, 2, 7, 100, 301, 2048):
        assert fht.scaled_width(w, alpha) == O.scaled_width(w, alpha)
    for h, w in ((256, 100), (7, 300), (2048, 2048)):
        for q in range(4):
            n = O.next_pow2(w if O.TRANSPOSED[q] else h)
            wa = O.scaled_width(h if O.TRANSPOSED[q] else w, alpha)
            assert fht.scaled_shape(h, w, q, alpha) == (n, wa + n)


@pytest.mark.parametrize("rng_", [(-15, 15), (75, 105), (-45, 45), (-60, 60), (10, 20),
                                  (-20, -10), (80, 100), (100, 120), (-5, 5), (0, 0),
                                  (20, 10), (-95, 0), (-85, 85), (30, 80)])
@pytest.mark.parametrize("hw", [(2048, 2048), (256, 100), (1, 1), (7, 300)])
def test_scale_range_matches_oracle(fht, rng_, hw):
    want = O.scale_range(float(rng_[0]), float(rng_[1]), *hw)
    if want is None:
        with pytest.raises(fht.FHTError):
            fht.scale_range(float(rng_[0]), float(rng_[1]), *hw)
        return
    got = fht.scale_range(float(rng_[0]), float(rng_[1]), *hw)
    assert got[0] == want[0] and got[3:] == want[3:]
    assert got[1] == want[1] and got[2] == want[2]   # the same double arithmetic


def test_scaled_bad_arguments_rejected_on_host(fht):
    L = fht.lib
    fake, null, st = ctypes.c_void_p(0x10000), ctypes.c_void_p(0), ctypes.c_void_p(0)
    U8, I32 = 0, 1
    wa = ctypes.c_int()
    assert L.fht_scaled_width(100, 0.0, ctypes.byref(wa)) == EINVAL
    assert L.fht_scaled_width(100, float("nan"), ctypes.byref(wa)) == EINVAL
    assert L.fht_scaled_width(100, 300.0, ctypes.byref(wa)) == EINVAL
    assert L.fht_scaled_width(4096, 16.0, ctypes.byref(wa)) == EINVAL   # 65536 > 32768
    assert L.fht_scaled_width(2048, 16.0, ctypes.byref(wa)) == 0 and wa.value == 32768
    # 8 x 8 image, alpha 2: W = 16 + 8 = 24
    args = lambda alpha, spl, lo, hi, pitch=24: (fake, U8, 8, 8, 8, 0, alpha, spl, lo, hi,  # noqa
                                                 fake, I32, pitch, null, 0, st)
    assert L.fht_forward_scaled(*args(2.0, 1.5, 0, 7)) == EINVAL
    assert L.fht_forward_scaled(*args(0.0, 0.0, 0, 7)) == EINVAL
    assert L.fht_forward_scaled(*args(2.0, 0.0, 3, 2)) == EINVAL
    assert L.fht_forward_scaled(*args(2.0, 0.0, 0, 8)) == EINVAL
    assert L.fht_forward_scaled(*args(2.0, 0.0, 0, 7, 23)) == EINVAL
    n = ctypes.c_size_t()
    assert L.fht_workspace_size_scaled(4096, 2048, 0, 2.0, U8, I32, ctypes.byref(n)) == 0
    # two passes: one full-width level of n x W (W = 4096 + 4096), uint16, then
    # the scaled copy of the image (h x w_alpha bytes)
    assert n.value == 4096 * 8192 * 2 + 4096 * 4096
    # alpha = 1: the sheared transform's levels, then the copy, its rows padded
    # to 16 bytes (Q0: 300 rows of 2001 -> 2016 uint8; Q2 scales the image's
    # row index: 300 rows of 2001 -> 2004 FP32 values)
    m = ctypes.c_size_t()
    F32 = 2
    for q, copy in ((0, 300 * 2016), (2, 300 * 2004 * 4)):
        dt = U8 if q == 0 else F32
        acc = I32 if q == 0 else F32
        assert L.fht_workspace_size_sheared(300, 2001, q, dt, acc, ctypes.byref(m)) == 0
        assert L.fht_workspace_size_scaled(300, 2001, q, 1.0, dt, acc, ctypes.byref(n)) == 0
        assert n.value == (m.value + 255) // 256 * 256 + copy, q


@pytest.mark.parametrize("q", [0, 1, 2, 3])
@pytest.mark.parametrize("hw", [(9, 14), (16, 5), (1, 1), (33, 20)])
def test_segment_matches_oracle(fht, q, hw):
    """fht_segment (host) against the oracle's point -> segment on every point
    of the quadrant."""
    h, w = hw
    n, W = O.quadrant_geometry(h, w, q)
    for t in range(n):
        for x in range(W):
            assert fht.segment(h, w, t, x, fht.LAYOUT_QUADRANT, q) == \
                O.point_segment(h, w, q, t, x), (t, x)


@pytest.mark.parametrize("hw", [(9, 14), (5, 3), (12, 20)])
def test_segment_full_layout_and_fhtshift(fht, hw):
    """Full layout: the count is the full transform of an all-ones image at the
    point (also after fhtshift, with shifted=1), and the run's pixel sum the
    full transform of a random image."""
    h, w = hw
    ones = O.full(np.ones((h, w), np.uint8))
    ones_s = O.fhtshift_full(ones, h, w)
    img = random_image(h, w, "u8", seed=h)
    F = O.full(img)
    R, W = O.full_geometry(h, w)
    rowmap = O.full_row_map(h, w)
    hp, wp = O.next_pow2(h), O.next_pow2(w)
    for r in range(R):
        q, t = rowmap[r]
        n = hp if q < 2 else wp
        for x in range(W):
            seg = fht.segment(h, w, r, x)
            cnt = 0 if seg is None else seg[0]
            assert cnt == ones[r, x], (r, x)
            segs = fht.segment(h, w, r, x, shifted=True)
            assert (0 if segs is None else segs[0]) == ones_s[r, x], (r, x)
            if seg is None:
                assert F[r, x] == 0
                continue
            _, a, b = seg
            tr = q >= 2
            ya, yb = (a[1], b[1]) if tr else (a[0], b[0])
            tot = 0
            for y in range(ya, yb + 1):
                c = (x + O.SIGMA[q] * O.offset(n, t, y)) % W
                rr, cc = (c, y) if tr else (y, c)
                tot += int(img[rr, cc])
            assert tot == F[r, x], (r, x)


def test_segment_bad_arguments(fht):
    L = fht.lib
    v = [ctypes.c_int() for _ in range(5)]
    refs = [ctypes.byref(x) for x in v]
    assert L.fht_segment(8, 8, 0, 0, 8, 0, 0, *refs) == EINVAL      # t >= n
    assert L.fht_segment(8, 8, 0, 0, 0, 16, 0, *refs) == EINVAL     # col >= W
    assert L.fht_segment(8, 8, 1, 0, 29, 0, 0, *refs) == EINVAL     # full row out of range
    assert L.fht_segment(8, 8, 0, 4, 0, 0, 0, *refs) == EINVAL      # quadrant
    assert L.fht_row_argmax(ctypes.c_void_p(0x1000), 0, 4, 4, 4, ctypes.c_void_p(0x1000),
                            ctypes.c_void_p(0x1000), ctypes.c_void_p(0)) == EINVAL  # u8
    assert L.fht_row_argmax(ctypes.c_void_p(0x1000), 1, 4, 4, 3, ctypes.c_void_p(0x1000),
                            ctypes.c_void_p(0x1000), ctypes.c_void_p(0)) == EINVAL  # pitch


def test_debug_hook_is_debug_build_only(fht):
    """The release build compiles no bounds checks: its test hook reports
    FHT_EUNSUPPORTED, and FHT_EBOUNDS has a name."""
    if fht.DEBUG:
        pytest.skip("the debug build is loaded")
    assert fht.lib.fht_debug_test_hooks(0) == 4
    assert b"debug build" in fht.lib.fht_status_string(6)
