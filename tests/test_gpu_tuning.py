"""Every tuning the autotuner can pick gives the oracle's results bit for
bit: 4, 5 or 6 butterfly levels fused per pass (so 2, 3 or 4 passes, and
intermediate levels of other depths and types than the default's) with
tile widths 1..3, on quadrants of 2^7 .. 2^13 rows -- uint8 into int32 in all
four quadrants, FP32, slope ranges, the FP32 adjoint of a quadrant and the
full image with its adjoint."""

import numpy as np
import pytest
import torch

import oracle as O
from workloads import edges_and_lines, random_image

pytestmark = pytest.mark.gpu

KS = range(7, 14)


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


@pytest.fixture
def tuned(fht, request):
    saved = {K: fht.get_tuning(K) for K in KS}
    levels, tiles = request.param
    for K in KS:
        fht.set_tuning(K, levels, *tiles)
    yield request.param
    for K, t in saved.items():
        fht.set_tuning(K, *t)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def i32(a):
    return a.astype(np.int64).astype(np.int32)


SETTINGS = [(4, (1, 1)), (4, (3, 2)), (5, (1, 1)), (5, (2, 3)), (6, (3, 3))]


@pytest.mark.parametrize("tuned", SETTINGS, indirect=True)
def test_quadrants_and_ranges(fht, tuned):
    for h, w in [(100, 300), (700, 90), (1500, 1100), (2500, 300)]:
        img = edges_and_lines(h, w, seed=h + w)
        x = dev(img)
        for q in range(4):
            H = O.quadrant(img, q)
            assert (host(fht.forward(x, q)) == i32(H)).all(), (tuned, h, w, q)
            n = H.shape[0]
            lo, hi = n // 5, n // 2 + 3
            assert (host(fht.forward_range(x, q, lo, hi)) == i32(H[lo:hi + 1])).all()


@pytest.mark.parametrize("tuned", SETTINGS, indirect=True)
def test_float_forward_and_adjoint(fht, tuned):
    for h, w in [(300, 129), (1100, 700)]:
        f = random_image(h, w, "f32", seed=h)
        x = dev(f)
        for q in (0, 3):
            assert (host(fht.forward(x, q, acc=torch.float32)) ==
                    O.quadrant(f, q, "f32")).all(), (tuned, h, w, q)
            n, W = fht.query_shape(h, w, q)
            g = np.random.default_rng(q).standard_normal((n, W)).astype(np.float32)
            got = host(fht.adjoint(dev(g), h, w, fht.LAYOUT_QUADRANT, q))
            assert (got == O.adjoint_quadrant(g, h, w, q, "f32")).all(), (tuned, h, w, q)


@pytest.mark.parametrize("tuned", [(4, (2, 2)), (5, (1, 3))], indirect=True)
def test_full_image_and_adjoint(fht, tuned):
    h, w = 1500, 1100
    img = edges_and_lines(h, w, seed=7)
    x = dev(img)
    F = O.full(img)
    assert (host(fht.full_quadrants(x)) == i32(F)).all()
    assert (host(fht.full_quadrants(x, apply_fhtshift=True)) ==
            i32(O.fhtshift_full(F, h, w))).all()
    R, C = fht.full_shape(h, w)
    g = np.random.default_rng(8).standard_normal((R, C)).astype(np.float32)
    assert (host(fht.adjoint(dev(g), h, w, fht.LAYOUT_FULL)) == O.adjoint_full(g, h, w, "f32")).all()


@pytest.mark.parametrize("tuned", [(4, (1, 1))], indirect=True)
def test_8192_rows_four_passes(fht, tuned):
    """2^13 rows at four levels per pass: passes of 4, 3, 3 and 3 levels."""
    img = edges_and_lines(5000, 40, seed=13)
    assert (host(fht.forward(dev(img), 0)) == i32(O.quadrant(img, 0))).all()


def test_autotuner_picks_the_fastest_and_sets_it(fht):
    """A short sweep on one size: the table names the candidate with the
    smallest summed time, the library is left set to it, and the default's
    time is reported beside it."""
    from paper_1811_06378_gb300 import autotune
    saved = fht.get_tuning(9)
    try:
        cands = [(6, 1, 1), (5, 2, 1), (4, 1, 2)]
        res = autotune.tune(ks=[9], reps=3, warmup=1, candidates=cands)
        e = res["table"]["9"]
        times = {tuple(c[:3]): c[3] for c in res["candidates"]["9"]}
        assert set(times) == set(cands)
        best = (e["max_levels"], e["tile_u8"], e["tile_wide"])
        assert times[best] == min(times.values()) == e["us"]
        assert e["default_us"] == times[(6, 1, 1)]
        assert fht.get_tuning(9) == best
    finally:
        fht.set_tuning(9, *saved)
