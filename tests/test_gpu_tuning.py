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


BATCHED = [
    {"ctas_per_sm": 3},
    {"units_per_item": 1, "tile_u8": 1, "tile_wide": 3},
    {"units_per_item": 16, "tile_u8": 3, "tile_wide": 2, "ctas_per_sm": 3},
    {"first_levels": {7: 1, 8: 6, 9: 3, 10: 6, 11: 5, 12: 6}},
    {"first_levels": {7: 6, 8: 2, 9: 6, 10: 4, 11: 6, 12: 6}, "ctas_per_sm": 3},
]


@pytest.mark.parametrize("bt", BATCHED)
def test_batched_tunings_match_the_oracle(fht, bt):
    """Every batched tuning the autotuner can pick (CTAs per SM, units per
    item, tile widths, first-pass depth per size) gives the oracle's results
    bit for bit: a uint8 batch of one- and two-pass images of every size
    class up to 4096 rows, and an FP32 adjoint batch."""
    from workloads import edge_batch
    saved = fht.get_batched_tuning()
    try:
        fht.set_batched_tuning(None)
        fht.set_batched_tuning(bt)
        shapes = [(1, 1), (40, 70), (64, 64), (100, 300), (200, 129), (300, 90), (600, 1000),
                  (1000, 77), (1500, 200), (4000, 33)]
        imgs = [dev(a) for a in edge_batch(shapes, seed=77)]
        plan = fht.BatchPlan(shapes, 1)
        outs = plan.forward(imgs)
        assert plan.status() == 0
        for x, o in zip(imgs, outs):
            assert (host(o) == i32(O.quadrant(x.cpu().numpy(), 1))).all(), tuple(x.shape)
        fshapes = shapes[:8]
        fplan = fht.BatchPlan(fshapes, 2, torch.float32, torch.float32)
        rng = np.random.default_rng(78)
        grads = [dev(rng.standard_normal(sh).astype(np.float32)) for sh in fplan.out_shapes]
        gouts = fplan.adjoint(grads)
        assert fplan.status() == 0
        for (h, w), g, o in zip(fshapes, grads, gouts):
            want = O.adjoint_quadrant(g.cpu().numpy(), h, w, 2, "f32")
            assert np.array_equal(host(o), want), (h, w)
    finally:
        fht.set_batched_tuning(None)
        fht.set_batched_tuning(saved)


def test_batched_autotuner_keeps_results_and_sets_the_best(fht):
    """A short batched sweep on a small batch: every candidate's results
    equal the default's (checked inside), the best is left in force and the
    default's time is reported."""
    from paper_1811_06378_gb300 import autotune
    saved = fht.get_batched_tuning()
    try:
        res = autotune.tune_batched(count=24, seed=5, reps=2, warmup=1)
        assert res["us"] <= res["default_us"]
        got = fht.get_batched_tuning()
        want = res["tuning"]
        assert got["ctas_per_sm"] == want["ctas_per_sm"]
        assert got["units_per_item"] == want["units_per_item"]
        assert {str(k): v for k, v in got["first_levels"].items()} == want["first_levels"]
    finally:
        fht.set_batched_tuning(None)
        fht.set_batched_tuning(saved)


def test_batched_tuning_changes_the_plan_workspace(fht):
    """The first pass's depth sets the intermediate level's compact width:
    for one 1024 x 300 uint8 image (K = 10), w_c + 2^f columns (pitch
    rounded to 64) of uint16, plus the plan's fixed tables."""
    saved = fht.get_batched_tuning()
    sizes = {}
    try:
        for f in (4, 5, 6):
            fht.set_batched_tuning(None)
            fht.set_batched_tuning({"first_levels": {10: f}})
            sizes[f] = fht.BatchPlan([(1024, 300)], 0).workspace_bytes
    finally:
        fht.set_batched_tuning(None)
        fht.set_batched_tuning(saved)
    pitch = lambda f: -(-(300 + (1 << f)) // 64) * 64   # noqa: E731
    assert sizes[5] - sizes[4] == 1024 * (pitch(5) - pitch(4)) * 2
    assert sizes[6] - sizes[5] == 1024 * (pitch(6) - pitch(5)) * 2
