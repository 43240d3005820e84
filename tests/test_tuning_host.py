"""The tuning entry points without a GPU: argument checks, set / get /
restore, workspace sizes that follow the pass split, and an autotuner table
applied through the binding."""

import json

import pytest
import torch


@pytest.fixture(scope="module")
def fht():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1811_06378_gb300 as m
    return m


@pytest.fixture
def restore(fht):
    saved = {K: fht.get_tuning(K) for K in range(1, 16)}
    yield
    for K, t in saved.items():
        fht.set_tuning(K, *t)


def test_bad_tunings_rejected(fht, restore):
    for K, t in [(0, (6, 1, 1)), (16, (6, 1, 1)), (12, (3, 1, 1)), (12, (7, 1, 1)),
                 (12, (6, 0, 1)), (12, (6, 1, 4))]:
        with pytest.raises(fht.FHTError):
            fht.set_tuning(K, *t)
    assert fht.lib.fht_get_tuning(12, None) == 1


def test_set_get_and_default(fht, restore):
    fht.set_tuning(12, None)
    default = fht.get_tuning(12)
    assert default[0] == 6
    fht.set_tuning(12, 4, 2, 3)
    assert fht.get_tuning(12) == (4, 2, 3)
    assert fht.get_tuning(11) == fht.get_tuning(11)   # other sizes untouched
    fht.set_tuning(12, None)
    assert fht.get_tuning(12) == default


def test_workspace_follows_the_split(fht, restore):
    """4096 rows: six levels per pass leave one intermediate level (uint16 for
    a uint8 image), four levels per pass two (uint16, then int32)."""
    args = (4096, 4096, fht.LAYOUT_QUADRANT, 0, torch.uint8, torch.int32)
    fht.set_tuning(12, 6, 1, 1)
    six = fht.workspace_size(*args)
    assert six == 4096 * (4096 + 64) * 2
    fht.set_tuning(12, 4, 1, 1)
    four = fht.workspace_size(*args)
    # row pitches rounded up to 64 elements: 4096 + 16 -> 4160, 4096 + 256
    assert four == 4096 * 4160 * 2 + 4096 * 4352 * 4
    # 64 rows: one pass of six levels needs no intermediate; 4 + 2 levels do
    small = (64, 64, fht.LAYOUT_QUADRANT, 0, torch.uint8, torch.int32)
    fht.set_tuning(6, 6, 1, 1)
    assert fht.workspace_size(*small) == 0
    fht.set_tuning(6, 4, 1, 1)
    assert fht.workspace_size(*small) == 64 * 128 * 2


def test_table_is_applied(fht, restore, tmp_path):
    from paper_1811_06378_gb300 import autotune
    table = {"table": {"9": {"max_levels": 5, "tile_u8": 3, "tile_wide": 2, "us": 1.0,
                             "default_us": 2.0},
                       "13": {"max_levels": 4, "tile_u8": 1, "tile_wide": 3, "us": 1.0,
                              "default_us": 1.0}}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    autotune.load(str(path))
    assert fht.get_tuning(9) == (5, 3, 2) and fht.get_tuning(13) == (4, 1, 3)


def test_shipped_table_is_valid(fht, restore):
    """The package's own table (if present) names only valid tunings."""
    import os
    if not os.path.exists(fht.TUNING_FILE):
        pytest.skip("no shipped table")
    saved_b = fht.get_batched_tuning()
    res = fht.load_tuning(fht.TUNING_FILE)
    for k, e in res["table"].items():
        assert fht.get_tuning(int(k)) == (e["max_levels"], e["tile_u8"], e["tile_wide"])
    if "batched" in res:
        want = dict(res["batched"]["tuning"])
        want["first_levels"] = {int(k): v for k, v in want["first_levels"].items()}
        assert fht.get_batched_tuning() == want
    fht.set_batched_tuning(None)
    fht.set_batched_tuning(saved_b)


def _model_forward_workspace(h, w, q, levels, acc_u16_ok):
    """Workspace of a forward quadrant plan, modelled from the documented
    layout: the K levels split into ceil(K / levels) near-equal passes (the
    larger ones first); every intermediate level keeps the columns
    x < w_c + 2^k (compact columns), row pitch rounded up to 64 elements,
    256-byte aligned; uint16 only for the first level of a uint8 image into
    int32 (exact while it sums at most 2^8 rows), else 4 bytes; levels
    alternate between two buffers."""
    hc, wc = (w, h) if q >= 2 else (h, w)
    n = 1
    while n < hc:
        n *= 2
    K = n.bit_length() - 1
    W = wc + n
    if K == 0:
        return 0
    P = -(-K // levels)
    m = [K // P + (1 if p < K % P else 0) for p in range(P)]
    al = lambda v, a: -(-v // a) * a   # noqa: E731
    slot = [0, 0]
    k = 0
    for p in range(1, P):
        k += m[p - 1]
        elem = 2 if (acc_u16_ok and k <= 8 and p == 1) else 4
        pitch = al(min(W, wc + (1 << k)), 64)
        slot[(p - 1) % 2] = max(slot[(p - 1) % 2], al(n * pitch * elem, 256))
    return slot[0] + slot[1]


@pytest.mark.parametrize("levels", [4, 5, 6])
def test_forward_workspace_matches_the_layout_model(fht, restore, levels):
    """For every split, the library's forward plans take exactly the
    workspace the documented level layout gives (uint8 into int32 and into
    float32, all quadrants, 2^1 .. 2^15 rows)."""
    for K in range(1, 16):
        fht.set_tuning(K, levels, 1, 1)
    for h, w in [(1, 1), (3, 40), (100, 300), (700, 90), (1500, 1100), (5000, 40),
                 (32768, 7), (9, 20000)]:
        for q in range(4):
            for acc, u16 in ((torch.int32, True), (torch.float32, False)):
                got = fht.workspace_size(h, w, fht.LAYOUT_QUADRANT, q, torch.uint8, acc)
                assert got == _model_forward_workspace(h, w, q, levels, u16), (h, w, q, acc)


@pytest.fixture
def restore_batched(fht):
    saved = fht.get_batched_tuning()
    yield
    fht.set_batched_tuning(None)
    fht.set_batched_tuning(saved)


def test_batched_tuning_set_get_and_checks(fht, restore_batched):
    fht.set_batched_tuning(None)
    d = fht.get_batched_tuning()
    assert d == {"units_per_item": 4, "tile_u8": 2, "tile_wide": 1, "ctas_per_sm": 2,
                 "first_levels": {}}
    fht.set_batched_tuning({"units_per_item": 8, "ctas_per_sm": 3, "first_levels": {10: 6}})
    got = fht.get_batched_tuning()
    assert got["units_per_item"] == 8 and got["ctas_per_sm"] == 3
    assert got["first_levels"] == {10: 6} and got["tile_u8"] == 2
    for bad in ({"units_per_item": 0}, {"units_per_item": 17}, {"tile_u8": 4},
                {"tile_wide": 0}, {"ctas_per_sm": 1}, {"ctas_per_sm": 4},
                {"first_levels": {10: 3}}, {"first_levels": {7: 7}}):
        with pytest.raises(fht.FHTError):
            fht.set_batched_tuning(bad)
        assert fht.get_batched_tuning() == got   # a rejected tuning changes nothing
    fht.set_batched_tuning(None)
    assert fht.get_batched_tuning() == d


def test_table_with_batched_part_is_applied(fht, restore, restore_batched, tmp_path):
    from paper_1811_06378_gb300 import autotune
    table = {"table": {}, "batched": {"tuning": {"units_per_item": 2, "tile_u8": 1,
                                                 "tile_wide": 3, "ctas_per_sm": 3,
                                                 "first_levels": {"9": 4}},
                                      "us": 1.0, "default_us": 2.0}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    autotune.load(str(path))
    assert fht.get_batched_tuning() == {"units_per_item": 2, "tile_u8": 1, "tile_wide": 3,
                                        "ctas_per_sm": 3, "first_levels": {9: 4}}
