"""The GPU level steps of the sharded quadrant (fht_forward_padded,
fht_merge_strips) against the oracle, on one GPU: every strip's first
K - log2(P) levels, the all-to-all done by slicing (each block goes where the
exchange would put it; nothing waits on another launch), then every rank's
last log2(P) levels. The concatenated blocks must be the oracle's quadrant bit
for bit. The exchange itself runs over torch.distributed in
tests/test_sharded_gloo.py."""

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


def _sharded_on_one_gpu(sharded, img_t, h, w, q, P, acc):
    plan = sharded.ShardPlan(h, w, q, P)
    locals_ = [sharded.local_levels_gpu(plan.strip_of(img_t, r), plan, acc) for r in range(P)]
    blocks = []
    for b in range(P):
        parts = torch.stack([L[b * plan.block:(b + 1) * plan.block] for L in locals_])
        blocks.append(sharded.merge_levels_gpu(parts, plan, b))
    return torch.cat(blocks).cpu().numpy()


@pytest.mark.parametrize("P", [1, 2, 4, 8])
@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_sharded_levels_u8_bit_exact(fht, P, q):
    from paper_1811_06378_gb300 import sharded
    h, w = (1500, 700) if q < 2 else (700, 1500)   # 2048 padded rows: a short last strip
    img = edges_and_lines(h, w, seed=q + 10 * P)
    got = _sharded_on_one_gpu(sharded, torch.from_numpy(img).cuda(), h, w, q, P, torch.int32)
    assert (got == O.quadrant(img, q).astype(np.int64).astype(np.int32)).all()


@pytest.mark.parametrize("P", [2, 8])
def test_sharded_levels_f32_and_4096(fht, P):
    from paper_1811_06378_gb300 import sharded
    img = random_image(300, 257, "f32", seed=P)
    got = _sharded_on_one_gpu(sharded, torch.from_numpy(img).cuda(), 300, 257, 1, P,
                              torch.float32)
    assert np.array_equal(got, O.quadrant(img, 1, "f32"))
    img = edges_and_lines(4096, 4096, seed=4096)
    got = _sharded_on_one_gpu(sharded, torch.from_numpy(img).cuda(), 4096, 4096, 0, P,
                              torch.int32)
    assert (got == O.quadrant(img, 0)).all()


def test_padded_forward_is_forward_at_its_own_size(fht):
    """With n = next_pow2(rows) and W = w_c + n the padded forward is the plain
    quadrant; a wider W and a taller n give the oracle's transform of the
    zero-padded image on that width."""
    img = edges_and_lines(200, 130, seed=3)
    x = torch.from_numpy(img).cuda()
    for q in range(4):
        n, W = fht.query_shape(200, 130, q)
        assert torch.equal(fht.forward_padded(x, q, n, W), fht.forward(x, q))
        got = fht.forward_padded(x, q, 2 * n, W + n + 5).cpu().numpy()
        src = img.T if q >= 2 else img
        want = O.butterfly(O.padded(src, 2 * n, W + n + 5, "i64"), O.SIGMA[q], "i64")
        assert (got == want).all(), q
    empty = x[:0]
    z = fht.forward_padded(empty, 0, 64, 200)
    assert z.shape == (64, 200) and int(z.abs().sum()) == 0
