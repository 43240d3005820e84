"""One image's quadrant over several ranks (paper_1811_06378_gb300.sharded):
row strips, their first K - log2(P) levels, one all-to-all, the last log2(P)
levels. Here the ranks are gloo processes on the CPU and both level steps are
the oracle's: each rank's slope rows must equal the oracle's whole quadrant
bit for bit, in integers and in FP32 (the same additions in the same order).
The GPU level steps are checked against the oracle in
tests/test_gpu_sharded.py."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_local(strip: torch.Tensor, plan, acc):
    """The strip's first K - log2(P) levels by the oracle: its plain
    butterfly, padded to n_s rows on the whole image's width W."""
    import oracle as O
    kind = "f32" if acc == torch.float32 else "i64"
    src = strip.numpy().T if plan.q >= 2 else strip.numpy()
    P = O.padded(src, plan.n_s, plan.W, kind)
    return torch.from_numpy(O.butterfly(P, O.SIGMA[plan.q], kind))


def _oracle_merge(parts: torch.Tensor, plan, rank):
    """The last log2(P) levels by the oracle: for every tau of the block, the
    P strips' rows tau, row p rotated left by sigma*tau*p (read at
    x + sigma*tau*p), through the plain P-row butterfly."""
    import oracle as O
    a = parts.numpy()
    sg = O.SIGMA[plan.q]
    kind = "f32" if a.dtype == np.float32 else "i64"
    out = []
    for r in range(a.shape[1]):
        tau = rank * plan.block + r
        rows = np.stack([np.roll(a[p, r], -sg * tau * p) for p in range(a.shape[0])])
        out.append(O.butterfly(rows, sg, kind))
    return torch.from_numpy(np.concatenate(out))


def _rank(rank, world, port, cases, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1811_06378_gb300 import sharded
    from workloads import edges_and_lines, random_image
    ok = []
    for h, w, q, kind in cases:
        img = (random_image(h, w, "f32", seed=h + w + q) if kind == "f32"
               else edges_and_lines(h, w, seed=h + w + q))
        acc = torch.float32 if kind == "f32" else torch.int64
        plan = sharded.ShardPlan(h, w, q, world)
        strip = plan.strip_of(torch.from_numpy(img), rank)
        got = sharded.forward_sharded(strip, plan, rank, acc=acc, local=_oracle_local,
                                      merge=_oracle_merge).numpy()
        t_lo, t_hi = plan.slopes(rank)
        want = O.quadrant(img, q, kind)[t_lo:t_hi + 1]
        ok.append(bool(got.shape == want.shape and np.array_equal(got, want)))
    results[rank] = ok
    dist.destroy_process_group()


CASES = [(64, 50, 0, "i64"), (64, 50, 1, "i64"), (70, 64, 2, "i64"), (37, 64, 3, "i64"),
         (100, 33, 0, "i64"), (128, 200, 1, "f32"), (90, 120, 3, "f32")]


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_quadrant_equals_the_whole_quadrant(world):
    """Ragged images (the last strips short or empty), all four quadrants,
    int64 and FP32: every rank's slope rows are the oracle's."""
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(world, port, CASES, results), nprocs=world, join=True)
        res = dict(results)
    for r in range(world):
        assert res[r] == [True] * len(CASES), (r, res[r])


def test_shard_plan_geometry():
    """Strips, owned slopes and the exchange size per pair (n*W/P^2)."""
    from paper_1811_06378_gb300 import sharded
    p = sharded.ShardPlan(3000, 700, 0, 4)
    assert (p.n, p.W, p.n_s, p.block) == (4096, 4796, 1024, 256)
    assert [p.strip(r) for r in range(4)] == [(0, 1024), (1024, 2048), (2048, 3000),
                                              (3072, 3000)]
    assert p.slopes(3) == (3072, 4095)
    assert p.exchange_elements() == 4096 * 4796 // 16
    p2 = sharded.ShardPlan(700, 3000, 2, 2)   # Q2: strips are image columns
    assert (p2.n, p2.W, p2.n_s) == (4096, 4796, 2048)
    img = torch.zeros((700, 3000))
    assert tuple(p2.strip_of(img, 1).shape) == (700, 952)
    with pytest.raises(ValueError):
        sharded.ShardPlan(4, 4, 0, 4)   # n = 4 < 16
    with pytest.raises(ValueError):
        sharded.ShardPlan(64, 64, 0, 3)
