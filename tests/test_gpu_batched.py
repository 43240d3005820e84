"""The batched persistent launch against the oracle (bit-exact, every image),
under CUDA-graph capture and replay, and its bounded dependency waits."""

import numpy as np
import pytest
import torch

import oracle as O
from workloads import batch_shapes, edge_batch, random_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


def _mixed_shapes():
    # single-pass (n <= 64) and two-pass images, ragged sizes, a 1 x 1 image
    return [(1, 1), (3, 70), (64, 64), (65, 33), (100, 300), (257, 129), (512, 1000),
            (1000, 77), (33, 1024), (1024, 1024)]


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_batched_u8_matches_per_image(fht, q):
    shapes = _mixed_shapes()
    imgs = [torch.from_numpy(a).cuda() for a in edge_batch(shapes, seed=q)]
    plan = fht.BatchPlan(shapes, q)
    outs = plan.forward(imgs)
    assert plan.status() == 0
    for x, o in zip(imgs, outs):
        want = O.quadrant(x.cpu().numpy(), q)
        assert (o.cpu().numpy().astype(np.int64) == want).all(), tuple(x.shape)


def test_batched_f32_matches_per_image(fht):
    shapes = [(50, 60), (128, 128), (300, 200)]
    imgs = [torch.from_numpy(random_image(h, w, "f32", seed=h)).cuda() for h, w in shapes]
    plan = fht.BatchPlan(shapes, 0, torch.float32, torch.float32)
    outs = plan.forward(imgs)
    for x, o in zip(imgs, outs):
        want = O.quadrant(x.cpu().numpy(), 0, "f32")
        assert np.array_equal(o.cpu().numpy(), want), tuple(x.shape)


def test_batched_512_images_graph_replay(fht):
    """The 512-image batch (sides log-uniform in [64, 1024], 8% edges) in one
    launch captured in a CUDA graph; replays are idempotent and every image
    equals the oracle's quadrant bit for bit."""
    shapes = batch_shapes(512, seed=3)
    imgs = [torch.from_numpy(a).cuda() for a in edge_batch(shapes, seed=3)]
    plan = fht.BatchPlan(shapes, 0)
    ws = plan.workspace("cuda")
    outs = [torch.zeros(sh, dtype=torch.int32, device="cuda") for sh in plan.out_shapes]
    plan.forward(imgs, outs, ws)          # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.forward(imgs, outs, ws, stream=s)
    for o in outs:
        o.fill_(-1)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    for j, (x, o) in enumerate(zip(imgs, outs)):
        want = O.quadrant(x.cpu().numpy(), 0)
        assert (o.cpu().numpy().astype(np.int64) == want).all(), (j, tuple(x.shape))


def test_batched_adjoint_512_images_graph_replay(fht):
    """The FP32 adjoint plan of the same 512 shapes, captured and replayed:
    every image gradient equals the oracle's FP32 transpose bit for bit."""
    shapes = batch_shapes(512, seed=3)
    plan = fht.BatchPlan(shapes, 0, torch.float32, torch.float32)
    gen = torch.Generator(device="cuda").manual_seed(512)
    grads = [torch.randn(sh, generator=gen, device="cuda") for sh in plan.out_shapes]
    ws = plan.workspace("cuda")
    outs = [torch.empty(sh, dtype=torch.float32, device="cuda") for sh in shapes]
    plan.adjoint(grads, outs, ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.adjoint(grads, outs, ws, stream=s)
    for o in outs:
        o.fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    for j, ((h, w), gr, o) in enumerate(zip(shapes, grads, outs)):
        want = O.adjoint_quadrant(gr.cpu().numpy(), h, w, 0, "f32")
        assert np.array_equal(o.cpu().numpy(), want), (j, h, w)


def test_batched_wait_timeout_is_reported(fht):
    """An unsatisfiable dependency (test hook) makes the bounded waits run
    out: the launch ends, reports FHT_ETIMEOUT, and the context stays usable."""
    shapes = [(256, 256), (300, 100)]     # two passes each: second passes wait
    imgs = [torch.from_numpy(a).cuda() for a in edge_batch(shapes, seed=9)]
    plan = fht.BatchPlan(shapes, 0)
    plan.set_test_hooks(wait_budget_cycles=2_000_000, dep_bias=1)   # ~1 ms per wait
    plan.forward(imgs)
    assert plan.status() == 5
    plan.set_test_hooks(wait_budget_cycles=4_000_000_000, dep_bias=0)
    outs = plan.forward(imgs)
    assert plan.status() == 0
    for x, o in zip(imgs, outs):
        assert (o.cpu().numpy().astype(np.int64) == O.quadrant(x.cpu().numpy(), 0)).all()


def test_batched_back_to_back_calls_keep_their_descriptors(fht):
    """Five direct calls on one plan and stream, different images and outputs,
    no synchronisation between them: each launch uses its own call's
    descriptors (the plan's staging tables, used in turn, are not rewritten
    before the copy of the call that used them last has run)."""
    shapes = [(300, 200), (64, 700), (513, 90)]
    sets = [[torch.from_numpy(x).cuda() for x in edge_batch(shapes, seed=21 + k)]
            for k in range(5)]
    plan = fht.BatchPlan(shapes, 1)
    ws = plan.workspace("cuda")
    torch.cuda._sleep(50_000_000)   # keep the stream busy so the copies are still queued
    outs = [plan.forward(imgs, workspace=ws) for imgs in sets]
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    for imgs, o in zip(sets, outs):
        for x, y in zip(imgs, o):
            assert (y.cpu().numpy().astype(np.int64) == O.quadrant(x.cpu().numpy(), 1)).all()


def test_batched_graph_keeps_captured_descriptors(fht):
    """A direct call after a capture does not change what the graph replays."""
    shapes = [(200, 300), (129, 64)]
    a = [torch.from_numpy(x).cuda() for x in edge_batch(shapes, seed=31)]
    b = [torch.from_numpy(x).cuda() for x in edge_batch(shapes, seed=32)]
    plan = fht.BatchPlan(shapes, 0)
    ws_g = plan.workspace("cuda")
    ws_d = plan.workspace("cuda")
    oa = [torch.empty(fht.query_shape(h, w, 0), dtype=torch.int32, device="cuda")
          for h, w in shapes]
    plan.forward(a, oa, ws_g)   # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.forward(a, oa, ws_g, stream=s)
    ob = plan.forward(b, workspace=ws_d)
    for o in oa:
        o.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    for x, o in zip(a, oa):
        assert (o.cpu().numpy().astype(np.int64) == O.quadrant(x.cpu().numpy(), 0)).all()
    for x, o in zip(b, ob):
        assert (o.cpu().numpy().astype(np.int64) == O.quadrant(x.cpu().numpy(), 0)).all()


def test_batched_two_captures_keep_their_own_descriptors(fht):
    """Two graphs captured from one plan with different images and outputs,
    replayed in turn (and again after a direct call): each graph runs the
    descriptors of its own capture."""
    shapes = [(200, 300), (129, 64), (700, 90)]
    a = [torch.from_numpy(x).cuda() for x in edge_batch(shapes, seed=41)]
    b = [torch.from_numpy(x).cuda() for x in edge_batch(shapes, seed=42)]
    c = [torch.from_numpy(x).cuda() for x in edge_batch(shapes, seed=43)]
    plan = fht.BatchPlan(shapes, 2)
    ws_a, ws_b, ws_c = (plan.workspace("cuda") for _ in range(3))
    oa = [torch.empty(fht.query_shape(h, w, 2), dtype=torch.int32, device="cuda")
          for h, w in shapes]
    ob = [torch.empty_like(o) for o in oa]
    plan.forward(a, oa, ws_a)   # warm-up outside the captures
    torch.cuda.synchronize()
    graphs = []
    for imgs, outs, ws in ((a, oa, ws_a), (b, ob, ws_b)):
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.forward(imgs, outs, ws, stream=s)
        graphs.append(g)
    for rep in range(2):
        for o in oa + ob:
            o.fill_(-1)
        graphs[0].replay()
        graphs[1].replay()
        torch.cuda.synchronize()
        assert plan.status(ws_a) == 0 and plan.status(ws_b) == 0
        for imgs, outs in ((a, oa), (b, ob)):
            for x, o in zip(imgs, outs):
                want = O.quadrant(x.cpu().numpy(), 2)
                assert (o.cpu().numpy().astype(np.int64) == want).all(), (rep, tuple(x.shape))
        oc = plan.forward(c, workspace=ws_c)   # a direct call between the replays
        for x, o in zip(c, oc):
            assert (o.cpu().numpy().astype(np.int64) == O.quadrant(x.cpu().numpy(), 2)).all()


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_batched_adjoint_matches_per_image_and_oracle(fht, q):
    """fht_adjoint_batched over mixed sizes (one- and two-pass images,
    ragged sides, a 1 x 1 image) equals the oracle's FP32 transpose bit for
    bit on every image; a forward call on the same plan and workspace in
    between leaves it unchanged."""
    shapes = _mixed_shapes()
    plan = fht.BatchPlan(shapes, q, torch.float32, torch.float32)
    rng = np.random.default_rng(40 + q)
    grads = [torch.from_numpy(rng.standard_normal(sh).astype(np.float32)).cuda()
             for sh in plan.out_shapes]
    ws = plan.workspace("cuda")
    outs = plan.adjoint(grads, workspace=ws)
    assert plan.status(ws) == 0
    imgs = [torch.from_numpy(random_image(h, w, "f32", seed=h + w)).cuda() for h, w in shapes]
    plan.forward(imgs, workspace=ws)
    again = plan.adjoint(grads, workspace=ws)
    assert plan.status(ws) == 0
    for (h, w), g, o, o2 in zip(shapes, grads, outs, again):
        want = O.adjoint_quadrant(g.cpu().numpy(), h, w, q, "f32")
        assert np.array_equal(o.cpu().numpy(), want), (h, w)
        assert np.array_equal(o2.cpu().numpy(), want), (h, w)


def test_batched_adjoint_is_transpose_of_batched_forward(fht):
    """<H x, g> = <x, H^T g> per image, both sides from the batched calls
    (FP64 sums of FP32 results, within the FP32 bound 1e-5 * sum|terms|)."""
    shapes = batch_shapes(64, seed=5)
    plan = fht.BatchPlan(shapes, 2, torch.float32, torch.float32)
    rng = np.random.default_rng(11)
    xs = [torch.from_numpy(rng.standard_normal(sh).astype(np.float32)).cuda() for sh in shapes]
    gs = [torch.from_numpy(rng.standard_normal(sh).astype(np.float32)).cuda()
          for sh in plan.out_shapes]
    ws = plan.workspace("cuda")
    hx = plan.forward(xs, workspace=ws)
    htg = plan.adjoint(gs, workspace=ws)
    for x, g, a, b in zip(xs, gs, hx, htg):
        lhs = float((a.double() * g.double()).sum())
        rhs = float((x.double() * b.double()).sum())
        scale = float((a.double().abs() * g.double().abs()).sum())
        assert abs(lhs - rhs) <= 1e-5 * scale


def test_batched_adjoint_graph_replay(fht):
    """The batched adjoint captured in a CUDA graph replays the captured
    descriptors."""
    shapes = [(200, 300), (129, 64), (40, 1000)]
    plan = fht.BatchPlan(shapes, 1, torch.float32, torch.float32)
    rng = np.random.default_rng(3)
    gs = [torch.from_numpy(rng.standard_normal(sh).astype(np.float32)).cuda()
          for sh in plan.out_shapes]
    ws = plan.workspace("cuda")
    outs = [torch.empty(sh, dtype=torch.float32, device="cuda") for sh in shapes]
    plan.adjoint(gs, outs, ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.adjoint(gs, outs, ws, stream=s)
    for o in outs:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    for (h, w), gr, o in zip(shapes, gs, outs):
        want = O.adjoint_quadrant(gr.cpu().numpy(), h, w, 1, "f32")
        assert np.array_equal(o.cpu().numpy(), want), (h, w)
