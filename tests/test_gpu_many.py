"""Uniform batches (forward_many / adjoint_many, one launch per pass for B
same-size FP32 images) against the oracle's FP32 recursion, bit for bit, on
every image of every batch."""

import numpy as np
import pytest
import torch

import oracle as O
from workloads import ellipse_phantom, random_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fht():
    import paper_1811_06378_gb300 as m
    return m


def _batch(B, h, w, seed):
    return torch.from_numpy(np.stack([random_image(h, w, "f32", seed=seed + b)
                                      for b in range(B)])).cuda()


@pytest.mark.parametrize("B,h,w", [(1, 37, 53), (5, 100, 130), (3, 257, 64), (4, 64, 300)])
def test_forward_many_full_and_quadrants(fht, B, h, w):
    x = _batch(B, h, w, seed=h)
    xs = x.cpu().numpy()
    got = fht.forward_many(x, fht.LAYOUT_FULL).cpu().numpy()
    for b in range(B):
        assert np.array_equal(got[b], O.full(xs[b], "f32")), b
    for q in range(4):
        got = fht.forward_many(x, fht.LAYOUT_QUADRANT, q).cpu().numpy()
        for b in range(B):
            assert np.array_equal(got[b], O.quadrant(xs[b], q, "f32")), (q, b)


@pytest.mark.parametrize("B,h,w", [(1, 37, 53), (5, 100, 130), (3, 257, 64)])
def test_adjoint_many_full_and_quadrants(fht, B, h, w):
    R, W = fht.full_shape(h, w)
    g = torch.randn((B, R, W), device="cuda", generator=torch.Generator("cuda").manual_seed(h))
    got = fht.adjoint_many(g, h, w, fht.LAYOUT_FULL).cpu().numpy()
    gs = g.cpu().numpy()
    for b in range(B):
        assert np.array_equal(got[b], O.adjoint_full(gs[b], h, w, "f32")), b
    for q in range(4):
        n, Wq = fht.query_shape(h, w, q)
        gq = torch.randn((B, n, Wq), device="cuda")
        got = fht.adjoint_many(gq, h, w, fht.LAYOUT_QUADRANT, q).cpu().numpy()
        gqs = gq.cpu().numpy()
        for b in range(B):
            assert np.array_equal(got[b], O.adjoint_quadrant(gqs[b], h, w, q, "f32")), (q, b)


def test_many_with_pitches_and_gaps(fht):
    """Images, Hough images and gradients as views: padded rows and gaps
    between batch items; the bytes around every view stay untouched."""
    B, h, w = 3, 90, 70
    src = torch.full((B + 1, h + 5, w + 9), 7.0, device="cuda")
    x = src[1:, 2:2 + h, 3:3 + w]
    x.copy_(_batch(B, h, w, seed=5))
    R, W = fht.full_shape(h, w)
    obuf = torch.full((B, R + 3, W + 5), -3.0, device="cuda")
    out = obuf[:, 1:1 + R, 2:2 + W]
    fht.forward_many(x, fht.LAYOUT_FULL, out=out)
    xs = x.cpu().numpy()
    for b in range(B):
        assert np.array_equal(out[b].cpu().numpy(), O.full(xs[b], "f32"))
    mask = torch.ones_like(obuf, dtype=torch.bool)
    mask[:, 1:1 + R, 2:2 + W] = False
    assert bool((obuf[mask] == -3.0).all())
    gbuf = torch.full((B, h + 4, w + 6), 11.0, device="cuda")
    gi = gbuf[:, 2:2 + h, 1:1 + w]
    fht.adjoint_many(out, h, w, fht.LAYOUT_FULL, out=gi)
    outs = out.cpu().numpy()
    for b in range(B):
        assert np.array_equal(gi[b].cpu().numpy(), O.adjoint_full(outs[b], h, w, "f32"))
    mask = torch.ones_like(gbuf, dtype=torch.bool)
    mask[:, 2:2 + h, 1:1 + w] = False
    assert bool((gbuf[mask] == 11.0).all())


def test_many_at_1024_matches_single_and_autograd(fht):
    """The differentiable path's batch (3 x 1024^2 phantoms): FHTFunction on
    (B, h, w) runs the uniform batches; forward and gradient equal the
    oracle's FP32 full image and FP32 transpose on every image."""
    x = torch.from_numpy(np.stack([ellipse_phantom(1024, seed=100 + b)
                                   for b in range(3)])).cuda().requires_grad_(True)
    y = fht.FHTFunction.apply(x)
    xs = x.detach().cpu().numpy()
    ys = y.detach().cpu().numpy()
    for b in range(3):
        assert np.array_equal(ys[b], O.full(xs[b], "f32")), b
    g = torch.randn_like(y)
    (y * g).sum().backward()
    gs = g.cpu().numpy()
    grads = x.grad.cpu().numpy()
    for b in range(3):
        assert np.array_equal(grads[b], O.adjoint_full(gs[b], 1024, 1024, "f32")), b
