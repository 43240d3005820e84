"""The differentiable path at its workload size: 64 FP32 1024 x 1024
random-ellipse phantoms, loss ||F x - F x_true||^2 over the full Hough image,
x starting at zero, 50 gradient-descent steps through FHTFunction (forward
kernels + hand-written adjoint). The step size is 1 / (2 lambda_max(F^T F)),
lambda_max by 30 power iterations, so the loss can only go down."""

import numpy as np
import pytest
import torch

from workloads import ellipse_phantom

pytestmark = pytest.mark.gpu


def test_reconstruction_64_phantoms():
    import paper_1811_06378_gb300 as fht
    B, n = 64, 1024
    x_true = torch.from_numpy(np.stack([ellipse_phantom(n, seed=100 + i) for i in range(B)])).cuda()
    F = fht.FHTFunction.apply
    with torch.no_grad():
        b = F(x_true)
        # lambda_max of F^T F by power iteration on one image (same operator for all)
        v = torch.randn((n, n), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        for _ in range(30):
            v = fht.adjoint(fht.full_quadrants(v / v.norm(), acc=torch.float32), n, n)
        lam = float(v.norm())
    lr = 1.0 / (2.0 * lam)
    x = torch.zeros_like(x_true, requires_grad=True)
    losses = []
    for _ in range(50):
        loss = ((F(x) - b) ** 2).sum()
        losses.append(float(loss))
        (g,) = torch.autograd.grad(loss, x)
        with torch.no_grad():
            x -= lr * g
    assert all(l1 <= l0 * (1 + 1e-6) for l0, l1 in zip(losses, losses[1:])), losses[:5]
    assert losses[-1] < 0.5 * losses[0]
    # the reconstruction moves toward the phantoms
    err0 = float(x_true.norm())
    err = float((x.detach() - x_true).norm())
    assert err < err0
