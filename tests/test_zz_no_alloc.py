"""fht_forward_static: the forward transform for callers that cannot allocate
device memory (code confined to a memory pool or budget it does not own,
hosts that forbid allocation after start-up).

It keeps its intermediate levels in a fixed device array inside the library
that every call shares and that keeps the last call's contents, so its output
is compared with fht_forward's on several calls in a row, through the C ABI,
and with the oracle. The tolerance is the one the parity tests use:
bit-exact (integer and FP32 results run the same additions in the same
order)."""

import ctypes

import numpy as np
import pytest
import torch

import oracle as O

from workloads import edges_and_lines, random_image

pytestmark = pytest.mark.gpu

FHT_OK, FHT_ENOMEM = 0, 2
_DT = {torch.uint8: 0, torch.int32: 1, torch.float32: 2}


def _static_fn():
    import paper_1811_06378_gb300 as fht
    fn = fht.lib.fht_forward_static
    vp, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    fn.restype = i
    fn.argtypes = [vp, i, i, i, i64, i, vp, i, i64, vp]
    return fht, fn


def _call_static(fn, img, q, out):
    h, w = img.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(ctypes.c_void_p(img.data_ptr()), _DT[img.dtype], h, w, img.stride(0), q,
              ctypes.c_void_p(out.data_ptr()), _DT[out.dtype], out.stride(0), stream)


def test_static_scratch_forward_matches_workspace_forward():
    fht, fn = _static_fn()
    cases = [
        (edges_and_lines(4096, 4096, seed=11), 0, torch.int32),   # the largest that fits
        (random_image(700, 513, "u8", seed=3), 2, torch.int32),   # transposed quadrant
        (random_image(300, 257, "f32", seed=4), 1, torch.float32),
        (edges_and_lines(4096, 4096, seed=12), 3, torch.int32),
    ]
    for img_np, q, acc in cases:
        img = torch.from_numpy(img_np).cuda()
        want = fht.forward(img, q, acc=acc)
        oracle = O.quadrant(img_np, q, "f32" if acc == torch.float32 else "i64")
        n, W = fht.query_shape(*img_np.shape, q)
        for _ in range(2):   # two calls in a row on the same shared scratch
            out = torch.full((n, W), -7, dtype=acc, device="cuda")
            assert _call_static(fn, img, q, out) == FHT_OK
            torch.cuda.synchronize()
            assert torch.equal(out, want), (img_np.shape, q)
            assert np.array_equal(out.cpu().numpy(), oracle.astype(out.cpu().numpy().dtype)), \
                (img_np.shape, q)


def test_static_scratch_rejects_oversized_requests():
    fht, fn = _static_fn()
    # an 8192 x 8192 float32 quadrant needs far more than the fixed 64 MiB
    need = fht.workspace_size(8192, 8192, fht.LAYOUT_QUADRANT, 0, torch.float32,
                              torch.float32)
    assert need > 64 << 20
    img = torch.zeros((8192, 8192), dtype=torch.float32, device="cuda")
    out = torch.full((8192, 16384), 3.0, dtype=torch.float32, device="cuda")
    assert _call_static(fn, img, 0, out) == FHT_ENOMEM
    torch.cuda.synchronize()
    assert bool((out == 3.0).all())   # nothing was enqueued
