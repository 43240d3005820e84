"""The concurrent schedule of the full layout (the default; FHT_CONCURRENT=0
turns it off: the four quadrants on four streams, each with its own workspace slice, the adjoint's
final passes chained in quadrant order) gives the serial schedule's results
bit for bit: the full image with and without the fused fhtshift, and the FP32
full adjoint (whose quadrant contributions must still be added in the order
Q0, Q1, Q2, Q3), called directly and replayed from a captured CUDA graph.
The library creates its streams on the first such call that is not being
captured; a graph captured before then holds the serial schedule, checked
too. The setting is read when the library loads, so each schedule runs in a
child process."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

H, W = 1500, 1100   # 2048 padded rows and columns: two passes per quadrant

CHILD = r"""
import sys
import numpy as np
import torch
import paper_1811_06378_gb300 as fht
from workloads import edges_and_lines
H, W = int(sys.argv[2]), int(sys.argv[3])
img = torch.from_numpy(edges_and_lines(H, W, seed=31)).cuda()
R, C = fht.full_shape(H, W)
g = torch.from_numpy(np.random.default_rng(32).standard_normal((R, C)).astype(np.float32)).cuda()
ws = torch.empty(max(fht.workspace_size(H, W, fht.LAYOUT_FULL, 0, torch.uint8, torch.int32),
                     fht.workspace_size(H, W, fht.LAYOUT_FULL, 0, torch.float32, torch.float32)),
                 dtype=torch.uint8, device="cuda")
F = torch.empty((R, C), dtype=torch.int32, device="cuda")
Fs = torch.empty_like(F)
A = torch.empty((H, W), dtype=torch.float32, device="cuda")
def step():
    fht.full_quadrants(img, out=F, workspace=ws)
    fht.full_quadrants(img, out=Fs, apply_fhtshift=True, workspace=ws)
    fht.adjoint(g, H, W, fht.LAYOUT_FULL, out=A, workspace=ws)
def direct():
    step()
    torch.cuda.synchronize()
    return [F.cpu().numpy(), Fs.cpu().numpy(), A.cpu().numpy()]
def replayed():
    for t in (F, Fs, A):
        t.fill_(0)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    return [F.cpu().numpy(), Fs.cpu().numpy(), A.cpu().numpy()]
if sys.argv[4] == "capture_first":
    r = replayed()
    d = direct()
else:
    d = direct()
    r = replayed()
np.savez(sys.argv[1], *d, *r, g=g.cpu().numpy())
"""


@pytest.mark.parametrize("concurrent,order", [("1", "direct_first"), ("1", "capture_first"),
                                              ("0", "direct_first")])
def test_full_layout_schedules_are_bit_exact(concurrent, order, tmp_path):
    import oracle as O
    from workloads import edges_and_lines
    path = str(tmp_path / "out.npz")
    env = dict(os.environ, FHT_CONCURRENT=concurrent, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD, path, str(H), str(W), order], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(path)
    img = edges_and_lines(H, W, seed=31)
    F = O.full(img)
    want = [F.astype(np.int64).astype(np.int32),
            O.fhtshift_full(F, H, W).astype(np.int64).astype(np.int32),
            O.adjoint_full(got["g"], H, W, "f32")]
    for k in range(6):
        assert (got[f"arr_{k}"] == want[k % 3]).all(), (concurrent, k)
