"""The bounds-checked debug build (compiled with -DFHT_DEBUG, loaded with
FHT_DEBUG=1): every global load and store of the pass kernels is checked
against the buffers its pass may touch. Run through every entry point, it
refuses nothing and still gives the oracle's results; with the test hook
recording destination spans shorter than the buffers, it refuses the last
stores (skipping them: nothing outside a buffer is touched) and
fht_device_status reports FHT_EBOUNDS. The library is built here, in a
directory of its own; each run is a child process (the build to load is
chosen when the package is imported)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
import torch
import oracle as O
import paper_1811_06378_gb300 as fht
from paper_1811_06378_gb300 import sharded
from workloads import edges_and_lines, random_image, edge_batch
assert fht.DEBUG
i32 = lambda a: a.astype(np.int64).astype(np.int32)
img = edges_and_lines(300, 257, seed=1)
x = torch.from_numpy(img).cuda()
for q in range(4):
    assert (fht.forward(x, q).cpu().numpy() == i32(O.quadrant(img, q))).all(), q
base = edges_and_lines(160, 300, seed=2)
view = torch.from_numpy(base).cuda()[5:150, 3:203]
assert (fht.forward(view, 1).cpu().numpy() == i32(O.quadrant(base[5:150, 3:203], 1))).all()
assert (fht.forward_range(x, 1, 3, 200).cpu().numpy() == O.range_slice(img, 1, 3, 200)).all()
F = fht.full_quadrants(x, apply_fhtshift=True).cpu().numpy()
assert (F == i32(O.fhtshift_full(O.full(img), 300, 257))).all()
g = torch.from_numpy(np.random.default_rng(3).standard_normal(fht.full_shape(300, 257))
                     .astype(np.float32)).cuda()
assert np.array_equal(fht.adjoint(g, 300, 257).cpu().numpy(),
                      O.adjoint_full(g.cpu().numpy(), 300, 257, "f32"))
gq = torch.from_numpy(np.random.default_rng(4).standard_normal(fht.query_shape(300, 257, 2))
                      .astype(np.float32)).cuda()
assert np.array_equal(fht.adjoint(gq, 300, 257, fht.LAYOUT_QUADRANT, 2).cpu().numpy(),
                      O.adjoint_quadrant(gq.cpu().numpy(), 300, 257, 2, "f32"))
assert (fht.forward_sheared(x, 3, -0.4).cpu().numpy() == i32(O.sheared_quadrant(img, 3, -0.4))).all()
assert (fht.forward_scaled(x, 2, 1.7, 0.3).cpu().numpy() ==
        i32(O.scaled_quadrant(img, 2, 1.7, 0.3))).all()
assert (fht.forward_op(x, 0, fht.OP_MAX).cpu().numpy() == O.quadrant_op(img, 0, 1)).all()
f = random_image(90, 70, "f32", seed=5)
fb = torch.from_numpy(np.stack([f, f * 2])).cuda()
got = fht.forward_many(fb, fht.LAYOUT_FULL).cpu().numpy()
assert np.array_equal(got[1], O.full(f * 2, "f32"))
shapes = [(40, 70), (100, 300), (300, 90), (600, 1000)]
imgs = [torch.from_numpy(a).cuda() for a in edge_batch(shapes, seed=6)]
plan = fht.BatchPlan(shapes, 2)
for a, o in zip(imgs, plan.forward(imgs)):
    assert (o.cpu().numpy() == i32(O.quadrant(a.cpu().numpy(), 2))).all()
fplan = fht.BatchPlan(shapes, 3, torch.float32, torch.float32)
grads = [torch.randn(sh, device="cuda") for sh in fplan.out_shapes]
for (h, w), gg, o in zip(shapes, grads, fplan.adjoint(grads)):
    assert np.array_equal(o.cpu().numpy(), O.adjoint_quadrant(gg.cpu().numpy(), h, w, 3, "f32"))
big = edges_and_lines(4096, 700, seed=7)
xb = torch.from_numpy(big).cuda()
assert (fht.forward(xb, 0).cpu().numpy() == O.quadrant(big, 0)).all()   # the staged final pass
for q, (h, w) in ((0, (4096, 700)), (2, (700, 4096))):   # the staged adjoint final passes
    gb = torch.from_numpy(np.random.default_rng(8 + q).standard_normal(fht.query_shape(h, w, q))
                          .astype(np.float32)).cuda()
    assert np.array_equal(fht.adjoint(gb, h, w, fht.LAYOUT_QUADRANT, q).cpu().numpy(),
                          O.adjoint_quadrant(gb.cpu().numpy(), h, w, q, "f32"))
p = sharded.ShardPlan(1500, 700, 1, 4)
Ls = [sharded.local_levels_gpu(p.strip_of(torch.from_numpy(big[:1500]).cuda(), r), p,
                               torch.int32) for r in range(4)]
blocks = [sharded.merge_levels_gpu(torch.stack([L[b * p.block:(b + 1) * p.block] for L in Ls]),
                                   p, b) for b in range(4)]
assert (torch.cat(blocks).cpu().numpy() == O.quadrant(big[:1500], 1)).all()
assert fht.device_status() == fht.FHT_OK, "an access in bounds was refused"
# the hook: destination spans 64 bytes short -> the last stores are refused
assert fht.lib.fht_debug_test_hooks(64) == 0
fht.forward(x, 0)
fht.adjoint(g, 300, 257)
assert fht.device_status() == fht.FHT_EBOUNDS
assert fht.lib.fht_debug_test_hooks(0) == 0
assert (fht.forward(x, 0).cpu().numpy() == i32(O.quadrant(img, 0))).all()
assert fht.device_status() == fht.FHT_OK
print("debug build ok")
"""


def test_debug_build_checks_every_entry_point():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__._builder().build(debug=True)
    env = dict(os.environ, FHT_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-1000:], r.stderr[-3000:])
    assert "debug build ok" in r.stdout
