"""Tile width and kernel form of the fused passes: any FHT_TUNE setting gives
the same result, and so do both forms of the final pass from a uint16 level
(FHT_STAGED: the persistent staged kernel by default, or one item per CTA).

FHT_TUNE="a,b" sets how many warp-widths of source columns one tile's first
block of levels covers (a: first passes over uint8 images, whose shared tile
holds uint16; b: tiles of 4-byte values). Wider tiles re-read less of the
halo but need more shared memory; a width whose tile does not fit one block's
shared memory is narrowed at launch. The setting is read when the library
loads, so each setting runs in a child process and its result is compared
bit for bit with the oracle. The child also checks that the device recorded
no error."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
import paper_1811_06378_gb300 as fht
from workloads import edges_and_lines, random_image
img = edges_and_lines(1500, 1100, seed=21)
f = random_image(700, 900, "f32", seed=22)
out = [fht.forward(torch.from_numpy(img).cuda(), q).cpu().numpy() for q in range(4)]
out += [fht.forward(torch.from_numpy(f).cuda(), q, acc=torch.float32).cpu().numpy()
        for q in (0, 2)]
assert fht.device_status() == fht.FHT_OK
np.savez(sys.argv[1], *out)
"""


@pytest.mark.parametrize("tune", ["1,1", "3,3", "2,2"])
def test_tile_width_setting_is_bit_exact(tune, tmp_path):
    import oracle as O
    from workloads import edges_and_lines, random_image
    path = str(tmp_path / "out.npz")
    env = dict(os.environ, FHT_TUNE=tune, FHT_TUNE_FILE="none", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD, path], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(path)
    img = edges_and_lines(1500, 1100, seed=21)
    f = random_image(700, 900, "f32", seed=22)
    for q in range(4):
        want = O.quadrant(img, q).astype(np.int64).astype(np.int32)
        assert (got[f"arr_{q}"] == want).all(), (tune, q)
    for i, q in enumerate((0, 2)):
        assert (got[f"arr_{4 + i}"] == O.quadrant(f, q, kind="f32")).all(), (tune, q)


CHILD_4096 = r"""
import sys
import numpy as np
import torch
import paper_1811_06378_gb300 as fht
from workloads import edges_and_lines
out = [fht.forward(torch.from_numpy(edges_and_lines(h, w, seed=h + w)).cuda(), q).cpu().numpy()
       for h, w, q in ((2500, 300, 0), (2500, 300, 1), (300, 2500, 2), (300, 2500, 3))]
np.savez(sys.argv[1], *out)
"""


@pytest.mark.parametrize("staged", ["0", "1"])
def test_final_pass_from_uint16_level_both_forms(staged, tmp_path):
    """The final pass of a 4096-row quadrant of a uint8 image runs as the
    persistent staged kernel (default) or, with FHT_STAGED=0, as the
    one-item-per-CTA kernel; both give the oracle's result bit for bit."""
    import oracle as O
    from workloads import edges_and_lines
    path = str(tmp_path / "out.npz")
    env = dict(os.environ, FHT_STAGED=staged, FHT_TUNE_FILE="none", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD_4096, path], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(path)
    for i, (h, w, q) in enumerate(((2500, 300, 0), (2500, 300, 1), (300, 2500, 2),
                                   (300, 2500, 3))):
        want = O.quadrant(edges_and_lines(h, w, seed=h + w), q)
        assert (got[f"arr_{i}"] == want.astype(np.int64).astype(np.int32)).all(), (staged, q)


CHILD_NVTX = r"""
import sys
import numpy as np
import torch
import paper_1811_06378_gb300 as fht
from workloads import edges_and_lines
img = edges_and_lines(700, 500, seed=5)
x = torch.from_numpy(img).cuda()
out = [fht.full_quadrants(x).cpu().numpy(), fht.forward_range(x, 1, 3, 300).cpu().numpy()]
g = torch.from_numpy(np.random.default_rng(6).standard_normal(fht.full_shape(700, 500))
                     .astype(np.float32)).cuda()
out.append(fht.adjoint(g, 700, 500).cpu().numpy())
out.append(g.cpu().numpy())
assert fht.device_status() == fht.FHT_OK
np.savez(sys.argv[1], *out)
"""


def test_nvtx_ranges_leave_results_unchanged(tmp_path):
    """FHT_NVTX=1 wraps every launch in an NVTX range (for nsys and ncu
    --nvtx filtering); the results stay the oracle's."""
    import oracle as O
    from workloads import edges_and_lines
    path = str(tmp_path / "out.npz")
    env = dict(os.environ, FHT_NVTX="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD_NVTX, path], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(path)
    img = edges_and_lines(700, 500, seed=5)
    assert (got["arr_0"] == O.full(img).astype(np.int64).astype(np.int32)).all()
    assert (got["arr_1"] == O.range_slice(img, 1, 3, 300)).all()
    assert np.array_equal(got["arr_2"], O.adjoint_full(got["arr_3"], 700, 500, "f32"))
