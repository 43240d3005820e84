"""The boundary is a C ABI: include/fht.h compiles as strict C99 and a plain C
program linked against libfht.so calls the host-side entry points (geometry,
slope ranges, the shear range, a Hough point's segment, tuning, status
strings) and gets the oracle's answers and the documented errors. No GPU."""

import os
import shutil
import subprocess

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fht.h"

int main(void) {
    int r = 0, c = 0, q = 0, t = 0, lo[4], hi[4];
    double spl = 0.0;
    fht_quadrant sq = FHT_Q0;
    int n = 0, r0 = 0, c0 = 0, r1 = 0, c1 = 0;
    fht_tuning tu;
    if (fht_full_shape(2048, 2048, &r, &c) != FHT_OK) return 1;
    printf("full %d %d\n", r, c);
    if (fht_query_shape(300, 129, FHT_Q2, &r, &c) != FHT_OK) return 1;
    printf("quadrant %d %d\n", r, c);
    if (fht_full_row_to_quadrant(16, 16, 31, &q, &t) != FHT_OK) return 1;
    printf("row %d %d\n", q, t);
    if (fht_angle_to_slopes(-15.0, 15.0, 2048, 2048, lo, hi) != FHT_OK) return 1;
    printf("slopes %d %d %d %d %d %d %d %d\n", lo[0], hi[0], lo[1], hi[1], lo[2], hi[2],
           lo[3], hi[3]);
    if (fht_shear_range(-30.0, 10.0, 256, 256, &sq, &spl, &r, &c) != FHT_OK) return 1;
    printf("shear %d %.12f %d %d\n", (int)sq, spl, r, c);
    if (fht_segment(16, 32, FHT_LAYOUT_QUADRANT, FHT_Q0, 15, 40, 0, &n, &r0, &c0, &r1, &c1)
        != FHT_OK)
        return 1;
    printf("segment %d %d %d %d %d\n", n, r0, c0, r1, c1);
    if (fht_get_tuning(12, &tu) != FHT_OK) return 1;
    printf("tuning %d\n", tu.max_levels);
    tu.max_levels = 3;   /* out of range */
    printf("bad_tuning %d\n", (int)fht_set_tuning(12, &tu));
    printf("bad_shape %d\n", (int)fht_full_shape(0, 8, &r, &c));
    printf("status %s|%s\n", fht_status_string(FHT_OK), fht_status_string(FHT_EINVAL));
    return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import __graft_entry__
    lib = __graft_entry__._builder().build()
    d = tmp_path_factory.mktemp("cabi")
    src, exe = d / "t.c", d / "t"
    src.write_text(PROGRAM)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", os.path.dirname(lib), "-lfht",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    return dict(line.split(" ", 1) for line in out.stdout.strip().splitlines())


def test_geometry_from_c(program):
    assert program["full"] == "%d %d" % O.full_geometry(2048, 2048)
    assert program["quadrant"] == "%d %d" % O.quadrant_geometry(300, 129, 2)
    assert program["row"] == "%d %d" % O.full_row_map(16, 16)[31]


def test_ranges_from_c(program):
    lo, hi = O.angle_to_slopes(-15.0, 15.0, 2048, 2048)
    assert program["slopes"] == " ".join(str(v) for pair in zip(lo, hi) for v in pair)
    q, spl, t_lo, t_hi = O.shear_range(-30.0, 10.0, 256, 256)
    got = program["shear"].split()
    assert (int(got[0]), int(got[2]), int(got[3])) == (q, t_lo, t_hi)
    assert abs(float(got[1]) - spl) < 1e-12


def test_segment_tuning_and_errors_from_c(program):
    count, (r0, c0), (r1, c1) = O.point_segment(16, 32, 0, 15, 40)
    assert program["segment"] == f"{count} {r0} {c0} {r1} {c1}"
    assert program["tuning"] in ("4", "5", "6")
    assert program["bad_tuning"] == "1" and program["bad_shape"] == "1"
    ok, einval = program["status"].split("|")
    assert ok and einval and ok != einval
