"""Autotuner of the fused butterfly passes.

For every quadrant size n = 2^K it times each candidate tuning on the GPU --
the most levels one pass fuses (4, 5 or 6: the K levels become
ceil(K / max_levels) passes) and the tile widths in warp-widths of source
columns for first passes over uint8 images and for passes with 4-byte shared
tiles (1..3 each) -- and keeps the fastest. Every candidate computes the same
result bit for bit; only the time differs.

The objective for one K is the sum of the median CUDA-event times of the
plain quadrant calls the library's workloads are made of, on seeded n x n
inputs resident on the device: the uint8 -> int32 forward of Q0, the FP32
forward of Q0 and the FP32 adjoint of Q0.

The result is a JSON table {"table": {K: {max_levels, tile_u8, tile_wide,
us, default_us}}, ...}; `load` applies one to the library (fht_set_tuning),
and the package loads its own table (tuning_gb300.json) when it is imported,
or the one named by FHT_TUNE_FILE (FHT_TUNE_FILE=none loads nothing).

    python -m paper_1811_06378_gb300.autotune --out table.json --sizes 7-13
"""

from __future__ import annotations

import argparse
import json
import os
import statistics

import torch

import paper_1811_06378_gb300 as fht

CANDIDATES = [(L, a, b) for L in (6, 5, 4) for a in (1, 2, 3) for b in (1, 2, 3)]
DEFAULT = (6, 1, 1)


def _median_us(fn, reps: int, warmup: int) -> float:
    for _ in range(warmup):
        fn()
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for a, b in evs:
        a.record(st)
        fn()
        b.record(st)
    torch.cuda.synchronize()
    return 1e3 * statistics.median(a.elapsed_time(b) for a, b in evs)


def _workload(K: int, device):
    """The three timed calls on seeded n x n inputs (n = 2^K), each with a
    workspace sized for the tuning in force when it is built."""
    n = 1 << K
    g = torch.Generator(device=device).manual_seed(K)
    img8 = (torch.rand((n, n), generator=g, device=device) < 0.05).to(torch.uint8)
    imgf = torch.rand((n, n), generator=g, device=device)
    rows, cols = fht.query_shape(n, n, fht.Q0)
    out_i = torch.empty((rows, cols), dtype=torch.int32, device=device)
    out_f = torch.empty((rows, cols), dtype=torch.float32, device=device)
    grad = torch.randn((rows, cols), generator=g, device=device)
    gimg = torch.empty((n, n), dtype=torch.float32, device=device)

    def calls():
        ws = torch.empty(max(fht.workspace_size(n, n, fht.LAYOUT_QUADRANT, fht.Q0, torch.uint8,
                                                torch.int32),
                             fht.workspace_size(n, n, fht.LAYOUT_QUADRANT, fht.Q0,
                                                torch.float32, torch.float32), 1),
                         dtype=torch.uint8, device=device)
        return [lambda: fht.forward(img8, fht.Q0, out=out_i, workspace=ws),
                lambda: fht.forward(imgf, fht.Q0, acc=torch.float32, out=out_f, workspace=ws),
                lambda: fht.adjoint(grad, n, n, fht.LAYOUT_QUADRANT, fht.Q0, out=gimg,
                                    workspace=ws)]
    return calls


def tune(ks=range(7, 14), reps: int = 15, warmup: int = 3, device="cuda",
         candidates=CANDIDATES, log=None) -> dict:
    """Time every candidate for every K; returns the JSON-ready result and
    leaves the library set to the best tuning of each K."""
    device = torch.device(device)
    table, tried = {}, {}
    for K in ks:
        calls_for = _workload(K, device)
        times = []
        for cand in candidates:
            fht.set_tuning(K, *cand)
            calls = calls_for()
            t = sum(_median_us(c, reps, warmup) for c in calls)
            times.append((t, cand))
            if log:
                log(f"K={K} {cand}: {t:.1f} us")
        best_t, best = min(times)
        default_t = next(t for t, c in times if c == DEFAULT)
        fht.set_tuning(K, *best)
        table[str(K)] = {"max_levels": best[0], "tile_u8": best[1], "tile_wide": best[2],
                         "us": best_t, "default_us": default_t}
        tried[str(K)] = [[*c, t] for t, c in times]
        torch.cuda.empty_cache()
    return {"device": torch.cuda.get_device_name(device),
            "objective": "sum of median times (us) of the uint8->int32 forward, the FP32 "
                         "forward and the FP32 adjoint of Q0 on an n x n input, n = 2^K",
            "reps": reps, "table": table, "candidates": tried}


def load(path_or_result) -> dict:
    """Apply a table (a JSON path or `tune`'s result) to the library."""
    if isinstance(path_or_result, (str, os.PathLike)):
        return fht.load_tuning(os.fspath(path_or_result))
    for k, e in path_or_result["table"].items():
        fht.set_tuning(int(k), int(e["max_levels"]), int(e["tile_u8"]), int(e["tile_wide"]))
    return path_or_result


def _parse_ks(spec: str):
    lo, _, hi = spec.partition("-")
    return range(int(lo), int(hi or lo) + 1)


def main():
    ap = argparse.ArgumentParser(description="autotune the fused passes per quadrant size")
    ap.add_argument("--out", required=True)
    ap.add_argument("--sizes", default="7-13", help="range of K (n = 2^K), e.g. 7-13")
    ap.add_argument("--reps", type=int, default=15)
    args = ap.parse_args()
    for K in _parse_ks(args.sizes):   # time from the defaults, not a loaded table
        fht.set_tuning(K, None)
    res = tune(_parse_ks(args.sizes), reps=args.reps, log=print)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    for k, e in res["table"].items():
        print(f"K={k}: levels {e['max_levels']}, tiles {e['tile_u8']},{e['tile_wide']}: "
              f"{e['us']:.1f} us (default {e['default_us']:.1f} us)")


if __name__ == "__main__":
    main()
