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

The persistent batched kernel has its own plan (fht_batched_tuning): units
of work per claimed item, tile widths, CTAs per SM (its register budget) and,
per image size 2^K, how many of the K levels the first of its two passes
fuses ("stages per CTA"). `tune_batched` searches it coordinate by
coordinate on a batch of uint8 edge maps with sides log-uniform in
[64, 1024] (the benchmark's batch), objective the sum of the median times of
the batch's uint8 -> int32 forward and its FP32 adjoint, every candidate's
results checked bit for bit against the default plan's.

The result is a JSON table {"table": {K: {max_levels, tile_u8, tile_wide,
us, default_us}}, "batched": {"tuning": {...}, "us", "default_us"}, ...};
`load` applies one to the library (fht_set_tuning, fht_set_batched_tuning),
and the package loads its own table (tuning_gb300.json) when it is imported,
or the one named by FHT_TUNE_FILE (FHT_TUNE_FILE=none loads nothing).

    python -m paper_1811_06378_gb300.autotune --out table.json --sizes 7-13
    python -m paper_1811_06378_gb300.autotune --out table.json --batched
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


def _batch_workload(count: int, seed: int, device):
    """`count` uint8 edge maps (8% edges) with sides log-uniform in [64, 1024],
    their FP32 quadrant gradients, and the calls that time them."""
    import numpy as np
    rng = np.random.default_rng(seed)
    shapes = [(int(h), int(w)) for h, w in
              np.round(np.exp(rng.uniform(np.log(64), np.log(1024), size=(count, 2))))]
    g = torch.Generator(device=device).manual_seed(seed)
    imgs = [(torch.rand(sh, generator=g, device=device) < 0.08).to(torch.uint8) for sh in shapes]
    grads = [torch.randn(fht.query_shape(h, w, fht.Q0), generator=g, device=device)
             for h, w in shapes]
    return shapes, imgs, grads


def _time_batch(shapes, imgs, grads, reps, warmup, device):
    """(us, outputs) of the batch's uint8 forward plus its FP32 adjoint
    under the batched tuning in force."""
    plan = fht.BatchPlan(shapes, fht.Q0)
    ws = plan.workspace(device)
    outs = [torch.empty(sh, dtype=torch.int32, device=device) for sh in plan.out_shapes]
    fplan = fht.BatchPlan(shapes, fht.Q0, torch.float32, torch.float32)
    fws = fplan.workspace(device)
    gouts = [torch.empty(sh, dtype=torch.float32, device=device) for sh in shapes]
    t = _median_us(lambda: plan.forward(imgs, outs, ws), reps, warmup)
    t += _median_us(lambda: fplan.adjoint(grads, gouts, fws), reps, warmup)
    if plan.status(ws) != 0 or fplan.status(fws) != 0:
        raise RuntimeError("a batched wait ran out of its budget")
    return t, outs, gouts


def tune_batched(count: int = 512, seed: int = 3, reps: int = 10, warmup: int = 3,
                 device="cuda", log=None) -> dict:
    """Coordinate search of the batched plan; leaves the library set to the
    best tuning found and returns the JSON-ready result."""
    device = torch.device(device)
    shapes, imgs, grads = _batch_workload(count, seed, device)
    ks = sorted({max(0, (max(h, 1) - 1).bit_length()) for h, _ in shapes})
    fht.set_batched_tuning(None)
    best = fht.get_batched_tuning()
    default_t, ref_o, ref_g = _time_batch(shapes, imgs, grads, reps, warmup, device)
    best_t = default_t
    if log:
        log(f"batched default {best}: {default_t:.1f} us")
    coords = [("ctas_per_sm", [2, 3]), ("units_per_item", [1, 2, 4, 8, 16]),
              ("tile_u8", [1, 2, 3]), ("tile_wide", [1, 2, 3])]
    coords += [(("first_levels", K), list(range(K - 6, 7))) for K in ks if 7 <= K <= 12]
    tried = []
    for key, values in coords:
        for v in values:
            cand = {**best, "first_levels": dict(best["first_levels"])}
            if isinstance(key, tuple):
                cand["first_levels"][key[1]] = v
            else:
                cand[key] = v
            if cand == best:
                continue
            fht.set_batched_tuning(None)
            fht.set_batched_tuning(cand)
            t, o, g = _time_batch(shapes, imgs, grads, reps, warmup, device)
            same = all(torch.equal(a, b) for a, b in zip(o, ref_o)) and \
                all(torch.equal(a, b) for a, b in zip(g, ref_g))
            if not same:
                raise RuntimeError(f"batched tuning {cand} changed the results")
            tried.append([json.dumps(cand, sort_keys=True), t])
            if log:
                log(f"batched {key}={v}: {t:.1f} us")
            if t < best_t:
                best_t, best = t, cand
        torch.cuda.empty_cache()
    fht.set_batched_tuning(None)
    fht.set_batched_tuning(best)
    return {"tuning": {**best, "first_levels": {str(k): v for k, v in best["first_levels"].items()}},
            "us": best_t, "default_us": default_t, "images": count, "seed": seed,
            "objective": "sum of median times (us) of the batch's uint8->int32 forward "
                         "and FP32 adjoint (Q0), sides log-uniform in [64, 1024]",
            "candidates": tried}


def load(path_or_result) -> dict:
    """Apply a table (a JSON path or `tune`'s result) to the library."""
    if isinstance(path_or_result, (str, os.PathLike)):
        return fht.load_tuning(os.fspath(path_or_result))
    for k, e in path_or_result["table"].items():
        fht.set_tuning(int(k), int(e["max_levels"]), int(e["tile_u8"]), int(e["tile_wide"]))
    if "batched" in path_or_result:   # replaces the batched tuning in force
        fht.set_batched_tuning(None)
        fht.set_batched_tuning(path_or_result["batched"]["tuning"])
    return path_or_result


def _parse_ks(spec: str):
    lo, _, hi = spec.partition("-")
    return range(int(lo), int(hi or lo) + 1)


def main():
    ap = argparse.ArgumentParser(description="autotune the fused passes per quadrant size")
    ap.add_argument("--out", required=True)
    ap.add_argument("--sizes", default="7-13", help="range of K (n = 2^K), e.g. 7-13")
    ap.add_argument("--reps", type=int, default=15)
    ap.add_argument("--batched", action="store_true",
                    help="tune the batched plan only and merge it into --out (kept "
                         "per-size table, if the file exists)")
    args = ap.parse_args()
    if args.batched:
        res = {}
        if os.path.exists(args.out):
            with open(args.out) as f:
                res = json.load(f)
        res["batched"] = tune_batched(log=print)
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
        b = res["batched"]
        print(f"batched: {b['tuning']}: {b['us']:.1f} us (default {b['default_us']:.1f} us)")
        return
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
