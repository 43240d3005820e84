#!/usr/bin/env python3
"""Benchmark of the GB300 fast Hough transform hot path.

One step = every row of the hot path on one resident 4096 x 4096 uint8 edge
map (5% Bernoulli edge pixels + 4 rasterised lines, seed 4096 + rank):

  1. fht_full_quadrants   four quadrants, int32, written into the
                          16381 x 8192 full Hough image (Section 3.3)
  2. fhtshift             standalone regrouping of that image (Section 5)
  3. fht_forward_range    slopes of [-15, 15] degrees (Q0 t<=1097, Q1 1<=t<=1097)
  4. fht_adjoint          FP32 back-projection of a resident 16381 x 8192 FP32
                          gradient onto the image (the transform's transpose)

value = input megapixels per second over the whole step (all ranks).
Timing: CUDA events on the stream the kernels run on, L2 flushed (a 512 MiB
write) before every timed step, W >= 3 warm-up steps. The timed region
replays the step captured as one CUDA graph (the four quadrants of the
full-layout calls on four streams); the per-kernel launch times behind the
roofline come from a second region of the same K steps launched call by call,
every launch timed alone with the library's per-launch CUDA events. The
roofline is that of the unit of work the dominant kernel serves (one
quadrant transform or adjoint): its algorithmic bytes (input read once,
output written once) over the summed time of that unit's kernels. Per-row
times, the plain single-quadrant forward (the headline FHT at 4096^2 int32)
and the batched path are reported under "rows".

Rows also include the batched path: 512 uint8 edge maps with sides
log-uniform in [64, 1024] in one persistent launch, against one fht_forward
call per image, and its FP32 adjoint the same way; the [-15, 15] degree range
as one sheared quadrant (Section 4); the maximum along the patterns of Q0;
the per-row maxima of the full image; one gradient step of the 64 x 1024^2
reconstruction.

Multi-GPU: replicas only (each rank transforms its own image, no collective
on the data path); value sums all ranks, time is the max over ranks.

cpu_baseline: the CPU oracle (plain C butterfly + numpy assembly, as it
stands) on one step of the same workload, its independent units (quadrants,
range quadrants, quadrant adjoints) on a process per host core (up to the
number of units), and again on one core; nproc and the CPU model recorded.

--impl reference times the same oracle harness on the host cores, each step
the same rows on a power-of-two crop of the image sized so that the whole run
takes about 90 s.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("FHT Mpix/s and HBM GB/s (% of 8 TB/s) at 4096² int32; "
          "batched & adjoint vs plain")
UNIT = "Mpix/s"
SIDE = 4096
RANGE_DEG = (-15.0, 15.0)
FLUSH_BYTES = 512 << 20
NOMINAL_HBM_GBS = 8000.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--side", type=int, default=SIDE,
                    help="image side (default 4096; smaller only for profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rows", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, fl in enumerate(flags)
                          if fl.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def kernel_source_hash() -> str:
    """Hash of the library's CUDA and host sources (csrc/; the public header
    holds declarations and comments only); a committed ncu summary is only
    used while the code it measured is unchanged."""
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_1811_06378_gb300", "csrc", "*")))
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel: str, side: int):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum +
    dram__bytes_write.sum) from profiles/ncu_traffic.json, or None when no
    capture of this kernel and workload exists for the current sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash() or rec.get("side") != side:
        return None
    k = rec.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_launch"])


def reduce_max_ms(total_ms: float, world: int, device) -> float:
    """The slowest rank's timed total (replicas run concurrently; the job takes
    as long as its slowest rank)."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(world: int, pixels_per_rank_step: int, ms_per_step: float) -> float:
    """Input megapixels per second summed over all ranks (weak scaling: every
    rank transforms its own image each step)."""
    return world * pixels_per_rank_step / 1e6 / (ms_per_step / 1e3)


def bind_near_gpu(index: int):
    """Keep this process on the CPU cores local to GPU `index` (its sysfs
    local_cpulist), so that the pinned host buffers of the end-to-end region
    and the copies through them stay on the GPU's NUMA node. Best effort:
    returns the cores used, or None when the topology is not readable."""
    try:
        import torch
        p = torch.cuda.get_device_properties(index)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
            return sorted(cpus)
    except Exception:
        return None
    return None


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


# ---------------------------------------------------------------- oracle step
#
# The CPU baseline runs the oracle as it stands (test infrastructure, never
# tuned for this), on the step's independent units: the four quadrants of the
# full image, the range quadrants and the four quadrant adjoints, each one
# call of an existing oracle function. With one worker they run one after
# another; with several, in a process pool (spawned: this process has
# already initialised CUDA). The image, the gradient and the results live in
# shared memory, so no array is pickled; the main process assembles the full
# image (rows by the oracle's row map), applies fhtshift and sums the
# adjoint's quadrant parts in the order Q0, Q1, Q2, Q3.

def _shm_array(name, shape, dtype):
    from multiprocessing import shared_memory
    import numpy as np
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf)


def _oracle_unit(args):
    """One unit of the step by the oracle, in a worker (or in-process)."""
    import numpy as np
    import oracle as O
    kind, q, side, names, lo, hi = args
    h = w = side
    R, Wf = O.full_geometry(h, w)
    shm_i, img = _shm_array(names["img"], (h, w), np.uint8)
    try:
        if kind == "full":
            # quadrant q of the full layout (a square power-of-two image: the
            # quadrant's own width is the full layout's) into its full rows
            shm_f, F = _shm_array(names["F"], (R, Wf), np.int64)
            H = O.quadrant(img, q)
            for r, (qq, t) in enumerate(O.full_row_map(h, w)):
                if qq == q:
                    F[r] = H[t]
            del F
            shm_f.close()
        elif kind == "range":
            O.range_slice(img, q, lo, hi)
        else:
            shm_g, G = _shm_array(names["G"], (R, Wf), np.float32)
            shm_p, parts = _shm_array(names["parts"], (4, h, w), np.float32)
            rows = [(r, t) for r, (qq, t) in enumerate(O.full_row_map(h, w)) if qq == q]
            n, W = O.quadrant_geometry(h, w, q)
            Gq = np.zeros((n, W), dtype=np.float32)
            for r, t in rows:
                Gq[t] = G[r]
            parts[q] = O.adjoint_quadrant(Gq, h, w, q, "f32")
            del G, parts
            shm_g.close()
            shm_p.close()
    finally:
        del img
        shm_i.close()
    return kind, q


class OracleStep:
    """The step's rows by the oracle on a side x side edge map (side a power
    of two), on `workers` processes."""

    def __init__(self, side: int, workers: int):
        import numpy as np
        from multiprocessing import shared_memory
        import oracle as O
        from workloads import edges_and_lines
        self.side, self.workers = side, workers
        h = w = side
        R, Wf = O.full_geometry(h, w)
        self.R, self.Wf = R, Wf
        lo, hi = O.angle_to_slopes(*RANGE_DEG, h, w)
        self.ranges = [(q, lo[q], hi[q]) for q in range(4) if lo[q] >= 0]
        self.shm = {}
        for key, nbytes in (("img", h * w), ("F", R * Wf * 8), ("G", R * Wf * 4),
                            ("parts", 4 * h * w * 4)):
            self.shm[key] = shared_memory.SharedMemory(create=True, size=nbytes)
        self.names = {k: v.name for k, v in self.shm.items()}
        img = np.ndarray((h, w), np.uint8, buffer=self.shm["img"].buf)
        img[:] = edges_and_lines(h, w, p_edge=0.05, n_lines=4, seed=4096)
        G = np.ndarray((R, Wf), np.float32, buffer=self.shm["G"].buf)
        G[:] = np.random.default_rng(0).standard_normal((R, Wf)).astype(np.float32)
        del img, G
        self.pool = None
        if workers > 1:
            # an executor, not a Pool: a worker that dies makes the call fail
            # instead of being restarted for ever
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            self.pool = ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
            # start every worker (interpreter, numpy, oracle library) before timing
            list(self.pool.map(_warm_worker, range(workers)))

    def units(self):
        side, names = self.side, self.names
        jobs = [("full", q, side, names, 0, 0) for q in range(4)]
        jobs += [("range", q, side, names, lo, hi) for q, lo, hi in self.ranges]
        jobs += [("adjoint", q, side, names, 0, 0) for q in range(4)]
        # the largest units first, so that the pool's tail is short
        return sorted(jobs, key=lambda j: j[0] == "range")

    def run(self):
        import numpy as np
        import oracle as O
        jobs = self.units()
        if self.pool is not None:
            list(self.pool.map(_oracle_unit, jobs))
        else:
            for j in jobs:
                _oracle_unit(j)
        F = np.ndarray((self.R, self.Wf), np.int64, buffer=self.shm["F"].buf)
        O.fhtshift_full(F, self.side, self.side)
        parts = np.ndarray((4, self.side, self.side), np.float32, buffer=self.shm["parts"].buf)
        acc = parts[0].copy()
        for q in (1, 2, 3):
            acc = (acc + parts[q]).astype(np.float32)
        del F, parts
        return acc

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()
        for v in self.shm.values():
            v.close()
            v.unlink()


def _warm_worker(_):
    import oracle as O
    O.offset(4, 1, 1)
    return os.getpid()


def host_cpu():
    """Host cores this process may use and the CPU model."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return cores, model or "unknown"


def time_oracle_step(side: int, workers: int, reps: int = 1) -> float:
    """Seconds per oracle step (median of reps) on `workers` processes."""
    st = OracleStep(side, workers)
    try:
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            st.run()
            times.append(time.perf_counter() - t0)
    finally:
        st.close()
    return statistics.median(times)


def cpu_baseline(side: int):
    cores, model = host_cpu()
    n_units = 4 + 2 + 4
    workers = max(1, min(cores, n_units))
    t_all = time_oracle_step(side, workers)
    t_one = time_oracle_step(side, 1)
    return {"value": side * side / 1e6 / t_all, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"one step (all four rows) on the same {side}x{side} edge map by the "
                      f"oracle (plain C butterfly + numpy assembly), its {n_units} independent "
                      f"units (4 full-image quadrants, 2 range quadrants, 4 adjoint quadrants) "
                      f"on {workers} worker processes: {t_all:.2f} s",
            "nproc": cores, "cpu_model": model,
            "single_core": {"value": side * side / 1e6 / t_one, "unit": UNIT, "cores": 1,
                            "seconds": t_one}}


def run_reference(args):
    ws, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores, model = host_cpu()
    workers = max(1, min(cores, 10))
    # size the per-step crop so that warm-up + timed steps stay near 90 s
    budget_s = 90.0
    t256 = time_oracle_step(256, workers)
    crop = 256
    while crop < args.side and (args.steps + args.warmup) * t256 * (2 * crop / 256) ** 2 \
            * math.log2(2 * crop) / 8 <= budget_s:
        crop *= 2
    st = OracleStep(crop, workers)
    try:
        for _ in range(args.warmup):
            st.run()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            st.run()
            times.append(time.perf_counter() - t0)
    finally:
        st.close()
    ms = 1e3 * sum(times) / len(times)
    value = crop * crop / 1e6 / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.side}x{args.side} u8 edge map (5% edges + 4 lines): "
                               "full 4-quadrant image, fhtshift, [-15,15] deg range, "
                               "FP32 full adjoint", "sample_crop": f"{crop}x{crop}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"each step = all rows on a {crop}x{crop} crop, its 10 "
                                   f"independent units on {workers} worker processes",
                         "nproc": cores, "cpu_model": model},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch
    import paper_1811_06378_gb300 as fht
    from workloads import edges_and_lines

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    near_cpus = bind_near_gpu(local)
    stream = torch.cuda.current_stream()
    S = args.side

    img_h = edges_and_lines(S, S, p_edge=0.05, n_lines=4, seed=4096 + rank)
    img = torch.from_numpy(img_h).to(dev)
    R, Wf = fht.full_shape(S, S)
    lo, hi = fht.angle_to_slopes(*RANGE_DEG, S, S)
    used = [q for q in range(4) if lo[q] >= 0]
    F = torch.empty((R, Wf), dtype=torch.int32, device=dev)
    Fs = torch.empty_like(F)
    n0, W0 = fht.query_shape(S, S, 0)
    rng_out = {q: torch.empty((hi[q] - lo[q] + 1, fht.query_shape(S, S, q)[1]),
                              dtype=torch.int32, device=dev) for q in used}
    gen = torch.Generator(device=dev).manual_seed(7 + rank)
    grad = torch.randn((R, Wf), generator=gen, device=dev, dtype=torch.float32)
    gimg = torch.empty((S, S), dtype=torch.float32, device=dev)
    # one workspace per row (the full-layout ones hold a slice per quadrant)
    ws_full = torch.empty(max(fht.workspace_size(S, S, fht.LAYOUT_FULL, 0, torch.uint8,
                                                 torch.int32), 1),
                          dtype=torch.uint8, device=dev)
    ws_rng = torch.empty(max(fht.workspace_size(S, S, fht.LAYOUT_QUADRANT, q, torch.uint8,
                                                torch.int32) for q in (0, 1)),
                         dtype=torch.uint8, device=dev)
    ws_adj = torch.empty(max(fht.workspace_size(S, S, fht.LAYOUT_FULL, 0, torch.float32,
                                                torch.float32), 1),
                         dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    H0 = torch.empty((n0, W0), dtype=torch.int32, device=dev)

    def row_full():
        fht.full_quadrants(img, out=F, workspace=ws_full)

    def row_shift():
        fht.fhtshift(F, S, S, fht.LAYOUT_FULL, out=Fs)

    def row_range():
        for q in used:
            fht.forward_range(img, q, lo[q], hi[q], out=rng_out[q], workspace=ws_rng)

    def row_adjoint():
        fht.adjoint(grad, S, S, fht.LAYOUT_FULL, out=gimg, workspace=ws_adj)

    def step():
        # the rows one after another on one stream (the full-layout calls run
        # their four quadrants concurrently inside the library). Running the
        # rows themselves on three streams as well was measured slower (1.053
        # against 1.030 ms per step): the quadrants already fill the GPU.
        row_full()
        row_shift()
        row_range()
        row_adjoint()

    def timed(fn, reps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for i in range(reps):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
            fn()
            ends[i].record(stream)
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in zip(starts, ends)]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # The step as one CUDA graph: every library call is capturable, and the
    # replay removes the host's launch gaps between the step's kernels.
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream()
    cap0 = fht.launch_count()
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream):
            step()
    torch.cuda.synchronize()
    launches_per_step = fht.launch_count() - cap0
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: K replays of the captured step
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = timed(graph.replay, args.steps)
    launches = launches_per_step * args.steps
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    # ---- per-launch kernel times (roofline): the same K steps launched call
    # by call, every launch bracketed by the library's CUDA events on its own
    # stream (the events cost a few microseconds per launch, so this region
    # is not the one `value` comes from)
    fht.profile_begin()
    prof_step_ms = timed(step, args.steps)
    prof = fht.profile_end()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None

    total_ms = reduce_max_ms(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_mpix_s(world, S * S, ms_per_step)
    prof_total_ms = sum(prof_step_ms)
    peak, peak_kind = load_peaks()
    rows = {}   # filled by the per-row section below

    # ---- roofline. The dominant kernel is the one with the largest share of
    # the profiled step. It serves a unit of the step's work -- one quadrant
    # transform, one quadrant adjoint, the range transform of one quadrant,
    # the fhtshift of the full image -- whose algorithmic bytes are fixed by
    # the transform's definition: the input read once and the output written
    # once (h*w*in_bytes + n*W*4 per quadrant; n*W*4 + h*w*4 per quadrant
    # adjoint). achieved = those bytes / the summed time of all the kernels
    # of that unit (their per-launch CUDA-event times, each launch alone).
    # The pass-counted figure (the level each launch reads as stored plus
    # the level it writes, over that launch's time) is kept beside it.
    nq, Wq = fht.query_shape(S, S, 0)   # every quadrant of the square full layout
    rng_rows = sum(t.shape[0] for t in rng_out.values())
    families = {
        "adjoint quadrant (FP32 gradient -> image gradient)": (
            lambda k: k.startswith("adjoint_fused"), 4, nq * Wq * 4 + S * S * 4),
        "forward quadrant (uint8 -> int32)": (
            lambda k: k.startswith("forward_fused") and not k.endswith("_range"), 4,
            S * S + nq * Wq * 4),
        "range quadrant (uint8 -> int32 slopes of [-15, 15] deg)": (
            lambda k: k.endswith("_range"), len(used),
            (len(used) * S * S + rng_rows * Wq * 4) / max(len(used), 1)),
        "fhtshift of the full image": (lambda k: k.startswith("fhtshift"), 1, 2 * R * Wf * 4),
    }
    steps = args.steps
    units = {}
    for fam, (match, per_step, unit_bytes) in families.items():
        ks = [k for k in prof if match(k)]
        if not ks:
            continue
        fam_ms = sum(prof[k][1] for k in ks) / steps          # per step
        unit_ms = fam_ms / per_step
        traffic_parts = [traffic_per_launch(k, S) for k in ks]
        traffic = None
        if all(t is not None for t in traffic_parts):
            traffic = sum(t * prof[k][0] / steps for t, k in zip(traffic_parts, ks)) / per_step
        units[fam] = {"kernels": ks, "units_per_step": per_step,
                      "alg_bytes_per_unit": unit_bytes, "unit_ms": unit_ms,
                      "achieved_gbs": unit_bytes / (unit_ms / 1e3) / 1e9,
                      "frac": unit_bytes / (unit_ms / 1e3) / 1e9 / peak,
                      "dram_bytes_per_unit": traffic}
    dom_name, (dom_launches, dom_ms, dom_bytes) = max(prof.items(), key=lambda kv: kv[1][1])
    dom_fam = next((f for f, v in units.items() if dom_name in v["kernels"]), None)
    avg_ms = dom_ms / max(dom_launches, 1)
    pass_bytes = dom_bytes / max(dom_launches, 1)
    pass_frac = pass_bytes / (avg_ms / 1e3) / 1e9 / peak
    if dom_fam is not None:
        u = units[dom_fam]
        achieved, frac, traffic = u["achieved_gbs"], u["frac"], u["dram_bytes_per_unit"]
        unit_note = dom_fam
    else:   # a kernel outside the step's units (not expected): its own launch
        achieved, frac, traffic = pass_bytes / (avg_ms / 1e3) / 1e9, pass_frac, None
        unit_note = "one launch (pass-counted bytes)"
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": frac, "traffic": traffic,
        "peak_kind": f"{peak_kind} copy bandwidth (burst)",
        "kernel": dom_name, "share_of_step": dom_ms / prof_total_ms,
        "unit_of_work": unit_note,
        "accounting": "algorithmic bytes of one unit (input read once, output written "
                      "once) over the summed per-launch times of that unit's kernels; "
                      "traffic = ncu DRAM read+write bytes of those kernels per unit",
        "launches_profiled": dom_launches, "avg_launch_ms": avg_ms,
        "frac_pass_counted": pass_frac, "pass_bytes_per_launch": pass_bytes,
    }
    kernels = {k: {"launches": v[0], "avg_us": 1e3 * v[1] / max(v[0], 1),
                   "pass_bytes_per_launch": v[2] / max(v[0], 1),
                   "pass_gbs": (v[2] / max(v[0], 1)) / (v[1] / max(v[0], 1) / 1e3) / 1e9,
                   "share_of_step": v[1] / prof_total_ms} for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{S}x{S} u8 edge map (5% edges + 4 lines): full "
                               "4-quadrant image, fhtshift, [-15,15] deg range, FP32 "
                               "full adjoint", "l2": "flushed before every timed step",
                   "parallelism": f"replicas x{world}",
                   "timing": "value: K replays of the step captured as one CUDA graph "
                             "(the quadrants of the full-layout calls on four streams); "
                             "roofline and kernels: a second region of the same K steps "
                             "launched call by call, every launch timed alone with "
                             "per-launch CUDA events",
                   "profiled_ms_per_step": prof_total_ms / args.steps,
                   "host_cores": (f"{len(near_cpus)} cores local to the GPU" if near_cpus
                                  else "unbound"),
                   "launches_per_step": launches_per_step,
                   "tuning": {"levels_per_pass_tile_u8_tile_wide":
                              list(fht.get_tuning(int(math.log2(fht.query_shape(S, S, 0)[0])))),
                              "batched": fht.get_batched_tuning(),
                              "table": os.environ.get("FHT_TUNE_FILE",
                                                      os.path.basename(fht.TUNING_FILE)
                                                      if os.path.exists(fht.TUNING_FILE)
                                                      else "none")}},
        "roofline": roofline,
        "gpu_launches": launches,
        "units": units,
        "kernels": kernels,
        "rows": rows,
        "clocks": clk,
    }

    # ---- end to end through the public API with host buffers. Every step
    # copies its own inputs (image, gradient) in from pinned host memory and
    # its results (full image, fhtshift image, range slices, image gradient)
    # out to pinned host memory. Three streams: host-to-device copies,
    # compute, device-to-host copies; each result's copy starts as soon as
    # its kernels are done, and the next step's inputs land in a second set of
    # device buffers while the current step computes.
    if not args.no_e2e:
        img_pin = torch.from_numpy(img_h).pin_memory()
        grad_pin = torch.empty((R, Wf), dtype=torch.float32).pin_memory()
        grad_pin.copy_(grad.cpu())
        host_out = {"F": torch.empty((R, Wf), dtype=torch.int32).pin_memory(),
                    "Fs": torch.empty((R, Wf), dtype=torch.int32).pin_memory(),
                    "g": torch.empty((S, S), dtype=torch.float32).pin_memory()}
        host_out.update({f"r{q}": torch.empty(tuple(rng_out[q].shape), dtype=torch.int32)
                         .pin_memory() for q in used})
        bufs = []
        for _ in range(2):
            bufs.append({"img": torch.empty_like(img), "grad": torch.empty_like(grad),
                         "F": torch.empty_like(F), "Fs": torch.empty_like(Fs),
                         "g": torch.empty_like(gimg),
                         **{f"r{q}": torch.empty_like(rng_out[q]) for q in used}})
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev = lambda: torch.cuda.Event()   # noqa: E731
        in_free = [None, None]    # compute of the buffer set's previous step is done
        out_free = [None, None]   # device-to-host copies of its previous step are done

        def e2e_step(i):
            b = bufs[i % 2]
            with torch.cuda.stream(s_in):
                if in_free[i % 2] is not None:
                    s_in.wait_event(in_free[i % 2])
                b["img"].copy_(img_pin, non_blocking=True)
                e_img = ev(); e_img.record(s_in)
                b["grad"].copy_(grad_pin, non_blocking=True)
                e_grad = ev(); e_grad.record(s_in)
            if out_free[i % 2] is not None:
                s_cmp.wait_event(out_free[i % 2])
            s_cmp.wait_event(e_img)
            fht.full_quadrants(b["img"], out=b["F"], workspace=ws_full, stream=s_cmp)
            e_f = ev(); e_f.record(s_cmp)
            fht.fhtshift(b["F"], S, S, fht.LAYOUT_FULL, out=b["Fs"], stream=s_cmp)
            e_fs = ev(); e_fs.record(s_cmp)
            for q in used:
                fht.forward_range(b["img"], q, lo[q], hi[q], out=b[f"r{q}"], workspace=ws_rng,
                                  stream=s_cmp)
            e_r = ev(); e_r.record(s_cmp)
            s_cmp.wait_event(e_grad)
            fht.adjoint(b["grad"], S, S, fht.LAYOUT_FULL, out=b["g"], workspace=ws_adj,
                        stream=s_cmp)
            e_g = ev(); e_g.record(s_cmp)
            in_free[i % 2] = e_g
            with torch.cuda.stream(s_out):
                s_out.wait_event(e_f)
                host_out["F"].copy_(b["F"], non_blocking=True)
                s_out.wait_event(e_fs)
                host_out["Fs"].copy_(b["Fs"], non_blocking=True)
                s_out.wait_event(e_r)
                for q in used:
                    host_out[f"r{q}"].copy_(b[f"r{q}"], non_blocking=True)
                s_out.wait_event(e_g)
                host_out["g"].copy_(b["g"], non_blocking=True)
                done = ev(); done.record(s_out)
            out_free[i % 2] = done

        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize()
        k = max(3, min(args.steps, 20))
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s_in)
        for i in range(k):
            e2e_step(i)
        t1.record(s_out)
        torch.cuda.synchronize()
        e_ms = t0.elapsed_time(t1) / k
        h2d = img.numel() + grad.numel() * 4
        d2h = sum(t.numel() * t.element_size() for t in host_out.values())
        line["e2e"] = {"value": world * S * S / 1e6 / (e_ms / 1e3), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": e_ms, "steps": k,
                       "streams": "host-to-device, compute and device-to-host copies "
                                  "on three streams, two device buffer sets"}
        del bufs

    # ---- per-row measurements (same flush discipline), after the end-to-end
    # region: their host-side loops and allocations come after its copies
    reps = max(10, min(args.steps, 50))
    if not args.no_rows:
        def row_entry(fn, alg_bytes, pixels):
            t = statistics.median(timed(fn, reps))
            return {"ms": t, "mpix_s": pixels / 1e6 / (t / 1e3),
                    "alg_gbs": alg_bytes / (t / 1e3) / 1e9,
                    "frac_of_measured_hbm": alg_bytes / (t / 1e3) / 1e9 / peak,
                    "frac_of_8tbs": alg_bytes / (t / 1e3) / 1e9 / NOMINAL_HBM_GBS}
        rows["forward_q0_int32"] = row_entry(
            lambda: fht.forward(img, 0, out=H0, workspace=ws_rng), S * S + n0 * W0 * 4, S * S)
        rows["full_quadrants_int32"] = row_entry(row_full, S * S + R * Wf * 4, S * S)
        rows["fhtshift_full_int32"] = row_entry(row_shift, 2 * R * Wf * 4, S * S)
        rows["range_pm15deg_int32"] = row_entry(
            row_range, S * S + sum(t.numel() for t in rng_out.values()) * 4, S * S)
        rows["adjoint_full_f32"] = row_entry(row_adjoint, R * Wf * 4 + S * S * 4, S * S)
        # batched: 512 uint8 edge maps, sides log-uniform in [64, 1024], each padded
        # to its own power of two, Q0 into int32 -- one persistent launch versus
        # one fht_forward call per image
        from workloads import batch_shapes, edge_batch
        shapes = batch_shapes(512, seed=3)
        bimgs = [torch.from_numpy(a).to(dev) for a in edge_batch(shapes, seed=3)]
        plan = fht.BatchPlan(shapes, 0)
        bws = plan.workspace(dev)
        bouts = [torch.empty(sh, dtype=torch.int32, device=dev) for sh in plan.out_shapes]
        bpix = sum(h * w for h, w in shapes)
        balg = bpix + sum(n * W * 4 for n, W in plan.out_shapes)
        pws = torch.empty(max(fht.workspace_size(1024, 1024, fht.LAYOUT_QUADRANT, 0,
                                                 torch.uint8, torch.int32), 1),
                          dtype=torch.uint8, device=dev)
        rows["batched_512_u8_q0"] = row_entry(lambda: plan.forward(bimgs, bouts, bws), balg, bpix)
        rows["per_image_512_u8_q0"] = row_entry(
            lambda: [fht.forward(x, 0, out=o, workspace=pws) for x, o in zip(bimgs, bouts)],
            balg, bpix)
        rows["batched_512_u8_q0"]["speedup_vs_per_image"] = (
            rows["per_image_512_u8_q0"]["ms"] / rows["batched_512_u8_q0"]["ms"])
        del bimgs, bouts, bws, plan
        # batched adjoint: FP32 gradients of the same 512 quadrants back onto
        # their images in one persistent launch, against one call per image
        fplan = fht.BatchPlan(shapes, 0, torch.float32, torch.float32)
        fws = fplan.workspace(dev)
        g512 = [torch.randn(sh, generator=gen, device=dev) for sh in fplan.out_shapes]
        gi512 = [torch.empty(sh, dtype=torch.float32, device=dev) for sh in shapes]
        badj = sum(n * W * 4 for n, W in fplan.out_shapes) + bpix * 4
        rows["batched_adjoint_512_f32_q0"] = row_entry(
            lambda: fplan.adjoint(g512, gi512, fws), badj, bpix)
        pws_f = torch.empty(max(fht.workspace_size(1024, 1024, fht.LAYOUT_QUADRANT, 0,
                                                   torch.float32, torch.float32), 1),
                            dtype=torch.uint8, device=dev)
        rows["per_image_adjoint_512_f32_q0"] = row_entry(
            lambda: [fht.adjoint(g, h, w, fht.LAYOUT_QUADRANT, 0, out=o, workspace=pws_f)
                     for (h, w), g, o in zip(shapes, g512, gi512)], badj, bpix)
        rows["batched_adjoint_512_f32_q0"]["speedup_vs_per_image"] = (
            rows["per_image_adjoint_512_f32_q0"]["ms"] / rows["batched_adjoint_512_f32_q0"]["ms"])
        del fplan, fws, g512, gi512
        # Section 4: the [-15, 15] degree range as ONE sheared quadrant (the
        # paper's shear in the first iteration), against the two pruned
        # quadrants of the range row above
        sq, spl, st0, st1 = fht.shear_range(*RANGE_DEG, S, S)
        sh_out = torch.empty((st1 - st0 + 1, fht.query_shape(S, S, sq)[1]), dtype=torch.int32,
                             device=dev)
        sh_ws = torch.empty(fht.workspace_size_sheared(S, S, sq, torch.uint8, torch.int32),
                            dtype=torch.uint8, device=dev)
        rows["sheared_range_pm15deg_int32"] = row_entry(
            lambda: fht.forward_sheared(img, sq, spl, st0, st1, out=sh_out, workspace=sh_ws),
            S * S + sh_out.numel() * 4, S * S)
        del sh_out, sh_ws
        # Section 4, both operations: the [-15, 15] degree range as ONE scaled
        # and sheared quadrant (alpha = 1/(2 tan 15 deg), spl = 1/2): every slope
        # row inside the range, angles resolved 1.87 times finer
        cq, ca, cs, c0, c1 = fht.scale_range(*RANGE_DEG, S, S)
        sc_out = torch.empty((c1 - c0 + 1, fht.scaled_shape(S, S, cq, ca)[1]),
                             dtype=torch.int32, device=dev)
        sc_ws = torch.empty(max(fht.workspace_size_scaled(S, S, cq, ca, torch.uint8,
                                                          torch.int32), 1),
                            dtype=torch.uint8, device=dev)
        rows["scaled_range_pm15deg_int32"] = row_entry(
            lambda: fht.forward_scaled(img, cq, ca, cs, c0, c1, out=sc_out, workspace=sc_ws),
            S * S + sc_out.numel() * 4, S * S)
        rows["scaled_range_pm15deg_int32"].update(
            {"alpha": ca, "spl": cs, "rows": c1 - c0 + 1, "cols": sc_out.shape[1]})
        del sc_out, sc_ws
        # other operations: the maximum along every pattern of Q0
        rows["max_q0_int32"] = row_entry(
            lambda: fht.forward_op(img, 0, fht.OP_MAX, out=H0, workspace=ws_adj),
            S * S + n0 * W0 * 4, S * S)
        # back to lines: the strongest line of every slope of the full image
        rows["row_argmax_full_int32"] = row_entry(lambda: fht.row_argmax(F), R * Wf * 4, S * S)
        # differentiable path: one gradient-descent step of the 64 x 1024^2 FP32
        # reconstruction (full-image forward + adjoint per image, plus the update)
        from workloads import ellipse_phantom
        B5, n5 = 64, 1024
        xt = torch.from_numpy(np.stack([ellipse_phantom(n5, seed=100 + i)
                                        for i in range(B5)])).to(dev)
        b5 = fht.FHTFunction.apply(xt)
        x5 = torch.zeros_like(xt)
        R5, W5 = fht.full_shape(n5, n5)

        def gd_step():
            with torch.no_grad():
                r = fht.FHTFunction.apply(x5) - b5
                g = fht.adjoint_many(r, n5, n5)
                x5.sub_(1e-6 * g)

        gd_alg = B5 * (2 * n5 * n5 * 4 + 2 * R5 * W5 * 4)
        rows["gd_step_64x1024_f32_eager"] = row_entry(gd_step, gd_alg, B5 * n5 * n5)
        # the same step replayed from a CUDA graph, as a training loop would run
        # it: its 64 images' 1024 small launches then leave no host gaps
        gd_stream = torch.cuda.Stream()
        gd_graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gd_stream):
            gd_step()
            gd_stream.synchronize()
            with torch.cuda.graph(gd_graph, stream=gd_stream):
                gd_step()
        torch.cuda.synchronize()
        rows["gd_step_64x1024_f32"] = row_entry(gd_graph.replay, gd_alg, B5 * n5 * n5)
        del xt, b5, x5, gd_graph

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(S)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
