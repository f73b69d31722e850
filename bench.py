"""Benchmark: DF Louvain update time per batch on a GB300.

Workload: R-MAT graph (a=0.57, b=0.19, c=0.19) with 2^22 vertices and
33,554,432 undirected unit-weight edges (self-loops and duplicates removed,
seeded vertex permutation), static Louvain once, then consecutive random
batch updates of 1e-3 x |E| edges (80% insertions between uniform vertex
pairs, 20% deletions of uniform existing edges), each one step =
dfl_apply_batch + dfl_update(DF).  Inputs of every step are already on the
device when the timed region starts; between timed steps L2 is flushed.

Prints one JSON line (see the keys below).  --impl reference times the CPU
oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

SCALE = 22
EDGES = 33_554_432
GRAPH_SEED = 2
BATCH_SEED = 200
BATCH_FRAC = 1e-3
SIZES = [1e-7, 1e-6, 1e-5, 1e-4, 1e-3]
METRIC = "ms/batch DF update (R-MAT 2^22, 1e-3|E| batches)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--scale", type=int, default=SCALE)
    p.add_argument("--edges", type=int, default=EDGES)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-sizes", action="store_true")
    p.add_argument("--profile-only", action="store_true",
                   help="a few steps for a profiler (no clocks, no CPU baseline)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(args, rank=0):
    g = synth.rmat(args.scale, args.edges, GRAPH_SEED)
    off, idx, w = synth.to_csr(g)
    return g, off, idx, w


def batch_size(g, frac):
    return max(1, int(round(frac * g.m)))


def run_oracle(g, off, idx, w, sizes_steps, seed):
    """Oracle timing: static once (not timed), then DF batches (timed each)."""
    import oracle
    oracle.build()
    o = oracle.Oracle(g.n, off, idx, w)
    t0 = time.perf_counter()
    o.static()
    static_s = time.perf_counter() - t0
    stream = synth.BatchStream(g, seed)
    times = []
    for size in sizes_steps:
        d, i = stream.next(size)
        t = time.perf_counter()
        rc = o.apply_batch(d, i)
        o.update(oracle.DF)
        times.append(time.perf_counter() - t)
        assert rc == 0
    return o, static_s, times


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g, off, idx, w = make_workload(args)
    size = batch_size(g, BATCH_FRAC)
    o, static_s, times = run_oracle(g, off, idx, w, [size] * (args.warmup + args.steps), BATCH_SEED)
    timed = times[args.warmup:]
    ms = 1e3 * sum(timed) / len(timed)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale} |E|={g.m} DF batches of {size} (1e-3|E|)",
                   "batch_edges": size, "static_s": static_s, "l2": "not applicable (CPU)"},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"{args.warmup}+{args.steps} DF batches of {size} edges after "
                                   f"static Louvain (static {static_s:.1f} s untimed)"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_2404_19634_gb300 as dfl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dfl.build()
    g, off, idx, w = make_workload(args, rank)
    size = batch_size(g, BATCH_FRAC)
    # a side stream: the library replays its captured local-moving iteration
    # (a CUDA graph) only on a non-default stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    opt = dfl.default_options(flags=dfl.FLAG_PROFILE)
    h = dfl.Dfl(g.n, off, idx, w, options=opt, stream=stream)
    torch.cuda.synchronize()
    # static Louvain (the paper's comparator), timed on its own
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.static()
    e1.record(stream)
    torch.cuda.synchronize()
    static_ms = e0.elapsed_time(e1)
    static_stats = h.stats()
    static_prof = h.profile(reset=True)

    bstream = synth.BatchStream(g, BATCH_SEED)
    nsteps = args.warmup + args.steps
    batches = [bstream.next(size) for _ in range(nsteps)]
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    dbatches = [(to_dev(d), to_dev(i)) for d, i in batches]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    torch.cuda.synchronize()

    def step(k):
        d, i = dbatches[k]
        h.apply_batch(d, i)
        h.update(dfl.DF)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    h.profile(reset=True)
    launches0 = h.stats()["kernel_launches"]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    clocks = Clocks(local)
    with clocks:
        for k in range(args.warmup, nsteps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(k)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    launches = h.stats()["kernel_launches"] - launches0
    prof = h.profile(reset=True)
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = total_ms / (args.steps * world)

    # roofline of the local-moving decide kernels (the hot loop)
    peak, peak_kind = peaks()
    mv = prof["move"]
    achieved = (mv["bytes"] / 1e9) / (mv["ms"] / 1e3) if mv["ms"] > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": "local-move decide",
                "peak_kind": peak_kind, "bytes_per_step": mv["bytes"] / args.steps,
                "kernel_ms_per_step": mv["ms"] / args.steps,
                "launches_per_step": mv["launches"] / args.steps}
    kernel_share = {k: round(v["ms"] / args.steps, 4) for k, v in prof.items()}

    extra = {}
    if not args.profile_only and not args.no_sizes and rank == 0:
        # per batch size (consecutive on the evolving graph), and static/ND on the
        # same graph for the paper's comparison
        for frac in SIZES:
            sz = batch_size(g, frac)
            ms = []
            for _ in range(3):
                d, i = bstream.next(sz)
                dd, di = to_dev(d), to_dev(i)
                torch.cuda.synchronize()
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.apply_batch(dd, di)
                h.update(dfl.DF)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            extra[f"{frac:g}"] = round(statistics.median(ms), 4)
        d, i = bstream.next(size)
        dd, di = to_dev(d), to_dev(i)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.apply_batch(dd, di)
        h.update(dfl.ND)
        b.record(stream)
        torch.cuda.synchronize()
        extra["nd_1e-3"] = round(a.elapsed_time(b), 4)
        nd_prof = h.profile(reset=True)["move"]
        extra["nd_move_gbs"] = round((nd_prof["bytes"] / 1e9) / (nd_prof["ms"] / 1e3), 1) if nd_prof["ms"] else None
    static_move = static_prof["move"]
    static_gbs = (static_move["bytes"] / 1e9) / (static_move["ms"] / 1e3) if static_move["ms"] else None

    # end to end through the public API with host buffers: pinned host batch in,
    # membership (4 bytes per vertex) out, every step
    e2e = None
    if not args.profile_only:
        out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        e2e_batches = [bstream.next(size) for _ in range(args.steps)]
        pin_d = [torch.from_numpy(np.ascontiguousarray(d).view(np.int32)).pin_memory() for d, _ in e2e_batches]
        pin_i = [torch.from_numpy(np.ascontiguousarray(i).view(np.int32)).pin_memory() for _, i in e2e_batches]
        h.set_options(dfl.default_options())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            h.apply_batch(pin_d[k], pin_i[k])
            h.update(dfl.DF)
            h.membership(out)
        torch.cuda.synchronize()
        e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 12 * size,
               "d2h_bytes_per_step": 4 * g.n}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.profile_only:
        # the oracle on the same graph and batch stream: static untimed, then
        # DF batches of the same size
        nb = 8
        o, static_s, times = run_oracle(g, off, idx, w, [size] * nb, BATCH_SEED)
        cpu = {"value": 1e3 * statistics.mean(times[2:]), "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"{nb - 2} DF batches of {size} edges (after 2 untimed) on the same "
                         f"graph, static Louvain untimed ({static_s:.1f} s)",
               "static_s": static_s}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale} |E|={g.m} DF batches of {size} (1e-3|E|)",
                       "graph": "R-MAT a=.57 b=.19 c=.19, 2^22 vertices, 33,554,432 edges, unit weights",
                       "batch_edges": size, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "static_ms": round(static_ms, 3), "static_passes": static_stats["iterations"],
                       "static_move_gbs": round(static_gbs, 1) if static_gbs else None,
                       "df_ms_by_batch_fraction": extra or None,
                       "step_ms_median": round(statistics.median(step_ms), 4),
                       "graph_captures": h.stats()["graph_captures"],
                       "graph_capture_ms": round(h.stats()["graph_capture_ms"], 2),
                       "kernel_ms_per_step": kernel_share},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
