"""Benchmark: DF Louvain update time per batch on a GB300.

Workload: R-MAT graph (a=0.57, b=0.19, c=0.19) with 2^22 vertices and
33,554,432 undirected unit-weight edges (self-loops and duplicates removed,
seeded vertex permutation), static Louvain once, then consecutive random
batch updates of 1e-3 x |E| edges (80% insertions between uniform vertex
pairs, 20% deletions of uniform existing edges), each one step = one
dfl_step call (dfl_apply_batch + dfl_update(DF), the update queued behind
the apply; the line's config also gives the same step as two calls).  Inputs of every step are already on the
device when the timed region starts; between timed steps L2 is flushed.

Prints one JSON line (see the keys below).  --impl reference times the CPU
oracle on the same workload instead.

--serve measures the serving form instead: 8 resident R-MAT graphs (2^18 to
2^23 vertices, edge factor 8) receive update requests as a Poisson stream of
2000 requests/s with batch sizes log-uniform in [10, 1e6] edges (80%
insertions, 20% deletions of existing edges), served three ways on fresh
copies of the same graphs: one request at a time (serial DF), concurrently
per graph without coalescing, and concurrently with coalescing.

--group measures the batched form instead: 64 planted-partition graphs
(10^4 to 10^6 vertices, log-uniform; 20 to 2000 blocks; mixing 0.1 to 0.5;
weights 1 to 16; 8 edges per vertex), each step one batch of 1e-4 x |E| per
graph (80% insertions with weights 1 to 16, 20% deletions), applied and
updated with DF for all graphs by one group handle, against the same
batches through one handle per graph, one graph after another.

--temporal measures DF on the temporal stream instead (2M vertices, 30M
interactions, base = the first 90%, sliding-window batches).

By default (one GPU, not --profile-only) the line also carries the group,
serving and temporal measurements as the sub-objects "group", "serve" and
"temporal" (each with its own clock record, end-to-end figure and
comparison with the serial baseline); their inputs are generated in spawned
worker processes while the DF steps run.  --no-extras leaves them out.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
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
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the decide
# kernels of one decide phase (one sub-step) of the default workload (R-MAT
# 2^22, 1e-3|E| batches), from single-pass ncu captures of the timed DF steps
# divided by their sub-steps: caches flushed before each launch (cold) and
# kept (warm).  They belong to the kernel sources whose hash is recorded;
# with other sources, or another workload, the line reports null.
DECIDE_TRAFFIC = {"sources_sha256": "49747fe3a5d5d7e0e78d8e35e7e6966bf97eedeb5f2ae2c3f18c4c55ae4207ab",
                  "cold": 53_582_293, "warm": 21_757_973,
                  "profile": "profiles/decide_traffic_rmat22_df.md"}
SIZES = [1e-7, 1e-6, 1e-5, 1e-4, 1e-3]
METRIC = "ms/batch DF update (R-MAT 2^22, 1e-3|E| batches)"
SERVE_SCALES = [18, 19, 19, 20, 21, 22, 22, 23]
SERVE_RATE = 2000.0
SERVE_SIZES = (10, 1_000_000)
SERVE_METRIC = "served updates/s with p50/p99 latency (8 resident R-MAT graphs, Poisson 2000 req/s)"
GROUP_GRAPHS = 64
GROUP_SEED = 4
GROUP_METRIC = "ms per step: DF update of 64 graphs, each with a 1e-4|E| batch (batched group launch)"


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
    p.add_argument("--serve", action="store_true", help="measure the serving form")
    p.add_argument("--serve-seconds", type=float, default=0.5,
                   help="length of the Poisson arrival window")
    p.add_argument("--group", action="store_true", help="measure the batched multi-graph form")
    p.add_argument("--aux", action="store_true",
                   help="measure what reusing K and Sigma saves (Section 4.2) for ND, DS and DF")
    p.add_argument("--temporal", action="store_true",
                   help="measure DF on the temporal stream (sliding-window batches)")
    p.add_argument("--launch", default="auto", choices=["auto", "host", "graph", "persistent"],
                   help="how a local-moving iteration is launched: the library's choice (default: "
                        "graph replay, host launches for updates below 256 batch edges), kernels "
                        "from the host (DFL_FLAG_NO_GRAPH), always a replayed CUDA graph "
                        "(DFL_FLAG_GRAPH) or one cooperative kernel (DFL_FLAG_PERSISTENT)")
    p.add_argument("--no-extras", action="store_true",
                   help="leave the group, serving and temporal sub-objects out of the default line")
    p.add_argument("--group-graphs", type=int, default=GROUP_GRAPHS)
    p.add_argument("--group-max-n", type=float, default=1e6)
    return p.parse_args()


LAUNCH_DESC = {"auto": "per-bin kernels, graph replay (host launches below 256 batch edges)",
               "host": "per-bin kernels launched from the host", "graph": "per-bin kernels, graph replay",
               "persistent": "one cooperative kernel per iteration"}


def whole_job_ms(total_ms: float, steps: int, world: int, device=None) -> float:
    """ms per batch of the whole job: every rank ran `steps` batches of its
    own replica; the job took as long as the slowest rank (max over ranks,
    on `device` for NCCL, on the CPU for gloo)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms / (steps * world)


def launch_flag(dfl, args):
    return {"auto": 0, "host": dfl.FLAG_NO_GRAPH, "graph": dfl.FLAG_GRAPH,
            "persistent": dfl.FLAG_PERSISTENT}[args.launch]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C/C++ source without comments, trailing blanks and empty lines (string
    and character literals kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            while i < n and text[i] != "\n":
                i += 1
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (ln.rstrip() for ln in "".join(out).split("\n"))
    return "\n".join(ln for ln in lines if ln)


def kernel_sources_sha() -> str:
    """sha256 over the code of the library's CUDA sources (file names and
    contents without comments and empty lines: a capture stays valid across
    comment edits, not across code changes)."""
    d = os.path.join(ROOT, "paper_2404_19634_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh")):
            h.update(name.encode())
            with open(os.path.join(d, name), encoding="utf-8") as f:
                h.update(_code_only(f.read()).encode())
    return h.hexdigest()


def host_cpu() -> dict:
    """The host CPU model (lscpu) and its core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model or platform.processor() or platform.machine(), "host_cores": os.cpu_count()}


def _visible_device(gpu_index: int) -> str:
    """The NVML name of CUDA device `gpu_index`: its entry of
    CUDA_VISIBLE_DEVICES (an index or a GPU-/MIG- UUID), else the index."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    if vis:
        ent = [x.strip() for x in vis.split(",") if x.strip()]
        if gpu_index < len(ent):
            return ent[gpu_index]
    return str(gpu_index)


class NvmlReader:
    """Read-only NVML queries of one GPU through ctypes and the driver's
    libnvidia-ml: the current and maximum SM clock, the power draw and the
    active clock-event reasons.  Raises OSError where NVML is unavailable."""

    CLOCK_SM = 1  # nvmlClockType_t NVML_CLOCK_SM

    def __init__(self, gpu_index: int):
        import ctypes
        self.ct = ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError as e:
            raise OSError(f"libnvidia-ml: {e}") from None
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.lib = lib
        self.dev = ctypes.c_void_p()
        key = _visible_device(gpu_index)
        if key.startswith(("GPU-", "MIG-")):
            rc = lib.nvmlDeviceGetHandleByUUID(key.encode(), ctypes.byref(self.dev))
        elif key.isdigit():
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(int(key)), ctypes.byref(self.dev))
        else:
            rc = -1
        count = ctypes.c_uint(0)
        if rc != 0 and lib.nvmlDeviceGetCount_v2(ctypes.byref(count)) == 0 and count.value == 1:
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(0), ctypes.byref(self.dev))  # the only GPU
        if rc != 0:
            lib.nvmlShutdown()
            raise OSError(f"no NVML handle for device {key!r}")
        # the reasons query was renamed in later NVML versions; either returns the same bits
        self._reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        ok = lib.nvmlDeviceGetMaxClockInfo(self.dev, self.CLOCK_SM, ctypes.byref(mx)) == 0
        self.max_mhz = float(mx.value) if ok else None

    def sample(self):
        """(SM MHz, power W or None, reason bits) now, or None."""
        ct, lib = self.ct, self.lib
        clk, bits, mw = ct.c_uint(0), ct.c_ulonglong(0), ct.c_uint(0)
        if lib.nvmlDeviceGetClockInfo(self.dev, self.CLOCK_SM, ct.byref(clk)) != 0:
            return None
        if self._reasons(self.dev, ct.byref(bits)) != 0:
            return None
        pw = mw.value / 1000.0 if lib.nvmlDeviceGetPowerUsage(self.dev, ct.byref(mw)) == 0 else None
        return float(clk.value), pw, int(bits.value)

    def close(self):
        self.lib.nvmlShutdown()


class Clocks:
    """Samples the SM clock, power draw and clock-event reasons of one GPU
    while the timed steps run: in process through NVML every `period`
    seconds (one sample on entry, then from a thread, and one on exit), or, where
    NVML does not load, with nvidia-smi every 50 ms (entry waits for its
    first line, so it is sampling when the timed steps start)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits and the names reported for them
    REASON_BITS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
                   ("hw_thermal_slowdown", 0x40), ("hw_power_brake_slowdown", 0x80))

    def __init__(self, gpu_index: int, reader=None, period: float = 2e-3):
        self.gpu = gpu_index
        self.reader = reader
        self._own = False
        self.period = period
        self.proc = None
        self.lines = []
        self.samples = []  # NVML: (MHz, W or None, bits)
        self.source = None
        self._stop = threading.Event()
        self.t = None

    def __enter__(self):
        if self.reader is None:
            try:
                self.reader = NvmlReader(self.gpu)
                self._own = True
            except Exception:  # no NVML here: nvidia-smi below
                self.reader = None
        self._stop.clear()
        if self.reader is not None:
            self.source = "nvml"
            self._take()
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self._first = threading.Event()
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self._first.wait(5.0)
        except OSError:
            self.proc = None
        return self

    def _take(self):
        try:
            s = self.reader.sample()
        except Exception:  # a failed read costs a sample, never the run
            return
        if s is not None:
            self.samples.append(s)

    def _poll(self):
        while not self._stop.wait(self.period):
            self._take()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self._first.set()
        self._first.set()

    def __exit__(self, *a):
        if self.source == "nvml":
            self._stop.set()
            self.t.join(timeout=5)
            self._take()
            if self._own:
                try:
                    self.reader.close()
                except Exception:
                    pass
        elif self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, pw, mx, reasons = [], [], None, set()
        if self.source == "nvml":
            mx = self.reader.max_mhz
            for mhz, w, bits in self.samples:
                sm.append(mhz)
                if w is not None:
                    pw.append(w)
                reasons.update(nm for nm, b in self.REASON_BITS if bits & b)
        else:
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
                try:
                    pw.append(float(f[3]))
                except ValueError:
                    pass
                for k, nm in enumerate(names):
                    if f[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w": round(statistics.median(pw), 1) if pw else None, "source": self.source}


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
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, **host_cpu(), "kind": "oracle",
                         "sample": f"{args.warmup}+{args.steps} DF batches of {size} edges after "
                                   f"static Louvain (static {static_s:.1f} s untimed)",
                         "threads": "1 core used of the host's"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _temporal_inputs(_=None):
    """The temporal stream and its base graph (worker process)."""
    t0 = time.perf_counter()
    src, dst = synth.temporal_pa_stream_vec(TEMPORAL_N, TEMPORAL_STEPS, 0.3, 3)
    base_end = TEMPORAL_STEPS * 9 // 10
    g = synth.temporal_edges(src[:base_end], dst[:base_end], TEMPORAL_N)
    return src, dst, g, synth.to_csr(g), time.perf_counter() - t0


def _group_graph(args):
    k, count, n_hi = args
    n, blocks, mu, seed = synth.planted_group_params(count, 1e4, n_hi, GROUP_SEED)[k]
    g = synth.planted_partition(n, blocks, mu, 16.0, 16, seed)
    return g, (g.n, *synth.to_csr(g)), {"n": n, "blocks": blocks, "mu": round(mu, 4)}


def _serve_graph(k):
    g = synth.rmat(SERVE_SCALES[k], 8 << SERVE_SCALES[k], 300 + k)
    return g, (g.n, *synth.to_csr(g))


def start_inputs(pool, args) -> dict:
    """Submit the inputs of the group, serving and temporal measurements to
    `pool` (spawned workers), the largest first."""
    t0 = time.perf_counter()
    order = sorted(range(len(SERVE_SCALES)), key=lambda k: -SERVE_SCALES[k])
    serve = {k: pool.submit(_serve_graph, k) for k in order}
    temporal = pool.submit(_temporal_inputs)
    group = [pool.submit(_group_graph, (k, args.group_graphs, args.group_max_n)) for k in range(args.group_graphs)]
    return {"t0": t0, "serve": serve, "temporal": temporal, "group": group}


def roofline_record(mv: dict, steps: int, peak: float, peak_kind: str, traffic_ok: bool) -> dict:
    """The roofline of the local-moving decide phase.  One "launch" is one
    sub-step's decide phase -- its concurrent decide kernels from the first
    start to the last end, two CUDA events on the handle's stream -- and
    `mv` is dfl_profile's DFL_PROF_MOVE class over `steps` DF steps: the
    phases counted, their algorithmic bytes (counted on the device) and
    their milliseconds.  DRAM traffic comes from the ncu capture recorded
    in DECIDE_TRAFFIC while `traffic_ok` (the same kernel sources, the same
    workload), else null.  Every figure follows from the record's own
    fields: achieved = bytes_per_launch / ms_per_launch, frac = achieved /
    peak, traffic_ratio = traffic / bytes_per_launch."""
    nl = max(1, mv["launches"])
    bytes_launch = mv["bytes"] / nl
    ms_launch = mv["ms"] / nl
    achieved = (bytes_launch / 1e9) / (ms_launch / 1e3) if ms_launch > 0 else 0.0
    cold = DECIDE_TRAFFIC["cold"] if traffic_ok else None
    warm = DECIDE_TRAFFIC["warm"] if traffic_ok else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": cold,
            "kernel": "local-move decide phase (one sub-step: the concurrent decide kernels of its "
                      "four degree bins)",
            "timing": f"CUDA events around each decide phase, in {steps} further DF steps of the "
                      "same size (the timed steps carry no profiling events)",
            "peak_kind": peak_kind, "bytes_per_launch": bytes_launch, "ms_per_launch": ms_launch,
            "launches_per_step": mv["launches"] / steps,
            "bytes_per_step": mv["bytes"] / steps, "kernel_ms_per_step": mv["ms"] / steps,
            "traffic_warm": warm,
            "traffic_ratio": (cold / bytes_launch) if cold else None,
            "traffic_ratio_warm": (warm / bytes_launch) if warm else None,
            "traffic_source": (f"ncu capture of these kernel sources ({DECIDE_TRAFFIC['profile']}), "
                               "bytes per decide phase; not measured in this run") if traffic_ok else
                              "null: no capture of these kernel sources on this workload"}


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_2404_19634_gb300 as dfl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    extras = world == 1 and not args.profile_only and not args.no_extras
    pool, futs = None, None
    if extras:  # before any CUDA call: the workers are spawned, not forked
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        pool = ProcessPoolExecutor(max_workers=max(1, min(14, (os.cpu_count() or 2) - 2)),
                                   mp_context=mp.get_context("spawn"))
        futs = start_inputs(pool, args)
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dfl.build()
    g, off, idx, w = make_workload(args, rank)
    size = batch_size(g, BATCH_FRAC)
    # a side stream (graph replay, when chosen, needs a non-default stream)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pflag = launch_flag(dfl, args)
    # the static run times only its decide phase (two events per sub-step)
    opt = dfl.default_options(flags=dfl.FLAG_PROFILE_MOVE | pflag)
    h = dfl.Dfl(g.n, off, idx, w, options=opt, stream=stream)
    torch.cuda.synchronize()
    # static Louvain (the paper's comparator), timed on its own; a first,
    # untimed run makes the handle's buffers, so the timed one excludes
    # allocation as the paper's timings do (the result is the same)
    h.static()
    torch.cuda.synchronize()
    if futs:
        # the input workers occupy most host cores; every timed region waits
        # for them (a host starved of cores delays the launches and control
        # reads the GPU waits on)
        from concurrent.futures import wait
        wait([futs["temporal"], *futs["group"], *futs["serve"].values()])
        futs["ready_s"] = time.perf_counter() - futs["t0"]  # all inputs generated
    h.profile(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("static")
    e0.record(stream)
    h.static()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    static_ms = e0.elapsed_time(e1)
    static_stats = h.stats()
    static_prof = h.profile(reset=True)

    bstream = synth.BatchStream(g, BATCH_SEED)
    nsteps = args.warmup + args.steps
    # the timed steps carry no profiling events; the roofline's decide-phase
    # durations come from as many further steps with them (below)
    h.set_options(dfl.default_options(flags=pflag))
    batches = [bstream.next(size) for _ in range(nsteps + args.steps)]
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    dbatches = [(to_dev(d), to_dev(i)) for d, i in batches]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    torch.cuda.synchronize()

    def step(k):  # dfl_step: the batch apply with the DF update queued behind it
        d, i = dbatches[k]
        h.step(d, i, dfl.DF)

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
        torch.cuda.nvtx.range_push("df_steps")  # lets a profiler select the timed steps
        for k in range(args.warmup, nsteps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(k)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    launches = h.stats()["kernel_launches"] - launches0
    value = whole_job_ms(sum(step_ms), args.steps, world, dev)
    # the decide phase of the same kind of steps, timed on the device (two
    # events around each sub-step's concurrent decide kernels)
    h.set_options(dfl.default_options(flags=dfl.FLAG_PROFILE_MOVE | pflag))
    h.profile(reset=True)
    for k in range(nsteps, nsteps + args.steps):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    prof = h.profile(reset=True)
    h.set_options(dfl.default_options(flags=pflag))
    ms_per_step = value * world  # the slowest rank's ms per step

    # roofline of the local-moving decide phase (the hot loop)
    peak, peak_kind = peaks()
    default_workload = args.scale == SCALE and args.edges == EDGES
    roofline = roofline_record(prof["move"], args.steps, peak, peak_kind,
                               default_workload and DECIDE_TRAFFIC["sources_sha256"] == kernel_sources_sha())
    kernel_share = None

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
                h.step(dd, di, dfl.DF)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            extra[f"{frac:g}"] = round(statistics.median(ms), 4)
        # the same step as two calls (dfl_apply_batch, then dfl_update): one
        # host wait more
        ms = []
        for _ in range(5):
            d, i = bstream.next(size)
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
        extra["two_calls_1e-3"] = round(statistics.median(ms), 4)
        # an untimed ND update first (its iteration graph is captured once),
        # then one timed plainly and one with its decide phases timed alone
        for profiled in (None, False, True):
            d, i = bstream.next(size)
            dd, di = to_dev(d), to_dev(i)
            h.set_options(dfl.default_options(flags=pflag | (dfl.FLAG_PROFILE_MOVE if profiled else 0)))
            torch.cuda.synchronize()
            flush.zero_()
            h.profile(reset=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.step(dd, di, dfl.ND)
            b.record(stream)
            torch.cuda.synchronize()
            if profiled is not None:
                extra["nd_1e-3_profiled" if profiled else "nd_1e-3"] = round(a.elapsed_time(b), 4)
        nd_prof = h.profile(reset=True)["move"]
        h.set_options(dfl.default_options(flags=pflag))
        extra["nd_move_gbs"] = round((nd_prof["bytes"] / 1e9) / (nd_prof["ms"] / 1e3), 1) if nd_prof["ms"] else None
        extra["nd_move_frac"] = round(extra["nd_move_gbs"] / peak, 4) if extra["nd_move_gbs"] else None
    static_move = static_prof["move"]
    static_gbs = (static_move["bytes"] / 1e9) / (static_move["ms"] / 1e3) if static_move["ms"] else None
    # every kernel class timed (more events, so separate from the timed steps)
    if rank == 0:
        h.set_options(dfl.default_options(flags=dfl.FLAG_PROFILE | pflag))
        h.profile(reset=True)
        nprof = 5
        for _ in range(nprof):
            d, i = bstream.next(size)
            h.step(to_dev(d), to_dev(i), dfl.DF)
        torch.cuda.synchronize()
        kernel_share = {k: round(v["ms"] / nprof, 4) for k, v in h.profile(reset=True).items()}

    # end to end through the public API with host buffers: pinned host batch in,
    # membership (4 bytes per vertex) out, every step
    e2e = None
    if not args.profile_only:
        out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        e2e_batches = [bstream.next(size) for _ in range(args.steps)]
        pin_d = [torch.from_numpy(np.ascontiguousarray(d).view(np.int32)).pin_memory() for d, _ in e2e_batches]
        pin_i = [torch.from_numpy(np.ascontiguousarray(i).view(np.int32)).pin_memory() for _, i in e2e_batches]
        h.set_options(dfl.default_options(flags=pflag))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            h.step(pin_d[k], pin_i[k], dfl.DF)
            h.membership(out)
        torch.cuda.synchronize()
        e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 12 * size,
               "d2h_bytes_per_step": 4 * g.n}
    substeps = dfl.default_options().substeps
    h.close()
    del flush, dbatches

    subs = {}
    if extras:
        tg = time.perf_counter()
        src, dst, tgraph, tcsr, t_gen = futs["temporal"].result()
        subs["temporal"] = temporal_measure(args, src, dst, tgraph, tcsr, t_gen)
        del src, dst, tgraph, tcsr
        made = [f.result() for f in futs["group"]]
        subs["group"] = group_measure(args, made, futs["ready_s"])
        del made
        served = [futs["serve"][k].result() for k in range(len(SERVE_SCALES))]
        subs["serve"] = serve_measure(args, served, futs["ready_s"])
        del served
        pool.shutdown()
        subs["extras_wall_s"] = round(time.perf_counter() - tg, 1)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.profile_only:
        # the oracle on the same graph and batch stream: static untimed, then
        # DF batches of the same size
        nb = 8
        o, static_s, times = run_oracle(g, off, idx, w, [size] * nb, BATCH_SEED)
        cpu = {"value": 1e3 * statistics.mean(times[2:]), "unit": "ms", "cores": 1, **host_cpu(),
               "threads": "1 core used of the host's", "kind": "oracle",
               "sample": f"{nb - 2} DF batches of {size} edges (after 2 untimed) on the same "
                         f"graph, static Louvain untimed ({static_s:.1f} s)",
               "static_s": static_s}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale} |E|={g.m} DF batches of {size} (1e-3|E|)",
                       "graph": f"R-MAT a=.57 b=.19 c=.19, 2^{args.scale} vertices, {g.m:,} edges, unit weights",
                       "batch_edges": size, "l2": "flushed between timed steps (256 MB write)",
                       "step_call": "dfl_step (the batch apply with the DF update queued behind it, one call)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "iteration_launch": LAUNCH_DESC[args.launch],
                       "substeps": substeps,
                       "schedule": f"{substeps} synchronous hash-class sub-steps per local-moving iteration "
                                   "(a class decides against the state the previous class left)",
                       "static_ms": round(static_ms, 3), "static_note": "second run on the handle (buffers made)",
                       "static_passes": static_stats["iterations"],
                       "static_move_gbs": round(static_gbs, 1) if static_gbs else None,
                       "static_move_frac": round(static_gbs / peak, 4) if static_gbs else None,
                       "df_ms_by_batch_fraction": extra or None,
                       "step_ms_median": round(statistics.median(step_ms), 4),
                       "kernel_ms_per_step_profiled": kernel_share},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def group_measure(args, made, gen_s) -> dict:
    """The batched form (one group handle) against one handle per graph."""
    import torch

    import paper_2404_19634_gb300 as dfl

    G = len(made)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    dfl.build()
    graphs = [g for g, _, _ in made]
    csrs = [c for _, c, _ in made]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    nsteps = args.warmup + args.steps
    bstreams = [synth.BatchStream(g, 500 + k) for k, g in enumerate(graphs)]
    bsize = [max(1, int(round(1e-4 * g.m))) for g in graphs]
    batches = [[bs.next(sz, w_max=16) for bs, sz in zip(bstreams, bsize)] for _ in range(nsteps + 2)]
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)

    # one group handle: batches of all graphs in one device array each
    pflag = launch_flag(dfl, args)
    grp = dfl.DflGroup(csrs, options=dfl.default_options(flags=pflag), stream=stream)
    grp.static()  # untimed: makes the buffers (the timed runs exclude allocation)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as static_clocks:
        e0.record(stream)
        grp.static()
        e1.record(stream)
        torch.cuda.synchronize()
    group_static_ms = e0.elapsed_time(e1)
    static_passes = [grp.graph_stats(g)["passes"] for g in range(G)]
    static_final = [grp.graph_modularity(g)[1:] for g in range(G)]
    gbatches = []
    for step in batches:
        d = np.concatenate([b[0] for b in step])
        i = np.concatenate([b[1] for b in step])
        doff = np.concatenate([[0], np.cumsum([b[0].shape[0] for b in step])]).astype(np.uint64)
        ioff = np.concatenate([[0], np.cumsum([b[1].shape[0] for b in step])]).astype(np.uint64)
        gbatches.append(((to_dev(d), doff), (to_dev(i), ioff)))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def time_steps(run_step, first, count):
        ms = []
        for k in range(first, first + count):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run_step(k)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return ms

    def group_step(k):
        grp.apply_batches(*gbatches[k])
        grp.update(dfl.DF)

    # the autotuner picks bin limits and block size for the first step's frontier
    grp.apply_batches(*gbatches[0])
    tuning, tune_ms = grp.autotune(dfl.DF, reps=3)
    grp.update(dfl.DF)
    time_steps(group_step, 1, args.warmup)
    l0 = grp.stats()["kernel_launches"]
    with Clocks(0) as clocks:
        torch.cuda.nvtx.range_push("group_steps")
        group_ms = time_steps(group_step, 1 + args.warmup, args.steps)
        torch.cuda.nvtx.range_pop()
    group_launches = grp.stats()["kernel_launches"] - l0
    group_final = [grp.graph_modularity(g)[1:] for g in range(G)]
    group_memb = [grp.graph_membership(g).copy() for g in range(G)]
    passes = [grp.graph_stats(g)["passes"] for g in range(G)]
    # a step in which graphs aggregate: ND over every vertex with the next batch
    k_nd = nsteps + 1
    grp.apply_batches(*gbatches[k_nd])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    grp.update(dfl.ND)
    b.record(stream)
    torch.cuda.synchronize()
    group_nd_ms = a.elapsed_time(b)
    nd_passes = [grp.graph_stats(g)["passes"] for g in range(G)]
    nd_final = [grp.graph_modularity(g)[1:] for g in range(G)]

    # the same graphs, batches and tuning, one handle per graph, one after another
    hs = [dfl.Dfl(n, off, idx, w, options=dfl.default_options(flags=pflag), stream=stream)
          for n, off, idx, w in csrs]
    for hh in hs:
        hh.set_tuning(**tuning)
        hh.static()  # untimed: makes the buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for hh in hs:
        hh.static()
    torch.cuda.synchronize()
    serial_static_ms = 1e3 * (time.perf_counter() - t0)
    serial_static_final = [hh.modularity()[1:] for hh in hs]
    sbatches = [[(to_dev(d), to_dev(i)) for d, i in step] for step in batches]

    def serial_step(k):
        for hh, (d, i) in zip(hs, sbatches[k]):
            hh.step(d, i, dfl.DF)

    serial_step(0)
    time_steps(serial_step, 1, args.warmup)
    with Clocks(0) as serial_clocks:
        serial_ms = time_steps(serial_step, 1 + args.warmup, args.steps)
    serial_final = [hh.modularity()[1:] for hh in hs]
    identical = serial_final == group_final
    same_membership = all(np.array_equal(group_memb[g], hs[g].membership()) for g in range(G))
    for hh, (d, i) in zip(hs, sbatches[k_nd]):
        hh.apply_batch(d, i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for hh in hs:
        hh.update(dfl.ND)
    torch.cuda.synchronize()
    serial_nd_ms = 1e3 * (time.perf_counter() - t0)
    serial_nd_final = [hh.modularity()[1:] for hh in hs]
    for hh in hs:
        hh.close()

    # end to end: host batches in, every graph's membership out, each step
    e2e = None
    if not args.profile_only:
        host = []
        for _ in range(args.steps):
            step = [bs.next(sz, w_max=16) for bs, sz in zip(bstreams, bsize)]
            host.append(([b[0] for b in step], [b[1] for b in step]))
        out = [np.zeros(g.n, np.uint32) for g in graphs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, i in host:
            grp.apply_batches(d, i)
            grp.update(dfl.DF)
            for g in range(G):
                grp.graph_membership(g, out[g])
        torch.cuda.synchronize()
        e2e = {"value": 1e3 * (time.perf_counter() - t0) / args.steps, "unit": "ms",
               "h2d_bytes_per_step": int(np.mean([12 * sum(x.shape[0] for x in d + i) for d, i in host])),
               "d2h_bytes_per_step": 4 * sum(g.n for g in graphs)}
    grp.close()
    del flush, gbatches, sbatches
    value = statistics.mean(group_ms)
    return {
        "metric": GROUP_METRIC, "value": value, "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{G} planted-partition graphs, n log-uniform [1e4, {args.group_max_n:g}], "
                               "blocks [20, 2000], mu [0.1, 0.5], weights 1-16, 8 edges per vertex; "
                               "DF batches of 1e-4|E| per graph (80/20)",
                   "vertices": sum(g.n for g in graphs), "edges": sum(g.m for g in graphs),
                   "batch_edges_per_step": sum(d.shape[0] + i.shape[0] for d, i in batches[0]),
                   "l2": "flushed between timed steps (256 MB write)", "generation_s": round(gen_s, 1),
                   "iteration_launch": LAUNCH_DESC["host" if args.launch == "auto" else args.launch],
                   "passes_min_max": [min(passes), max(passes)]},
        "tuning": tuning, "autotune_decide_ms": round(tune_ms, 4),
        "serial_ms_per_step": statistics.mean(serial_ms),
        "speedup_vs_serial": statistics.mean(serial_ms) / value,
        "identical_to_serial": bool(identical and same_membership),
        "serial_tuning": "the group's autotuned tuning on every handle",
        "aggregating_steps": {
            "static": {"group_ms": round(group_static_ms, 2), "serial_ms": round(serial_static_ms, 2),
                       "passes_min_max": [min(static_passes), max(static_passes)],
                       "identical_to_serial": static_final == serial_static_final,
                       "clocks": static_clocks.summary()},
            "nd_update": {"group_ms": round(group_nd_ms, 2), "serial_ms": round(serial_nd_ms, 2),
                          "passes_min_max": [min(nd_passes), max(nd_passes)],
                          "identical_to_serial": nd_final == serial_nd_final}},
        "e2e": e2e,
        "gpu_launches": int(group_launches),
        "clocks": clocks.summary(),
        "serial_clocks": serial_clocks.summary(),
    }


def group_arm(args):
    t_gen = time.perf_counter()
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        made = pool.map(_group_graph, [(k, args.group_graphs, args.group_max_n) for k in range(args.group_graphs)])
    print(json.dumps(group_measure(args, made, time.perf_counter() - t_gen)), flush=True)


AUX_METRIC = "mean speedup of DF from reusing K and Sigma instead of recomputing them (Section 4.2)"
# The same run records, per mode and batch size, the fraction of vertices
# the first pass marked and processed: the affected-set comparison of DS and
# DF.


def aux_arm(args):
    """Each update with the auxiliary information reused (the default) and
    with K, 2m and Sigma recomputed from scratch first (DFL_FLAG_RECOMPUTE_AUX),
    alternating on the evolving graph: ND, DS and DF at every batch size."""
    import torch

    import paper_2404_19634_gb300 as dfl

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    dfl.build()
    g, off, idx, w = make_workload(args)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pflag = launch_flag(dfl, args)
    h = dfl.Dfl(g.n, off, idx, w, options=dfl.default_options(flags=pflag), stream=stream)
    h.static()
    bstream = synth.BatchStream(g, BATCH_SEED + 7)
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    reps = max(3, min(args.steps, 5))
    table = {}
    launches = 0
    for frac in SIZES:
        size = batch_size(g, frac)
        row = {}
        for name, mode in (("ND", dfl.ND), ("DS", dfl.DS), ("DF", dfl.DF)):
            ms = {False: [], True: []}
            ever, initial = [], []
            for _ in range(reps):
                for recompute in (False, True):
                    h.set_options(dfl.default_options(
                        flags=pflag | (dfl.FLAG_RECOMPUTE_AUX if recompute else 0)))
                    d, i = bstream.next(size)
                    dd, di = to_dev(d), to_dev(i)
                    l0 = h.stats()["kernel_launches"]
                    torch.cuda.synchronize()
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    h.apply_batch(dd, di)
                    h.update(mode)
                    b.record(stream)
                    torch.cuda.synchronize()
                    st = h.stats()
                    launches += st["kernel_launches"] - l0
                    ms[recompute].append(a.elapsed_time(b))
                    if not recompute:
                        ever.append(st["affected_ever"] / g.n)
                        initial.append(st["affected_initial"] / g.n)
            reuse, scratch = statistics.median(ms[False]), statistics.median(ms[True])
            # vertices processed by the first pass (the ever-affected set) and
            # marked initially, as fractions of |V| (Section 5.2's explanation)
            row[name] = {"reuse_ms": round(reuse, 4), "recompute_ms": round(scratch, 4),
                         "speedup": round(scratch / reuse, 3),
                         "affected_initial_frac": float(f"{statistics.median(initial):.4g}"),
                         "affected_ever_frac": float(f"{statistics.median(ever):.4g}")}
        table[f"{frac:g}"] = row
    h.close()
    mean = {m: round(statistics.mean(table[f"{f:g}"][m]["speedup"] for f in SIZES), 3) for m in ("ND", "DS", "DF")}
    line = {
        "metric": AUX_METRIC, "value": mean["DF"], "unit": "x", "n_gpus": 1, "steps": reps,
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale} |E|={g.m}, batches of 1e-7..1e-3|E| (80/20), "
                               f"{reps} updates per mode, size and variant (median)",
                   "l2": "flushed before each update (256 MB write)",
                   "iteration_launch": LAUNCH_DESC[args.launch],
                   "mean_speedup": mean, "by_batch_fraction": table,
                   "paper_context": "64-core CPU, graphs of Table 2: ND 11.8x, DS 2.9x, DF 48.5x"},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)


TEMPORAL_N = 2_000_000
TEMPORAL_STEPS = 30_000_000
TEMPORAL_METRIC = "ms/batch DF update, temporal PA stream (2M vertices, 30M interactions), sliding window"


def temporal_measure(args, src, dst, g, csr, gen_s) -> dict:
    """The temporal workload: base = the first 90% of the stream (weight =
    multiplicity, tau_agg = 1), then consecutive sliding-window batches of
    1e-5 and 1e-4 x interactions (insert the next ones, expire as many of the
    oldest), each applied and updated with DF; then the same from pinned
    host buffers with the membership read back (end to end)."""
    import torch

    import paper_2404_19634_gb300 as dfl

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    dfl.build()
    off, idx, w = csr
    base_end = TEMPORAL_STEPS * 9 // 10
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pflag = launch_flag(dfl, args)
    h = dfl.Dfl(g.n, off, idx, w, options=dfl.default_options(tau_agg=1.0, flags=pflag), stream=stream)
    h.static()  # untimed: makes the buffers (the timed run excludes allocation)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.static()
    e1.record(stream)
    torch.cuda.synchronize()
    static_ms = e0.elapsed_time(e1)
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    start, end = 0, base_end
    by_size = {}
    launches = 0
    clocks = Clocks(0)
    for frac in (1e-5, 1e-4):
        size = int(round(frac * TEMPORAL_STEPS))
        batches = []
        for _ in range(args.warmup + args.steps):
            batches.append(synth.window_batch(src, dst, start, end, size))
            start += size
            end += size
        dbatches = [(to_dev(d), to_dev(i)) for d, i in batches]
        ms = []
        for k, (d, i) in enumerate(dbatches):
            timed = k >= args.warmup
            if k == args.warmup:
                l0 = h.stats()["kernel_launches"]
                if frac == 1e-4:
                    clocks.__enter__()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.step(d, i, dfl.DF)
            b.record(stream)
            torch.cuda.synchronize()
            if timed:
                ms.append(a.elapsed_time(b))
        launches += h.stats()["kernel_launches"] - l0
        by_size[f"{frac:g}"] = {"batch_interactions": size, "ms_mean": round(statistics.mean(ms), 4),
                                "ms_median": round(statistics.median(ms), 4)}
    clocks.__exit__(None, None, None)
    # end to end at 1e-4: pinned host window batches in, membership out
    size = int(round(1e-4 * TEMPORAL_STEPS))
    host = []
    for _ in range(args.steps):
        d, i = synth.window_batch(src, dst, start, end, size)
        start += size
        end += size
        host.append((torch.from_numpy(np.ascontiguousarray(d).view(np.int32)).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(i).view(np.int32)).pin_memory()))
    out = torch.empty(g.n, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d, i in host:
        h.step(d, i, dfl.DF)
        h.membership(out)
    torch.cuda.synchronize()
    e2e = {"value": 1e3 * (time.perf_counter() - t0) / args.steps, "unit": "ms",
           "h2d_bytes_per_step": int(np.mean([12 * (d.shape[0] + i.shape[0]) for d, i in host])),
           "d2h_bytes_per_step": 4 * g.n}
    h.close()
    del flush
    value = by_size["0.0001"]["ms_mean"]
    return {
        "metric": TEMPORAL_METRIC, "value": value, "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"temporal PA stream, {TEMPORAL_N:,} vertices, {TEMPORAL_STEPS:,} interactions "
                               "(30% repeats), base = first 90%, window batches of 1e-4 x interactions",
                   "base_edges": g.m, "tau_agg": 1.0, "generation_s": round(gen_s, 1),
                   "l2": "flushed between timed steps (256 MB write)",
                   "iteration_launch": LAUNCH_DESC[args.launch],
                   "static_ms": round(static_ms, 2), "df_by_batch_fraction": by_size,
                   "df_vs_static_1e-4": round(static_ms / value, 1)},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
    }


def temporal_arm(args):
    print(json.dumps(temporal_measure(args, *_temporal_inputs())), flush=True)


def serve_measure(args, made, gen_s) -> dict:
    """The serving form: serial per-request DF, overlapped per graph without
    coalescing (results identical to serial), and overlapped with coalescing."""
    import torch

    import paper_2404_19634_gb300 as dfl
    from paper_2404_19634_gb300 import serve

    torch.cuda.set_device(0)
    dfl.build()
    t_gen = time.perf_counter()
    graphs = [g for g, _ in made]
    csrs = [c for _, c in made]
    pools = [synth.EdgePool(g, 400 + k) for k, g in enumerate(graphs)]
    warm = [(0.0, g, 1000) for _ in range(max(1, args.warmup)) for g in range(len(graphs))]
    sched = synth.poisson_requests(len(graphs), SERVE_RATE, args.serve_seconds, *SERVE_SIZES, seed=500)
    reqs = serve.make_requests(pools, warm + sched)
    wreq, treq = reqs[:len(warm)], reqs[len(warm):]
    gen_s += time.perf_counter() - t_gen
    edges = [int(r.dels.shape[0] + r.ins.shape[0]) for r in treq]

    def run(mode):
        srv = serve.Server.from_graphs(csrs, mem_cap=150 << 30)
        srv.replay(wreq, [(r.graph, [r.rid]) for r in wreq])
        torch.cuda.synchronize()
        l0 = sum(h.stats()["kernel_launches"] for h in srv.handles)
        with Clocks(0) as clk:
            if mode == "serial":
                res = srv.serve_serial(treq)
            else:
                res = srv.serve(treq, coalesce=(mode == "coalesce"))
            torch.cuda.synchronize()
        launches = sum(h.stats()["kernel_launches"] for h in srv.handles) - l0
        final = [h.modularity() for h in srv.handles]
        srv.close()
        out = res.summary()
        out["gpu_launches"] = launches
        out["clocks"] = clk.summary()
        return res, out, final

    ser, ser_sum, ser_final = run("serial")
    ovl, ovl_sum, ovl_final = run("overlap")
    coa, coa_sum, coa_final = run("coalesce")
    ovl_sum["identical_to_serial"] = all((a.num, a.den) == (b.num, b.den)
                                         for a, b in zip(ovl.records, ser.records))
    ovl_sum["final_q_minus_serial"] = [round(a[0] - b[0], 9) for a, b in zip(ovl_final, ser_final)]
    coa_sum["final_q_minus_serial"] = [round(a[0] - b[0], 9) for a, b in zip(coa_final, ser_final)]
    coa_sum["max_requests_per_update"] = max(len(ids) for _, ids in coa.groups)
    mean_edges = float(np.mean(edges)) if edges else 0.0

    def vs(x):
        return {"updates_per_s": x["requests_per_s"] / ser_sum["requests_per_s"],
                "p50": ser_sum["p50_ms"] / x["p50_ms"], "p99": ser_sum["p99_ms"] / x["p99_ms"]}

    return {
        "metric": SERVE_METRIC, "value": coa_sum["requests_per_s"], "unit": "updates/s",
        "n_gpus": 1, "steps": len(treq), "warmup": len(wreq),
        "ms_per_step": 1e3 * coa_sum["wall_s"] / max(1, len(treq)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "8 R-MAT graphs (a=.57 b=.19 c=.19) of 2^18,2^19,2^19,2^20,2^21,2^22,"
                               "2^22,2^23 vertices, 8 edges per vertex; Poisson requests",
                   "rate_per_s": SERVE_RATE, "arrival_window_s": args.serve_seconds,
                   "window_note": "shorter than the 10 s the workload names, so that generating the "
                                  "batches fits a bench run",
                   "batch_edges": "log-uniform [10, 1e6], 80% insertions / 20% deletions",
                   "requests": len(treq), "mean_batch_edges": round(mean_edges, 1),
                   "warmup": f"{len(wreq)} requests of 1000 edges, served serially, untimed",
                   "mem_cap_bytes": 150 << 30, "generation_s": round(gen_s, 1),
                   "l2": "not flushed (the 8 graphs total 1.5e8 edges, far above L2)"},
        "serial": ser_sum, "overlap": ovl_sum, "coalesce": coa_sum,
        "speedup_vs_serial": {"overlap_identical_results": vs(ovl_sum), "coalesce": vs(coa_sum)},
        "e2e": {"value": coa_sum["requests_per_s"], "unit": "updates/s",
                "h2d_bytes_per_step": 12 * mean_edges, "d2h_bytes_per_step": 32},
        "gpu_launches": coa_sum["gpu_launches"],
        "clocks": coa_sum["clocks"],
    }


def serve_arm(args):
    t_gen = time.perf_counter()
    # the graphs are generated in parallel host processes (spawned, so that
    # no child inherits a CUDA context)
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(SERVE_SCALES), os.cpu_count() or 1)) as pool:
        made = pool.map(_serve_graph, range(len(SERVE_SCALES)))
    print(json.dumps(serve_measure(args, made, time.perf_counter() - t_gen)), flush=True)


def main():
    args = parse()
    if args.serve:
        serve_arm(args)
        return
    if args.group:
        group_arm(args)
        return
    if args.temporal:
        temporal_arm(args)
        return
    if args.aux:
        aux_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
