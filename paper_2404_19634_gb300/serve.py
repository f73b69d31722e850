"""Continuous-batching update server for resident graphs.

Each graph stays resident on the GPU in its own handle (graph, K, Sigma and
membership), each on its own CUDA stream.  Update requests (a batch of edge
deletions and insertions for one graph) arrive over time; the server

  * admits a request when a slot and enough device memory are free (the
    memory estimate covers the batch's staging and working buffers; the cap
    defaults to 150 GB),
  * coalesces the requests that queued up for one graph while its previous
    update ran: their batches are applied in arrival order (dfl_apply_batch
    calls) and one DF update follows, as the API allows -- the last batch and
    the update as one dfl_step call,
  * runs different graphs' updates at the same time: one worker thread per
    graph drives its handle through the C ABI (ctypes releases the GIL), so
    their kernels overlap on the device,
  * optionally refreshes a graph with static Louvain after every
    `refresh_every` of its updates: DF (like DS) can miss a community that a
    long run of deletions splits or an outlier that drifts away, and a
    periodic static run -- every 1000 batches, say -- restores the quality
    (the remedy the paper proposes with its correctness argument,
    Section 7.5).

Results are deterministic: a request's result (the modularity numerator and
denominator after the update that served it, and the membership) depends only
on its graph's earlier requests and on how they were grouped, never on what
other graphs were doing -- `replay` recomputes any grouping one update at a
time for comparison.  `serve_serial` is the plain baseline: one request at a
time, in arrival order, one update per request.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import DF, Dfl, default_options


@dataclass
class Request:
    rid: int
    graph: int
    arrival: float          # seconds after the start of serving
    dels: np.ndarray        # (k, 3) uint32 rows (u, v, w)
    ins: np.ndarray


@dataclass
class Record:
    rid: int
    graph: int
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    group: int = -1         # id of the update that served the request
    num: int = 0            # modularity numerator / denominator after that update
    den: int = 0
    q: float = 0.0
    membership: object = None  # copy of C after that update (keep_membership)
    refreshed: bool = False    # static Louvain ran after that update (refresh_every)
    failed: bool = False       # its graph's worker raised before serving it

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class ServeResult:
    records: list
    groups: list = field(default_factory=list)  # per update: graph and request ids, in order
    wall: float = 0.0

    def summary(self) -> dict:
        served = [r for r in self.records if not r.failed]
        lat = np.array([r.latency for r in served]) * 1e3
        edges = sum(getattr(r, "edges", 0) for r in served)
        return {"requests": len(served), "failed": len(self.records) - len(served),
                "updates": len(self.groups),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None,
                "requests_per_s": len(served) / self.wall if self.wall else None,
                "wall_s": self.wall, "edges": edges}


def batch_bytes(req: Request) -> int:
    """Device memory a request needs while it is applied: staging copy of the
    edges, both arcs with keys and weights, and the pair table."""
    ne = int(req.dels.shape[0] + req.ins.shape[0])
    return 12 * ne + 2 * ne * (8 + 4) + 4 * 2 * ne * 40 + (1 << 16)


class Server:
    """Resident graphs plus the serving loop (see the module docstring)."""

    def __init__(self, handles, resident_bytes: int = 0, mem_cap: int = 150 << 30,
                 slots: int | None = None, keep_membership: bool = False, refresh_every: int = 0):
        """handles: one object per graph with the Dfl methods apply_batch,
        update, static, modularity and membership, each already past
        dfl_static.  refresh_every > 0: static Louvain after every that many
        updates of a graph (counted per server)."""
        self.handles = list(handles)
        self.refresh_every = int(refresh_every)
        self.updates = [0] * len(self.handles)
        self.resident = resident_bytes
        self.mem_cap = mem_cap
        self.slots = slots or len(self.handles)
        self.keep_membership = keep_membership
        self.peak = {"busy": 0, "mem": 0}

    @classmethod
    def from_graphs(cls, graphs, options=None, **kw) -> "Server":
        """Resident Dfl handles for CSR graphs (n, offsets, indices, weights),
        each on its own CUDA stream, after static Louvain."""
        import torch

        streams = [torch.cuda.Stream() for _ in graphs]
        opt = options if options is not None else default_options()
        handles = [Dfl(n, off, idx, w, options=opt, stream=s)
                   for (n, off, idx, w), s in zip(graphs, streams)]
        for h in handles:
            h.static()
        torch.cuda.synchronize()
        srv = cls(handles, sum(8 * h.stats()["arc_pool"] + 64 * h.n for h in handles), **kw)
        srv.streams = streams
        return srv

    def close(self):
        for h in self.handles:
            h.close()

    # -- one update ---------------------------------------------------------
    def _run_group(self, g: int, group: list, t0: float, recs: dict, gid: int):
        h = self.handles[g]
        start = time.perf_counter() - t0
        if hasattr(h, "step"):
            for r in group[:-1]:
                h.apply_batch(r.dels, r.ins)
            h.step(group[-1].dels, group[-1].ins, DF)
        else:
            for r in group:
                h.apply_batch(r.dels, r.ins)
            h.update(DF)
        self.updates[g] += 1
        refreshed = self.refresh_every > 0 and self.updates[g] % self.refresh_every == 0
        if refreshed:
            h.static()
        q, num, den = h.modularity()
        finish = time.perf_counter() - t0
        memb = h.membership() if self.keep_membership else None
        for r in group:
            rec = recs[r.rid]
            rec.start, rec.finish, rec.group = start, finish, gid
            rec.num, rec.den, rec.q = num, den, q
            rec.membership = memb
            rec.refreshed = refreshed

    # -- continuous batching ------------------------------------------------
    def serve(self, requests: list, coalesce: bool = True) -> ServeResult:
        """Serve `requests` (sorted by arrival) with one worker per graph.

        If a graph's worker raises, its slot and memory are given back, the
        other graphs go on being served, that graph's unserved requests are
        marked failed, and serve() raises the first error once every worker
        has stopped (the partial result is attached as `.result`)."""
        ng = len(self.handles)
        queues = [deque() for _ in range(ng)]
        cv = threading.Condition()
        state = {"done": False, "mem": 0, "busy": 0, "gid": 0}
        recs = {r.rid: Record(r.rid, r.graph, r.arrival) for r in requests}
        for r in requests:
            recs[r.rid].edges = int(r.dels.shape[0] + r.ins.shape[0])
        groups = []
        errors = []
        failed = [False] * ng
        t0 = time.perf_counter()

        def worker(g):
            admitted, need, take = False, 0, []
            try:
                while True:
                    with cv:
                        while not queues[g] and not state["done"]:
                            cv.wait()
                        if not queues[g] and state["done"]:
                            return
                        # admission: a free slot and room in the memory cap for
                        # the queued requests (as many as fit, in arrival
                        # order; one alone is admitted once the GPU is idle)
                        while True:
                            room = self.mem_cap - self.resident - state["mem"]
                            take, need = [], 0
                            for r in queues[g]:
                                b = batch_bytes(r)
                                if need + b > room or (take and not coalesce):
                                    break
                                take.append(r)
                                need += b
                            if state["busy"] < self.slots and (take or state["busy"] == 0):
                                if not take:
                                    take, need = [queues[g][0]], batch_bytes(queues[g][0])
                                break
                            cv.wait()
                        for _ in take:
                            queues[g].popleft()
                        state["busy"] += 1
                        state["mem"] += need
                        admitted = True
                        self.peak["busy"] = max(self.peak["busy"], state["busy"])
                        self.peak["mem"] = max(self.peak["mem"], state["mem"])
                        gid = state["gid"]
                        state["gid"] += 1
                        groups.append((gid, g, [r.rid for r in take]))
                    self._run_group(g, take, t0, recs, gid)
                    with cv:
                        state["busy"] -= 1
                        state["mem"] -= need
                        admitted = False
                        take = []
                        cv.notify_all()
            except Exception as e:  # surfaced after the join
                with cv:
                    errors.append(e)
                    if admitted:  # give back exactly what this update held
                        state["busy"] -= 1
                        state["mem"] -= need
                    failed[g] = True
                    for r in list(take) + list(queues[g]):
                        recs[r.rid].failed = True
                    queues[g].clear()
                    cv.notify_all()

        threads = [threading.Thread(target=worker, args=(g,), daemon=True) for g in range(ng)]
        for t in threads:
            t.start()
        for r in requests:  # release each request at its arrival time
            delay = r.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            with cv:
                if failed[r.graph]:
                    recs[r.rid].failed = True
                else:
                    queues[r.graph].append(r)
                cv.notify_all()
        with cv:
            state["done"] = True
            cv.notify_all()
        for t in threads:
            t.join()
        groups.sort()
        result = ServeResult([recs[r.rid] for r in requests], [(g, ids) for _, g, ids in groups],
                             time.perf_counter() - t0)
        if errors:
            errors[0].result = result
            raise errors[0]
        return result

    # -- baselines ------------------------------------------------------------
    def serve_serial(self, requests: list) -> ServeResult:
        """One request at a time in arrival order, one update each."""
        recs = {r.rid: Record(r.rid, r.graph, r.arrival) for r in requests}
        for r in requests:
            recs[r.rid].edges = int(r.dels.shape[0] + r.ins.shape[0])
        groups = []
        t0 = time.perf_counter()
        for gid, r in enumerate(requests):
            delay = r.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            self._run_group(r.graph, [r], t0, recs, gid)
            groups.append((r.graph, [r.rid]))
        return ServeResult([recs[r.rid] for r in requests], groups, time.perf_counter() - t0)

    def replay(self, requests: list, groups: list) -> ServeResult:
        """Recompute a grouping one update at a time (no timing)."""
        by_id = {r.rid: r for r in requests}
        recs = {r.rid: Record(r.rid, r.graph, r.arrival) for r in requests}
        t0 = time.perf_counter()
        for gid, (g, ids) in enumerate(groups):
            self._run_group(g, [by_id[i] for i in ids], t0, recs, gid)
        return ServeResult([recs[r.rid] for r in requests], groups, time.perf_counter() - t0)


def make_requests(pools, schedule) -> list:
    """Requests from (arrival, graph, size) triples; each graph's batches come
    from its own edge pool in arrival order."""
    out = []
    for rid, (t, g, size) in enumerate(schedule):
        d, i = pools[g].next(size)
        out.append(Request(rid, g, t, d, i))
    return out
