"""Host logic of the serving loop (admission, coalescing, ordering), with
stand-in handles on the CPU: each records the batches it was given and
sleeps inside update() so that graphs' work overlaps in time."""
import threading
import time

import numpy as np

from paper_2404_19634_gb300 import serve


class FakeHandle:
    def __init__(self, g, delay=0.004):
        self.g = g
        self.delay = delay
        self.pending = []
        self.history = []  # request sizes per update, in order
        self.lock = threading.Lock()
        self.active = 0

    def apply_batch(self, dels, ins):
        self.pending.append(int(dels.shape[0] + ins.shape[0]))

    def update(self, mode):
        with self.lock:
            self.active += 1
            assert self.active == 1, "one update at a time per graph"
        time.sleep(self.delay)
        self.history.append(tuple(self.pending))
        self.pending = []
        with self.lock:
            self.active -= 1

    def static(self):
        self.history.append("static")

    def modularity(self):
        # a value that depends on the whole grouping history of this graph
        num = hash(tuple(self.history)) & 0xFFFFFFFF
        return num / 2**32, num, 2**32

    def membership(self):
        return np.array([len(self.history)], np.uint32)


def requests(num_graphs=4, count=120, seed=3):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for rid in range(count):
        t += rng.exponential(1 / 5000)
        g = int(rng.integers(0, num_graphs))
        k = int(rng.integers(1, 50))
        out.append(serve.Request(rid, g, t, np.zeros((k // 5, 3), np.uint32),
                                 np.zeros((k - k // 5, 3), np.uint32)))
    return out


def check_groups(reqs, res, coalesce=True):
    seen = []
    for g, ids in res.groups:
        assert all(reqs[i].graph == g for i in ids)
        seen += ids
        if not coalesce:
            assert len(ids) == 1
    assert sorted(seen) == [r.rid for r in reqs], "every request served exactly once"
    for g in {r.graph for r in reqs}:
        order = [i for gg, ids in res.groups if gg == g for i in ids]
        assert order == sorted(order), "a graph's requests are applied in arrival order"
    for rec in res.records:
        assert rec.finish >= rec.start >= rec.arrival - 1e-3


def test_coalescing_overlap_and_replay():
    reqs = requests()
    srv = serve.Server([FakeHandle(g) for g in range(4)])
    res = srv.serve(reqs, coalesce=True)
    check_groups(reqs, res)
    assert len(res.groups) < len(reqs), "queued requests were coalesced"
    assert srv.peak["busy"] > 1, "graphs' updates overlapped"
    # the same grouping replayed one update at a time gives the same results
    again = serve.Server([FakeHandle(g, 0.0) for g in range(4)]).replay(reqs, res.groups)
    assert [(r.num, r.den, r.group) for r in again.records] == \
           [(r.num, r.den, r.group) for r in res.records]
    s = res.summary()
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_no_coalescing_matches_serial():
    reqs = requests(count=60)
    a = serve.Server([FakeHandle(g) for g in range(4)]).serve(reqs, coalesce=False)
    check_groups(reqs, a, coalesce=False)
    b = serve.Server([FakeHandle(g, 0.0) for g in range(4)]).serve_serial(reqs)
    assert [(r.num, r.den) for r in a.records] == [(r.num, r.den) for r in b.records]


def test_slots_and_memory_cap():
    reqs = requests(count=80)
    one = max(serve.batch_bytes(r) for r in reqs)
    srv = serve.Server([FakeHandle(g) for g in range(4)], resident_bytes=1000,
                       mem_cap=1000 + 2 * one, slots=2)
    res = srv.serve(reqs, coalesce=True)
    check_groups(reqs, res)
    assert srv.peak["busy"] <= 2
    assert srv.peak["mem"] <= 2 * one


def test_oversized_request_runs_alone():
    reqs = requests(count=20)
    srv = serve.Server([FakeHandle(g) for g in range(4)], resident_bytes=0, mem_cap=1)
    res = srv.serve(reqs, coalesce=True)
    check_groups(reqs, res)
    assert srv.peak["busy"] == 1
    assert all(len(ids) == 1 for _, ids in res.groups)


def test_periodic_static_refresh():
    """refresh_every=k: static Louvain after every k-th update of a graph,
    counted per graph, and the same under replay of the same grouping."""
    reqs = requests(num_graphs=3, count=90, seed=8)
    srv = serve.Server([FakeHandle(g, 0.0) for g in range(3)], refresh_every=4)
    res = srv.serve(reqs)
    check_groups(reqs, res)
    for g, h in enumerate(srv.handles):
        updates = [x for x in h.history if x != "static"]
        assert len(updates) == srv.updates[g]
        # a static run follows exactly every 4th update
        pos = [k for k, x in enumerate(h.history) if x == "static"]
        assert len(pos) == len(updates) // 4
        for j, p in enumerate(pos):
            assert sum(1 for x in h.history[:p] if x != "static") == 4 * (j + 1)
    flagged = {rid for rid, rec in enumerate(res.records) if rec.refreshed}
    by_group = {gid: ids for gid, (g, ids) in enumerate(res.groups)}
    assert flagged and all(res.records[i].refreshed == res.records[ids[0]].refreshed
                           for ids in by_group.values() for i in ids)
    again = serve.Server([FakeHandle(g, 0.0) for g in range(3)], refresh_every=4).replay(reqs, res.groups)
    assert [(r.num, r.refreshed) for r in again.records] == [(r.num, r.refreshed) for r in res.records]


class FailingHandle(FakeHandle):
    """Raises on its `fail_at`-th update (0-based)."""

    def __init__(self, g, fail_at, delay=0.002):
        super().__init__(g, delay)
        self.fail_at = fail_at
        self.calls = 0

    def update(self, mode):
        self.calls += 1
        if self.calls - 1 == self.fail_at:
            self.pending = []
            raise RuntimeError(f"graph {self.g} failed")
        super().update(mode)


def test_worker_error_gives_back_its_slot_and_memory():
    """A graph whose update raises: its slot and memory return to the pool
    (the other graphs are still served, also with one slot in all), its
    unserved requests are marked failed, and serve() raises the error with
    the partial result attached."""
    import pytest
    reqs = requests(num_graphs=3, count=90, seed=5)
    one = max(serve.batch_bytes(r) for r in reqs)
    handles = [FakeHandle(0), FailingHandle(1, fail_at=2), FakeHandle(2)]
    srv = serve.Server(handles, resident_bytes=0, mem_cap=3 * one, slots=1)
    with pytest.raises(RuntimeError, match="graph 1 failed") as ei:
        srv.serve(reqs, coalesce=False)
    res = ei.value.result
    ok = [r for r in res.records if r.graph != 1]
    assert ok and all(not r.failed and r.finish >= r.arrival for r in ok), \
        "the other graphs were served after the failure"
    g1 = [r for r in res.records if r.graph == 1]
    assert sum(not r.failed for r in g1) == 2 and all(r.failed for r in g1[2:])
    s = res.summary()
    assert s["failed"] == len(g1) - 2 and s["p50_ms"] >= 0


class StepHandle(FakeHandle):
    """Has dfl_step: a coalesced group's earlier batches are applied, the
    last one goes with the update."""

    def __init__(self, g, delay=0.002):
        super().__init__(g, delay)
        self.calls = []

    def apply_batch(self, dels, ins):
        self.calls.append("apply")
        super().apply_batch(dels, ins)

    def update(self, mode):
        self.calls.append("update")
        super().update(mode)

    def step(self, dels, ins, mode):
        self.calls.append("step")
        super().apply_batch(dels, ins)
        super().update(mode)


def test_worker_steps_with_the_last_batch_of_a_group():
    reqs = requests(num_graphs=2, count=60, seed=11)
    hs = [StepHandle(g) for g in range(2)]
    res = serve.Server(hs).serve(reqs, coalesce=True)
    check_groups(reqs, res)
    for h in hs:
        assert "update" not in h.calls  # every update went with a batch through step
        n_groups = sum(1 for g, _ in res.groups if g == h.g)
        assert h.calls.count("step") == n_groups
        sizes = [len(ids) for g, ids in res.groups if g == h.g]
        assert h.calls.count("apply") == sum(s - 1 for s in sizes)
        # within each update: the group's earlier batches, then the step
        i = 0
        for s in sizes:
            assert h.calls[i:i + s] == ["apply"] * (s - 1) + ["step"]
            i += s
