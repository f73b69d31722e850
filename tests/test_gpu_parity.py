"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer state must match bit for bit: the slack CSR as sorted adjacency,
K, Sigma, 2m, membership, frontiers and the first-pass trace (vertices
processed, movers and the exact 128-bit sum S of the movers' dQ numerators
per iteration).  Modularity must match within 1e-12 relative; its exact
integer numerator and denominator must be equal.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2404_19634_gb300 as mod
    mod.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


_STREAMS = []


def pair(dfl, orc, g, substeps=4, tau_agg=0.8, graph=True, **kw):
    """GPU handle and oracle on the same graph.  The handle runs on a side
    stream; with graph=True it replays its captured local-moving iteration
    (DFL_FLAG_GRAPH), with graph=False every kernel is launched from the
    host (the default)."""
    import torch
    off, idx, w = synth.to_csr(g)
    flags = kw.pop("flags", 0) | (32 if graph else 4)  # DFL_FLAG_GRAPH / DFL_FLAG_NO_GRAPH
    opt = dfl.default_options(substeps=substeps, tau_agg=tau_agg, flags=flags, **kw)
    s = torch.cuda.Stream()
    _STREAMS.append(s)
    a = dfl.Dfl(g.n, off, idx, w, options=opt, stream=s)
    b = orc.Oracle(g.n, off, idx, w)
    b.set_options(substeps=substeps, tau_agg=tau_agg,
                  **{k: v for k, v in kw.items() if k in ("max_iterations", "max_passes")})
    return a, b


def same_state(a, b, stats=True):
    Ca, Cb = a.membership(), b.membership()
    assert np.array_equal(Ca, Cb), f"membership differs at {np.flatnonzero(Ca != Cb)[:10]}"
    Ka, Sa, ma = a.weights()
    Kb, Sb, mb = b.weights()
    assert ma == mb
    assert np.array_equal(Ka, Kb), "K differs"
    assert np.array_equal(Sa, Sb), "Sigma differs"
    qa, na, da = a.modularity()
    qb, nb, db = b.modularity()
    assert (na, da) == (nb, db)
    assert abs(qa - qb) <= 1e-12 * max(1.0, abs(qb))
    if stats:
        sa, sb = a.stats(), b.stats()
        assert sa["passes"] == sb["passes"] and sa["iterations"] == sb["iterations"]
        assert sa["affected_initial"] == sb["affected_initial"]
        assert sa["affected_ever"] == sb["affected_ever"]
        assert a.trace() == b.trace()


def same_graph(a, b):
    for x, y in zip(a.graph(), b.graph()):
        assert np.array_equal(x, y), "graph differs"


# ---------------------------------------------------------------------------

def test_static_sbm_10k(dfl, orc):
    g = synth.sbm(10000, 50, 0.02, 0.0002, 1)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    same_state(a, b)
    same_graph(a, b)


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sbm_batch_update(dfl, orc, mode, graph):
    """10,000-vertex SBM, static, then one 100-edge batch (80% insertions,
    20% deletions) updated with ND, DS or DF."""
    g = synth.sbm(10000, 50, 0.02, 0.0002, 1)
    dels, ins = synth.random_batch(g.n, g, 80, 20, 11)
    a, b = pair(dfl, orc, g, graph=graph)
    a.static()
    b.static()
    assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
    same_graph(a, b)
    same_state(a, b, stats=False)  # K, Sigma after the batch, before the update
    Fa, Ra = a.mark(mode)
    Fb, Rb = b.mark(mode)
    assert np.array_equal(Fa, Fb) and np.array_equal(Ra, Rb)
    a.update(mode)
    b.update(mode)
    same_state(a, b)


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("substeps", [1, 2, 4, 8])
@pytest.mark.parametrize("scale", [10, 13])
def test_rmat_stream(dfl, orc, substeps, scale, graph):
    g = synth.rmat(scale, 8 << scale, 30 + scale)
    a, b = pair(dfl, orc, g, substeps=substeps, graph=graph)
    a.static()
    b.static()
    same_state(a, b)
    stream = synth.BatchStream(g, 99)
    for t, size in enumerate([3, 40, 500, 3000]):
        dels, ins = stream.next(size)
        assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
        mode = [2, 0, 1, 2][t]
        a.update(mode)
        b.update(mode)
        same_state(a, b)
    same_graph(a, b)


def test_weighted_graph_partial_deletions(dfl, orc):
    rng = np.random.default_rng(5)
    g = synth.planted_partition(3000, 40, 0.3, 12, 16, 6)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    for t in range(5):
        off, idx, w = b.graph()
        edges = [(i, int(idx[k]), int(w[k])) for i in range(g.n)
                 for k in range(int(off[i]), int(off[i + 1])) if i < idx[k]]
        pick = rng.choice(len(edges), 60, replace=False)
        dels = np.array([(edges[p][0], edges[p][1], int(rng.integers(0, edges[p][2] + 1)))
                         for p in pick], np.uint32)
        ins = np.stack([rng.integers(0, g.n, 200), rng.integers(0, g.n, 200),
                        rng.integers(1, 17, 200)], 1).astype(np.uint32)
        ins = ins[ins[:, 0] != ins[:, 1]]
        ins = np.concatenate([ins, ins[:5]])  # repeated insertions add up
        assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
        same_graph(a, b)
        a.update(t % 3)
        b.update(t % 3)
        same_state(a, b)


@pytest.mark.parametrize("graph", [True, False])
def test_high_degree_bins(dfl, orc, graph):
    """Hubs of degree ~300, ~5,000 and ~20,000 exercise the block kernels
    with shared-memory and global-memory tables."""
    rng = np.random.default_rng(8)
    n = 40000
    base = synth.planted_partition(n, 100, 0.2, 6, 1, 3)
    us, vs = [base.u], [base.v]
    for hub, deg in [(5, 300), (17, 5000), (123, 20000)]:
        nb = rng.choice(n, deg, replace=False)
        nb = nb[nb != hub]
        us.append(np.full(nb.shape[0], hub, np.uint32))
        vs.append(nb.astype(np.uint32))
    u = np.concatenate(us)
    v = np.concatenate(vs)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = np.unique((lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64))
    g = synth.EdgeList(n, (key >> np.uint64(32)).astype(np.uint32),
                       (key & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                       np.ones(key.shape[0], np.uint32))
    a, b = pair(dfl, orc, g, graph=graph)
    a.static()
    b.static()
    same_state(a, b)
    stream = synth.BatchStream(g, 4)
    dels, ins = stream.next(2000)
    ins = np.concatenate([ins, np.array([[17, 9, 1], [123, 77, 2], [5, 31, 1]], np.uint32)])
    assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
    a.update(0)
    b.update(0)
    same_state(a, b)
    same_graph(a, b)


def test_move_iteration_random_states(dfl, orc):
    rng = np.random.default_rng(11)
    g = synth.rmat(11, 12 << 11, 4)
    for k in (1, 4):
        a, b = pair(dfl, orc, g, substeps=k)
        for _ in range(3):
            C = rng.integers(0, g.n // 8, g.n).astype(np.uint32)
            F = (rng.random(g.n) < 0.6).astype(np.uint8)
            R = (rng.random(g.n) < 0.9).astype(np.uint8)
            a.set_membership(C)
            b.set_membership(C)
            Fa, ma, Sa = a.move_iteration(F, R)
            Fb, mb, Sb = b.move_iteration(F, R)
            assert np.array_equal(ma, mb)
            assert np.array_equal(Fa, Fb)
            assert Sa == Sb
            same_state(a, b, stats=False)


def test_aggregation_export(dfl, orc):
    rng = np.random.default_rng(3)
    g = synth.sbm(3000, 30, 0.04, 0.002, 9)
    a, b = pair(dfl, orc, g)
    for C in [rng.integers(0, 3000, 3000), np.repeat(np.arange(30), 100), np.zeros(3000)]:
        C = C.astype(np.uint32)
        a.set_membership(C)
        b.set_membership(C)
        for x, y in zip(a.aggregate(), b.aggregate()):
            assert np.array_equal(x, y)


def test_louvain_from_random_frontier(dfl, orc):
    rng = np.random.default_rng(12)
    g = synth.sbm(5000, 25, 0.03, 0.001, 13)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    F = (rng.random(g.n) < 0.3).astype(np.uint8)
    R = (rng.random(g.n) < 0.7).astype(np.uint8)
    a.louvain_from(F, R)
    b.louvain_from(F, R)
    same_state(a, b)


def test_temporal_aggregation_tolerance_disabled(dfl, orc):
    """tau_agg = 1 (Section 5.1.2, real-world dynamic graphs): the low-shrink
    test of Alg. 4 is disabled, so passes only stop on convergence."""
    src, dst = synth.temporal_pa_stream(3000, 40000, 0.3, 21)
    base = synth.temporal_edges(src[:36000], dst[:36000], 3000)
    a, b = pair(dfl, orc, base, tau_agg=1.0)
    a.static()
    b.static()
    same_state(a, b)
    for t in range(4):
        s = slice(36000 + t * 1000, 36000 + (t + 1) * 1000)
        ins = np.stack([src[s], dst[s], np.ones(1000, np.uint32)], 1)
        ins = ins[ins[:, 0] != ins[:, 1]]
        old = slice(t * 1000, (t + 1) * 1000)
        exp = np.stack([src[old], dst[old], np.ones(1000, np.uint32)], 1)
        exp = exp[exp[:, 0] != exp[:, 1]]
        # expire the oldest interactions (weight 1 each); group repeats
        lo, hi = np.minimum(exp[:, 0], exp[:, 1]), np.maximum(exp[:, 0], exp[:, 1])
        key, cnt = np.unique((lo.astype(np.uint64) << np.uint64(32)) | hi, return_counts=True)
        dels = np.stack([(key >> np.uint64(32)).astype(np.uint32),
                         (key & np.uint64(0xFFFFFFFF)).astype(np.uint32), cnt.astype(np.uint32)], 1)
        assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
        a.update(2)
        b.update(2)
        same_state(a, b)


def test_empty_and_degenerate(dfl, orc):
    g = synth.sbm(1000, 10, 0.08, 0.004, 23)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    C0 = a.membership().copy()
    empty = np.zeros((0, 3), np.uint32)
    assert a.apply_batch(empty, empty) == 0 and b.apply_batch(empty, empty) == 0
    a.update(2)
    b.update(2)
    same_state(a, b)
    assert np.array_equal(a.membership(), C0)
    assert a.stats()["affected_ever"] == 0
    # a graph without edges
    e = synth.EdgeList(50, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    a, b = pair(dfl, orc, e)
    a.static()
    b.static()
    same_state(a, b)
    assert a.modularity()[0] == 0.0
    assert a.apply_batch(empty, np.array([[1, 2, 3]], np.uint32)) == 0
    b.apply_batch(empty, np.array([[1, 2, 3]], np.uint32))
    a.update(2)
    b.update(2)
    same_state(a, b)
    # two vertices
    t = synth.EdgeList(2, np.array([0], np.uint32), np.array([1], np.uint32), np.array([1], np.uint32))
    a, b = pair(dfl, orc, t)
    a.static()
    b.static()
    same_state(a, b)


def test_batch_errors_leave_state_unchanged(dfl, orc):
    g = synth.sbm(500, 5, 0.1, 0.01, 3)
    a, b = pair(dfl, orc, g)
    with pytest.raises(dfl.DflError):
        a.update(2)
    assert a.apply_batch(None, np.array([[0, 1, 1]], np.uint32), check=False) == -7
    a.static()
    b.static()
    before_g = a.graph()
    before_w = a.weights()
    u, v = int(g.u[0]), int(g.v[0])
    off, idx, _ = synth.to_csr(g)
    absent = next((x, y) for x in range(g.n) for y in range(x + 1, g.n)
                  if y not in set(idx[int(off[x]):int(off[x + 1])]))
    cases = [
        ([], [(0, 0, 1)], -1),
        ([], [(0, g.n, 1)], -1),
        ([], [(0, 1, 0)], -1),
        ([(u, v, 0), (v, u, 0)], [], -1),
        ([absent + (0,)], [], -2),
        ([(u, v, 2)], [], -2),
        ([], [(u, v, 0xFFFFFFFF)], -3),
        ([absent + (0,)], [(0, 0, 1)], -1),
    ]
    for d, i, code in cases:
        d = np.array(d, np.uint32).reshape(-1, 3)
        i = np.array(i, np.uint32).reshape(-1, 3)
        assert a.apply_batch(d, i, check=False) == code
        assert b.apply_batch(d, i) == code
        for x, y in zip(before_g, a.graph()):
            assert np.array_equal(x, y)
        after = a.weights()
        assert np.array_equal(before_w[0], after[0]) and np.array_equal(before_w[1], after[1])
    same_state(a, b, stats=False)


def test_invalid_graph_rejected(dfl):
    off = np.array([0, 1, 1], np.uint64)  # arc (0,1) without (1,0)
    with pytest.raises(dfl.DflError):
        dfl.Dfl(2, off, np.array([1], np.uint32), np.array([1], np.uint32))
    off = np.array([0, 1, 2], np.uint64)  # unequal weights
    with pytest.raises(dfl.DflError):
        dfl.Dfl(2, off, np.array([1, 0], np.uint32), np.array([1, 2], np.uint32))


def test_device_buffers_and_stream(dfl, orc):
    import torch
    g = synth.sbm(4000, 20, 0.04, 0.002, 31)
    off, idx, w = synth.to_csr(g)
    s = torch.cuda.Stream()
    dev = lambda x: torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else x.view(np.int32)).cuda()
    a = dfl.Dfl(g.n, dev(off), dev(idx), dev(w), stream=s)
    b = orc.Oracle(g.n, off, idx, w)
    a.static()
    b.static()
    dels, ins = synth.random_batch(g.n, g, 200, 50, 2)
    a.apply_batch(dev(np.ascontiguousarray(dels)), dev(np.ascontiguousarray(ins)))
    b.apply_batch(dels, ins)
    a.update(2)
    b.update(2)
    out = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    a.membership(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), b.membership())
    same_state(a, b)


def test_long_stream_tombstones_and_rebuilds(dfl, orc):
    """Many batches on a small graph: deletions leave tombstones, re-inserted
    edges revive them, hot vertices overflow their append tail and are
    rebuilt; the graph and the state must track the oracle throughout."""
    rng = np.random.default_rng(17)
    g = synth.planted_partition(600, 12, 0.25, 6, 4, 2)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    deleted = []
    for t in range(40):
        off, idx, w = b.graph()
        edges = [(i, int(idx[k]), int(w[k])) for i in range(g.n)
                 for k in range(int(off[i]), int(off[i + 1])) if i < idx[k]]
        pick = rng.choice(len(edges), min(25, len(edges)), replace=False)
        dels = [(edges[p][0], edges[p][1], 0 if rng.random() < 0.7 else int(rng.integers(1, edges[p][2] + 1)))
                for p in pick]
        ins = []
        hot = int(rng.integers(0, 8))  # a few vertices receive many new edges
        for _ in range(30):
            j = int(rng.integers(0, g.n))
            if j != hot:
                ins.append((hot, j, int(rng.integers(1, 4))))
        for _ in range(20):
            x, y = int(rng.integers(0, g.n)), int(rng.integers(0, g.n))
            if x != y:
                ins.append((x, y, 1))
        if deleted:  # re-insert some previously deleted edges (tombstone revival)
            for p in rng.choice(len(deleted), min(10, len(deleted)), replace=False):
                ins.append(deleted[p])
        deleted += [(u, v, 1) for (u, v, _) in dels]
        d = np.array(dels, np.uint32).reshape(-1, 3)
        i = np.array(ins, np.uint32).reshape(-1, 3)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        same_graph(a, b)
        if t % 5 == 4:
            a.update(t % 3)
            b.update(t % 3)
            same_state(a, b)


@pytest.mark.parametrize("count", [3500, 5000])
def test_one_row_gets_thousands_of_edges(dfl, orc, count):
    """3,500 new arcs of one row are sorted in shared memory by the rebuild;
    5,000 exceed that and take the sort-based batch apply."""
    g = synth.sbm(6000, 30, 0.01, 0.001, 41)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    rng = np.random.default_rng(2)
    nb = rng.choice(np.arange(1, g.n), count, replace=False)
    ins = np.stack([np.zeros(count, np.int64), nb, rng.integers(1, 5, count)], 1).astype(np.uint32)
    off, idx, w = synth.to_csr(g)
    row0 = idx[int(off[0]):int(off[1])]
    dels = np.array([[0, int(x), 0] for x in row0[:3]], np.uint32).reshape(-1, 3)
    assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
    same_graph(a, b)
    a.update(2)
    b.update(2)
    same_state(a, b)
    # delete most of that row again, then re-insert part of it
    dels = np.stack([np.zeros(3000, np.int64), nb[:3000], np.zeros(3000, np.int64)], 1).astype(np.uint32)
    assert a.apply_batch(dels, np.zeros((0, 3), np.uint32)) == 0
    assert b.apply_batch(dels, np.zeros((0, 3), np.uint32)) == 0
    ins = np.stack([np.zeros(500, np.int64), nb[:500], np.ones(500, np.int64)], 1).astype(np.uint32)
    assert a.apply_batch(np.zeros((0, 3), np.uint32), ins) == 0 and b.apply_batch(np.zeros((0, 3), np.uint32), ins) == 0
    same_graph(a, b)
    a.update(1)
    b.update(1)
    same_state(a, b)


def test_giant_vertex_many_distinct_communities(dfl, orc):
    """A vertex of degree 20,000 whose neighbours sit in 20,000 different
    communities: its chunked decision needs several merge passes."""
    n = 20001
    u = np.zeros(20000, np.uint32)
    v = np.arange(1, n, dtype=np.uint32)
    # a sparse ring among the leaves, weights vary
    ring = np.arange(1, n - 1, dtype=np.uint32)
    g = synth.EdgeList(n, np.concatenate([u, ring]), np.concatenate([v, ring + 1]),
                       np.concatenate([np.ones(20000, np.uint32), (ring % 7 + 1).astype(np.uint32)]))
    for k in (1, 4):
        a, b = pair(dfl, orc, g, substeps=k)
        C = np.arange(n, dtype=np.uint32)
        a.set_membership(C)
        b.set_membership(C)
        F = np.ones(n, np.uint8)
        R = np.ones(n, np.uint8)
        Fa, ma, Sa = a.move_iteration(F, R)
        Fb, mb, Sb = b.move_iteration(F, R)
        assert np.array_equal(ma, mb) and np.array_equal(Fa, Fb) and Sa == Sb
        same_state(a, b, stats=False)
        a.static()
        b.static()
        same_state(a, b)


def test_profiled_graph_replay(dfl, orc):
    """Profiling events inside the captured iteration graph are recorded and
    harvested; results stay identical."""
    g = synth.rmat(12, 8 << 12, 5)
    a, b = pair(dfl, orc, g, flags=1)  # DFL_FLAG_PROFILE
    a.static()
    b.static()
    stream = synth.BatchStream(g, 6)
    for _ in range(3):
        d, i = stream.next(200)
        a.apply_batch(d, i)
        b.apply_batch(d, i)
        a.update(2)
        b.update(2)
        same_state(a, b)
    prof = a.profile()
    assert prof["move"]["ms"] > 0 and prof["move"]["bytes"] > 0 and prof["bin0"]["launches"] > 0


@pytest.mark.parametrize("graph", [True, False])
def test_decide_phase_profile_only(dfl, orc, graph):
    """DFL_FLAG_PROFILE_MOVE times the decide phase alone: the move class
    gets time and bytes, no other class is timed; results stay identical."""
    g = synth.rmat(12, 8 << 12, 7)
    a, b = pair(dfl, orc, g, graph=graph, flags=64)  # DFL_FLAG_PROFILE_MOVE
    a.static()
    b.static()
    a.profile(reset=True)
    stream = synth.BatchStream(g, 8)
    for _ in range(3):
        d, i = stream.next(300)
        a.apply_batch(d, i)
        b.apply_batch(d, i)
        a.update(2)
        b.update(2)
        same_state(a, b)
    prof = a.profile()
    assert prof["move"]["ms"] > 0 and prof["move"]["bytes"] > 0 and prof["move"]["launches"] > 0
    assert all(v["ms"] == 0 for k, v in prof.items() if k != "move")


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_recomputed_auxiliary_information_same_results(dfl, orc, mode):
    """DFL_FLAG_RECOMPUTE_AUX recomputes K, Sigma and 2m from scratch before
    every update (the ablation of Section 4.2): the state must still equal
    the oracle's, which updates K and Sigma incrementally (Alg. 7)."""
    g = synth.rmat(12, 8 << 12, 9)
    a, b = pair(dfl, orc, g, flags=128)  # DFL_FLAG_RECOMPUTE_AUX
    a.static()
    b.static()
    stream = synth.BatchStream(g, 10)
    for size in (30, 600):
        d, i = stream.next(size, w_max=5)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        a.update(mode)
        b.update(mode)
        same_state(a, b)


def test_compaction_and_checkpoint_continue_exactly(dfl, orc, tmp_path):
    """A long stream leaves relocated rows' slots behind; dfl_compact gives
    them back without changing anything later updates compute.  A
    checkpoint (graph, membership, tuning) saved to disk and restored into a
    new handle continues exactly like the original."""
    rng = np.random.default_rng(23)
    g = synth.planted_partition(800, 16, 0.25, 6, 4, 3)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    a.set_tuning(bin_warp=4, bin_warp_hash=64, bin_block=1024, block_threads=128)

    def batch(t):
        off, idx, w = b.graph()
        edges = [(i, int(idx[k]), int(w[k])) for i in range(g.n)
                 for k in range(int(off[i]), int(off[i + 1])) if i < idx[k]]
        pick = rng.choice(len(edges), min(30, len(edges)), replace=False)
        dels = np.array([(edges[p][0], edges[p][1], 0) for p in pick], np.uint32).reshape(-1, 3)
        hot = int(rng.integers(0, 10))
        ins = [(hot, int(j), 1) for j in rng.integers(0, g.n, 60) if j != hot]
        ins += [(int(x), int(y), 2) for x, y in rng.integers(0, g.n, (30, 2)) if x != y]
        return dels, np.array(ins, np.uint32).reshape(-1, 3)

    for t in range(30):
        d, i = batch(t)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        if t % 3 == 2:
            a.update(2)
            b.update(2)
    same_state(a, b)
    arcs = a.num_arcs()
    before, after = a.compact()
    assert after < before and a.num_arcs() == arcs
    same_graph(a, b)
    same_state(a, b, stats=False)
    path = str(tmp_path / "state.npz")
    dfl.save_checkpoint(path, a.checkpoint())
    import torch
    s = torch.cuda.Stream()
    c = dfl.Dfl.restore(dfl.load_checkpoint(path), options=dfl.default_options(), stream=s)
    assert c.tuning() == a.tuning()
    same_graph(c, b)
    same_state(c, b, stats=False)
    for t in range(6):
        d, i = batch(t)
        for x in (a, b, c):
            assert x.apply_batch(d, i) == 0
        for x in (a, b, c):
            x.update(t % 3)
        same_state(a, b)
        same_state(c, b)
    same_graph(a, b)
    same_graph(c, b)
    c.close()


def test_weights_near_the_2m_limit(dfl, orc):
    """Edge weights in the hundreds of thousands with 2m just below 2^32:
    every gain numerator factor (2m, K_i, Sigma_c, K_{i->c}) is close to its
    2^32 bound, so products reach 2^63; results must still equal the
    oracle's, and a batch that would take 2m to 2^32 is refused."""
    rng = np.random.default_rng(29)
    base = synth.planted_partition(2000, 20, 0.2, 10, 1, 7)
    m = base.m
    w = rng.integers(1, 2 * ((1 << 32) - 1) // (2 * m) - 1, m).astype(np.uint64)
    scale = ((1 << 32) - 2 * 400000 - 64) / (2.0 * float(w.sum()))
    w = np.maximum(1, (w * scale).astype(np.uint64)).astype(np.uint32)
    g = synth.EdgeList(base.n, base.u, base.v, w)
    assert 2 * int(w.astype(np.uint64).sum()) < (1 << 32) - 2 * 400000
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    same_state(a, b)
    assert a.weights()[2] > (1 << 31)
    off, idx, _ = synth.to_csr(g)
    for t in range(3):
        dels = np.array([(int(g.u[k]), int(g.v[k]), 0) for k in rng.choice(m, 20, replace=False)], np.uint32)
        x = rng.integers(0, g.n, (10, 2))
        x = x[x[:, 0] != x[:, 1]]
        ins = np.concatenate([x, rng.integers(1, 40000, (x.shape[0], 1))], 1).astype(np.uint32)
        if t:
            dels = np.zeros((0, 3), np.uint32)  # only the first batch deletes (edges may be gone later)
        assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
        a.update([2, 1, 0][t])
        b.update([2, 1, 0][t])
        same_state(a, b)
    big = np.array([[0, 1, 0xFFFFFFFF // 2]], np.uint32)
    assert a.apply_batch(np.zeros((0, 3), np.uint32), big, check=False) == -3  # DFL_ERR_OVERFLOW
    assert b.apply_batch(np.zeros((0, 3), np.uint32), big) == -3
    same_state(a, b, stats=False)
