"""Launch-shape tuning, the autotuner and graph groups against the oracle.

A tuning only moves vertices between decide kernels, so every tuning must
give the oracle's exact state.  A group must give each of its graphs what
the oracle gives that graph alone: membership (labels local to the graph),
K, Sigma, 2m, the exact modularity numerator and denominator, and the
per-graph pass and iteration counts.
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


def _stream():
    import torch
    s = torch.cuda.Stream()
    _STREAMS.append(s)
    return s


def same(a, b):
    Ca, Cb = a.membership(), b.membership()
    assert np.array_equal(Ca, Cb), f"membership differs at {np.flatnonzero(Ca != Cb)[:10]}"
    Ka, Sa, ma = a.weights()
    Kb, Sb, mb = b.weights()
    assert ma == mb and np.array_equal(Ka, Kb) and np.array_equal(Sa, Sb)
    qa, na, da = a.modularity()
    qb, nb, db = b.modularity()
    assert (na, da) == (nb, db)
    assert abs(qa - qb) <= 1e-12 * max(1.0, abs(qb))
    sa, sb = a.stats(), b.stats()
    assert sa["passes"] == sb["passes"] and sa["iterations"] == sb["iterations"]


DEFAULT_TUNING = dict(bin_warp=8, bin_warp_hash=256, bin_block=4096, block_threads=256)
TUNINGS = [
    dict(bin_warp=32, bin_warp_hash=256, bin_block=4096, block_threads=256),
    dict(bin_warp=8, bin_warp_hash=64, bin_block=1024, block_threads=128),
    dict(bin_warp=16, bin_warp_hash=128, bin_block=16384, block_threads=512),
    dict(bin_warp=0, bin_warp_hash=0, bin_block=0, block_threads=256),      # all chunked
    dict(bin_warp=0, bin_warp_hash=256, bin_block=256, block_threads=128),  # warp tables only
    dict(bin_warp=32, bin_warp_hash=32, bin_block=32, block_threads=512),
    dict(bin_warp=4, bin_warp_hash=256, bin_block=4096, block_threads=256),  # 8 vertices a warp
    dict(bin_warp=5, bin_warp_hash=40, bin_block=2048, block_threads=256),   # 4 a warp, odd limits
]


@pytest.mark.parametrize("tuning", range(len(TUNINGS)))
@pytest.mark.parametrize("graph", [True, False])
def test_tuning_same_results(dfl, orc, tuning, graph):
    g = synth.rmat(13, 8 << 13, 41)
    off, idx, w = synth.to_csr(g)
    opt = dfl.default_options(flags=32 if graph else 4)
    a = dfl.Dfl(g.n, off, idx, w, options=opt, stream=_stream())
    a.set_tuning(**TUNINGS[tuning])
    assert a.tuning() == TUNINGS[tuning]
    b = orc.Oracle(g.n, off, idx, w)
    a.static()
    b.static()
    same(a, b)
    stream = synth.BatchStream(g, 7)
    for t, size in enumerate([50, 800, 4000]):
        d, i = stream.next(size)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        a.update([2, 1, 0][t])
        b.update([2, 1, 0][t])
        same(a, b)


def test_tuning_rejects_out_of_range(dfl):
    g = synth.rmat(8, 8 << 8, 3)
    off, idx, w = synth.to_csr(g)
    a = dfl.Dfl(g.n, off, idx, w, stream=_stream())
    for bad in [dict(bin_warp=33), dict(bin_warp_hash=300), dict(bin_warp=32, bin_warp_hash=16),
                dict(bin_block=100), dict(block_threads=64)]:
        with pytest.raises(dfl.DflError) as e:
            a.set_tuning(**bad)
        assert e.value.code == -1
    assert a.tuning() == DEFAULT_TUNING


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_autotune_keeps_state_and_results(dfl, orc, mode):
    g = synth.rmat(14, 8 << 14, 43)
    off, idx, w = synth.to_csr(g)
    a = dfl.Dfl(g.n, off, idx, w, stream=_stream())
    b = orc.Oracle(g.n, off, idx, w)
    a.static()
    b.static()
    stream = synth.BatchStream(g, 8)
    for t in range(3):
        d, i = stream.next(2000)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        C0 = a.membership()
        K0, S0, m0 = a.weights()
        tuning, ms = a.autotune(mode, reps=2)
        assert ms > 0 and set(tuning) == set(TUNINGS[0])  # the same fields
        assert a.tuning() == tuning
        # the autotuner computed decisions but applied none of them
        K1, S1, m1 = a.weights()
        assert np.array_equal(C0, a.membership())
        assert np.array_equal(K0, K1) and np.array_equal(S0, S1) and m0 == m1
        a.update(mode)
        b.update(mode)
        same(a, b)


# ---------------------------------------------------------------------------
# groups

def group_graphs():
    gs = [g for g, _ in synth.planted_group(5, 500, 6000, 17)]
    gs.append(synth.rmat(11, 8 << 11, 44))                        # skewed degrees
    gs.append(synth.EdgeList(7, np.array([0, 2], np.uint32), np.array([1, 3], np.uint32),
                             np.array([5, 1], np.uint32)))         # tiny, converges at once
    gs.append(synth.EdgeList(4, np.zeros(0, np.uint32), np.zeros(0, np.uint32),
                             np.zeros(0, np.uint32)))             # no edges
    return gs


def group_pair(dfl, orc, gs, **kw):
    csrs = [(g.n, *synth.to_csr(g)) for g in gs]
    opt = dfl.default_options(**kw)
    grp = dfl.DflGroup(csrs, options=opt, stream=_stream())
    orcs = []
    for n, off, idx, w in csrs:
        o = orc.Oracle(n, off, idx, w)
        o.set_options(**{k: v for k, v in kw.items() if k in ("max_iterations", "max_passes", "substeps",
                                                                "tau_agg")})
        orcs.append(o)
    return grp, orcs


def same_group(grp, orcs):
    K, S, _ = grp.weights()
    start = 0
    for g, o in enumerate(orcs):
        n = grp.sizes[g]
        C = grp.graph_membership(g)
        Co = o.membership()
        assert np.array_equal(C, Co), f"graph {g}: membership differs at {np.flatnonzero(C != Co)[:10]}"
        Ko, So, mo = o.weights()
        assert np.array_equal(K[start:start + n], Ko), f"graph {g}: K differs"
        assert np.array_equal(S[start:start + n], So), f"graph {g}: Sigma differs"
        q, num, den = grp.graph_modularity(g)
        qo, numo, deno = o.modularity()
        assert (num, den) == (numo, deno), f"graph {g}: modularity differs"
        assert abs(q - qo) <= 1e-12 * max(1.0, abs(qo))
        so, sg = o.stats(), grp.graph_stats(g)
        assert sg["passes"] == so["passes"] and sg["iterations"] == so["iterations"], f"graph {g}"
        start += n


@pytest.mark.parametrize("graph", [True, False])
def test_group_matches_each_graph_alone(dfl, orc, graph):
    gs = group_graphs()
    grp, orcs = group_pair(dfl, orc, gs, flags=32 if graph else 4)
    grp.static()
    for o in orcs:
        o.static()
    same_group(grp, orcs)
    streams = [synth.BatchStream(g, 60 + k) if g.m >= 8 else None for k, g in enumerate(gs)]
    for t, frac in enumerate([1e-3, 1e-2, 5e-2, 1e-2]):
        mode = [2, 2, 1, 0][t]
        dels, ins = [], []
        for k, g in enumerate(gs):
            if streams[k] is None:
                dels.append(np.zeros((0, 3), np.uint32))
                ins.append(np.zeros((0, 3), np.uint32))
                continue
            d, i = streams[k].next(max(1, int(frac * g.m)), w_max=16)
            dels.append(d)
            ins.append(i)
        grp.apply_batches(dels, ins)
        for o, d, i in zip(orcs, dels, ins):
            assert o.apply_batch(d, i) == 0
        grp.update(mode)
        for o in orcs:
            o.update(mode)
        same_group(grp, orcs)


def test_group_substeps_and_passes(dfl, orc):
    gs = [g for g, _ in synth.planted_group(4, 2000, 20000, 23)]
    for substeps, passes in [(1, 10), (8, 2)]:
        grp, orcs = group_pair(dfl, orc, gs, substeps=substeps, max_passes=passes)
        grp.static()
        for o in orcs:
            o.static()
        same_group(grp, orcs)


def test_group_device_batch_and_autotune(dfl, orc):
    import torch
    gs = [g for g, _ in synth.planted_group(6, 1000, 30000, 29)]
    grp, orcs = group_pair(dfl, orc, gs)
    grp.static()
    for o in orcs:
        o.static()
    streams = [synth.BatchStream(g, 80 + k) for k, g in enumerate(gs)]
    for t in range(3):
        pairs = [s.next(max(1, int(1e-3 * g.m)), w_max=16) for s, g in zip(streams, gs)]
        d = np.concatenate([p[0] for p in pairs])
        i = np.concatenate([p[1] for p in pairs])
        doff = np.concatenate([[0], np.cumsum([p[0].shape[0] for p in pairs])]).astype(np.uint64)
        ioff = np.concatenate([[0], np.cumsum([p[1].shape[0] for p in pairs])]).astype(np.uint64)
        dd = torch.from_numpy(d.view(np.int32)).cuda()
        di = torch.from_numpy(i.view(np.int32)).cuda()
        grp.apply_batches((dd, doff), (di, ioff))
        for o, p in zip(orcs, pairs):
            assert o.apply_batch(*p) == 0
        if t == 1:
            tuning, ms = grp.autotune(2, reps=2)
            assert ms > 0
        grp.update(2)
        for o in orcs:
            o.update(2)
        same_group(grp, orcs)


def test_group_bad_batch_changes_nothing(dfl, orc):
    gs = [g for g, _ in synth.planted_group(3, 500, 2000, 31)]
    grp, orcs = group_pair(dfl, orc, gs)
    grp.static()
    for o in orcs:
        o.static()
    C0 = grp.membership()
    K0, S0, _ = grp.weights()
    n1 = gs[1].n
    dels = [np.zeros((0, 3), np.uint32)] * 3
    ins = [np.array([[0, 1, 1]], np.uint32), np.array([[0, n1, 1]], np.uint32),
           np.array([[0, 1, 1]], np.uint32)]
    assert grp.apply_batches(dels, ins, check=False) == -1  # id beyond graph 1's size
    ins[1] = np.array([[0, 0, 1]], np.uint32)
    assert grp.apply_batches(dels, ins, check=False) == -1  # self-loop
    e = gs[2]
    dels[2] = np.array([[int(e.u[0]), int(e.v[0]), int(e.w[0]) + 1]], np.uint32)
    ins[1] = np.array([[0, 1, 1]], np.uint32)
    assert grp.apply_batches(dels, ins, check=False) == -2  # more weight than present
    K1, S1, _ = grp.weights()
    assert np.array_equal(C0, grp.membership())
    assert np.array_equal(K0, K1) and np.array_equal(S0, S1)
    grp.update(2)
    for o in orcs:
        o.update(2)
    same_group(grp, orcs)
    with pytest.raises(dfl.DflError) as ex:
        dfl.Dfl.static(grp)  # single-graph calls are refused on a group
    assert ex.value.code == -7


def test_group_with_a_graph_of_no_vertices(dfl, orc):
    gs = [g for g, _ in synth.planted_group(2, 500, 3000, 37)]
    empty = synth.EdgeList(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    csrs = [(g.n, *synth.to_csr(g)) for g in [gs[0], empty, gs[1]]]
    grp = dfl.DflGroup(csrs, stream=_stream())
    orcs = [orc.Oracle(n, off, idx, w) for n, off, idx, w in (csrs[0], csrs[2])]
    grp.static()
    for o in orcs:
        o.static()
    assert grp.graph_membership(1).shape == (0,)
    assert grp.graph_modularity(1)[1:] == (0, 0)
    for g, o in ((0, orcs[0]), (2, orcs[1])):
        assert np.array_equal(grp.graph_membership(g), o.membership())
        assert grp.graph_modularity(g)[1:] == o.modularity()[1:]


def test_group_recomputed_auxiliary_information(dfl, orc):
    """A group with DFL_FLAG_RECOMPUTE_AUX (K, every graph's 2m and Sigma
    recomputed before each update) gives each graph the oracle's state."""
    gs = [g for g, _ in synth.planted_group(3, 2000, 20000, 31)]
    grp, orcs = group_pair(dfl, orc, gs, flags=128)
    grp.static()
    for o in orcs:
        o.static()
    streams = [synth.BatchStream(g, 70 + k) for k, g in enumerate(gs)]
    for mode in (2, 1):
        batches = [st.next(max(1, g.m // 500), w_max=16) for st, g in zip(streams, gs)]
        grp.apply_batches([b[0] for b in batches], [b[1] for b in batches])
        for o, (d, i) in zip(orcs, batches):
            assert o.apply_batch(d, i) == 0
        grp.update(mode)
        for o in orcs:
            o.update(mode)
        same_group(grp, orcs)


def test_group_of_graphs_each_near_the_2m_limit(dfl, orc):
    """Two graphs whose own 2m is just below 2^32 (the union's is above):
    each graph is checked against its own bound and scored with its own 2m."""
    rng = np.random.default_rng(31)
    gs = []
    for k in range(2):
        base = synth.planted_partition(1500, 15, 0.2, 10, 1, 40 + k)
        w = rng.integers(1, 400000, base.m).astype(np.uint64)
        scale = ((1 << 32) - (1 << 21)) / (2.0 * float(w.sum()))
        w = np.maximum(1, (w * scale).astype(np.uint64)).astype(np.uint32)
        gs.append(synth.EdgeList(base.n, base.u, base.v, w))
    grp, orcs = group_pair(dfl, orc, gs)
    grp.static()
    for o in orcs:
        o.static()
    same_group(grp, orcs)
    batches = []
    for g in gs:
        x = rng.integers(0, g.n, (12, 2))
        x = x[x[:, 0] != x[:, 1]]
        ins = np.concatenate([x, rng.integers(1, 30000, (x.shape[0], 1))], 1).astype(np.uint32)
        batches.append((np.zeros((0, 3), np.uint32), ins))
    grp.apply_batches([b[0] for b in batches], [b[1] for b in batches])
    for o, (d, i) in zip(orcs, batches):
        assert o.apply_batch(d, i) == 0
    grp.update(2)
    for o in orcs:
        o.update(2)
    same_group(grp, orcs)
