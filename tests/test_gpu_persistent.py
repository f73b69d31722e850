"""The persistent iteration kernel (DFL_FLAG_PERSISTENT) against the oracle.

With the flag every local-moving iteration is one cooperative launch whose
blocks take work units from a counter and meet at grid barriers between
sub-steps.  The decisions are the same exact integer computations as in the
per-bin kernels, so the state must match the oracle bit for bit on every
degree class: segments, warp tables, block tables (shared and global) and
chunked giant vertices, with and without the part blocks.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

PERSISTENT = 16  # DFL_FLAG_PERSISTENT


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


def pair(dfl, orc, g, substeps=4, tau_agg=0.8, **kw):
    import torch
    off, idx, w = synth.to_csr(g)
    opt = dfl.default_options(substeps=substeps, tau_agg=tau_agg, flags=PERSISTENT, **kw)
    s = torch.cuda.Stream()
    _STREAMS.append(s)
    a = dfl.Dfl(g.n, off, idx, w, options=opt, stream=s)
    b = orc.Oracle(g.n, off, idx, w)
    b.set_options(substeps=substeps, tau_agg=tau_agg)
    return a, b


def ran_persistent(a):
    """Every local-moving iteration was one launch of the iteration kernel:
    no per-bin decide or commit launches were issued."""
    p = a.profile()
    assert p["move"]["launches"] == sum(a.stats()["iterations"]) > 0
    assert all(p[k]["launches"] == 0 for k in ("bin0", "bin1", "bin2", "bin3", "commit"))


def same_state(a, b, stats=True):
    Ca, Cb = a.membership(), b.membership()
    assert np.array_equal(Ca, Cb), f"membership differs at {np.flatnonzero(Ca != Cb)[:10]}"
    Ka, Sa, ma = a.weights()
    Kb, Sb, mb = b.weights()
    assert ma == mb and np.array_equal(Ka, Kb) and np.array_equal(Sa, Sb)
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


@pytest.mark.parametrize("substeps", [1, 2, 4, 8])
def test_rmat_stream(dfl, orc, substeps):
    g = synth.rmat(13, 8 << 13, 43)
    a, b = pair(dfl, orc, g, substeps=substeps)
    a.static()
    b.static()
    same_state(a, b)
    ran_persistent(a)
    stream = synth.BatchStream(g, 3)
    for t, size in enumerate([20, 300, 3000]):
        d, i = stream.next(size)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        a.update([2, 0, 1][t])
        b.update([2, 0, 1][t])
        same_state(a, b)


def test_hubs_in_every_bin(dfl, orc):
    """Hubs of degree ~300, ~5,000 and ~20,000 next to a planted partition."""
    rng = np.random.default_rng(8)
    n = 40000
    base = synth.planted_partition(n, 100, 0.2, 6, 1, 3)
    us, vs = [base.u], [base.v]
    for hub, deg in [(5, 300), (17, 5000), (123, 20000), (999, 9000)]:
        nb = rng.choice(n, deg, replace=False)
        nb = nb[nb != hub]
        us.append(np.full(nb.shape[0], hub, np.uint32))
        vs.append(nb.astype(np.uint32))
    u, v = np.concatenate(us), np.concatenate(vs)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = np.unique((lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64))
    g = synth.EdgeList(n, (key >> np.uint64(32)).astype(np.uint32),
                       (key & np.uint64(0xFFFFFFFF)).astype(np.uint32), np.ones(key.shape[0], np.uint32))
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    same_state(a, b)
    ran_persistent(a)
    stream = synth.BatchStream(g, 4)
    d, i = stream.next(2000)
    i = np.concatenate([i, np.array([[17, 9, 1], [123, 77, 2], [5, 31, 1]], np.uint32)])
    assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
    a.update(0)
    b.update(0)
    same_state(a, b)


def test_giant_vertex_with_part_blocks(dfl, orc):
    """Degree 20,000 with every neighbour in its own community: more than
    4,096 distinct communities send the vertex to the part blocks."""
    n = 20001
    ring = np.arange(1, n - 1, dtype=np.uint32)
    g = synth.EdgeList(n, np.concatenate([np.zeros(20000, np.uint32), ring]),
                       np.concatenate([np.arange(1, n, dtype=np.uint32), ring + 1]),
                       np.concatenate([np.ones(20000, np.uint32), (ring % 7 + 1).astype(np.uint32)]))
    for k in (1, 4):
        a, b = pair(dfl, orc, g, substeps=k)
        a.static()
        b.static()
        same_state(a, b)
        ran_persistent(a)


@pytest.mark.parametrize("tuning", [
    dict(bin_warp=32, bin_warp_hash=256, bin_block=4096, block_threads=256),
    dict(bin_warp=0, bin_warp_hash=0, bin_block=0, block_threads=256),      # all chunked
    dict(bin_warp=16, bin_warp_hash=128, bin_block=16384, block_threads=512),
    dict(bin_warp=4, bin_warp_hash=64, bin_block=1024, block_threads=128),
])
def test_tunings(dfl, orc, tuning):
    g = synth.rmat(13, 8 << 13, 41)
    a, b = pair(dfl, orc, g)
    a.set_tuning(**tuning)
    a.static()
    b.static()
    same_state(a, b)
    stream = synth.BatchStream(g, 7)
    for t, size in enumerate([50, 4000]):
        d, i = stream.next(size)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        a.update([2, 0][t])
        b.update([2, 0][t])
        same_state(a, b)


def test_group(dfl, orc):
    """Graphs of a group converge at different iterations; the persistent
    kernel skips finished graphs like the per-bin kernels do."""
    from test_gpu_group import group_graphs, group_pair, same_group
    gs = group_graphs()
    grp, orcs = group_pair(dfl, orc, gs, flags=PERSISTENT)
    grp.static()
    for o in orcs:
        o.static()
    same_group(grp, orcs)
    streams = [synth.BatchStream(g, 60 + k) if g.m >= 8 else None for k, g in enumerate(gs)]
    for t, frac in enumerate([1e-3, 5e-2]):
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
        grp.update([2, 0][t])
        for o in orcs:
            o.update([2, 0][t])
        same_group(grp, orcs)


def test_empty_batch_and_tiny_graphs(dfl, orc):
    g = synth.sbm(1000, 10, 0.08, 0.004, 23)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    empty = np.zeros((0, 3), np.uint32)
    assert a.apply_batch(empty, empty) == 0 and b.apply_batch(empty, empty) == 0
    a.update(2)
    b.update(2)
    same_state(a, b)
    assert a.stats()["affected_ever"] == 0
    e = synth.EdgeList(50, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    a, b = pair(dfl, orc, e)
    a.static()
    b.static()
    same_state(a, b)
    assert a.apply_batch(empty, np.array([[1, 2, 3]], np.uint32)) == 0
    b.apply_batch(empty, np.array([[1, 2, 3]], np.uint32))
    a.update(2)
    b.update(2)
    same_state(a, b)
