"""The seeded input generators produce the workloads they state: simple
undirected graphs of the stated sizes and structure, symmetric CSR, and
batches that are valid when they arrive.  Bounds on random quantities are
five standard deviations or looser."""
import math

import numpy as np
import pytest

import synth


def simple_undirected(g):
    """Each edge once with u < v, ids below n, no duplicates, weights >= 1."""
    assert g.u.dtype == g.v.dtype == g.w.dtype == np.uint32
    assert np.all(g.u < g.v) and (g.m == 0 or int(g.v.max()) < g.n)
    key = (g.u.astype(np.uint64) << np.uint64(32)) | g.v.astype(np.uint64)
    assert np.unique(key).shape[0] == g.m
    assert np.all(g.w >= 1)


def test_rmat_sizes_and_skew():
    g = synth.rmat(14, 8 << 14, 2)
    simple_undirected(g)
    assert g.n == 1 << 14 and g.m == 8 << 14 and np.all(g.w == 1)
    deg = np.bincount(np.concatenate([g.u, g.v]).astype(np.int64), minlength=g.n)
    # a heavy tail: the largest degree is over 100x the mean, the top 1% of
    # vertices hold over a fifth of the arcs, and many vertices are isolated
    assert deg.max() > 100 * deg.mean()
    assert np.sort(deg)[::-1][: g.n // 100].sum() > 0.2 * deg.sum()
    assert (deg == 0).sum() > 0.1 * g.n
    again = synth.rmat(14, 8 << 14, 2)
    assert np.array_equal(g.u, again.u) and np.array_equal(g.v, again.v)
    other = synth.rmat(14, 8 << 14, 3)
    assert not np.array_equal(g.u, other.u)


def test_sbm_block_structure():
    """10,000 vertices, 50 blocks of 200, p_in 0.02, p_out 0.0002: about
    19,900 edges inside blocks and 9,800 between them."""
    n, blocks, p_in, p_out = 10_000, 50, 0.02, 0.0002
    g = synth.sbm(n, blocks, p_in, p_out, 1)
    simple_undirected(g)
    s = n // blocks
    intra = int(((g.u // s) == (g.v // s)).sum())
    pairs_in = blocks * s * (s - 1) // 2
    pairs_out = n * (n - 1) // 2 - pairs_in
    for got, pairs, p in ((intra, pairs_in, p_in), (g.m - intra, pairs_out, p_out)):
        mean = pairs * p
        assert abs(got - mean) <= 5 * math.sqrt(pairs * p * (1 - p))


def test_planted_partition_mixing_and_weights():
    n, blocks, mu, deg, w_max = 20_000, 40, 0.3, 16, 16
    g = synth.planted_partition(n, blocks, mu, deg, w_max, 7)
    simple_undirected(g)
    block_of = np.repeat(np.arange(blocks), n // blocks)
    assert g.m == round(n * (1 - mu) * deg / 2) + round(n * mu * deg / 2)
    assert abs(float((block_of[g.u] != block_of[g.v]).mean()) - mu) < 1e-3
    assert g.w.min() == 1 and g.w.max() == w_max
    counts = np.bincount(g.w, minlength=w_max + 1)[1:]
    assert np.all(np.abs(counts - g.m / w_max) <= 5 * math.sqrt(g.m / w_max))


def test_to_csr_is_symmetric_and_sorted():
    g = synth.planted_partition(3000, 10, 0.2, 8, 5, 2)
    off, idx, w = synth.to_csr(g)
    assert off.dtype == np.uint64 and idx.dtype == np.uint32 and w.dtype == np.uint32
    assert off[0] == 0 and off[-1] == 2 * g.m and np.all(np.diff(off.astype(np.int64)) >= 0)
    rows = np.repeat(np.arange(g.n, dtype=np.uint64), np.diff(off.astype(np.int64)))
    fwd = (rows << np.uint64(32)) | idx.astype(np.uint64)
    assert np.all(np.diff(fwd.astype(np.int64)) > 0)  # sorted rows, no duplicate arcs
    back = (idx.astype(np.uint64) << np.uint64(32)) | rows
    order = np.argsort(back)
    assert np.array_equal(back[order], fwd) and np.array_equal(w[order], w)  # (j, i) has (i, j)'s weight
    ref = {(int(a), int(b)): int(c) for a, b, c in zip(g.u, g.v, g.w)}
    for k in range(0, 2 * g.m, 97):
        i, j = int(rows[k]), int(idx[k])
        assert ref[(min(i, j), max(i, j))] == int(w[k])


def test_batch_stream_is_valid_when_applied():
    """80/20 insertions/deletions; every deletion removes a base edge still
    present (no base edge is deleted twice across the stream); insertions
    join distinct vertices with weights in 1..w_max."""
    g = synth.rmat(10, 4 << 10, 5)
    bs = synth.BatchStream(g, 9)
    present = set(zip(g.u.tolist(), g.v.tolist()))
    deleted = set()
    for size, w_max in ((1, 1), (10, 1), (333, 4), (1000, 16)):
        d, i = bs.next(size, w_max=w_max)
        assert i.shape == (round(0.8 * size), 3) and d.shape == (size - round(0.8 * size), 3)
        for u, v, w in d.tolist():
            assert w == 0 and (u, v) in present and (u, v) not in deleted
            deleted.add((u, v))
        assert np.all(i[:, 0] != i[:, 1]) and int(i[:, :2].max(initial=0)) < g.n
        assert np.all((i[:, 2] >= 1) & (i[:, 2] <= w_max))
    with pytest.raises(ValueError):
        bs.next(10 * g.m)


def test_edge_pool_deletions_exist_in_the_evolved_graph():
    """Each deletion removes weight that the graph holds after every earlier
    batch of the same pool (base edges plus earlier insertions)."""
    g = synth.rmat(9, 4 << 9, 6)
    pool = synth.EdgePool(g, 3)
    held = {}
    for u, v in zip(g.u.tolist(), g.v.tolist()):
        held[(u, v)] = held.get((u, v), 0) + 1
    for size in (5, 50, 500, 3000, 3000):
        d, i = pool.next(size)
        assert i.shape[0] == round(0.8 * size)
        for u, v, w in d.tolist():
            assert u < v and w >= 1 and held.get((u, v), 0) >= w
            held[(u, v)] -= w
        for u, v, _ in i.tolist():
            key = (min(u, v), max(u, v))
            held[key] = held.get(key, 0) + 1
        assert sum(held.values()) == pool.size


def test_poisson_requests_rate_and_sizes():
    rate, dur, lo, hi = 2000.0, 5.0, 10, 10**6
    r = synth.poisson_requests(8, rate, dur, lo, hi, 500)
    assert abs(len(r) - rate * dur) <= 5 * math.sqrt(rate * dur)
    t = np.array([x[0] for x in r])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < dur
    graphs = np.bincount([x[1] for x in r], minlength=8)
    assert np.all(np.abs(graphs - len(r) / 8) <= 5 * math.sqrt(len(r) / 8))
    sizes = np.array([x[2] for x in r])
    assert sizes.min() >= lo and sizes.max() <= hi
    # log-uniform: the logarithm is uniform, so its median is the midpoint
    assert abs(np.median(np.log(sizes)) - 0.5 * (math.log(lo) + math.log(hi))) < 0.25


def test_planted_group_parameters_of_the_64_graph_workload():
    """64 graphs, n log-uniform in [1e4, 1e6] (15,696,720 vertices in all),
    blocks in [20, 2000] and at most n / 32, mixing in [0.1, 0.5]."""
    p = synth.planted_group_params(64, 1e4, 1e6, 4)
    assert len(p) == 64 and sum(n for n, _, _, _ in p) == 15_696_720
    for n, blocks, mu, _ in p:
        assert 1e4 <= n <= 1e6
        assert blocks <= max(2, n // 32) and (blocks >= 20 or blocks == n // 32)
        assert 0.1 <= mu <= 0.5
    logs = np.log([n for n, _, _, _ in p])
    # uniform on [log 1e4, log 1e6]: mean log 1e5, sd (log 100)/sqrt(12)/sqrt(64)
    assert abs(logs.mean() - math.log(1e5)) <= 5 * math.log(100) / math.sqrt(12 * 64)
