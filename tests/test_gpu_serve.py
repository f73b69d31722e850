"""Serving loop on the GPU: every request's result (the exact modularity
numerator and denominator, and the membership, after the update that served
it) is the same when its graph is served alone, one update at a time, as in
the concurrent mix with other graphs; and coalesced groups equal the oracle
applying the same batches and one DF update per group."""
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


SCALES = [11, 12, 12, 13]


def workload(seed=7, rate=6000.0, duration=0.04, hi=4000):
    graphs = [synth.rmat(s, 8 << s, 100 + k) for k, s in enumerate(SCALES)]
    csrs = [(g.n, *synth.to_csr(g)) for g in graphs]
    from paper_2404_19634_gb300 import serve
    sched = synth.poisson_requests(len(graphs), rate, duration, 10, hi, seed)
    pools = [synth.EdgePool(g, 50 + k) for k, g in enumerate(graphs)]
    return csrs, serve.make_requests(pools, sched)


def same_records(a, b):
    for x, y in zip(a.records, b.records):
        assert x.rid == y.rid
        assert (x.num, x.den) == (y.num, y.den), f"request {x.rid}: modularity differs"
        assert np.array_equal(x.membership, y.membership), f"request {x.rid}: membership differs"


def test_mix_equals_alone(dfl):
    from paper_2404_19634_gb300 import serve
    csrs, reqs = workload()
    assert len(reqs) > 100
    srv = serve.Server.from_graphs(csrs, keep_membership=True)
    mix = srv.serve(reqs, coalesce=True)
    srv.close()
    assert len(mix.groups) < len(reqs)
    assert srv.peak["busy"] > 1, "updates of different graphs overlapped"
    # each graph alone, its own requests with the same grouping
    for g, csr in enumerate(csrs):
        mine = [r for r in reqs if r.graph == g]
        local = [serve.Request(r.rid, 0, r.arrival, r.dels, r.ins) for r in mine]
        groups = [(0, ids) for gg, ids in mix.groups if gg == g]
        one = serve.Server.from_graphs([csr], keep_membership=True)
        alone = one.replay(local, groups)
        one.close()
        sub = serve.ServeResult([mix.records[r.rid] for r in mine])
        same_records(sub, alone)


def test_overlap_without_coalescing_equals_serial(dfl):
    from paper_2404_19634_gb300 import serve
    csrs, reqs = workload(seed=8, rate=3000.0, duration=0.03)
    a_srv = serve.Server.from_graphs(csrs, keep_membership=True)
    a = a_srv.serve(reqs, coalesce=False)
    a_srv.close()
    b_srv = serve.Server.from_graphs(csrs, keep_membership=True)
    b = b_srv.serve_serial(reqs)
    b_srv.close()
    assert all(len(ids) == 1 for _, ids in a.groups)
    same_records(a, b)


def test_coalesced_groups_match_oracle(dfl, oracle_mod):
    from paper_2404_19634_gb300 import serve
    csrs, reqs = workload(seed=9, rate=8000.0, duration=0.02, hi=2000)
    srv = serve.Server.from_graphs(csrs, keep_membership=True)
    mix = srv.serve(reqs, coalesce=True)
    srv.close()
    by_id = {r.rid: r for r in reqs}
    for g, (n, off, idx, w) in enumerate(csrs):
        o = oracle_mod.Oracle(n, off, idx, w)
        o.static()
        for gg, ids in mix.groups:
            if gg != g:
                continue
            for i in ids:
                assert o.apply_batch(by_id[i].dels, by_id[i].ins) == 0
            o.update(2)  # DF
            q, num, den = o.modularity()
            rec = mix.records[ids[-1]]
            assert (rec.num, rec.den) == (num, den)
            assert abs(rec.q - q) <= 1e-12 * max(1.0, abs(q))
            assert np.array_equal(rec.membership, o.membership())


def test_periodic_static_refresh_matches_oracle(dfl, oracle_mod):
    """refresh_every=3: after every third update of a graph the server runs
    static Louvain on the current graph; the oracle replaying the same
    groups and refreshes gives every recorded result."""
    from paper_2404_19634_gb300 import serve
    csrs, reqs = workload(seed=12, rate=8000.0, duration=0.02, hi=2000)
    srv = serve.Server.from_graphs(csrs, keep_membership=True, refresh_every=3)
    mix = srv.serve(reqs, coalesce=True)
    srv.close()
    assert any(rec.refreshed for rec in mix.records)
    by_id = {r.rid: r for r in reqs}
    for g, (n, off, idx, w) in enumerate(csrs):
        o = oracle_mod.Oracle(n, off, idx, w)
        o.static()
        k = 0
        for gg, ids in mix.groups:
            if gg != g:
                continue
            for i in ids:
                assert o.apply_batch(by_id[i].dels, by_id[i].ins) == 0
            o.update(2)  # DF
            k += 1
            rec = mix.records[ids[-1]]
            assert rec.refreshed == (k % 3 == 0)
            if rec.refreshed:
                o.static()
            q, num, den = o.modularity()
            assert (rec.num, rec.den) == (num, den)
            assert np.array_equal(rec.membership, o.membership())
