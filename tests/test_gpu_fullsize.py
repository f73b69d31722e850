"""Full-size parity on the benchmark workload: R-MAT with 2^22 vertices and
33,554,432 edges, static Louvain, then DF updates of 1e-3 and 1e-5 x |E| edge
batches, in the launch configuration the benchmark times (side stream, host
launches).  The oracle runs the same steps; membership, K, Sigma, 2m, modularity
and the first-pass trace must match exactly.  About two minutes (most of it
in the CPU oracle)."""
import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_rmat22_static_and_df_batches_match_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    import paper_2404_19634_gb300 as dfl
    dfl.build()
    oracle.build()
    g = synth.rmat(22, 33_554_432, 2)
    off, idx, w = synth.to_csr(g)
    s = torch.cuda.Stream()
    a = dfl.Dfl(g.n, off, idx, w, stream=s)
    b = oracle.Oracle(g.n, off, idx, w)
    a.static()
    b.static()
    stream = synth.BatchStream(g, 200)

    def check():
        assert np.array_equal(a.membership(), b.membership())
        Ka, Sa, ma = a.weights()
        Kb, Sb, mb = b.weights()
        assert ma == mb and np.array_equal(Ka, Kb) and np.array_equal(Sa, Sb)
        qa, na, da = a.modularity()
        qb, nb, db = b.modularity()
        assert (na, da) == (nb, db) and abs(qa - qb) <= 1e-12
        assert a.trace() == b.trace()
        sa, sb = a.stats(), b.stats()
        assert sa["iterations"] == sb["iterations"]
        assert sa["affected_ever"] == sb["affected_ever"]

    check()
    for size in (33_554, 335, 33_554):
        d, i = stream.next(size)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        a.update(dfl.DF)
        b.update(oracle.DF)
        check()
    assert a.num_arcs() == int(b.graph()[0][-1])


def test_temporal_stream_2m_vertices_matches_oracle():
    """Temporal workload at full size: 2,000,000 vertices, 30,000,000
    preferential-attachment interactions with 30% repeats; the first 90% form
    the base graph (multiplicity = weight, tau_agg = 1 as for the paper's
    temporal graphs), then batches of 1e-5 and 1e-4 x 30M insertions with as
    many expiries of the oldest interactions, each updated with DF."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    import paper_2404_19634_gb300 as dfl
    dfl.build()
    oracle.build()
    n, steps = 2_000_000, 30_000_000
    src, dst = synth.temporal_pa_stream_vec(n, steps, 0.3, 3)
    base_end = steps * 9 // 10
    g = synth.temporal_edges(src[:base_end], dst[:base_end], n)
    off, idx, w = synth.to_csr(g)
    s = torch.cuda.Stream()
    a = dfl.Dfl(g.n, off, idx, w, options=dfl.default_options(tau_agg=1.0), stream=s)
    b = oracle.Oracle(g.n, off, idx, w)
    b.set_options(tau_agg=1.0)
    a.static()
    b.static()

    def check():
        assert np.array_equal(a.membership(), b.membership())
        Ka, Sa, ma = a.weights()
        Kb, Sb, mb = b.weights()
        assert ma == mb and np.array_equal(Ka, Kb) and np.array_equal(Sa, Sb)
        qa, na, da = a.modularity()
        qb, nb, db = b.modularity()
        assert (na, da) == (nb, db) and abs(qa - qb) <= 1e-12
        assert a.trace() == b.trace()
        assert a.stats()["iterations"] == b.stats()["iterations"]

    check()
    start, end = 0, base_end
    for size in (300, 3000, 300, 3000):
        dels, ins = synth.window_batch(src, dst, start, end, size)
        start += size
        end += size
        assert a.apply_batch(dels, ins) == 0 and b.apply_batch(dels, ins) == 0
        a.update(dfl.DF)
        b.update(oracle.DF)
        check()
    assert a.num_arcs() == int(b.graph()[0][-1])


def test_group_64_graphs_sampled_against_oracle():
    """The batched workload at full size: 64 planted-partition graphs (n
    log-uniform in [1e4, 1e6], 15.7 M vertices in total) in one group, static
    Louvain, then one DF step with a 1e-4 x |E_g| batch per graph.  The oracle
    runs four of the graphs alone (the smallest, the largest and two between);
    each must match exactly, including its pass and iteration counts."""
    import multiprocessing as mp
    import os

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    import paper_2404_19634_gb300 as dfl
    dfl.build()
    oracle.build()
    G = 64
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        made = pool.starmap(synth.planted_group_member, [(k, G, 1e4, 1e6, 4) for k in range(G)])
    graphs = [g for g, _ in made]
    csrs = [c for _, c in made]
    s = torch.cuda.Stream()
    grp = dfl.DflGroup(csrs, stream=s)
    grp.static()
    streams = [synth.BatchStream(g, 500 + k) for k, g in enumerate(graphs)]
    batches = [st.next(max(1, int(round(1e-4 * g.m))), w_max=16) for st, g in zip(streams, graphs)]
    grp.apply_batches([b[0] for b in batches], [b[1] for b in batches])
    grp.update(dfl.DF)
    K, S, _ = grp.weights()
    starts = np.concatenate([[0], np.cumsum([g.n for g in graphs])])
    order = np.argsort([g.n for g in graphs])
    for k in (order[0], order[G // 3], order[2 * G // 3], order[-1]):
        n, off, idx, w = csrs[k]
        o = oracle.Oracle(n, off, idx, w)
        o.static()
        assert o.apply_batch(*batches[k]) == 0
        o.update(oracle.DF)
        assert np.array_equal(grp.graph_membership(k), o.membership()), f"graph {k}: membership"
        Ko, So, _ = o.weights()
        assert np.array_equal(K[starts[k]:starts[k + 1]], Ko) and np.array_equal(S[starts[k]:starts[k + 1]], So)
        q, num, den = grp.graph_modularity(k)
        qo, numo, deno = o.modularity()
        assert (num, den) == (numo, deno) and abs(q - qo) <= 1e-12
        so, sg = o.stats(), grp.graph_stats(k)
        assert sg["passes"] == so["passes"] and sg["iterations"] == so["iterations"]


def test_serving_8_graphs_sampled_against_oracle():
    """The serving workload at full size: 8 resident R-MAT graphs (2^18 to
    2^23 vertices, 8 edges per vertex) and the Poisson request log of the
    bench (2,000 requests/s over 0.5 s, batches log-uniform in [10, 1e6]
    edges), served with coalescing.  The oracle replays the smallest graph's
    requests with the same grouping: every result of that graph (exact
    modularity numerator and denominator) and its final membership must
    match."""
    import multiprocessing as mp
    import os
    import sys

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    import paper_2404_19634_gb300 as dfl
    from paper_2404_19634_gb300 import serve
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dfl.build()
    oracle.build()
    with mp.get_context("spawn").Pool(min(len(bench.SERVE_SCALES), os.cpu_count() or 1)) as pool:
        made = pool.map(bench._serve_graph, range(len(bench.SERVE_SCALES)))
    graphs = [g for g, _ in made]
    csrs = [c for _, c in made]
    del made
    pools = [synth.EdgePool(g, 400 + k) for k, g in enumerate(graphs)]
    sched = synth.poisson_requests(len(graphs), bench.SERVE_RATE, 0.5, *bench.SERVE_SIZES, seed=500)
    reqs = serve.make_requests(pools, sched)
    srv = serve.Server.from_graphs(csrs)
    res = srv.serve(reqs, coalesce=True)
    final0 = srv.handles[0].membership().copy()
    srv.close()
    assert len(res.groups) < len(reqs)
    by_id = {r.rid: r for r in reqs}
    o = oracle.Oracle(*csrs[0])
    o.static()
    checked = 0
    for g, ids in res.groups:
        if g != 0:
            continue
        for i in ids:
            assert o.apply_batch(by_id[i].dels, by_id[i].ins) == 0
        o.update(2)  # DF
        q, num, den = o.modularity()
        rec = res.records[ids[-1]]
        assert (rec.num, rec.den) == (num, den), f"request {ids[-1]}"
        checked += len(ids)
    assert checked > 50  # requests of graph 0, in a few coalesced updates
    assert np.array_equal(final0, o.membership())
