"""Failure detection without a GPU fault.

Two host-side hooks make the failures happen:
  - DFL_FLAG_TEST_UNREACHABLE_BARRIER gives the persistent iteration kernel's
    grid barriers a wait that nothing completes and a poll limit of a few
    milliseconds: every block gives up and returns, and the call must come
    back with DFL_ERR_TIMEOUT, after which the context, the stream and the
    handle still work (nothing is left in flight);
  - dfl_test_fail_allocations(k) makes every device allocation after the
    next k fail as if the GPU were full: for every k up to the first success,
    dfl_create must return no handle, dfl_apply_batch must leave the graph,
    K, Sigma and 2m unchanged, and dfl_static must fail cleanly so that a
    later call starts over -- and what finally succeeds must equal the
    oracle.
No test traps, faults or hangs a GPU.
"""
import time

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
    yield mod
    mod.test_fail_allocations(-1)


def state(h):
    off, idx, w = h.graph()
    K, S, m2 = h.weights()
    return off, idx, w, K, S, m2


def same(a, b):
    return all(np.array_equal(x, y) if isinstance(x, np.ndarray) else x == y for x, y in zip(a, b))


def test_barrier_timeout_returns_and_everything_still_works(dfl, oracle_mod):
    import torch
    g = synth.sbm(3000, 15, 0.03, 0.002, 21)
    off, idx, w = synth.to_csr(g)
    stream = torch.cuda.Stream()
    opt = dfl.default_options(flags=dfl.FLAG_PERSISTENT | dfl.FLAG_TEST_UNREACHABLE_BARRIER)
    h = dfl.Dfl(g.n, off, idx, w, options=opt, stream=stream)
    t0 = time.perf_counter()
    with pytest.raises(dfl.DflError) as ei:
        h.static()
    assert ei.value.code == -6, ei.value  # DFL_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 20.0
    torch.cuda.synchronize()  # nothing of the failed call is left running
    # no communities after the failed run ...
    with pytest.raises(dfl.DflError) as ei:
        h.membership()
    assert ei.value.code == -7
    # ... until a static run on the same handle and stream, which matches the oracle
    h.set_options(dfl.default_options(flags=dfl.FLAG_PERSISTENT))
    h.static()
    ref = oracle_mod.Oracle(g.n, off, idx, w)
    ref.static()
    assert np.array_equal(h.membership(), ref.membership())
    assert h.modularity()[1:] == ref.modularity()[1:]
    # and the stream serves other work
    x = torch.arange(1000, device="cuda")
    with torch.cuda.stream(stream):
        y = (x * 2).sum()
    stream.synchronize()
    assert int(y) == 999000
    h.close()


def test_create_fails_cleanly_at_every_allocation(dfl, oracle_mod):
    import torch
    g = synth.sbm(2000, 10, 0.04, 0.003, 22)
    off, idx, w = synth.to_csr(g)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    h = None
    for k in range(400):
        dfl.test_fail_allocations(k)
        try:
            h = dfl.Dfl(g.n, off, idx, w)
        except dfl.DflError as e:
            assert e.code == -4, e  # DFL_ERR_NOMEM
            failures += 1
            continue
        finally:
            dfl.test_fail_allocations(-1)
        break
    assert h is not None and failures > 10
    h.static()
    ref = oracle_mod.Oracle(g.n, off, idx, w)
    ref.static()
    assert np.array_equal(h.membership(), ref.membership())
    h.close()
    torch.cuda.synchronize()
    # the failed creations left nothing allocated (allow for allocator slack)
    assert free0 - torch.cuda.mem_get_info()[0] < 64 << 20


def test_apply_batch_fails_cleanly_at_every_allocation(dfl, oracle_mod):
    g = synth.rmat(13, 8 << 13, 31)
    off, idx, w = synth.to_csr(g)
    h = dfl.Dfl(g.n, off, idx, w)
    h.static()
    ref = oracle_mod.Oracle(g.n, off, idx, w)
    ref.static()
    bs = synth.BatchStream(g, 32)
    # a first batch sizes the scratch; the second is larger, so it must grow it,
    # and it piles insertions onto a few rows so that rows are rebuilt
    d0, i0 = bs.next(200)
    assert h.apply_batch(d0, i0) == 0 and ref.apply_batch(d0, i0) == 0
    h.update(dfl.DF)
    ref.update(oracle_mod.DF)
    d1, i1 = bs.next(3000)
    rng = np.random.default_rng(5)
    hub = np.stack([np.zeros(600, np.uint32), rng.choice(np.arange(1, g.n, dtype=np.uint32), 600, replace=False),
                    np.ones(600, np.uint32)], axis=1)
    i1 = np.concatenate([i1, hub])
    before = state(h)
    failures = 0
    for k in range(200):
        dfl.test_fail_allocations(k)
        try:
            rc = h.apply_batch(d1, i1, check=False)
        finally:
            dfl.test_fail_allocations(-1)
        if rc == 0:
            break
        assert rc == -4, rc
        failures += 1
        assert same(state(h), before), f"state changed by a failed apply (k={k})"
    assert rc == 0 and failures > 0
    assert ref.apply_batch(d1, i1) == 0
    h.update(dfl.DF)
    ref.update(oracle_mod.DF)
    assert same(state(h), (*ref.graph(), *ref.weights()))
    assert np.array_equal(h.membership(), ref.membership())
    # the failed attempts left no residue for later batches either
    d2, i2 = bs.next(500)
    assert h.apply_batch(d2, i2) == 0 and ref.apply_batch(d2, i2) == 0
    h.update(dfl.DF)
    ref.update(oracle_mod.DF)
    assert np.array_equal(h.membership(), ref.membership())
    assert h.modularity()[1:] == ref.modularity()[1:]
    h.close()


def test_static_fails_cleanly_at_every_allocation(dfl, oracle_mod):
    # small limits put vertices and communities in every degree bin, so the
    # first static run allocates the largest-degree tables and aggregation's
    # giant-community tables as well
    g = synth.rmat(13, 8 << 13, 33)
    off, idx, w = synth.to_csr(g)
    h = dfl.Dfl(g.n, off, idx, w)
    h.set_tuning(bin_warp=8, bin_warp_hash=32, bin_block=96, block_threads=128)
    failures = 0
    for k in range(400):
        dfl.test_fail_allocations(k)
        try:
            h.static()
            ok = True
        except dfl.DflError as e:
            assert e.code == -4, e
            failures += 1
            ok = False
        finally:
            dfl.test_fail_allocations(-1)
        if ok:
            break
    assert ok and failures > 3
    assert h.stats()["passes"] >= 2  # the run that succeeded aggregated
    ref = oracle_mod.Oracle(g.n, off, idx, w)
    ref.static()
    assert np.array_equal(h.membership(), ref.membership())
    assert h.modularity()[1:] == ref.modularity()[1:]
    # an update that fails leaves no communities; static starts over
    bs = synth.BatchStream(g, 34)
    d, i = bs.next(300)
    assert h.apply_batch(d, i) == 0 and ref.apply_batch(d, i) == 0
    dfl.test_fail_allocations(0)
    try:
        failed = False
        try:
            h.update(dfl.ND)
        except dfl.DflError as e:
            failed = e.code == -4
    finally:
        dfl.test_fail_allocations(-1)
    if failed:  # (an update that needs no new buffer succeeds instead)
        with pytest.raises(dfl.DflError) as ei:
            h.modularity()
        assert ei.value.code == -7
        h.static()
        ref.static()
    else:
        ref.update(oracle_mod.ND)
    assert np.array_equal(h.membership(), ref.membership())
    h.close()


def test_step_fails_cleanly_at_every_allocation(dfl, oracle_mod):
    """dfl_step on a fresh handle: allocations fail either before the apply is
    enqueued (nothing changes) or after it, while local-moving sizes its
    buffers with the apply unsettled (the batch is applied, the communities
    are dropped as a failed dfl_update drops them).  Either way the handle
    recovers and matches the oracle."""
    import torch
    g = synth.rmat(13, 8 << 13, 35)
    off, idx, w = synth.to_csr(g)
    s = torch.cuda.Stream()
    opt = dfl.default_options(flags=32)  # graph replay: the update is queued behind the apply
    ref = oracle_mod.Oracle(g.n, off, idx, w)
    ref.static()
    bs = synth.BatchStream(g, 36)
    d, i = bs.next(3000)
    seen = set()
    for k in range(400):
        h = dfl.Dfl(g.n, off, idx, w, options=opt, stream=s)
        h.static()
        before = state(h)
        dfl.test_fail_allocations(k)
        try:
            rc = h.step(d, i, dfl.DF, check=False)
        finally:
            dfl.test_fail_allocations(-1)
        if rc == 0:
            break
        assert rc == -4, rc
        try:
            h.membership()
            kept = True
        except dfl.DflError as e:
            assert e.code == -7
            kept = False
        if kept:  # nothing of the batch was written
            seen.add("unchanged")
            assert same(state(h), before)
            assert h.step(d, i, dfl.DF) == 0
        else:  # the batch was applied, the update failed
            seen.add("applied")
            o2 = oracle_mod.Oracle(g.n, off, idx, w)
            o2.static()
            assert o2.apply_batch(d, i) == 0
            assert same(state(h)[:4], (*o2.graph(), o2.weights()[0]))
            h.static()
            o2.static()
            assert np.array_equal(h.membership(), o2.membership())
        h.close()
    else:
        raise AssertionError("dfl_step never succeeded")
    assert seen == {"unchanged", "applied"}  # failures before and after the enqueue
    assert ref.apply_batch(d, i) == 0
    ref.update(oracle_mod.DF)
    assert same(state(h), (*ref.graph(), *ref.weights()))
    assert np.array_equal(h.membership(), ref.membership())
    h.close()
