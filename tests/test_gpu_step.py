"""dfl_step: a batch apply and the DF update queued behind it in one call.

The step must equal dfl_apply_batch + dfl_update, and hence the oracle's
apply + update, bit for bit: graph, K, Sigma, 2m, membership, modularity,
pass and iteration counts, affected counts and the first-pass trace.  The
batch's validation is read only after the update's first iteration has run,
so these cases also cover what the step does when the batch is not written:
an invalid batch leaves everything as it was (earlier pending batches
included), and a batch that needs a larger arc pool or the sort-based path
is applied again by the two-call path.
"""
import numpy as np
import pytest

import synth
from test_gpu_parity import pair, same_graph, same_state

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


def step_both(a, b, d, i, mode=2):
    assert a.step(d, i, mode) == 0
    assert b.apply_batch(d, i) == 0
    b.update(mode)


@pytest.mark.parametrize("flags", [32, 4, 16])  # graph replay, host launches, persistent kernel
def test_step_stream_matches_oracle(dfl, orc, flags):
    """R-MAT 2^13, batches from 3 to 3,000 edges: the single-block apply,
    the multi-kernel apply, host-launched and replayed iterations."""
    g = synth.rmat(13, 8 << 13, 41)
    a, b = pair(dfl, orc, g, graph=bool(flags & 32), flags=flags & ~36)
    a.static()
    b.static()
    bs = synth.BatchStream(g, 42)
    for size in (3, 300, 600, 3000, 40, 2000):
        d, i = bs.next(size)
        step_both(a, b, d, i)
        same_graph(a, b)
        same_state(a, b)


def test_step_other_modes_and_empty(dfl, orc):
    g = synth.sbm(4000, 20, 0.02, 0.001, 43)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    bs = synth.BatchStream(g, 44)
    for mode in (0, 1, 2):
        d, i = bs.next(500)
        step_both(a, b, d, i, mode)
        same_state(a, b)
    # an empty batch is an update of what is pending (nothing)
    z = np.zeros((0, 3), np.uint32)
    step_both(a, b, z, z)
    same_state(a, b)


def test_step_invalid_batch_changes_nothing(dfl, orc):
    g = synth.rmat(12, 8 << 12, 45)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    bs = synth.BatchStream(g, 46)
    # a batch applied on its own stays pending across the failed steps
    d0, i0 = bs.next(700)
    assert a.apply_batch(d0, i0) == 0 and b.apply_batch(d0, i0) == 0
    before = (a.graph(), a.weights(), a.membership())
    d1, i1 = bs.next(2000)
    bad_label = i1.copy()
    bad_label[5, 1] = g.n + 3                    # a vertex id >= n
    missing = np.array([[0, 1, 0]], np.uint32)   # (absent unless the graph has it)
    off, idx, _ = synth.to_csr(g)
    if 1 in idx[off[0]:off[1]]:
        missing = np.array([[0, g.n - 1, 0]], np.uint32)
    huge = i1.copy()
    huge[7, 2] = 0xFFFFFFFF                      # weight overflow with a repeat of the pair
    huge = np.concatenate([huge, huge[7:8]])
    for dd, ii, code in ((d1, bad_label, -1), (missing, i1, -2), (d1, huge, -3)):
        for n_small in (False, True):  # the multi-kernel apply and the single-block one
            if n_small:
                dd2, ii2 = dd[:10], ii[:200] if code != -3 else np.concatenate([ii[:100], ii[7:8]])
                if code == -1:
                    ii2 = ii2.copy()
                    ii2[5, 1] = g.n + 3
            else:
                dd2, ii2 = dd, ii
            rc = a.step(dd2, ii2, check=False)
            assert rc == code, (rc, code, n_small)
            after = (a.graph(), a.weights(), a.membership())
            for x, y in zip(before[0], after[0]):
                assert np.array_equal(x, y)
            for x, y in zip(before[1], after[1]):
                assert np.array_equal(np.asarray(x), np.asarray(y))
            assert np.array_equal(before[2], after[2])
    # the pending batch is still pending: the next step updates for both
    step_both(a, b, d1, i1)
    same_graph(a, b)
    same_state(a, b, stats=False)
    assert np.array_equal(a.membership(), b.membership())


def test_step_pool_growth_and_sorted_path(dfl, orc):
    """After dfl_compact the arc pool has little room: a hub batch relocates
    rows beyond it (the step's apply settles as 'grow, then again').  A row
    gaining more than 4,096 arcs takes the sort-based apply."""
    g = synth.rmat(13, 6 << 13, 47)
    a, b = pair(dfl, orc, g)
    a.static()
    b.static()
    a.compact()
    rng = np.random.default_rng(48)
    for hub_edges in (3000, 5000):
        hub = np.stack([np.full(hub_edges, 7, np.uint32),
                        rng.choice(np.arange(8, g.n, dtype=np.uint32), hub_edges, replace=False),
                        np.ones(hub_edges, np.uint32)], axis=1)
        z = np.zeros((0, 3), np.uint32)
        step_both(a, b, z, hub)
        same_graph(a, b)
        same_state(a, b)
