"""dfl_modularity_csr_noalloc: the allocation-free modularity entry point.

It is for callers that cannot allocate device memory while it runs (their
device memory belongs to another allocator, or cudaMalloc/cudaFree would
stall a latency-critical path), so it keeps its scratch in a fixed array
inside the library.  These checks call it through the C ABI and compare it
with dfl_modularity on a handle holding the same graph and membership and
with the CPU oracle's exact modularity numerator and denominator, on calls
in a row (a later call must not see an earlier call's leftovers, also when
the earlier one used more of the scratch), and check its error returns.
This file is collected last on purpose.
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


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    view = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)
    return torch.from_numpy(view).cuda()


def call(dfl, n, off, idx, w, C):
    import torch
    out = dfl.modularity_csr_noalloc(n, to_dev(off), to_dev(idx), to_dev(w), to_dev(C))
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_handle_and_oracle_twice(dfl, oracle_mod):
    g = synth.sbm(6000, 30, 0.02, 0.001, 77)
    off, idx, w = synth.to_csr(g)
    h = dfl.Dfl(g.n, off, idx, w)
    ref = oracle_mod.Oracle(g.n, off, idx, w)
    rng = np.random.default_rng(3)
    memberships = [rng.integers(0, 40, g.n).astype(np.uint32),          # many small labels
                   np.repeat(np.arange(30), 200).astype(np.uint32)]   # the planted blocks
    for C in memberships:
        h.set_membership(C)
        ref.set_membership(C)
        q_ref, num_ref, den_ref = h.modularity()
        q_orc, num_orc, den_orc = ref.modularity()
        rc, q, num, den = call(dfl, g.n, off, idx, w, C)
        assert rc == 0
        assert (num, den) == (num_ref, den_ref) == (num_orc, den_orc)
        assert abs(q - q_ref) <= 1e-12 * max(1.0, abs(q_ref))
        assert abs(q - q_orc) <= 1e-12 * max(1.0, abs(q_orc))


def test_noalloc_small_call_after_a_larger_one(dfl, oracle_mod):
    # the first call fills scratch entries the second call's n does not cover
    big = synth.sbm(20000, 40, 0.004, 0.0005, 5)
    small = synth.sbm(700, 7, 0.05, 0.004, 6)
    rng = np.random.default_rng(9)
    for g, labels in ((big, 19000), (small, 650), (big, 300), (small, 7)):
        off, idx, w = synth.to_csr(g)
        C = rng.integers(0, labels, g.n).astype(np.uint32)
        ref = oracle_mod.Oracle(g.n, off, idx, w)
        ref.set_membership(C)
        _, num_orc, den_orc = ref.modularity()
        rc, _, num, den = call(dfl, g.n, off, idx, w, C)
        assert rc == 0
        assert (num, den) == (num_orc, den_orc)


def test_noalloc_error_returns(dfl):
    g = synth.sbm(500, 5, 0.05, 0.005, 8)
    off, idx, w = synth.to_csr(g)
    C = np.zeros(g.n, np.uint32)
    # a label >= n
    bad = C.copy()
    bad[17] = g.n
    assert call(dfl, g.n, off, idx, w, bad)[0] == -1
    # a neighbour id >= n
    bidx = idx.copy()
    bidx[3] = g.n + 5
    assert call(dfl, g.n, off, bidx, w, C)[0] == -1
    # decreasing offsets (within the arrays)
    boff = off.copy()
    boff[10], boff[11] = boff[11], boff[10]
    if boff[10] != boff[11]:
        assert call(dfl, g.n, boff, idx, w, C)[0] == -1
    # 2m reaching 2^32: two arcs of weight 2^31
    two = (np.array([0, 1, 2], np.uint64), np.array([1, 0], np.uint32),
           np.array([1 << 31, 1 << 31], np.uint32))
    assert call(dfl, 2, *two, np.zeros(2, np.uint32))[0] == -3
    # and a valid call right after the failures still matches
    rc, _, num, den = call(dfl, g.n, off, idx, w, C)
    assert rc == 0 and num == 0 and den > 0  # one community: Q = 0


def test_noalloc_rejects_sizes_beyond_its_scratch(dfl):
    import torch
    n = dfl.NOALLOC_MAX_VERTICES + 1
    z64 = torch.zeros(2, dtype=torch.int64, device="cuda")
    z32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, _, _, _ = dfl.modularity_csr_noalloc(n, z64, z32, z32, z32)
    assert rc == -1
    # host buffers are refused by the binding: the C function reads device memory
    with pytest.raises(TypeError):
        dfl.modularity_csr_noalloc(4, np.zeros(5, np.uint64), np.zeros(1, np.uint32),
                                   np.zeros(1, np.uint32), np.zeros(4, np.uint32))
