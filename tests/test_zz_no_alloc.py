"""dfl_modularity_csr_noalloc: the allocation-free modularity entry point.

It is for callers that cannot allocate device memory while it runs (their
device memory belongs to another allocator, or cudaMalloc/cudaFree would
stall a latency-critical path), so it keeps its scratch in a fixed array
inside the library.  These checks compare it, through the C ABI, with
dfl_modularity on a handle holding the same graph and membership, on two
calls in a row (the second must not see the first call's leftovers).
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


def test_noalloc_matches_handle_modularity_twice(dfl):
    import torch
    g = synth.sbm(6000, 30, 0.02, 0.001, 77)
    off, idx, w = synth.to_csr(g)
    h = dfl.Dfl(g.n, off, idx, w)
    rng = np.random.default_rng(3)
    memberships = [rng.integers(0, 40, g.n).astype(np.uint32),          # many small labels
                   np.repeat(np.arange(30), 200).astype(np.uint32)]   # the planted blocks
    doff, didx, dw = to_dev(off), to_dev(idx), to_dev(w)
    for C in memberships:
        h.set_membership(C)
        q_ref, num_ref, den_ref = h.modularity()
        rc, q, num, den = dfl.modularity_csr_noalloc(g.n, doff, didx, dw, to_dev(C))
        torch.cuda.synchronize()
        assert rc == 0
        assert (num, den) == (num_ref, den_ref)
        assert abs(q - q_ref) <= 1e-12 * max(1.0, abs(q_ref))


def test_noalloc_rejects_sizes_beyond_its_scratch(dfl):
    n = dfl.NOALLOC_MAX_VERTICES + 1
    # the size check comes before any device access
    rc, _, _, _ = dfl.modularity_csr_noalloc(n, np.zeros(2, np.uint64), np.zeros(1, np.uint32),
                                             np.zeros(1, np.uint32), np.zeros(1, np.uint32))
    assert rc == -1
