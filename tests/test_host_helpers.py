"""Host-side helpers that need no GPU: checkpoint files and the per-graph
generator of the batched workload."""
import numpy as np

import synth


def test_checkpoint_file_round_trip(tmp_path):
    import paper_2404_19634_gb300 as dfl
    g = synth.sbm(300, 6, 0.1, 0.01, 4)
    off, idx, w = synth.to_csr(g)
    ck = {"n": g.n, "offsets": off, "indices": idx, "weights": w,
          "membership": np.arange(g.n, dtype=np.uint32)[::-1].copy(),
          "tuning": {"bin_warp": 4, "bin_warp_hash": 64, "bin_block": 1024, "block_threads": 128}}
    path = str(tmp_path / "ck.npz")
    dfl.save_checkpoint(path, ck)
    back = dfl.load_checkpoint(path)
    assert back["n"] == ck["n"] and back["tuning"] == ck["tuning"]
    for k in ("offsets", "indices", "weights", "membership"):
        assert np.array_equal(back[k], ck[k]) and back[k].dtype == ck[k].dtype


def test_group_member_is_the_group_graph():
    whole = synth.planted_group(4, 2000, 20000, 9)
    for k in range(4):
        g, (n, off, idx, w) = synth.planted_group_member(k, 4, 2000, 20000, 9)
        ref = whole[k][0]
        assert g.n == ref.n == n
        assert np.array_equal(g.u, ref.u) and np.array_equal(g.v, ref.v) and np.array_equal(g.w, ref.w)
        o2, i2, w2 = synth.to_csr(ref)
        assert np.array_equal(off, o2) and np.array_equal(idx, i2) and np.array_equal(w, w2)
