"""Host-side helpers that need no GPU: checkpoint files and the per-graph
generator of the batched workload."""
import numpy as np
import pytest

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


class _FakeNvml:
    """Stands in for the NVML reader: a fixed sequence of (MHz, W, reason bits)."""

    def __init__(self, seq):
        self.seq = list(seq)
        self.k = 0
        self.max_mhz = 2070.0

    def sample(self):
        s = self.seq[min(self.k, len(self.seq) - 1)]
        self.k += 1
        return s


def test_clock_sampler_summary_from_nvml_readings():
    import time

    import bench
    fake = _FakeNvml([(2070.0, 900.0, 0x0), (1980.0, 1390.0, 0x4), (2070.0, 1000.0, 0x1)])
    with bench.Clocks(0, reader=fake, period=1e-3) as c:
        time.sleep(0.05)
    s = c.summary()
    assert s["source"] == "nvml" and s["samples"] >= 3 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # the idle bit (0x1) is not a slowdown
    assert s["sm_mhz"] == 2070.0 and s["power_w"] == 1000.0
    fake = _FakeNvml([(1500.0, None, 0x8 | 0x20 | 0x40 | 0x80)])
    with bench.Clocks(0, reader=fake) as c:
        pass
    s = c.summary()
    assert s["samples"] == 2 and s["power_w"] is None  # one on entry, one on exit
    assert s["reasons"] == ["hw_power_brake_slowdown", "hw_slowdown", "hw_thermal_slowdown",
                            "sw_thermal_slowdown"]


def test_clock_sampler_without_a_gpu():
    """Where neither NVML nor nvidia-smi answers, the sampler reports no
    samples instead of failing the run."""
    import shutil

    import pytest

    import bench
    try:
        bench.NvmlReader(0).close()
        pytest.skip("NVML answers here")
    except (OSError, AttributeError):
        pass
    if shutil.which("nvidia-smi"):
        pytest.skip("nvidia-smi present")
    with bench.Clocks(0) as c:
        pass
    s = c.summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "power_w": None,
                 "source": None}


def test_visible_device_names(monkeypatch):
    import bench
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES", raising=False)
    assert bench._visible_device(0) == "0"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-abc, 5")
    assert bench._visible_device(0) == "GPU-abc" and bench._visible_device(1) == "5"
    assert bench._visible_device(2) == "2"


def test_clock_sampler_survives_a_failing_reader():
    import bench

    class Broken:
        max_mhz = None

        def sample(self):
            raise RuntimeError("driver went away")

    with bench.Clocks(0, reader=Broken(), period=1e-3) as c:
        pass
    assert c.summary()["samples"] == 0


def test_buffer_marshalling_checks_types():
    """Tensors are passed by pointer, so their element width must match;
    arrays of other integer types are converted; floats are refused."""
    import torch

    import paper_2404_19634_gb300 as dfl
    ok = torch.zeros((4, 3), dtype=torch.int32)
    p, mk, keep = dfl._buf(ok, np.uint32)
    assert p.value == ok.data_ptr() and mk == dfl.MEM_HOST and keep is ok
    assert dfl._buf(torch.zeros(5, dtype=torch.int64), np.uint64)[0].value is not None
    for bad, want in ((torch.zeros((4, 3), dtype=torch.int64), np.uint32),
                      (torch.zeros(4, dtype=torch.float32), np.uint32),
                      (torch.zeros(4, dtype=torch.int32), np.uint64)):
        with pytest.raises(TypeError):
            dfl._buf(bad, want)
    with pytest.raises(ValueError):
        dfl._buf(torch.zeros((3, 4), dtype=torch.int32).t(), np.uint32)
    with pytest.raises(TypeError):
        dfl._buf(np.ones(3, np.float64), np.uint32)
    p, mk, a = dfl._buf(np.arange(3, dtype=np.int64), np.uint32)
    assert mk == dfl.MEM_HOST and a.dtype == np.uint32 and list(a) == [0, 1, 2]
    assert dfl._buf(None, np.uint32) == (None, dfl.MEM_HOST, None)
