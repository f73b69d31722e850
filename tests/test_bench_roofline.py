"""The bench's roofline record: every figure follows from the record's own
fields, and DRAM traffic is reported only for the kernel sources it was
captured on (CPU only)."""
import math

import bench


def test_roofline_record_is_self_consistent():
    mv = {"launches": 80, "bytes": 80 * 12_000_000.0, "ms": 80 * 0.045}
    r = bench.roofline_record(mv, 20, 6795.8, "measured", True)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["bytes_per_launch"], 12_000_000.0)
    assert math.isclose(r["ms_per_launch"], 0.045)
    assert math.isclose(r["achieved"], r["bytes_per_launch"] / 1e9 / (r["ms_per_launch"] / 1e3))
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    assert r["launches_per_step"] == 4.0
    assert math.isclose(r["bytes_per_step"], 4 * 12_000_000.0)
    assert math.isclose(r["kernel_ms_per_step"], 4 * 0.045)
    assert r["traffic"] == bench.DECIDE_TRAFFIC["cold"]
    assert r["traffic_warm"] == bench.DECIDE_TRAFFIC["warm"]
    assert math.isclose(r["traffic_ratio"], r["traffic"] / r["bytes_per_launch"])
    assert math.isclose(r["traffic_ratio_warm"], r["traffic_warm"] / r["bytes_per_launch"])


def test_roofline_traffic_only_for_the_captured_sources():
    mv = {"launches": 4, "bytes": 4e7, "ms": 0.2}
    r = bench.roofline_record(mv, 1, 6800.0, "fallback", False)
    assert r["traffic"] is None and r["traffic_ratio"] is None and r["traffic_warm"] is None
    assert r["traffic_source"].startswith("null")


def test_roofline_without_timing_does_not_divide_by_zero():
    r = bench.roofline_record({"launches": 0, "bytes": 0.0, "ms": 0.0}, 1, 6800.0, "measured", False)
    assert r["achieved"] == 0.0 and r["frac"] == 0.0


def test_source_hash_ignores_comments_not_code():
    src = 'int f(int a) {  // the sum\n  /* block\n comment */ return a + 1;\n}\nconst char* s = "// kept";\n'
    code = bench._code_only(src)
    assert "the sum" not in code and "block" not in code
    assert '"// kept"' in code and "return a + 1;" in code
    assert bench._code_only(src.replace("the sum", "a sum").replace("\n}", "\n\n}")) == code
    assert bench._code_only(src.replace("a + 1", "a + 2")) != code
