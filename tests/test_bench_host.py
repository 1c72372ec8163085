"""Host-side pieces of bench.py (no GPU): the clock summary keeps only the
samples of the timed region, and a recorded ncu traffic figure is used only
while the kernel's launch shape and source hash match."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_keeps_the_timed_region():
    b = load_bench()
    c = b.ClockSampler(0)
    # rows: [host time, sm MHz, max MHz, power, hw, hw_thermal, sw_thermal, sw_power_cap]
    c.rows = [[1.0, "1200", "2070", "300", "Not Active", "Not Active", "Not Active", "Not Active"],
              [2.0, "2070", "2070", "900", "Not Active", "Not Active", "Not Active", "Active"],
              [2.5, "2060", "2070", "950", "Not Active", "Not Active", "Not Active", "Not Active"],
              [4.0, "900", "2070", "200", "Active", "Not Active", "Not Active", "Not Active"]]
    s = c.stop(1.5, 3.0)
    assert s["samples"] == 2 and s["in_timed_region"]
    assert s["sm_mhz"] == 2065.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    # nothing inside the region: every sample, marked as such
    s = c.stop(10.0, 11.0)
    assert s["samples"] == 4 and not s["in_timed_region"]
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_recorded_traffic_needs_the_same_kernel(tmp_path, monkeypatch):
    b = load_bench()
    kinfo = {"variant": "staged", "depth": 1, "cols_per_cta": 128, "strips": 47, "strip_rows": "absolute"}
    rec = {"w/fp32": {"kernel_info": kinfo, "kernel_sha": b.kernel_hash("staged"), "dram_bytes_per_launch": 123}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(b, "TRAFFIC_FILE", str(f))
    assert b.recorded_traffic("fp32", "w", kinfo) == 123.0
    assert b.recorded_traffic("fp32", "w", dict(kinfo, strips=46)) is None
    assert b.recorded_traffic("fp16s", "w", kinfo) is None
    rec["w/fp32"]["kernel_sha"] = "0" * 16
    f.write_text(json.dumps(rec))
    assert b.recorded_traffic("fp32", "w", kinfo) is None

