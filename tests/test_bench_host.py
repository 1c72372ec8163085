"""Host-side pieces of bench.py (no GPU): the clock summary keeps only the
samples of the timed region, a recorded ncu traffic figure is used only
while the kernel's launch shape and source hash match, and the all-core
oracle baseline runs one spawned process per core."""
import importlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    # imported by its own name, so that spawned worker processes can find
    # the functions they run
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


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
    assert s["too_short_to_sample"] and s["timed_region_s"] == 1.0
    assert "too_short_to_sample" not in c.stop(1.5, 3.0)


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



def test_oracle_on_several_host_cores():
    """The all-core oracle baseline: spawned processes, one per core, each on
    its own copy of the crop; the figure counts every process's updates over
    the slowest one's time."""
    b = load_bench()
    w = b.workload()
    value, slowest, n_fluid = b.oracle_all_cores(w, 16, 1, 2, 2)
    assert n_fluid == int((w.mask[:, :16] == 0).sum())
    assert slowest > 0 and value == 2 * n_fluid * 2 / slowest / 1e9
    n, model = b.host_cores()
    assert n >= 1 and isinstance(model, str)


def test_reference_line_has_the_native_config(monkeypatch, capsys):
    """The reference arm prints its line on the native arm's `config` (the
    workload; how each arm runs it goes in its own keys) with the contract's
    keys; the oracle timing itself is replaced by a stub here."""
    import argparse
    b = load_bench()
    w = b.workload()

    class Sample:
        cols = 64

    monkeypatch.setattr(b, "oracle_sample_for", lambda w, s: Sample())
    monkeypatch.setattr(b, "oracle_all_cores", lambda w, cols, warmup, steps, procs: (0.04, 2.5, 123))
    assert b.reference_arm(argparse.Namespace(steps=4, warmup=3)) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["config"] == b.workload_config(w, 1)
    assert line["impl"] == "reference" and line["metric"] == b.METRIC and line["unit"] == b.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 4 and line["warmup"] == 3
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["fluid_nodes"] == int((w.mask == 0).sum())


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    """Launched under torchrun with several ranks, only rank 0 times the
    oracle and prints the line; the other ranks exit 0 without work."""
    import argparse
    b = load_bench()
    called = []
    monkeypatch.setattr(b, "oracle_all_cores", lambda *a: called.append(a) or (0.04, 2.5, 123))
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert b.reference_arm(argparse.Namespace(steps=4, warmup=3)) == 0
    assert called == [] and capsys.readouterr().out == ""
