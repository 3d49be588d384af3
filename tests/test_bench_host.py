"""Host logic of bench.py that needs no GPU: the clock summary behind the
"clocks" key, the guard that ties the committed ncu figures (DRAM bytes,
executed FLOPs) to the kernel sources they were taken on, and the defaults
that the timing rules fix (at least 3 warm-up steps, one GPU)."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

FLOPS_PER_PAIR = 4 * 165 + 19


def _row(sm, mx, active=("Not Active",) * 5):
    return "0, %s, %s, 900.5, %s\n" % (sm, mx, ", ".join(active))


def test_clock_summary_median_max_and_reasons():
    lines = [_row(2070, 2070), _row(2055, 2070), "garbled line\n",
             _row(1980, 2070, ("Active", "Not Active", "Not Active", "Not Active", "Active")),
             _row("[N/A]", 2070)]
    c = bench.clock_summary(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == 2055.0  # median of the numeric samples
    assert c["sm_max_mhz"] == 2070.0
    # the reason columns after 'active' are hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.clock_summary([_row(1500, 2070, ("Active", "Active", "Active", "Not Active", "Not Active"))])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.clock_summary([]) is None
    assert bench.clock_summary(["no, samples\n"]) is None


def test_recorded_capture_follows_the_kernel_sources(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")))
    for prec in ("mixed", "fp64"):
        monkeypatch.setattr(bench, "kernel_source_sha", lambda: rec[prec]["kernel_src_sha"])
        cap = bench.recorded_capture(prec)
        assert cap["dram_bytes_per_launch"] == bench.recorded_traffic(prec) > 0
        monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
        assert bench.recorded_capture(prec) == {} and bench.recorded_traffic(prec) is None
    assert bench.recorded_capture("fp16") == {}


def test_committed_capture_is_plausible():
    """Executed FLOPs within a factor of the defining formulation's 679 and
    DRAM traffic at least the unique FP32 source records of the large
    workload (32 768 records of 64 bytes)."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")))
    m, f = rec["mixed"], rec["fp64"]
    assert 0.5 * FLOPS_PER_PAIR < m["executed_fp32_flops_per_pair"] < FLOPS_PER_PAIR
    assert m["executed_fp64_flops_per_pair"] < 0.01 * FLOPS_PER_PAIR  # the near field is rare
    assert 0.5 * FLOPS_PER_PAIR < f["executed_fp64_flops_per_pair"] < 1.5 * FLOPS_PER_PAIR
    assert f["executed_fp32_flops_per_pair"] == 0.0
    for e in (m, f):
        assert e["dram_bytes_per_launch"] >= 32768 * 64
        assert len(e["kernel_src_sha"]) == 16
        assert "ncu" in e["command"] and "--clock-control none" in e["command"]
        assert "--clock-control none" in e["executed_command"]


def test_defaults_follow_the_timing_rules(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.precision == "mixed"
    assert a.warmup >= 3 and a.steps >= 1 and a.e2e_steps >= 2
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "4", "--warmup", "3"])
    a = bench.parse()
    assert a.impl == "reference" and a.steps == 4 and a.warmup == 3
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "other"])
    with pytest.raises(SystemExit):
        bench.parse()
