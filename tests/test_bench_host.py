"""Host-side logic of bench.py (no GPU): the clock summary of the timed
region and the committed DRAM-traffic record of the roofline line."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_takes_the_window_median_and_the_active_reasons(bench):
    c = bench.Clocks(0)
    idle = ["Not Active"] * 4
    c.rows = [
        (0.5, ["2070", "2070"] + idle),                                          # before the window
        (1.0, ["1900", "2070", "Not Active", "Not Active", "Not Active", "Active"]),
        (1.5, ["2070", "2070", "Not Active", "Active", "Not Active", "Not Active"]),
        (2.0, ["[N/A]", "2070"] + idle),                                         # unparsable: skipped
        (3.0, ["100", "2070", "Active", "Active", "Active", "Active"]),          # after the window
    ]
    s = c.summary(0.9, 2.5)
    assert s["samples"] == 2
    assert s["sm_mhz"] == pytest.approx(1985.0)
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_of_an_empty_window(bench):
    c = bench.Clocks(0)
    c.rows = [(5.0, ["2070", "2070", "Active", "Active", "Active", "Active"])]
    s = c.summary(0.0, 1.0)
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []


def test_traffic_record_is_near_the_algorithmic_bytes():
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    for f in rec["sources"]:
        assert os.path.isfile(os.path.join(ROOT, f)), f
    n = 512 ** 3
    # step A reads q and writes D'' and three packed 2-bit maps: 8.75 B/pt; its
    # tiles re-read a one-point y halo and a four-point x halo (+13 % of q)
    r = rec["kernels"]["detect"]["dram_bytes_per_launch"] / (8.75 * n)
    assert 0.95 < r < 1.15
    # near reads the packed codes and writes the packed S: 0.5 B/pt (part of it left in L2)
    assert rec["kernels"]["near"]["dram_bytes_per_launch"] <= 0.5 * n * 1.05


def test_traffic_is_withheld_once_a_source_changes(bench, monkeypatch):
    monkeypatch.setattr(bench, "src_hash", lambda files: "0" * 16)
    assert bench.ncu_traffic("detect") is None
    assert bench.ncu_traffic("near") is None
