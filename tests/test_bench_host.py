"""Host-side helpers of bench.py (no GPU): the clock-sample summary that goes
into the JSON line's "clocks" object, and the scaling of the committed ncu
traffic record to the timed launch."""
import json
import os
import sys

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

ROW = "0, {sm}, 2070, 900.5, {active}, {hw}, {hwt}, {swt}, {cap}"


def row(sm=2070, active="0x0", hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ROW.format(sm=sm, active=active, hw=hw, hwt=hwt, swt=swt, cap=cap)


def test_median_clock_and_no_reasons():
    text = "\n".join(row(sm=s) for s in (2070, 1965, 2040, 2070, 1980))
    d = bench.parse_clock_samples(text)
    assert d == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_every_reason_active_in_any_sample_is_reported():
    text = "\n".join([row(), row(cap="Active"), row(hwt="Active"), row(), row(hw="Active", swt="Active")])
    d = bench.parse_clock_samples(text)
    assert d["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_unreadable_rows_are_skipped():
    text = "\n".join(["index, clocks.current.sm [MHz], ...", row(sm="[N/A]"), "garbage", row(sm=1500), ""])
    d = bench.parse_clock_samples(text)
    assert d["samples"] == 1 and d["sm_mhz"] == 1500.0
    assert bench.parse_clock_samples("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_record_is_scaled_by_keys_and_dropped_after_a_kernel_change(tmp_path):
    path = str(tmp_path / "traffic.json")
    assert bench.ncu_traffic(1000, path)[0] is None  # no record
    rec = {"bytes_per_launch": 760, "n": 64, "note": "capture", "source_sha256": bench.source_hash(bench.SCATTER_SRC)}
    with open(path, "w") as f:
        json.dump({"scatter": rec}, f)
    assert bench.ncu_traffic(256, path) == (4 * 760, "capture")
    rec["source_sha256"] = "0" * 64  # taken on another version of the kernel
    with open(path, "w") as f:
        json.dump({"scatter": rec}, f)
    got, why = bench.ncu_traffic(256, path)
    assert got is None and "changed" in why


def test_committed_traffic_record_is_plausible():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["scatter"]
    # 16-bit keys + 32-bit values: a pass reads and writes 6 bytes per key
    assert 0.5 < rec["bytes_per_launch"] / (12 * rec["n"]) < 1.5
