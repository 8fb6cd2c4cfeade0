"""Host logic of bench.py that needs no GPU: the clock record taken during the timed region and the
guard that drops the ncu traffic figure once the kernel's sources change."""
import json
import os

import pytest

import bench


class _Running:
    """Stands in for the nvidia-smi process handle; summary() only checks that sampling ran."""


def _clocks_from(rows, tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.proc = _Running()
    return c.summary()


def test_clock_summary_takes_the_median_and_collects_active_reasons(tmp_path):
    idle = "Not Active"
    rows = [
        "2070, 2070, 400.5, 0x0, %s, %s, %s, %s" % (idle, idle, idle, idle),
        "2055, 2070, 612.0, 0x4, %s, %s, %s, Active" % (idle, idle, idle),
        "garbage line",
        "2070, 2070, 598.2, 0x0, %s, %s, %s, %s" % (idle, idle, idle, idle),
        "[N/A], 2070, 10, 0x0, a, b, c, d",
    ]
    s = _clocks_from(rows, tmp_path)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["power_w_max"] == 612.0
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clock_summary_reports_thermal_slowdown(tmp_path):
    idle = "Not Active"
    s = _clocks_from(["1500, 2070, 900, 0x20, %s, Active, %s, %s" % (idle, idle, idle)], tmp_path)
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples(tmp_path):
    assert _clocks_from([], tmp_path)["reasons"] == ["no samples"]
    c = bench.Clocks(0)
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_ncu_traffic_is_dropped_when_the_kernel_sources_change(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.txt")) as f:
        rec = json.load(f)["kernels"]["mg_fine"]
    monkeypatch.setattr(bench, "src_hash", lambda files=None: rec["source_hash"])
    assert bench.ncu_traffic("mg_fine") == rec["dram_bytes_per_launch_full_size"]
    monkeypatch.setattr(bench, "src_hash", lambda files=None: "0" * 16)
    assert bench.ncu_traffic("mg_fine") is None
    assert bench.ncu_traffic("no_such_group") is None


def test_source_hash_covers_only_the_named_files():
    rec_files = ["stencil4.cu", "common.cuh", "solver.cuh"]
    assert bench.src_hash(rec_files) == bench.src_hash(list(reversed(rec_files)))
    assert bench.src_hash(rec_files) != bench.src_hash(rec_files[:2])
    with pytest.raises(FileNotFoundError):
        bench.src_hash(["no_such_file.cu"])
