"""Host logic of bench.py that needs no GPU: the clock record taken during the timed region, the
guard that drops the ncu traffic figure once the kernel's sources change, and the roofline object
(the dominant group and the whole-step byte sums)."""
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


def _measurement(precision="fp32"):
    """A made-up measurement: two kernel groups and the momentum solve over 20 steps."""
    groups = {
        "mg_fine": {"launches": 700, "launches_incl_empty": 960, "avg_launch_ms": 3.3, "bytes_per_launch": 2.2e9,
                    "achieved_gbs": 2.2e9 / 3.3e-3 / 1e9, "frac": 0.1},
        "cg_update": {"launches": 350, "launches_incl_empty": 480, "avg_launch_ms": 0.75, "bytes_per_launch": 4.8e9,
                      "achieved_gbs": 4.8e9 / 0.75e-3 / 1e9, "frac": 0.94},
        "momentum_per_step": {"launches": 20, "avg_launch_ms": 120.0, "bytes_per_launch": 2.3e11,
                              "achieved_gbs": 2.3e11 / 0.12 / 1e9, "frac": 0.28},
    }
    return {"groups": groups, "peak": (6784.5, "measured"), "steps": 20, "cells": 201326592, "ms_per_step": 363.4,
            "precision": precision, "shares": {}, "solve": {"inner_iters_per_step": 17.2, "refinements_per_step": 1.0}}


def test_roofline_takes_the_group_with_the_largest_total_time_and_sums_the_step():
    m = _measurement()
    r = bench.roofline_of(m, "no_such_workload")
    # mg_fine: 700 x 3.3 ms > cg_update: 350 x 0.75 ms; the momentum solve is a per-step group, not a kernel
    assert r["kernel"] == "mg_fine"
    assert r["frac"] == pytest.approx(2.2e9 / 3.3e-3 / 1e9 / 6784.5)
    assert r["traffic"] is None
    step = r["step"]
    alg = (700 * 2.2e9 + 350 * 4.8e9 + 20 * 2.3e11) / 20
    assert step["algorithmic_bytes_per_step"] == pytest.approx(alg)
    assert step["frac"] == pytest.approx(alg / 0.3634 / 1e9 / 6784.5)
    model = (119 + 41 * 17.2 + 41 * 1.0) * 201326592
    assert step["cg_model_bytes_per_step"] == pytest.approx(model)
    assert step["cg_model_frac"] == pytest.approx(model / 0.3634 / 1e9 / 6784.5)


def test_step_model_of_the_fp64_path():
    r = bench.roofline_of(_measurement("fp64"), "no_such_workload")
    assert r["step"]["cg_model_bytes_per_step"] == pytest.approx((235 + 81 * 17.2) * 201326592)
