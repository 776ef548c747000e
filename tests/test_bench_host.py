"""Host-side pieces of bench.py (no GPU): the clock record taken during the
timed region and the roofline denominator."""
import json
import os
import stat

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

ROW = "0, {sm}, 2070, {pw}, {act}, {hw}, {hwt}, {swt}, {cap}"


def _row(sm, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active", pw=900.0):
    return ROW.format(sm=sm, pw=pw, act="0x0000000000000000", hw=hw, hwt=hwt, swt=swt, cap=cap)


def test_clock_summary_takes_the_median_under_load_and_every_reason():
    rows = [_row(345), _row(345)] + [_row(2070)] * 5 + [_row(1965, cap="Active"), _row(2055, hw="Active"),
                                                           "0, [N/A], 2070, [N/A], x, x, x, x, x", "garbage"]
    d = bench.ClockSampler.summarize("\n".join(rows) + "\n")
    assert d["sm_max_mhz"] == 2070.0
    assert d["sm_mhz"] == 2070.0                 # idle samples (below 30 % of max) left out
    assert d["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert d["samples"] == 9                     # the unparsable rows are skipped
    d = bench.ClockSampler.summarize("\n".join([_row(2070, hwt="Active"), _row(2070, swt="Active")]))
    assert d["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize("") is None


def test_clock_sampler_runs_nvidia_smi_and_stops_it(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    lines = "\\n".join([_row(2070)] * 3 + [_row(1800, cap="Active")])
    fake.write_text(f"#!/bin/sh\nprintf '{lines}\\n'\nexec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler()
    s.start()
    import time
    time.sleep(0.5)
    d = s.stop()
    assert d == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler()
    s.start()
    assert s.stop() is None


def test_roofline_peak_is_the_measured_copy_bandwidth():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        hbm = float(json.load(f)["hbm_gbs"])
    assert bench.measured_peaks() == (hbm, "measured")


def test_recorded_traffic_matches_the_capture_of_the_run_shape(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    caps = [{"kernel": "k_step_tma", "tile": [32, 8], "zdepth": 8, "order": "costliest", "cells": 1000,
             "dram_bytes_per_launch": 111},
            {"kernel": "k_step_tma", "tile": [32, 8], "zdepth": 0, "order": "costliest", "cells": 1000,
             "dram_bytes_per_launch": 222}]
    (tmp_path / "profiles" / "traffic_w.json").write_text(json.dumps(caps))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))

    class Args:
        zdepth = 0
        order = ""

    def rec(kname="k_step_tma", tile=(32, 8), zdepth=0, order=0, cells=1000, n_kernels=1):
        return {"tune": {"zdepth": zdepth, "order": order}, "n_kernels": n_kernels, "kname": kname,
                "tiles": [list(tile)], "cells": cells}

    assert bench.recorded_traffic(Args, "w", rec()) == 222
    assert bench.recorded_traffic(Args, "w", rec(zdepth=8)) == 111
    assert bench.recorded_traffic(Args, "w", rec(zdepth=16)) is None      # no capture of that shape
    assert bench.recorded_traffic(Args, "w", rec(order=1)) is None        # another item order
    assert bench.recorded_traffic(Args, "w", rec(cells=999)) is None      # another grid size
    assert bench.recorded_traffic(Args, "w", rec(kname="k_step_pair")) is None
    assert bench.recorded_traffic(Args, "w", rec(n_kernels=2)) is None    # two kernels: no single figure
    assert bench.recorded_traffic(Args, "none", rec()) is None            # no capture file
    # a single record (not a list) still works
    (tmp_path / "profiles" / "traffic_w.json").write_text(json.dumps(caps[0]))
    assert bench.recorded_traffic(Args, "w", rec(zdepth=8)) == 111
