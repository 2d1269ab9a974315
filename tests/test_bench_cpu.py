"""Host logic of bench.py that decides what its JSON line reports (CPU only).

  * The clock record: only samples inside the timed window count, the SM
    clock is their median, and every throttle reason seen there is listed.
  * The DRAM traffic figure: it is read from the committed ncu summary only
    while the kernel source still has the hash the summary was taken on.
  * The roofline denominator: the measured peaks when present, else the
    documented fallback, labelled as such.
"""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler.__new__(bench.ClockSampler)  # no nvidia-smi process
    s.proc = None
    s.lines = lines
    return s


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.00, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_clock_summary_keeps_the_timed_window_only():
    lines = [(9.0, _row(900, 2070, hw="Active")),      # before the window: ignored
             (10.0, _row(2070, 2070)),
             (10.5, _row(2040, 2070, cap="Active")),
             (11.0, _row(2010, 2070)),
             (11.05, _row(2070, 2070)),                 # within the 0.1 s grace after t1
             (12.0, _row(1000, 2070, hwt="Active"))]    # after the window: ignored
    out = _sampler(lines).summary(10.0, 11.0)
    assert out["samples"] == 4
    assert out["sm_mhz"] == pytest.approx(2055.0)       # median of 2070, 2040, 2010, 2070
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_lists_every_slowdown_and_skips_unreadable_fields():
    lines = [(1.0, _row("[N/A]", 2070, hw="Active")),
             (1.1, _row(1500, "[N/A]", swt="Active")),
             (1.2, "garbled line\n")]
    out = _sampler(lines).summary(0.0, 2.0)
    assert out["samples"] == 2
    assert out["sm_mhz"] == 1500.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _sampler([]).summary(0.0, 1.0) is None


def _traffic_tree(tmp_path, src_text, recorded_sha):
    src = tmp_path / "kernel.cu"
    src.write_text(src_text)
    (tmp_path / "profiles").mkdir()
    entry = {"source": "kernel.cu", "source_sha": recorded_sha,
             "dram_bytes_per_launch_full": 123456}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"fam": entry}))


def test_traffic_is_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    text = "// kernel as profiled\n"
    sha = hashlib.sha256(text.encode()).hexdigest()[:16]
    _traffic_tree(tmp_path, text, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("fam") == 123456
    assert bench.ncu_traffic("other_family") is None
    (tmp_path / "kernel.cu").write_text(text + "// changed since\n")
    assert bench.ncu_traffic("fam") is None


def test_committed_traffic_table_matches_its_sources():
    # Every family in the committed table names a source that exists, and the
    # full-size traffic is within a few percent of the algorithmic bytes.
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        table = json.load(fh)
    for fam, e in table.items():
        assert os.path.exists(os.path.join(ROOT, e["source"])), fam
        assert 1.0 <= e["dram_bytes_per_launch_full"] / e["alg_bytes_per_launch_full"] < 1.05, fam
        assert os.path.exists(os.path.join(ROOT, e["profile"])), fam


def test_peaks_fall_back_when_not_measured(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0}))
    peaks, kind = bench.measured_peaks()
    assert kind == "measured" and peaks["hbm_gbs"] == 7000.0
