"""Host logic of bench.py that decides whether a number is valid: the
nvidia-smi clock and throttle-reason parser, where the clock samples go, and
the algorithmic bytes of the headline roofline entry."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    cs = bench.ClockSampler(str(path), 0)
    cs.p = object()  # as if nvidia-smi had run and written the file
    return cs.summary()


def test_clock_summary_takes_the_median_and_active_reasons_only(tmp_path):
    na = "Not Active"
    rows = [
        f"0, 2070, 2070, 900.1, 0x0, {na}, {na}, {na}, {na}",
        f"0, 1950, 2070, 1390.0, 0x4, {na}, {na}, {na}, Active",
        f"0, 2070, 2070, 1010.5, 0x0, {na}, {na}, {na}, {na}",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, x, x, x, x",
    ]
    s = _summary(tmp_path, rows)
    assert s["sm_mhz"] == 2070.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3


def test_clock_summary_reports_thermal_slowdown(tmp_path):
    na = "Not Active"
    s = _summary(tmp_path, [f"0, 1500, 2070, 1200.0, 0x40, {na}, Active, {na}, {na}"])
    assert s["reasons"] == ["hw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples(tmp_path):
    assert _summary(tmp_path, ["", "x"])["reasons"] == ["no samples"]
    assert bench.ClockSampler("unused", 0).summary()["reasons"] == ["nvidia-smi unavailable"]


def test_clock_path_honours_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("CHEBRBM_CLOCKS_DIR", str(tmp_path))
    assert bench.clock_path("sym6", 3) == os.path.join(str(tmp_path), "clocks_sym6_r3.csv")
    monkeypatch.delenv("CHEBRBM_CLOCKS_DIR")
    assert os.path.basename(bench.clock_path("chain64", 0)) == "clocks_chain64_r0.csv"


def test_headline_roofline_bytes():
    # oreduce_tc on chain64: tanh theta complex64 [16384][128] = 16.78 MB,
    # spins int8 [16384][64] = 1.05 MB, g complex64 [16384] = 0.13 MB, and the
    # complex128 row of P = 64 + 128 + 64 * 128 sums out: 18.09 MB in all
    from paper_2103_08804_gb300 import synth
    wl = synth.WORKLOADS["chain64"]
    assert (wl.walkers, wl.N, wl.M) == (16384, 64, 128)
    assert bench.reduce_bytes(wl) == 16384 * 128 * 8 + 16384 * 64 + 16384 * 8 + 16 * 8384
    assert abs(bench.reduce_bytes(wl) / 1e6 - 18.09) < 0.005
    # the measured DRAM traffic of one launch is the algorithmic read volume
    traffic = bench.MEASURED_TRAFFIC[("mixed", "chain64")][0]
    assert abs(traffic - bench.reduce_bytes(wl)) / bench.reduce_bytes(wl) < 0.01
