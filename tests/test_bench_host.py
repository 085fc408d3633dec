"""Host logic of bench.py that decides whether a number is valid: the
nvidia-smi clock and throttle-reason parser, where the clock samples go, the
algorithmic work of the roofline entries, and the CG convergence summary."""

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


def test_fused_cg_roofline_work():
    # per CG iteration of the fused solve on the 16 x 16 lattice: T = tanh theta
    # complex64 [65536][256] = 134.2 MB and spins int8 [65536][256] = 16.8 MB
    # read once; the two contractions sigma V and sigma^T (conj(T) w) are
    # 4 B N M real flops each
    from paper_2103_08804_gb300 import synth
    wl = synth.WORKLOADS["square16"]
    assert (wl.walkers, wl.N, wl.M) == (65536, 256, 256)
    assert bench.fcg_bytes_per_iter(wl) == 65536 * 256 * 8 + 65536 * 256
    assert abs(bench.fcg_bytes_per_iter(wl) / 1e6 - 151.0) < 0.1
    assert bench.fcg_flops_per_iter(wl) == 8.0 * 65536 * 256 * 256


def test_plain_reduction_flops():
    # oreduce2 on chain64: per (walker, i, j) one real x complex FMA (4 flops),
    # per (walker, j) conj(T) g and its b-sum (8 flops), per (walker, i) 4 flops
    from paper_2103_08804_gb300 import synth
    wl = synth.WORKLOADS["chain64"]
    assert bench.reduce_flops(wl) == 16384 * (4 * 64 * 128 + 8 * 128 + 4 * 64)


def test_cg_summary_counts_truncated_solves():
    import numpy as np
    st = np.zeros((2, 3, 8))
    st[..., 5] = [[50, 12, 50], [50, 50, 7]]
    st[..., 6] = [[2e-4, 5e-5, 9e-5], [3e-3, 1e-4, 1e-5]]
    s = bench.cg_summary(st, 50, 1e-4)
    assert s["cg_iters_max"] == 50 and abs(s["cg_iters_mean"] - 219 / 6) < 1e-12
    # at the limit and above tolerance: (0,0) and (1,0); (0,2) met the tolerance
    assert abs(s["cg_truncated_fraction"] - 2 / 6) < 1e-12
    assert s["cg_rel_residual_max"] == 3e-3


def test_shift_rule_of_the_workloads():
    # 0.1 where the parameters reach the walker count (S singular), 1e-3
    # otherwise; the batch specs take it per sequence unless a shift is given
    from paper_2103_08804_gb300 import batch, synth
    assert synth.default_shift(8384, 8192) == 0.1
    assert synth.default_shift(8384, 16384) == 1e-3
    assert synth.WORKLOADS["square16"].shift == 0.1
    assert synth.WORKLOADS["square10"].shift == 1e-2
    assert synth.WORKLOADS["chain64"].shift == 1e-3
    specs = batch.momentum_scan_specs(L=8, alpha=2, chains=(48, 96), walkers=8192, n_moments=2,
                                      n_iter=1)
    shifts = {s.name: s.cfg.shift for s in specs}
    assert all(v == 0.1 for k, v in shifts.items() if k.startswith("square8"))
    assert shifts["chain48_q1.5708"] == 1e-3 and shifts["chain96_q1.5708"] == 0.1
    given = batch.momentum_scan_specs(L=4, alpha=2, chains=(), walkers=64, n_moments=2, n_iter=1,
                                      shift=0.5)
    assert all(s.cfg.shift == 0.5 for s in given)
