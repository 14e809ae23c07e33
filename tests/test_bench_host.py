"""Host-side pieces of bench.py that need no GPU: the clock and throttle
summary taken from nvidia-smi's CSV during the timed region, and the peak
table's fallback."""
import json

import bench


def _sampler_with(tmp_path, rows):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")
    return s


def test_clock_summary_median_max_and_reasons(tmp_path):
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["0", "1980", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
            ["0", "2055", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    out = _sampler_with(tmp_path, rows).summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    rows = [["0", "1500", "2070", "1000", "0x40", "Not Active", "Active", "Not Active", "Not Active"]]
    out = _sampler_with(tmp_path, rows).summary()
    assert out["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_samples(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "missing.csv")
    out = s.summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_summary_skips_malformed_rows(tmp_path):
    rows = [["0", "[N/A]", "2070"], ["0", "2070", "2070", "1", "0x0", "Not Active", "Not Active",
                                     "Not Active", "Not Active"]]
    out = _sampler_with(tmp_path, rows).summary()
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0


def test_peaks_fallback_when_file_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "none.json"))
    p, kind = bench.peaks()
    assert kind == "fallback" and p["hbm_gbs"] == 6800.0


def test_peaks_measured_file(monkeypatch, tmp_path):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 6794.0, "bf16_tflops": 1968.0}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    p, kind = bench.peaks()
    assert kind == "measured" and p["hbm_gbs"] == 6794.0


def test_alu_roofline_of_a_profile():
    # seven KKT applies of 103.8 MFLOP in 1.42 ms at 1.196 TFLOP/s
    p = {"launches": 7, "ms": 1.42, "bytes": 7 * 13.2e6, "flops": 7 * 103.8e6}
    r = bench.alu_roofline("kron_rank1_kernel", p, 1.196, "measured")
    assert r["launches_per_step"] == 7
    assert abs(r["avg_us"] - 1420.0 / 7) < 1e-9
    assert abs(r["achieved"] - 103.8e6 / (1.42e-3 / 7) / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / 1.196) < 1e-12
    assert r["algorithmic_bytes_per_launch"] == 13.2e6


def test_alu_roofline_absent_kernel():
    assert bench.alu_roofline("k", None, 1.0, "x") is None
    assert bench.alu_roofline("k", {"launches": 0, "ms": 0.0, "bytes": 0, "flops": 0}, 1.0, "x") is None
    assert bench.alu_roofline("k", {"launches": 1}, 1.0, "x") is None


def test_reference_arm_line():
    """`bench.py --impl reference` (the oracle on a bounded sample, host cores
    only) prints one JSON line with the contract's keys."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    # the small unit-cube workload keeps this CPU test short; the default
    # workload goes through the same code
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--config", "1", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True,
                         check=True, timeout=300, cwd=root)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["higher_is_better"] is False and line["value"] > 0
    assert line["config"]["workload"] == "unit_cube_p2_e16" and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_profiling_cases_parse(monkeypatch):
    # the single-measurement cases of the bench: the TT apply, the random-volume
    # solve, the timed steps alone, the parabolic solve and the FP32 applies
    for case in ("ttm", "c5solve", "step", "parabolic", "kron32"):
        monkeypatch.setattr("sys.argv", ["bench.py", "--only", case, "--nt", "4"])
        a = bench.parse()
        assert a.only == case and a.nt == 4 and a.gpus == 1
