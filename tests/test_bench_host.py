"""Host logic of bench.py on CPU: the clock sampler (driven by a stand-in for
nvidia-smi), the summary of its samples, and the ncu traffic lookup that is
valid only for the profiled kernel source."""
import json
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(sm, mx, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000004, " + ", ".join(flags) + "\n"


def test_summary_uses_the_timed_window_and_reports_reasons():
    lines = [(0.5, _line(2070, 2070)),                                 # before the window
             (1.0, _line(1800, 2070, ["sw_power_cap"])),
             (1.1, _line(1750, 2070, ["sw_power_cap"])),
             (1.2, _line(1900, 2070)),
             (1.3, "garbage\n"),                                        # malformed: skipped
             (1.4, "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active\n"),
             (3.0, _line(600, 2070, ["hw_slowdown"]))]                  # after the window
    got = bench.summarize_clock_samples(lines, (1.0, 2.0))
    assert got == {"sm_mhz": 1800.0, "sm_max_mhz": 2070.0, "samples": 3, "samples_in": "timed region",
                   "reasons": ["sw_power_cap"]}


def test_summary_falls_back_to_the_whole_run_and_to_none():
    lines = [(0.5, _line(2000, 2070, ["hw_thermal_slowdown"])), (0.6, _line(2010, 2070))]
    got = bench.summarize_clock_samples(lines, (5.0, 6.0))      # nothing inside the window
    assert got["samples_in"] == "whole run" and got["samples"] == 2
    assert got["reasons"] == ["hw_thermal_slowdown"] and got["sm_mhz"] == 2005.0
    assert bench.summarize_clock_samples([], None) is None
    assert bench.summarize_clock_samples([(1.0, "x\n")], None) is None


def test_clocks_sampler_with_a_stand_in_nvidia_smi(tmp_path, monkeypatch):
    # a stand-in on PATH that prints one sample every 20 ms until terminated
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!" + sys.executable + "\n"
                    "import sys, time\n"
                    "assert '--format=csv,noheader,nounits' in sys.argv\n"
                    "i = 0\n"
                    "while True:\n"
                    "    print(f'0, {1700 + i % 3}, 2070, 1000.0, 0x4, Not Active, Not Active, Not Active, Active', flush=True)\n"
                    "    i += 1\n"
                    "    time.sleep(0.02)\n")
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR | stat.S_IXGRP | stat.S_IXOTH)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.Clocks(0)
    c.start()
    assert c.lines, "the sampler waits for its first sample"
    t0 = time.perf_counter()
    time.sleep(0.3)
    c.window = (t0, time.perf_counter())
    got = c.stop()
    assert got["samples_in"] == "timed region" and got["samples"] >= 5
    assert 1700 <= got["sm_mhz"] <= 1702 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]


def test_clocks_without_nvidia_smi_reports_none(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None


def test_ncu_traffic_only_for_the_profiled_source(tmp_path):
    kernel = tmp_path / "kernel.cu"
    kernel.write_text("// some kernel source\n")
    rec = {"source_sha": bench.source_sha(str(kernel)), "per_launch_bytes": {"w1": 123.0}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    assert bench.ncu_traffic(str(kernel), "w1", str(path)) == 123.0
    assert bench.ncu_traffic(str(kernel), "other", str(path)) is None
    kernel.write_text("// the kernel changed since the capture\n")
    assert bench.ncu_traffic(str(kernel), "w1", str(path)) is None
    assert bench.ncu_traffic(str(kernel), "w1", str(tmp_path / "missing.json")) is None


def test_committed_traffic_record_matches_the_current_leaf_kernel():
    # the bench reports `traffic` only while the committed capture belongs to
    # the kernel source it runs
    kernel = os.path.join(ROOT, "paper_1205_2927_gb300", "csrc", "leaf_gemm.cu")
    assert bench.ncu_traffic(kernel, "n16384_d3_bn512_fp32") is not None
