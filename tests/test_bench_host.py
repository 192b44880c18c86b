"""Host-side logic of bench.py, on CPU: the clock record taken during the timed region (nvidia-smi lines
parsed into a median SM clock, the maximum clock and the throttle reasons seen), the peaks file and its
fallback, the kernel-source key of the measured traffic and the whole-job throughput."""
import os
import re
import stat
import time

import pytest

import bench

ROW = "0, {sm}, 2070, 950.25, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def _line(sm, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ROW.format(sm=sm, hw=hw, hwt=hwt, swt=swt, cap=cap)


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [_line(2070), _line(1980, cap="Active"), _line(2055), "", "garbage", _line(2070, hwt="active")]
    s = c.summary()
    assert s["samples"] == 4  # the empty and malformed lines are skipped
    assert s["sm_mhz"] == pytest.approx(2062.5)  # median of 1980, 2055, 2070, 2070
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.lines = ["[N/A], [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi anywhere on the path
    with bench.ClockSampler(0) as c:
        pass
    assert c.proc is None and c.summary()["samples"] == 0


def test_clock_sampler_reads_a_running_sampler(tmp_path, monkeypatch):
    """A stand-in nvidia-smi that prints three samples and keeps running until the sampler stops it."""
    fake = tmp_path / "nvidia-smi"
    lines = "\n".join(f'echo "{_line(sm)}"' for sm in (2070, 2040, 2055))
    fake.write_text("#!/bin/sh\n" + lines + "\nexec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    t0 = time.time()
    with bench.ClockSampler(3) as c:
        while len(c.lines) < 3 and time.time() - t0 < 10:
            time.sleep(0.02)
    assert c.proc.poll() is not None  # stopped on exit
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055.0 and s["reasons"] == []


def test_peaks_file_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6796.5, "bf16_tflops_sustained": 1742.1}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d = bench.measured_peaks()
    assert d["_source"] == "measured" and d["hbm_gbs"] == 6796.5
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    d = bench.measured_peaks()
    assert d["_source"] == "fallback"
    assert (d["hbm_gbs"], d["bf16_tflops"], d["bf16_tflops_sustained"]) == (6800.0, 1900.0, 1700.0)


def test_traffic_key_is_a_stable_source_hash():
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", h) and h == bench.kernel_source_hash()
    assert all(re.fullmatch(r"[0-9a-f]{16}", k) and v > 0 for k, v in bench.MEASURED_TRAFFIC.items())


def test_job_throughput_and_single_rank_max():
    # two ranks, each 2.0e12 flops per step in 500 ms: 8 TFLOP/s for the job
    assert bench.job_throughput(2, 2.0e12, 500.0) == pytest.approx(8.0)
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
