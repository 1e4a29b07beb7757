"""The benchmark's clock record, on the CPU: which GPU nvidia-smi is asked
about, and how the sampled lines become the "clocks" object (median SM clock
over the loaded samples, the maximum, and every throttle reason seen)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_smi_device_id(monkeypatch):
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES", raising=False)
    assert bench.smi_device_id(0) == "0" and bench.smi_device_id(3) == "3"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5")
    assert bench.smi_device_id(0) == "5"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-aaaa, GPU-bbbb")
    assert bench.smi_device_id(1) == "GPU-bbbb"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "2,7")
    assert bench.smi_device_id(1) == "7" and bench.smi_device_id(2) == "2"


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines, skip=0):
    c = bench.ClockSampler("0")
    c.proc = _Proc()
    c.lines = lines
    c.skip = skip
    return c


def _line(sm, smax=2070, reasons=("Not Active",) * 4):
    return f"0, {sm}, {smax}, 900.5, 0x0000000000000000, " + ", ".join(reasons) + "\n"


def test_clock_record(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    lines = [_line(300)] + [_line(2070)] * 5 + [_line(1980)] * 2 + [_line(400)]
    lines.append(_line(2000, reasons=("Not Active", "Not Active", "Not Active", "Active")))
    lines.append("garbage\n")
    rec = _sampler(lines, skip=1).stop()
    # the idle sample (400 MHz) is below half of the maximum and left out
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 9


def test_clock_record_without_samples(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    assert _sampler([]).stop()["reasons"] == ["no samples"]
    c = bench.ClockSampler("0")
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
