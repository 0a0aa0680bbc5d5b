"""Host logic of bench.py's clock record (no GPU): the median SM clock under
load, the maximum clock and the throttle reasons seen in the samples of
nvidia-smi's CSV output, which decide whether a timed run is kept."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _DoneThread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.proc, c.th, c.lines = _DoneProcess(), _DoneThread(), list(lines)
    return c


def test_median_clock_and_no_reasons():
    lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2070, 2070, 940.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    r = _sampler(lines).stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == [] and r["samples"] == 3


def test_throttle_reasons_are_collected_and_bad_lines_skipped():
    lines = ["0, 1800, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
             "garbage",
             "0, [N/A], 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 1500, 2070, 1390.0, 0x20, Active, Not Active, Active, Not Active"]
    r = _sampler(lines).stop()
    assert r["samples"] == 2
    assert r["sm_mhz"] == 1650.0
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_missing_nvidia_smi_is_reported():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
