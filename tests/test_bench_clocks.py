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


# --- forecast layout of a handle (bench --forecast-choice) -----------------
class _FakeHandle:
    """Stands in for MGEnKF: records the choice set or autotuned."""

    def __init__(self, tuned=(7, 9)):
        self.choice, self.tuned, self.calls = (-1, -1), tuned, []

    def forecast_autotune(self, reps=3):
        self.calls.append(("autotune", reps))
        self.choice = self.tuned
        return self.choice

    def set_forecast_choice(self, m, f):
        self.calls.append(("set", m, f))
        self.choice = (m, f)

    def forecast_choice(self):
        return self.choice


class _Args:
    def __init__(self, forecast_choice, workload="ns2d"):
        self.forecast_choice, self.workload = forecast_choice, workload


def test_forecast_choice_auto_tunes_and_explicit_sets():
    g = _FakeHandle()
    assert bench._forecast_choice(g, _Args("auto")) == (7, 9)
    assert g.calls == [("autotune", 3)]
    g = _FakeHandle()
    assert bench._forecast_choice(g, _Args("1,9")) == (1, 9)
    assert g.calls == [("set", 1, 9)]
    g = _FakeHandle()
    assert bench._forecast_choice(g, _Args("-1,-1")) == (-1, -1)
    g = _FakeHandle()  # Burgers: no layout, the choice flag is ignored
    assert bench._forecast_choice(g, _Args("1,9", workload="burgers_large")) == (-1, -1)
    assert g.calls == []


def test_layout_decodes_choices_like_the_binding():
    from paper_2012_10091_gb300 import build as B
    B.build()  # the binding loads the library at import (no GPU needed)
    from paper_2012_10091_gb300 import mgenkf as M
    lay = bench._layout(M, (7, 9))
    # choice c: rows (32, 16, 64, 128, 256, 24, 48, 20)[c % 8], narrow bands for c >= 8
    assert lay == {"members": {"segment_rows": 20, "narrow_bands": False},
                   "fine": {"segment_rows": 16, "narrow_bands": True}}
    assert bench._layout(M, (-1, -1)).startswith("2-D tile kernel")
    assert len(M.SEGMENT_ROWS) == len(M.NARROW_BANDS) == 16
