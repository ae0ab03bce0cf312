"""Host logic of bench.py that needs no GPU: the clock record keeps the
nvidia-smi samples taken inside the timed region."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(sm, power_cap="Not Active", hw="Not Active"):
    return f"{sm}, 2070, 900.0, {hw}, Not Active, Not Active, {power_cap}"


def test_clock_record_keeps_the_timed_window():
    ck = bench.ClockSampler(0)
    ck.proc = _FakeProc()
    ck.lines = [(1.0, _row(2070)), (2.0, _row(1500, power_cap="Active")), (3.0, _row(1600)),
                (9.0, _row(2070, hw="Active"))]
    ck.window = [1.5, 3.5]
    rec = ck.stop()
    assert rec["in_timed_region"] and rec["samples"] == 2
    assert rec["sm_mhz"] == 1550.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]          # the hw_slowdown sample lies outside


def test_clock_record_without_samples_in_the_window_uses_all():
    ck = bench.ClockSampler(0)
    ck.proc = _FakeProc()
    ck.lines = [(1.0, _row(2000)), (2.0, _row(2070)), (3.0, "garbled line")]
    ck.window = [5.0, 5.01]
    rec = ck.stop()
    assert not rec["in_timed_region"] and rec["samples"] == 2 and rec["sm_mhz"] == 2035.0


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
