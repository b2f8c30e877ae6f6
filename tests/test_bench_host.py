"""Host logic of bench.py that needs no GPU: the clock sampler keeps only the
samples taken inside the timed region and reads the throttle reasons."""
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


def _line(sm, smax, hw="Not Active", pcap="Not Active"):
    return f"{sm}, {smax}, 600.0, 0x0, {hw}, Not Active, Not Active, {pcap}"


def test_clock_sampler_keeps_only_the_timed_window():
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.t_begin = 100.0
    c.lines = [
        (99.0, _line(1200, 2070, hw="Active")),  # before the timed region: ignored
        (100.1, _line(2070, 2070)),
        (100.3, _line(2060, 2070, pcap="Active")),
        (100.5, _line(2070, 2070)),
        (1e12, _line(300, 2070)),  # long after: ignored
        (100.6, "garbled"),
    ]
    out = c.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
