"""bench.py's clock record: only samples that arrived while the timed region ran count, their
throttle reasons are recorded, and without such samples the whole sampler run is used (and
the record says so).  Host logic only, on CPU with synthetic nvidia-smi lines."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _Thread:
    def join(self, timeout=None):
        pass


def _line(mhz, thermal="Not Active", power="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return f"0, {mhz}, 2070, 900.5, 0x0, Not Active, Not Active, {thermal}, {power}"


def _sampler(lines):
    c = bench.Clocks(0)
    c.proc, c.t = _Proc(), _Thread()
    c.lines = list(lines)
    return c


def test_only_samples_inside_the_timed_region_count():
    c = _sampler([(0.0, _line(1000)), (1.00, _line(2070)), (1.02, _line(2050, power="Active")),
                  (1.04, _line(2070)), (5.0, _line(300, thermal="Active"))])
    c.mark(0.99, 1.03)
    r = c.stop()
    assert r["scope"] == "timed region"
    assert r["samples"] == 3                    # 1.00, 1.02 and 1.04 (one period of slack)
    assert r["sm_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]     # the idle-time thermal sample is outside


def test_falls_back_to_the_whole_run_and_flags_rejected_reasons():
    c = _sampler([(0.0, _line(1900)), (0.5, _line(1800, thermal="Active"))])
    c.mark(2.0, 2.1)
    r = c.stop()
    assert r["scope"] == "whole sampler run"
    assert r["samples"] == 2
    assert r["reasons"] == ["sw_thermal_slowdown"]


def test_no_sampler_gives_no_record():
    assert bench.Clocks(0).stop() is None
