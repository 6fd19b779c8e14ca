"""Host logic of bench.py's clock record (no GPU): samples are kept when
their nvidia-smi timestamps fall in the timed region, and throttle reasons
are collected from those samples only."""
import datetime
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _line(t, sm, reasons=()):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if n in reasons else "Not Active"
             for n in ("hw", "hwt", "swt", "pc")]
    return ", ".join([ts, str(sm), "2070", "900.0"] + flags)


def test_samples_inside_the_region_decide():
    c = bench.ClockSampler(0)
    base = 1.8e9
    c.lines = [_line(base, 1000, ("hwt",)), _line(base + 1.0, 2070), _line(base + 1.02, 2055),
               _line(base + 1.04, 2070, ("pc",)), _line(base + 2.0, 900)]
    c.t0, c.t1 = base + 0.99, base + 1.05
    s = c.summary()
    assert s["samples_in_timed_region"] == 3 and s["samples"] == 3
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]


def test_no_sample_in_region_falls_back_to_all():
    c = bench.ClockSampler(0)
    base = 1.8e9
    c.lines = [_line(base, 2070), _line(base + 0.5, 2060)]
    c.t0, c.t1 = base + 0.1, base + 0.2
    s = c.summary()
    assert s["samples_in_timed_region"] == 0 and s["samples"] == 2
    assert bench.ClockSampler(0).summary() is None
