"""The bench's clocks summary on CPU: samples are selected by nvidia-smi's own
timestamps, so only those inside the timed region count; a region shorter
than the sampling interval falls back to the two samples around it; a
throttle reason seen in the region is reported."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

T0 = datetime.datetime(2026, 1, 2, 3, 4, 5).timestamp()
OFF = "Not Active"


def _line(dt, sm, power_cap=False, thermal=False):
    ts = datetime.datetime.fromtimestamp(T0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = [OFF, "Active" if thermal else OFF, OFF, "Active" if power_cap else OFF]
    return f"{ts}, 0, {sm}, 2032, 412.25, 0x0000000000000000, " + ", ".join(flags) + "\n"


def _clocks(lines, region):
    c = bench.Clocks(0)
    c.lines = lines
    c.region = region
    return c.summary()


def test_only_samples_inside_the_region_count():
    lines = [_line(-0.5, 900, thermal=True), _line(0.10, 2032), _line(0.30, 1995, power_cap=True),
             _line(0.50, 2032), _line(2.0, 600, thermal=True)]
    s = _clocks(lines, (T0, T0 + 0.5))
    assert s["window"] == "timed region"
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"]          # the thermal samples lie outside


def test_short_region_takes_the_bracketing_samples():
    lines = [_line(-1.0, 700), _line(-0.05, 2010), _line(0.08, 2032), _line(1.0, 800)]
    s = _clocks(lines, (T0, T0 + 0.002))
    assert s["window"].startswith("the two samples bracketing")
    assert s["samples"] == 2 and s["sm_mhz"] == 2032.0


def test_unreadable_timestamps_use_every_sample():
    lines = [_line(0.0, 2000).replace(_line(0.0, 2000).split(",")[0], "n/a"), _line(0.1, 1800)]
    s = _clocks(lines, (T0, T0 + 1.0))
    assert s["window"].startswith("whole sampler run")
    assert s["samples"] == 2


def test_no_sampler_gives_none():
    assert _clocks([], None) is None
    assert bench.Clocks.parse("garbage") is None
