"""The bench's clock summary on CPU: only samples written after the sampler's first one (the start
of the timed region) count, throttle reasons are collected, and a region shorter than one sampling
interval falls back to the sample taken just before it."""
import os
import tempfile

import bench

PRE = "0, 2070, 2070, 310.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
IN = ("0, 1950, 2070, 1210.5, 0x4, Not Active, Not Active, Not Active, Active\n"
      "0, 2010, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
      "0, 1990, 2070, 1240.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")


def _sampler(text, skip):
    c = bench.ClockSampler(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write(text)
    c.skip = skip
    c.proc = object()  # stands for the nvidia-smi process (not used by the summary)
    return c


def test_samples_inside_the_region_only():
    s = _sampler(PRE + IN, len(PRE)).summary()
    assert s == {"sm_mhz": 1990.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_region_shorter_than_one_interval_uses_the_last_sample_before_it():
    s = _sampler(PRE, len(PRE)).summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 0}


def test_no_sampler_gives_no_summary():
    assert bench.ClockSampler(0).summary() is None
