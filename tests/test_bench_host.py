"""Host logic of bench.py that decides whether a measurement stands: the
clock record taken during the timed region (median SM clock, maximum clock,
throttle reasons seen) and the workload description of the JSON line."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def __init__(self):
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def wait(self, timeout=None):
        return 0


class _Thread:
    def join(self, timeout=None):
        pass


def _stopped(lines):
    c = bench.ClockSampler(0)
    c.proc, c.t, c.lines = _Proc(), _Thread(), list(lines)
    return c.stop(), c.proc


def _row(sm, mx=2070, power=900.0, active="0x0000000000000000", hw="Not Active", hwt="Not Active",
         swt="Not Active", cap="Not Active"):
    return "0, %s, %s, %s, %s, %s, %s, %s, %s" % (sm, mx, power, active, hw, hwt, swt, cap)


def test_median_clock_and_no_reason():
    rec, proc = _stopped([_row(2070), _row(1995), _row(2070), _row(2055), _row(2070)])
    assert proc.terminated
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_reasons_seen_in_any_sample_are_reported():
    rec, _ = _stopped([_row(2070), _row(1900, cap="Active"), _row(1500, hwt="Active"), _row(2070)])
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert rec["sm_mhz"] == 2070.0   # upper median of 1500, 1900, 2070, 2070
    assert rec["samples"] == 4


def test_unreadable_lines_are_skipped():
    rec, _ = _stopped(["", "No devices were found", "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, "
                       "Not Active, Not Active", _row(1980), "0, 1, 2"])
    assert rec == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1}


def test_no_sample_gives_no_record():
    assert _stopped([])[0] is None
    c = bench.ClockSampler(0)        # nvidia-smi could not be started
    assert c.stop() is None


def test_workload_description_names_the_measured_configuration():
    cfg = bench._workload_config()
    assert cfg["n_photons"] == bench.N_PHOTONS and cfg["tau"] == bench.TAU
    assert cfg["image"] == [bench.NZ, bench.NX] and cfg["n_radial"] == bench.N_RADIAL
    assert "flushed" in cfg["l2"]
    assert "%.0e photons" % bench.N_PHOTONS in cfg["workload"]


def test_single_process_job_rate():
    import torch
    rate, t_max, total = bench.job_rate(2.0, 5e9, 1, torch.device("cpu"))
    assert (t_max, total) == (2.0, 5e9) and rate == pytest.approx(2.5e9)
