"""bench.py's clock record: nvidia-smi samples are kept when their
timestamps fall inside the timed region (all of them, flagged, when none
does); the median SM clock, the maximum clock and the throttle reasons
active in the kept samples are reported.  No GPU and no nvidia-smi: the
sampler reads a file written here."""
import os
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(t, sm, reasons=("Not Active",) * 4):
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(int(t))) + ".%03d" % (
        int(round((t - int(t)) * 1000)) % 1000)
    return ", ".join([stamp, str(sm), "2070", "900.00", "0x0", *reasons]) + "\n"


def _sampler(rows, t0, t1):
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.writelines(rows)
    s.proc = _Done()
    s.t0, s.t1 = t0, t1
    return s


def test_samples_inside_the_timed_region_are_kept():
    t0 = time.time()
    active = ("Not Active", "Not Active", "Not Active", "Active")  # sw_power_cap
    rows = [_row(t0 - 0.5, 1200), _row(t0 + 0.10, 2070), _row(t0 + 0.15, 2055, active),
            _row(t0 + 0.20, 2070), _row(t0 + 1.5, 900)]
    rec = _sampler(rows, t0, t0 + 0.3).stop()
    assert rec["in_region"] and rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_without_a_sample_in_the_region_all_are_reported_and_flagged():
    t0 = time.time()
    rows = [_row(t0 - 0.5, 2070), _row(t0 + 0.9, 2070)]
    rec = _sampler(rows, t0, t0 + 0.01).stop()
    assert not rec["in_region"] and rec["samples"] == 2


def test_timestamp_parsing():
    t = time.time()
    assert abs(bench.ClockSampler._stamp(_row(t, 1)[:23]) - t) < 2e-3
    assert bench.ClockSampler._stamp("not a time") is None
