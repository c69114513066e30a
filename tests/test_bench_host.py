"""Host logic of bench.py that needs no GPU: the clock-log parsing that marks
a run as throttled or clean, and the whole-job value."""
import os

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _log(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_clock_log_clean_run(tmp_path):
    path = _log(tmp_path, [
        "0, 2070, 2070, 903.12, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 911.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 915.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 100.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",  # other GPU
    ])
    c = bench.clocks_stop(_FakeProc(), path, device_index=0)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    assert not os.path.exists(path)


def test_clock_log_reports_throttle_reasons(tmp_path):
    path = _log(tmp_path, [
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1500, 2070, 1400.0, 0x0000000000000048, Not Active, Active, Not Active, Active",
        "garbage line",
    ])
    c = bench.clocks_stop(_FakeProc(), path, device_index=0)
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert c["samples"] == 2 and c["sm_mhz"] == 1740.0


def test_clock_log_without_samples(tmp_path):
    assert bench.clocks_stop(_FakeProc(), _log(tmp_path, ["n/a"]), device_index=0) is None
    assert bench.clocks_stop(None, "unused") is None


def test_whole_job_value_counts_every_rank():
    # 4 ranks x 10 steps x 64 solves in 2.5 s of the slowest rank
    assert bench.whole_job_value(64, 10, 4, 2500.0) == 4 * 10 * 64 / 2.5
