"""Host-side logic of bench.py that needs no GPU: the clock sampler's parsing of
nvidia-smi output (median and maximum SM clock, throttle reasons) and the
whole-job rate."""
import bench


class FakeProc:
    def __init__(self, out):
        self.out = out
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.out, ""

    def kill(self):
        pass


def sampler_with(lines):
    s = bench.ClockSampler(0)
    s.proc = FakeProc("\n".join(lines) + "\n")
    return s


def test_clock_sampler_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1101.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = sampler_with(rows)
    out = s.stop()
    assert s.proc.terminated
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3


def test_clock_sampler_reports_thermal_and_hw_slowdown():
    rows = ["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active",
            "0, 1600, 2070, 1400, 0x48, Not Active, Not Active, Active, Not Active"]
    out = sampler_with(rows).stop()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1550.0


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    s.proc = None
    assert s.stop()["reasons"] == ["unsampled"]


def test_job_rate_counts_every_rank():
    assert bench.job_rate(1, 1000, 2.0) == 500.0
    assert bench.job_rate(4, 1000, 2.0) == 2000.0
