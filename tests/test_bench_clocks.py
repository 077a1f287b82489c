"""bench.py's clock sampler on CPU, against a fake NVML: the median SM clock,
the maximum, and which clock-event reasons a run saw (idle and other bits that
do not reject a run are not reported); and its fallback when NVML cannot find
the device. Nothing here touches a GPU."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeNVML:
    """The part of pynvml's interface the sampler uses; bit values as NVML's."""
    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonGpuIdle = 0x1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self, clocks, reasons, known_uuid="GPU-test"):
        self.clocks, self.reasons, self.known = clocks, reasons, known_uuid
        self.n = 0
        self.queried = []

    def nvmlInit(self):
        pass

    def nvmlDeviceGetHandleByUUID(self, uuid):
        if uuid != self.known:
            raise RuntimeError("NVML_ERROR_NOT_FOUND")
        return ("handle", uuid)

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        assert kind == self.NVML_CLOCK_SM
        return 2032

    def nvmlDeviceGetClockInfo(self, h, kind):
        assert h == ("handle", self.known) and kind == self.NVML_CLOCK_SM
        v = self.clocks[min(self.n, len(self.clocks) - 1)]
        self.queried.append("clock")
        return v

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.reasons[min(self.n, len(self.reasons) - 1)]
        self.n += 1
        return v


def _run(nv, uuid="GPU-test", seconds=0.08):
    s = bench.ClockSampler(0, tag="test", nvml=nv, uuid=uuid)
    with s:
        time.sleep(seconds)
    return s.summary()


def test_median_max_and_reasons():
    # five samples, then the last one repeats: median 2010, power cap seen, idle ignored
    nv = FakeNVML([2032, 2010, 1995, 2032, 2010], [0x0, 0x4, 0x1, 0x0, 0x1])
    r = _run(nv)
    assert r["source"].startswith("nvml")
    assert r["samples"] >= 5
    assert r["sm_max_mhz"] == 2032.0
    assert r["sm_mhz"] == 2010.0   # later samples repeat the last one (2010)
    assert r["reasons"] == ["sw_power_cap"]


def test_every_rejecting_reason_is_named():
    nv = FakeNVML([1500], [0x8 | 0x20 | 0x40])
    r = _run(nv)
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1500.0


def test_samples_every_10_ms():
    nv = FakeNVML([2032], [0])
    r = _run(nv, seconds=0.2)
    assert 8 <= r["samples"] <= 30   # ~20 at 10 ms


def test_device_not_found_falls_back_without_raising():
    nv = FakeNVML([2032], [0])
    r = _run(nv, uuid="GPU-other", seconds=0.01)
    assert not nv.queried            # NVML was never sampled
    assert r.get("source") != "nvml, 10 ms"
    assert "sm_mhz" in r and "reasons" in r
