"""Host logic of the benchmark that needs no GPU: the clock record keeps only the
nvidia-smi samples taken inside the timed region and reports the throttle reasons seen
there (a run that saw hw_slowdown or a thermal slowdown is rejected by the reader of the
record, sw_power_cap is kept and noted)."""
import datetime
import time

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _line(t, sm, power_cap="Not Active", hw="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, {sm}, 2070, 900.00, 0x0, {hw}, Not Active, Not Active, {power_cap}"


def _stop_at(sampler, t_end, monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    monkeypatch.setattr(bench.time, "time", lambda: t_end)
    return sampler.stop()


def test_samples_inside_the_region_only(monkeypatch):
    now = time.time()
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.t0 = now
    c.lines = [_line(now - 0.5, 1100, hw="Active"),          # before: ignored
               _line(now + 0.02, 1900, power_cap="Active"),
               _line(now + 0.04, 1950),
               _line(now + 0.30, 1200, hw="Active")]          # after: ignored
    rec = _stop_at(c, now + 0.10, monkeypatch)
    assert rec["samples"] == 2 and rec["window"] == "timed region"
    assert rec["sm_mhz"] == 1925.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_short_region_takes_the_next_sample(monkeypatch):
    now = time.time()
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.t0 = now
    c.lines = ["garbage line", _line(now - 0.1, 2070), _line(now + 0.015, 2055, hw="Active")]
    rec = _stop_at(c, now + 0.005, monkeypatch)
    assert rec["samples"] == 1 and rec["sm_mhz"] == 2055.0
    assert rec["reasons"] == ["hw_slowdown"]
    assert rec["window"].startswith("first sample after")


def test_no_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
