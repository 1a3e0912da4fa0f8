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


def test_accuracy_report_counts_queries_above_each_bar():
    # the benchmark's accuracy object: per bandwidth, the errors of the benchmarked form
    # and of the plain form against the oracle values, and how many queries break their
    # form's bar (error above it with kappa at or below the form's kappa0)
    import numpy as np
    import oracle
    rng = np.random.default_rng(1)
    X = rng.normal(size=(400, 3)).astype(np.float32)
    Q = rng.normal(size=(50, 3)).astype(np.float32)
    a = 0.5
    ref = oracle.kde(X, Q, a)
    tc = ref * (1 + 1e-6)
    tc[3] *= 1 + 5e-4      # breaks 1e-4 (kappa is small here)
    plain = ref * (1 - 2e-7)
    plain[7] *= 1 + 3e-5   # breaks 1e-5
    acc = bench.accuracy(X, Q, [a], ["gaussian"], [tc], [plain], [ref], 2)
    e = acc[0]
    assert e["queries"] == 50
    assert e["bench_form"]["above_0.0001"] == 1 and e["bench_form"]["above_0.0001_with_kappa_le_400"] == 1
    assert e["simt_f32"]["above_1e-05"] == 1 and e["simt_f32"]["above_1e-05_with_kappa_le_40"] == 1
    assert abs(e["bench_form"]["max_rel_err"] - 5e-4) < 2e-5


def test_roofline_uses_the_given_sm_count():
    r = bench.roofline_for("tc", 16, 1e10, 1.5, {"sm_mhz": 2000.0}, {"bf16_tflops": 1900.0}, 100)
    assert r["bound"] == "alu" and abs(r["peak"] - 32 * 100 * 2e9 / 1e12) < 1e-9
    r = bench.roofline_for("tc", 16, 1e10, 1.5, {"sm_mhz": 2000.0}, {"bf16_tflops": 1900.0}, 152, ex2_measured=9.5e12)
    assert abs(r["mufu_frac_of_probe"] - 1e10 / 1.5e-3 / 9.5e12) < 1e-9
