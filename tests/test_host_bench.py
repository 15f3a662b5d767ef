"""Host logic of the benchmark (no GPU): clock-sample parsing, the ncu traffic gate, peaks."""
import hashlib

import pytest

import bench


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _clocks_with(text):
    c = bench.Clocks.__new__(bench.Clocks)
    c.proc = _FakeSmi(text)
    return c


def test_clock_samples_median_under_load_and_reasons(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    rows = [
        "345, 2070, 120.5, Not Active, Not Active, Not Active, Not Active",  # idle sample
        "2070, 2070, 350.0, Not Active, Not Active, Not Active, Active",
        "2040, 2070, 360.2, Not Active, Not Active, Not Active, Active",
        "2055, 2070, 355.0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = _clocks_with("\n".join(rows)).stop()
    assert out["sm_mhz"] == 2055.0  # median of the loaded samples (the idle one is left out)
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 4
    assert out["power_w_max"] == 360.2


def test_clock_throttle_reasons_are_named(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    rows = ["1500, 2070, 900.0, Active, Not Active, Active, Not Active",
            "1510, 2070, 905.0, Not Active, Active, Not Active, Not Active"]
    out = _clocks_with("\n".join(rows)).stop()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clocks_without_samples_or_tool(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    assert _clocks_with("").stop() is None
    c = bench.Clocks.__new__(bench.Clocks)
    c.proc = None
    assert c.stop() is None


def test_ncu_traffic_only_for_the_captured_sources(monkeypatch, tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k": (1234, digest, ("k.cu",)), "none": (None, digest, ("k.cu",))})
    assert bench.ncu_traffic("k") == 1234
    assert bench.ncu_traffic("none") is None
    assert bench.ncu_traffic("other") is None
    src.write_text("kernel v2\n")  # the kernel changed since the capture
    assert bench.ncu_traffic("k") is None


def test_peaks_fall_back_without_the_measurement(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6793.8, "bf16_tflops": 1913.2}')
    peaks, src = bench.measured_peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 6793.8


def test_fp32_peak_from_unit_counts():
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784)


def test_aggregate_single_rank():
    assert bench.aggregate(2.0, 1) == (2.0, 500.0)
