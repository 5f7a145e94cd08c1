"""Host logic of bench.py that needs no GPU: the clock sampler's summary keeps the samples
taken during the timed region (fake sampler output, no NVML)."""
import importlib.util
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sampler(bench, lines, t0, t1):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc, s.error, s.lines, s.t0, s.t1 = None, None, lines, t0, t1
    return s


def test_summary_keeps_samples_inside_the_region():
    b = _bench()
    lines = ["max 2032", "s 0.99 1500 0 100.0", "s 1.00 2032 0 300.0", "s 1.01 2020 4 350.0", "s 1.02 2032 0 320.0",
             "s 1.10 900 64 90.0"]
    out = _sampler(b, lines, 1.0, 1.05).summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2032 and out["sm_max_mhz"] == 2032
    assert out["reasons"] == ["sw_power_cap"] and out["power_w_max"] == 350.0


def test_short_region_takes_the_next_sample():
    b = _bench()
    lines = ["max 2032", "s 0.99 1500 0 100.0", "s 1.03 2025 0 200.0", "s 1.04 2032 0 210.0"]
    out = _sampler(b, lines, 1.0, 1.01).summary()
    assert out["samples"] == 1 and out["sm_mhz"] == 2025


def test_no_samples_reports_unavailable():
    b = _bench()
    out = _sampler(b, ["max 2032"], 1.0, 1.01).summary()
    assert out["samples"] == 0 and out["reasons"] == ["unavailable"]
