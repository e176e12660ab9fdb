"""CPU test of the benchmark's clock record: nvidia-smi samples of the timed
region are parsed into the median SM clock, the maximum and the throttle
reasons seen, and the timing rule is applied to them."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _clk(bench, rows):
    c = bench.Clocks()
    c.samples = [[x.strip() for x in r.split(",")] for r in rows]
    return c.stop()


def test_clean_run_is_ok():
    b = _bench()
    rows = ["2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"] * 5
    out = _clk(b, rows)
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070 and out["reasons"] == []
    assert out["rule"] == "ok" and out["samples"] == 5


def test_power_cap_is_kept_and_noted():
    b = _bench()
    rows = ["1850, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"] * 3
    out = _clk(b, rows)
    assert out["reasons"] == ["sw_power_cap"] and out["rule"].startswith("ok")


def test_thermal_slowdown_rejects():
    b = _bench()
    rows = ["2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
            "1500, 2070, 900, 0x0, Not Active, Active, Not Active, Not Active"]
    out = _clk(b, rows)
    assert "hw_thermal_slowdown" in out["reasons"] and out["rule"].startswith("rejected")


def test_clock_lock_without_reason_rejects():
    b = _bench()
    rows = ["1200, 2070, 500, 0x0, Not Active, Not Active, Not Active, Not Active"] * 4
    out = _clk(b, rows)
    assert out["rule"].startswith("rejected: SM clock 1200")


def test_no_samples_is_unknown():
    b = _bench()
    out = _clk(b, [])
    assert out["rule"].startswith("unknown") and out["sm_mhz"] is None
