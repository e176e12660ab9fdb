"""CPU tests of the benchmark's DRAM traffic table: each entry holds the
bytes one pair visit moved in an ncu capture and the SHA-256 of the kernel
source it was captured from; the benchmark reports the traffic only while the
source still matches, so a stale figure can never appear in the line."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_kernel_class_has_a_traffic_entry():
    b = _bench()
    names = {"gram_f64", "inner_f64", "apply_f64", "gram_f32", "inner_f32", "apply_f32"}
    assert names <= set(b.TRAFFIC)


def test_traffic_entries_match_the_current_kernel_sources():
    # a kernel edited after its capture needs a new ncu capture (and hash)
    b = _bench()
    for name, ent in b.TRAFFIC.items():
        got = b.kernel_source_sha256(ent["source"], ent["kernel"])
        assert got is not None, "kernel %s not found in %s" % (ent["kernel"], ent["source"])
        assert got == ent["source_sha256"], "%s: %s changed since its DRAM capture" % (name, ent["kernel"])


def test_traffic_scales_with_the_visits_of_a_launch():
    b = _bench()
    for name, ent in b.TRAFFIC.items():
        one = b.traffic_per_launch(name, 1)
        assert one == ent["bytes_per_visit"] > 0
        assert b.traffic_per_launch(name, 64) == 64 * ent["bytes_per_visit"]
    assert b.traffic_per_launch("no_such_kernel", 64) is None


def test_a_changed_source_drops_the_traffic(monkeypatch):
    b = _bench()
    monkeypatch.setitem(b.TRAFFIC, "gram_f64", dict(b.TRAFFIC["gram_f64"], source_sha256="0" * 64))
    assert b.traffic_per_launch("gram_f64", 64) is None
