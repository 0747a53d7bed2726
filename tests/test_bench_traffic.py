"""The bench reports the frontier kernel's DRAM traffic from the committed ncu
summary only while that summary was taken on the current kernel source."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_follows_the_kernel_source_digest(tmp_path, monkeypatch):
    b = _bench()
    dig = b.kernel_source_digest()
    assert len(dig) == 16
    good = tmp_path / "good.txt"
    good.write_text(f"# comment: 1\nkernel_source_sha256_16: {dig}\ndram_bytes_per_launch: 12345\n")
    monkeypatch.setattr(b, "PROFILE", str(good))
    assert b.profiled_traffic() == 12345
    stale = tmp_path / "stale.txt"
    stale.write_text("kernel_source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 12345\n")
    monkeypatch.setattr(b, "PROFILE", str(stale))
    assert b.profiled_traffic() is None
    monkeypatch.setattr(b, "PROFILE", str(tmp_path / "missing.txt"))
    assert b.profiled_traffic() is None
