"""Host logic of bench.py that needs no GPU: the roofline's DRAM traffic is
reported only while the update kernel's sources match the capture it came
from, and the method's flop counts follow the step formulas."""
import hashlib
import os

import bench


def _sources_hash():
    h = hashlib.sha256()
    for f in bench.TRAFFIC_SOURCES:
        with open(os.path.join(bench.ROOT, "paper_2603_16644_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_traffic_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    good = tmp_path / "good.md"
    good.write_text(f"summary\n\ntraffic_bytes_per_launch: 123456789\nsource_sha16: {_sources_hash()}\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(good))
    assert bench.update_traffic() == 123456789.0
    stale = tmp_path / "stale.md"
    stale.write_text("traffic_bytes_per_launch: 123456789\nsource_sha16: 0000000000000000\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(stale))
    assert bench.update_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.update_traffic() is None


def test_committed_traffic_capture_parses():
    # the committed summary carries both machine-readable fields
    with open(bench.TRAFFIC_PROFILE) as f:
        text = f.read()
    assert "traffic_bytes_per_launch: " in text and "source_sha16: " in text


def test_method_flops_follow_the_step_formulas():
    m, n, s = 262144, 4096, 8192
    f = bench.method_flops(m, n, s, False)
    assert f["sketch"] == 2.0 * s * m * n
    assert f["trsm"] == float(m) * n * n
    assert f["gram"] == float(m) * n * n
    assert f["qr"] == 2.0 * n * n * (s - n / 3)
    assert abs(f["factor"] - n ** 3 / 3.0) < 1.0
