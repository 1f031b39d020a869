"""Host logic of the benchmark (no GPU): DRAM traffic figures are reported
only while the captured kernel's source is byte-identical (sha256); a changed
kernel reports none until it is captured again."""
import hashlib
import os

import bench


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {("w", "m2l"): ("k.cu", sha, 123.0e6)})
    assert bench.traffic_for("w", "m2l") == 123.0e6
    assert bench.traffic_for("w", "p2p") is None          # no capture for this stage
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for("w", "m2l") is None          # kernel changed since the capture
    os.remove(src)
    assert bench.traffic_for("w", "m2l") is None          # source gone

