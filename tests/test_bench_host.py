"""Host logic of the benchmark (no GPU): DRAM traffic figures are reported
only while the captured kernel's sources are byte-identical (sha256 over the
listed files, in order); a changed kernel or header reports none until it is
captured again."""
import hashlib
import os

import bench


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    src, hdr = tmp_path / "k.cu", tmp_path / "k.cuh"
    src.write_text("__global__ void k() {}\n")
    hdr.write_text("#pragma once\n")
    sha = hashlib.sha256(src.read_bytes() + hdr.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {("w", "m2l"): (("k.cu", "k.cuh"), sha, 123.0e6)})
    assert bench.traffic_for("w", "m2l") == 123.0e6
    assert bench.traffic_for("w", "p2p") is None          # no capture for this stage
    hdr.write_text("#pragma once\n// changed\n")
    assert bench.traffic_for("w", "m2l") is None          # a header changed since the capture
    hdr.write_text("#pragma once\n")
    assert bench.traffic_for("w", "m2l") == 123.0e6
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for("w", "m2l") is None          # kernel changed since the capture
    os.remove(src)
    assert bench.traffic_for("w", "m2l") is None          # source gone
