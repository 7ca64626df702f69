"""Host logic of the benchmark's roofline fields (no GPU): the DRAM traffic
comes from the committed ncu summary only while the kernel source is the
file it was captured on, and the peak comes from the measured-peaks file,
else from the stated fallback."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "kernels_pr.cu"
    src.write_bytes(b"// kernel, first version\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "summary.md"
    prof.write_text("kernels_pr.cu sha256: %s\n(notes)\ntraffic per 50-body launch: 123456789 bytes\n" % digest)
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(prof))
    assert bench._traffic_per_launch() == 123456789
    src.write_bytes(b"// kernel, edited after the capture\n")
    assert bench._traffic_per_launch() is None
    src.write_bytes(b"// kernel, first version\n")
    prof.write_text("kernels_pr.cu sha256: %s\n" % digest)   # no traffic line
    assert bench._traffic_per_launch() is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench._traffic_per_launch() is None


def test_peak_from_measured_file_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.5, "bf16_tflops": 1900.0}))
    assert bench._peaks() == (6783.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    assert bench._peaks() == (6800.0, "fallback")
