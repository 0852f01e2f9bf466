"""Host logic of bench.py that the JSON line rests on: the recorded DRAM
traffic is used only for the kernel source it was captured from, the peak
falls back when the measured file is absent, and throughput is whole-job
cells x steps over the slowest rank's time."""
import json

import pytest

import bench


def write_record(path, sha, bpc=147.9):
    path.write_text("# a capture\n\nkernel_source_sha256_16: %s\ndram_bytes_per_cell: %s\ncells_captured: 8388608\n"
                    % (sha, bpc))


def test_traffic_record_applies_only_to_the_captured_source(tmp_path, monkeypatch):
    rec = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    write_record(rec, bench.kernel_hash())
    assert bench.recorded_traffic(1000) == pytest.approx(147.9e3)
    write_record(rec, "0" * 16)                     # captured from another source: no traffic
    assert bench.recorded_traffic(1000) is None
    rec.write_text("kernel_source_sha256_16: %s\n" % bench.kernel_hash())   # no figure
    assert bench.recorded_traffic(1000) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.recorded_traffic(1000) is None


def test_kernel_hash_follows_the_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("a")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    h = bench.kernel_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    src.write_text("b")
    assert bench.kernel_hash() != h


def test_peak_is_measured_else_fallback(tmp_path, monkeypatch):
    peaks = tmp_path / "peaks.json"
    peaks.write_text(json.dumps({"hbm_gbs": 6780.7, "bf16_tflops": 1900}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(peaks))
    assert bench.hbm_peak() == (6780.7, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "absent.json"))
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")


def test_job_throughput_is_whole_job_over_the_slowest_rank():
    # 33.5 M cells, 2000 steps on each of 4 replicas in 1.7 s (the slowest rank)
    cells = 512 * 256 * 256
    v = bench.job_mlups(cells, 2000, 4, 1700.0)
    assert v == pytest.approx(cells * 2000 * 4 / 1.7 / 1e6)
