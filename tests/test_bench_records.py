"""The bench's measurement bookkeeping on CPU: an ncu traffic record is used
only for the kernel sources it was taken on, is scaled to one step, and feeds
the roofline's DRAM fraction; the whole-job rate and the FP64 arithmetic
roofline follow their definitions."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write_records(tmp_path, records):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "sem_step_kernel_traffic.json").write_text(json.dumps({"note": "test", "records": records}))


def _record(**kw):
    r = {"workload": "graded_512x512_p4", "precision": "fp32_kahan", "ordering": "hilbert", "stream_order": "step",
         "kernel": "sem_stream_kernel<5, float, MODE_KAHAN>", "steps_per_launch": 32,
         "dram_bytes_per_launch": 32 * 170e6, "kernel_sha256": "abc"}
    r.update(kw)
    return r


def test_record_matches_only_its_kernel_sources(tmp_path, monkeypatch):
    _write_records(tmp_path, [_record()])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "abc")
    # per step: the launch's bytes over the steps it ran
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_stream_kernel") == pytest.approx(170e6)
    # another workload, ordering, precision, kernel or metric source: no record
    assert bench.recorded_traffic("fp32_kahan", "random", "sem_stream_kernel") is None
    assert bench.recorded_traffic("fp64", "hilbert", "sem_stream_kernel") is None
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_step_kernel") is None
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_stream_kernel", metric="stored") is None
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_stream_kernel",
                                  workload="layered_4096x1024_p4") is None
    # the kernel sources changed since the capture: the record is not used
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "def")
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_stream_kernel") is None


def test_missing_or_broken_record_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_stream_kernel") is None
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "sem_step_kernel_traffic.json").write_text("{not json")
    assert bench.recorded_traffic("fp32_kahan", "hilbert", "sem_stream_kernel") is None


def test_hbm_roofline_dram_fraction(tmp_path, monkeypatch):
    _write_records(tmp_path, [_record()])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "abc")
    r = {"nodes": 4198401, "steps_per_launch": 20.0, "step_kernel_us": 40.0, "kernel": "sem_stream_kernel",
         "compulsory_bytes_per_step": 150e6}
    out = bench.hbm_roofline(r, "fp32_kahan", 6800.0, "measured", "graded_512x512_p4")
    algo = bench.ALGO_BYTES["fp32_kahan"]
    # achieved: algorithmic bytes of one launch over the launch's duration
    assert out["launch_us"] == pytest.approx(800.0)
    assert out["achieved"] == pytest.approx(algo * 4198401 * 20 / 800e-6 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 6800.0)
    # traffic per launch and the DRAM fraction from the record
    assert out["traffic"] == pytest.approx(170e6 * 20)
    assert out["dram_frac"] == pytest.approx(170e6 / 40e-6 / 1e9 / 6800.0)
    assert out["compulsory_frac"] == pytest.approx(150e6 / 40e-6 / 1e9 / 6800.0)


def test_job_rate_and_fp64_roofline():
    # weak scaling: every rank's nodes over the slowest rank's time
    assert bench.job_rate(4, 1000, 10, 2.0) == pytest.approx(20000.0)
    r = {"nodes": 1000000, "step_kernel_us": 100.0, "kernel": "sem_stream_kernel"}
    out = bench.fp64_roofline(r)
    tf = bench.FLOPS_FP64_LEAPFROG * 1e6 / 100e-6 / 1e12
    assert out["achieved"] == pytest.approx(tf)
    assert out["frac"] == pytest.approx(tf / bench.FP64_PEAK_TFLOPS)
    assert bench.cores_busy(12.0, 1.0) == 12 and bench.cores_busy(0.1, 1.0) == 1
    assert bench.rel_l2([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert bench.rel_l2([0.0], [0.0]) == 0.0
