"""Host-side logic of the benchmark, on the CPU: the defaults of the command
line, the peak lookup, the guard that reports a captured DRAM traffic only for
the kernel sources it was taken on, and the config object of the JSON line."""
import json

import bench


def test_defaults_run_one_gpu_with_enough_warmup():
    a = bench.parse([])
    assert a.gpus == 1 and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 1
    assert (a.width, a.height) == (1600, 900)


def test_measured_peak_reads_the_file_and_falls_back(tmp_path, monkeypatch):
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0}
    root = tmp_path / "repo"
    root.mkdir()
    (root / "MEASURED_PEAKS.json").write_text(json.dumps(peaks))
    monkeypatch.setattr(bench, "__file__", str(root / "bench.py"))
    assert bench.measured_peak("bf16_tflops") == 1800.0
    (root / "MEASURED_PEAKS.json").unlink()
    assert bench.measured_peak("bf16_tflops") == bench.FALLBACK_PEAKS["bf16_tflops"]


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    same = {"bytes": 123, "sources_sha256": bench.blend_sources_sha256()}
    monkeypatch.setattr(bench, "BLEND_BWD_TRAFFIC", same)
    assert bench.blend_bwd_traffic() == 123
    monkeypatch.setattr(bench, "BLEND_BWD_TRAFFIC", dict(same, sources_sha256="0" * 64))
    assert bench.blend_bwd_traffic() is None


def test_config_names_the_workload_without_model_keys():
    c = bench.workload_config(1600, 900, 2)
    assert "workload" in c and "1600x900" in c["workload"]
    assert c["views_per_step"] == 2 and c["surfels"] == bench.N_SURFELS
    assert not {"model", "global_batch", "seq_len"} & set(c)
    assert "L2" in c["l2"]
