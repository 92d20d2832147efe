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


def test_step_time_summary_shows_a_stall():
    s = bench.step_time_summary([2.0, 2.1, 1.9, 9.0], host_ms=15.2)
    assert s["median_ms"] == 2.1 and s["min_ms"] == 1.9 and s["max_ms"] == 9.0
    assert s["host_wall_ms_per_step"] == 3.8


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 lanes x 2 FLOPs x 2070 MHz
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.55) < 0.01


def test_stage_bytes_are_the_stated_per_unit_sums():
    b = bench.stage_bytes(N=10, C=4, V=3, K=7, ntiles=2, npix=5)
    assert b["preprocess"] == 10 * 48 + 4 * (4 + 192 + 112 + 56 + 8)
    assert b["sort"] == 4 * 152 + 7 * 44 + 2 * 20
    assert b["loss"] == 5 * 72
    assert b["preprocess_bwd"] == 4 * 8 + 3 * (64 + 3 * 232)
    assert b["densify"] == 10 * 118


def test_stage_roofline_fractions():
    info = {"n_candidates": 4, "n_visible": 3, "n_instances": 7, "tiles_x": 2, "tiles_y": 1,
            "pairs_evaluated": 100, "pairs_blended": 40, "bwd_pairs_evaluated": 90}
    r = bench.stage_roofline(info, {"loss": 1e-3, "blend_fwd": 1e-3}, 10, 5, 152, 2070.0, 1000.0)
    assert r["loss"]["frac"] == round(5 * 72 / 1e-6 / 1e9 / 1000.0, 4)
    flops = bench.FLOP_EVAL * 100 + bench.FLOP_BLEND * 40
    assert r["blend_fwd"]["flops"] == flops and "blend_bwd" not in r
