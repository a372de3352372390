"""Host helpers of bench.py that the JSON line is built from (no GPU needed): the algorithmic
work per pair, the code-only source hash that guards the recorded DRAM traffic, and the
reading of the measured peaks."""
import json
import math

import numpy as np

import bench
from paper_1507_05156_gb300 import inputs


def test_algorithmic_flops_per_pair_is_two_ffts_plus_pointwise_work():
    # 10 N log2 N (two 3-D FFTs at 5 N log2 N) + 16 N (pair product 6, kernel 2, MAC 8)
    for n in (12, 16, 20, 24):
        N = n ** 3
        assert bench.algorithmic_flops_per_pair(N) == 10.0 * N * math.log2(N) + 16.0 * N
    # the bench workload's figure per apply: 1,048,576 pairs at 20^3
    c = inputs.workload(1)
    assert c.pairs == 64 * 16 * 64 * 16
    assert abs(bench.algorithmic_flops_per_pair(8000) * c.pairs - 1.2216e12) < 1e9


def test_fp32_peak_is_lanes_times_clock():
    # SMs x 128 FP32 FMA lanes x 2 flop x clock, with the SM count of the device at hand
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(bench.fp32_peak_tflops(160, 2000.0) - 160 * 128 * 2 * 2.0e9 / 1e12) < 1e-9


def test_max_sm_clock_prefers_the_sampled_figure(tmp_path, monkeypatch):
    assert bench.max_sm_mhz({"sm_max_mhz": 1980.0})[0] == 1980.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"sm_max_mhz": 2070.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.max_sm_mhz({"sm_max_mhz": None}) == (2070.0, "MEASURED_PEAKS.json sm_max_mhz")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.max_sm_mhz(None)[0] == bench.DEFAULT_SM_MHZ


def test_bench_workload_is_the_largest_single_gpu_config():
    spec = inputs.WORKLOADS[bench.WORKLOAD]
    assert spec["grid"] == (24, 24, 24) and spec["kmesh"] == (8, 8, 8)
    assert spec["n_occ"] == 16 and spec["n_occ"] + spec["n_empty"] == 32
    pairs = 512 * 32 * 512 * 16
    assert pairs == 134_217_728
    # the reference arm's per-step sample: one target against REF_KPRIME k' of 16 bands
    assert bench.REF_KPRIME * 16 == 1024


def test_code_only_ignores_comments_and_blank_lines():
    a = "int x = 1;  // one\n/* block\n comment */\n\nint y = 2;\n"
    b = "int x = 1;\n// other words\nint y = 2;   \n"
    assert bench._code_only(a) == bench._code_only(b) == "int x = 1;\nint y = 2;"
    assert bench._code_only("int x = 1;\n") != bench._code_only("int x = 2;\n")


def test_kernel_source_sha_is_stable_and_short():
    s = bench.kernel_source_sha()
    assert s == bench.kernel_source_sha()
    assert len(s) == 16 and all(ch in "0123456789abcdef" for ch in s)


def test_measured_peak_reads_the_file_or_returns_none(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops": 1928.7, "hbm_gbs": "x"}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._measured_peak("bf16_tflops") == 1928.7
    assert bench._measured_peak("hbm_gbs") is None      # not a number
    assert bench._measured_peak("missing") is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench._measured_peak("bf16_tflops") is None


def test_workload_shapes_match_the_stated_configs():
    w = {k: inputs.WORKLOADS[k] for k in inputs.WORKLOADS}
    assert w[1]["grid"] == (20, 20, 20) and w[1]["kmesh"] == (4, 4, 4) and w[1]["n_occ"] == 16
    assert w[2]["grid"] == (24, 24, 24) and w[2]["kmesh"] == (8, 8, 8) and w[2]["n_occ"] + w[2]["n_empty"] == 32
    assert np.prod(w[0]["kmesh"]) == 8 and np.prod(w[4]["kmesh"]) == 27


def test_clock_summary_reads_median_clock_and_throttle_reasons():
    # nvidia-smi --format=csv,noheader,nounits lines: index, clocks.sm, clocks.max.sm, power,
    # active mask, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    s = bench.ClockSampler(0)
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line", ""]
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.lines = ["0, 1400, 2070, 500.0, 0x8, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
