"""Host-side arithmetic of bench.py without a GPU: the roofline records, the
conservation drift and the CPU description are computed from their stated
models (no device work)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_derived_peaks():
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(bench.FP32_PEAK_TFLOPS / 64)


def test_step_roofline_picks_the_larger_bound():
    n, pairs, cands = 1_000_000, 100_000_000, 450_000_000
    r = {"pairs": pairs, "candidates": cands}
    hbm = bench.peaks().get("hbm_gbs")
    out = bench.step_roofline(r, n, "fp32_mixed", ms_step=10.0)
    b = bench.STEP_BYTES["fp32_mixed"]
    assert out["bytes_per_step"] == b["particle"] * n + b["entry"] * pairs
    flops = bench.FLOPS["find"] * cands + sum(bench.FLOPS[k] for k in ("density", "iad", "momentum")) * pairs
    assert out["flops_per_step"] == flops
    alu_ms = (bench.FLOPS["find"] * cands + (flops - bench.FLOPS["find"] * cands)) / (
        bench.FP32_PEAK_TFLOPS * 1e12) * 1e3
    assert out["alu_ms"] == pytest.approx(alu_ms)
    if hbm:
        assert out["hbm_ms"] == pytest.approx(out["bytes_per_step"] / (hbm * 1e9) * 1e3)
        assert out["bound"] == ("alu" if out["alu_ms"] >= out["hbm_ms"] else "hbm")
    assert out["frac"] == pytest.approx(out["time_ms"] / 10.0)
    # FP64: the pair flops run on the FP64 pipe
    out64 = bench.step_roofline(r, n, "fp64", ms_step=100.0)
    pair64 = sum(bench.FLOPS64[k] for k in ("density", "iad", "momentum")) * pairs
    find_ms = bench.FLOPS["find"] * cands / (bench.FP32_PEAK_TFLOPS * 1e12) * 1e3
    assert out64["alu_ms"] == pytest.approx(find_ms + pair64 / (bench.FP64_PEAK_TFLOPS * 1e12) * 1e3)


def test_kernel_roofline_uses_the_slowest_stage():
    r = {"stages": {"sort": 1.0, "find": 6.0, "density": 2.0, "iad": 2.0, "momentum": 6.5,
                    "dt": 0.1, "update": 0.8},
         "pairs": 8.5e8, "candidates": 3.7e9}
    out = bench.roofline(r, 8_416_298, "fp32_mixed")
    assert out["kernel"] == "momentum (fp32_mixed)"
    assert out["flops_per_launch"] == pytest.approx(bench.FLOPS["momentum"] * 8.5e8)
    assert out["achieved"] == pytest.approx(bench.FLOPS["momentum"] * 8.5e8 / 6.5e-3 / 1e12)
    assert out["frac"] == pytest.approx(out["achieved"] / bench.FP32_PEAK_TFLOPS)
    r["stages"]["find"] = 7.0
    out = bench.roofline(r, 8_416_298, "fp32_mixed")
    assert out["kernel"] == "find (fp32_mixed)"
    assert out["flops_per_launch"] == pytest.approx(bench.FLOPS["find"] * 3.7e9)


def test_conservation_drift():
    d0 = [1.0, 2.0, 3.0, 4.0, 6.0, 0.0, 0.0, 0.0]
    d1 = [1.5, 2.0, 2.0, 4.5, 6.5, 0.0, 0.0, 0.0]
    out = bench.conservation(d0, d1, steps=4)
    assert out["energy_rel_change_per_step"] == pytest.approx((11.0 - 10.0) / 10.0 / 4)
    assert out["momentum_change"] == [0.5, 0.0, -1.0]


def test_traffic_record_matches_its_source_hash():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, rec in t.items():
        assert rec["bytes_per_launch"] == pytest.approx(
            rec["captured_bytes"] * rec["scaled_to_particles"] / rec["captured_particles"])
        # a record is reported only while its kernel sources are unchanged
        value = bench.traffic_for(key)
        assert value is None or value == rec["bytes_per_launch"]


def test_host_cpu_description():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["machine"]
