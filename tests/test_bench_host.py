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


def _run(stages=None):
    return {"stages": stages or {"sort": 1.0, "find": 6.0, "density": 2.0, "iad": 2.0,
                                 "momentum": 6.5, "dt": 0.1, "update": 0.8},
            "pairs": 8.5e8, "candidates": 3.7e9, "slots": 1.0e8, "words": 6.0e7}


def test_step_roofline_picks_the_larger_bound():
    n = 1_000_000
    r = _run()
    hbm = bench.peaks().get("hbm_gbs")
    out = bench.step_roofline(r, n, "fp32_mixed", ms_step=10.0)
    kb = bench.KERNEL_BYTES["fp32_mixed"]
    expect = bench.OTHER_BYTES * n + sum(
        kb[k]["particle"] * n + kb[k]["slot"] * r["slots"] + kb[k]["word"] * r["words"] +
        kb[k]["entry"] * r["pairs"] for k in bench.PAIR_KERNELS)
    assert out["bytes_per_step"] == pytest.approx(expect)
    flops = bench.FLOPS["find"] * r["candidates"] + sum(
        bench.FLOPS[k] for k in ("density", "iad", "momentum")) * r["pairs"]
    assert out["flops_per_step"] == pytest.approx(flops)
    assert out["alu_ms"] == pytest.approx(flops / (bench.FP32_PEAK_TFLOPS * 1e12) * 1e3)
    if hbm:
        assert out["hbm_ms"] == pytest.approx(out["bytes_per_step"] / (hbm * 1e9) * 1e3)
        assert out["bound"] == ("alu" if out["alu_ms"] >= out["hbm_ms"] else "hbm")
    assert out["frac"] == pytest.approx(out["time_ms"] / 10.0)
    # the survey's 25 kflop / 1.9 KB per particle model beside it
    sv = out["survey_model"]
    assert sv["alu_ms"] == pytest.approx(25_000 * n / (bench.FP32_PEAK_TFLOPS * 1e12) * 1e3)
    if hbm:
        assert sv["hbm_ms"] == pytest.approx(1_900 * n / (hbm * 1e9) * 1e3)
    assert sv["frac"] == pytest.approx(sv["time_ms"] / 10.0)
    # FP64: the pair flops run on the FP64 pipe, the lists and W_ab are counted per entry
    out64 = bench.step_roofline(r, n, "fp64", ms_step=100.0)
    pair64 = sum(bench.FLOPS64[k] for k in ("density", "iad", "momentum")) * r["pairs"]
    find_ms = bench.FLOPS["find"] * r["candidates"] / (bench.FP32_PEAK_TFLOPS * 1e12) * 1e3
    assert out64["alu_ms"] == pytest.approx(find_ms + pair64 / (bench.FP64_PEAK_TFLOPS * 1e12) * 1e3)
    kb64 = bench.KERNEL_BYTES["fp64"]
    assert out64["bytes_per_step"] == pytest.approx(bench.OTHER_BYTES * n + sum(
        kb64[k]["particle"] * n + kb64[k]["entry"] * r["pairs"] for k in bench.PAIR_KERNELS))


def test_kernel_rooflines_both_roofs():
    r = _run()
    n = 8_416_298
    ks = bench.kernel_rooflines(r, n, "fp32_mixed", fp32_measured=70.0)
    hbm = bench.peaks().get("hbm_gbs")
    units = {"find": r["candidates"], "density": r["pairs"], "iad": r["pairs"],
             "momentum": r["pairs"]}
    for k, v in ks.items():
        ms = r["stages"][k]
        tf = bench.FLOPS[k] * units[k] / (ms * 1e-3) / 1e12
        assert v["alu"]["achieved"] == pytest.approx(tf)
        assert v["alu"]["frac"] == pytest.approx(tf / bench.FP32_PEAK_TFLOPS)
        assert v["alu"]["frac_measured"] == pytest.approx(tf / 70.0)
        b = bench.kernel_bytes(r, n, "fp32_mixed", k)
        assert v["hbm"]["bytes_per_launch"] == pytest.approx(b)
        assert v["hbm"]["achieved"] == pytest.approx(b / (ms * 1e-3) / 1e9)
        if hbm:
            assert v["hbm"]["frac"] == pytest.approx(b / (ms * 1e-3) / 1e9 / hbm)
            assert v["bound"] == ("alu" if v["alu"]["frac"] >= v["hbm"]["frac"] else "hbm")
    # FP64: the pair kernels on the FP64 pipe, the search on the FP32 pipe
    ks64 = bench.kernel_rooflines(r, n, "fp64")
    assert ks64["momentum"]["alu"]["peak"] == bench.FP64_PEAK_TFLOPS
    assert ks64["find"]["alu"]["peak"] == bench.FP32_PEAK_TFLOPS
    assert "frac_measured" not in ks64["momentum"]["alu"]


def test_kernel_roofline_uses_the_slowest_stage():
    r = _run()
    out = bench.roofline(r, 8_416_298, "fp32_mixed", fp32_measured=70.0)
    assert out["kernel"] == "momentum (fp32_mixed)"
    assert out["bound"] == "alu"
    assert out["flops_per_launch"] == pytest.approx(bench.FLOPS["momentum"] * 8.5e8)
    assert out["achieved"] == pytest.approx(bench.FLOPS["momentum"] * 8.5e8 / 6.5e-3 / 1e12)
    assert out["frac"] == pytest.approx(out["achieved"] / bench.FP32_PEAK_TFLOPS)
    assert out["frac_measured"] == pytest.approx(out["achieved"] / 70.0)
    r["stages"]["find"] = 7.0
    out = bench.roofline(r, 8_416_298, "fp32_mixed")
    assert out["kernel"] == "find (fp32_mixed)"
    assert out["flops_per_launch"] == pytest.approx(bench.FLOPS["find"] * 3.7e9)


NCU_CSV = """==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","void sph::k_find_mask<false>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","1,000"
"0","1","python","h","void sph::k_find_mask<false>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","500"
"1","1","python","h","void sph::k_cellwarp<sph::DensityPass>(int)","1","7","(64, 1, 1)","(1064, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","4000"
"1","1","python","h","void sph::k_cellwarp<sph::DensityPass>(int)","1","7","(64, 1, 1)","(1064, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","1000"
"2","1","python","h","void sph::k_find_mask<false>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Kbyte","2"
"2","1","python","h","void sph::k_find_mask<false>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","600"
"3","1","python","h","void sph::k_find_mask<true>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","10"
"3","1","python","h","void sph::k_find_mask<true>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","0"
"3","1","python","h","void sph::k_find_mask<true>(int)","1","7","(128, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","nsecond","1200"
"""


def test_ncu_csv_traffic_per_stage(tmp_path):
    p = tmp_path / "x.csv"
    p.write_text(NCU_CSV)
    rows = bench.read_ncu_csv(str(p))
    assert [r[0] for r in rows] == [0, 1, 2, 3]
    assert rows[3][2]["gpu__time_duration.sum"] == 1200.0
    t = bench.stage_traffic(rows)
    # the last step starts at the search launch that follows another stage
    # (id 2): find = k_find_mask<false> (id 2) + <true> (id 3)
    assert t["find"] == pytest.approx(2000 + 600 + 10)
    assert "density" not in t and "momentum" not in t
    rows2 = rows + [(4, "void sph::k_cellwarp<sph::DensityPass>(int)",
                     {"dram__bytes_read.sum": 7.0, "dram__bytes_write.sum": 1.0}),
                    (5, "void sph::k_cellpass<sph::DensityPass>(int)",
                     {"dram__bytes_read.sum": 2.0, "dram__bytes_write.sum": 0.0})]
    t2 = bench.stage_traffic(rows2)
    assert t2["density"] == pytest.approx(10.0)      # two launches of one stage add up
    assert t2["find"] == pytest.approx(2610)


def test_committed_traffic_capture_scales_with_particles():
    path = os.path.join(ROOT, bench.TRAFFIC_META)
    if not os.path.exists(path):
        pytest.skip("no committed ncu traffic capture")
    meta = json.load(open(path))
    rows = bench.read_ncu_csv(os.path.join(ROOT, "profiles", meta["csv"]))
    per_stage = bench.stage_traffic(rows)
    assert set(per_stage) == {"find", "density", "iad", "momentum"}
    for stage, b in per_stage.items():
        v = bench.traffic_for(stage, 2 * meta["n_particles"])
        # reported only while the kernel sources are those the capture was taken on
        assert v is None or v == pytest.approx(2 * b)


def test_conservation_drift():
    d0 = [1.0, 2.0, 3.0, 4.0, 6.0, 0.0, 0.0, 0.0]
    d1 = [1.5, 2.0, 2.0, 4.5, 6.5, 0.0, 0.0, 0.0]
    out = bench.conservation(d0, d1, steps=4)
    assert out["energy_rel_change_per_step"] == pytest.approx((11.0 - 10.0) / 10.0 / 4)
    assert out["momentum_change"] == [0.5, 0.0, -1.0]


def test_host_cpu_description():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["machine"]
