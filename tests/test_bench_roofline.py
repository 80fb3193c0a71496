"""bench.py's roofline object (host logic, no GPU): the dominant kernel class is the one with the largest
measured time; `achieved` is that class's algorithmic bytes (or flops) per launch over its average launch
time, `frac` = achieved / peak with the peak the bound names, and measured DRAM traffic is attached only
for the default launch variants the counters were taken on."""
import math

import pytest

import bench

N, ORDER = 256, 6


def _alg():
    return bench.algorithmic(N, ORDER, [13, 13], real_medium=True, precision="fp16")


def _times(dominant):
    ms = {c: 1.0 for c in bench.CLASSES}
    ln = {c: 26 for c in bench.CLASSES}
    ms[dominant] = 5.0
    return ms, ln


def test_hbm_bound_class_reports_bytes_over_time():
    alg = _alg()
    ms, ln = _times("stencil")
    r = bench.roofline(ms, ln, alg, "fp16", ORDER, N, "default")
    pk, _ = bench.peaks()
    assert r["kernel"] == "stencil" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    avg_s = ms["stencil"] / ln["stencil"] / 1e3
    per_launch = alg["stencil"]["bytes"] / alg["stencil"]["launches"]
    assert math.isclose(r["achieved"] * 1e9 * avg_s, per_launch, rel_tol=1e-12)
    assert math.isclose(r["algorithmic_bytes_per_launch"], per_launch, rel_tol=1e-12)
    assert r["peak"] == pk["hbm_gbs"] and math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12)
    assert r["traffic"] == bench.MEASURED_TRAFFIC[("stencil", N, ORDER, "fp16")]
    # counters taken on the default variants say nothing about autotuned ones
    assert bench.roofline(ms, ln, alg, "fp16", ORDER, N, "autotuned")["traffic"] is None


@pytest.mark.parametrize("precision, ratio", [("fp16", 1.0), ("tf32", 1.1 / 2.25)])
def test_tensor_bound_class_reports_flops_against_its_dtype_peak(precision, ratio):
    alg = bench.algorithmic(N, ORDER, [13, 13], real_medium=True, precision=precision)
    ms, ln = _times("ypass")
    ln["ypass"] = 52
    r = bench.roofline(ms, ln, alg, precision, ORDER, N, "default")
    pk, _ = bench.peaks()
    assert r["kernel"] == "ypass" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["peak"], pk["bf16_tflops_sustained"] * ratio, rel_tol=1e-12)
    avg_s = ms["ypass"] / ln["ypass"] / 1e3
    assert math.isclose(r["achieved"] * 1e12 * avg_s, alg["ypass"]["flops"] / alg["ypass"]["launches"], rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12) and r["traffic"] is None


def test_no_timed_class_gives_no_roofline():
    alg = _alg()
    assert bench.roofline({c: 0.0 for c in bench.CLASSES}, {c: 0 for c in bench.CLASSES}, alg, "fp16", ORDER, N,
                          "default") is None
