"""Host logic of bench.py's roofline object: the dominant class is the one with the most device
time, each class is divided by the peak of the pipe it runs on, and FP64 classes of a mixed run
are not measured against the FP32 peak."""
import bench
from synthetic import WORKLOADS


def test_roofline_picks_dominant_class_and_its_pipe():
    kst = {"gemm": {"ms": 25_000.0, "flops": 5.0e14, "bytes": 0.0, "launches": 100},
           "jacobi": {"ms": 16_000.0, "flops": 5.1e14, "bytes": 0.0, "launches": 50},
           "gemm_fp64": {"ms": 6_600.0, "flops": 7.7e12, "bytes": 0.0, "launches": 28}}
    r = bench.roofline(kst, WORKLOADS["mixed_n256"], {}, "fallback")
    assert r["kernel"] == "gemm" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 20.0) < 1e-9
    assert abs(r["frac"] - 20.0 / bench.FFMA_TFLOPS_NOMINAL) < 1e-12
    by = {c["kernel"]: c for c in r["classes"]}
    assert by["gemm_fp64"]["peak"] == bench.DFMA_TFLOPS_NOMINAL
    assert 0.9 < by["gemm_fp64"]["frac"] < 1.0
    assert [c["kernel"] for c in r["classes"]] == ["gemm", "jacobi", "gemm_fp64"]


def test_roofline_fp64_workload_uses_dfma_peak():
    kst = {"gemm": {"ms": 1000.0, "flops": 1.0e12, "bytes": 0.0, "launches": 10}}
    r = bench.roofline(kst, WORKLOADS["fp64_n128"], {}, "fallback")
    assert r["peak"] == bench.DFMA_TFLOPS_NOMINAL and abs(r["frac"] - 0.8) < 1e-12
    assert bench.roofline({}, WORKLOADS["fp64_n128"], {}, "fallback") is None
