"""Host logic of bench.py's roofline object: the dominant class is the one with the most device
time, each class is divided by the peak of the pipe it runs on (tensor-core GEMM and Jacobi: the
useful 3xTF32 rate from the sustained BF16 figure, since they run inside a long step; sweeps: HBM
bandwidth; FP64 classes: DFMA; the other mixed-run classes: FFMA)."""
import bench
from synthetic import WORKLOADS

PIPES = bench.default_pipes({"hbm_gbs": 6000.0, "bf16_tflops": 1500.0, "bf16_tflops_sustained": 1200.0}, "test")


def test_roofline_picks_dominant_class_and_its_pipe():
    kst = {"gemm": {"ms": 25_000.0, "flops": 5.0e14, "bytes": 0.0, "launches": 100},
           "jacobi": {"ms": 16_000.0, "flops": 5.1e14, "bytes": 0.0, "launches": 50},
           "gemm_fp64": {"ms": 6_600.0, "flops": 7.7e12, "bytes": 0.0, "launches": 28}}
    r = bench.roofline(kst, WORKLOADS["mixed_n256"], PIPES)
    assert r["kernel"] == "gemm" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 20.0) < 1e-9
    assert abs(r["frac"] - 20.0 / bench.FFMA_TFLOPS_NOMINAL) < 1e-12
    by = {c["kernel"]: c for c in r["classes"]}
    assert by["gemm_fp64"]["peak"] == bench.DFMA_TFLOPS_NOMINAL
    assert 0.9 < by["gemm_fp64"]["frac"] < 1.0
    assert [c["kernel"] for c in r["classes"]] == ["gemm", "jacobi", "gemm_fp64"]


def test_roofline_fp64_workload_uses_dfma_peak():
    kst = {"gemm": {"ms": 1000.0, "flops": 1.0e12, "bytes": 0.0, "launches": 10}}
    r = bench.roofline(kst, WORKLOADS["fp64_n128"], PIPES)
    assert r["peak"] == bench.DFMA_TFLOPS_NOMINAL and abs(r["frac"] - 0.8) < 1e-12
    assert bench.roofline({}, WORKLOADS["fp64_n128"], PIPES) is None


def test_tensor_core_gemm_and_sweep_use_their_own_pipes():
    kst = {"gemm_tc": {"ms": 1000.0, "flops": 1.0e14, "bytes": 0.0, "launches": 10},
           "sweep": {"ms": 10.0, "flops": 0.0, "bytes": 3.0e10, "launches": 2}}
    r = bench.roofline(kst, WORKLOADS["mixed_n256"], PIPES)
    assert r["kernel"] == "gemm_tc" and r["bound"] == "tensor"
    assert abs(r["peak"] - 1200.0 * 1.1 / 2.25 / 3.0) < 1e-9
    assert abs(r["achieved"] - 100.0) < 1e-9
    sw = {c["kernel"]: c for c in r["classes"]}["sweep"]
    assert sw["bound"] == "hbm" and sw["unit"] == "GB/s" and abs(sw["achieved"] - 3000.0) < 1e-9
    assert abs(sw["frac"] - 0.5) < 1e-12


def test_tensor_core_jacobi_uses_the_tensor_pipe():
    """The blocked Jacobi step whose Gram and update products run on tcgen05 is divided by the
    3xTF32 useful rate, the CUDA-core one by the FFMA rate."""
    kst = {"jacobi_tc": {"ms": 2000.0, "flops": 2.0e14, "bytes": 0.0, "launches": 20},
           "jacobi": {"ms": 1000.0, "flops": 2.0e13, "bytes": 0.0, "launches": 5}}
    r = bench.roofline(kst, WORKLOADS["mixed_n256"], PIPES)
    assert r["kernel"] == "jacobi_tc" and r["bound"] == "tensor"
    assert abs(r["frac"] - 100.0 / (1200.0 * 1.1 / 2.25 / 3.0)) < 1e-12
    jb = {c["kernel"]: c for c in r["classes"]}["jacobi"]
    assert jb["bound"] == "alu" and jb["peak"] == bench.FFMA_TFLOPS_NOMINAL
