"""Time the library's batched complex GEMM (nudft2_la_gemm) on given shapes.

Usage: python -m paper_2607_00928_b300.microbench --m 2048 --n 2048 --k 2048 --batch 2 [--ops NN]
       [--prec fp32|fp64] [--reps 5] [--tensor-cores]

Prints one JSON line per run: device time per call (CUDA events on the launching stream, after
one untimed call) and the rate in TFLOP/s with 8 m n k flops per complex product.
--tensor-cores sets NH_GEMM_TC=1, which sends large FP32 batches to the tcgen05 kernel.
"""
from __future__ import annotations

import argparse
import json
import os


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=2048)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--k", type=int, default=2048)
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--ops", default="NN")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--tensor-cores", action="store_true")
    a = ap.parse_args()
    if a.tensor_cores:
        os.environ["NH_GEMM_TC"] = "1"
    import ctypes

    import torch

    from .binding import FP64, MIXED, _check, _stream, lib
    dt = torch.complex64 if a.prec == "fp32" else torch.complex128
    opa, opb = a.ops
    ra, ca = (a.m, a.k) if opa == "N" else (a.k, a.m)     # stored shapes (column major)
    rb, cb = (a.k, a.n) if opb == "N" else (a.n, a.k)
    A = torch.randn((a.batch, ca, ra), dtype=dt, device="cuda")   # (batch, cols, rows) = column major
    B = torch.randn((a.batch, cb, rb), dtype=dt, device="cuda")
    C = torch.zeros((a.batch, a.n, a.m), dtype=dt, device="cuda")
    ops = {"N": 0, "T": 1, "C": 2}

    def call():
        _check(lib().nudft2_la_gemm(FP64 if a.prec == "fp64" else MIXED, ops[opa], ops[opb], a.m, a.n, a.k, 1.0,
                                    ctypes.c_void_p(A.data_ptr()), ra, ra * ca, ctypes.c_void_p(B.data_ptr()), rb,
                                    rb * cb, 0.0, ctypes.c_void_p(C.data_ptr()), a.m, a.m * a.n, a.batch, _stream()))

    call()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        call()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = min(ts)
    fl = 8.0 * a.m * a.n * a.k * a.batch
    print(json.dumps({"m": a.m, "n": a.n, "k": a.k, "batch": a.batch, "ops": a.ops, "prec": a.prec,
                      "tensor_cores": a.tensor_cores, "ms": ms, "tflops": fl / ms / 1e9}), flush=True)


if __name__ == "__main__":
    main()
