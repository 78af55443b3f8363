"""bench.py's JSON line on the host: the control flow of the GPU arm (warm-up steps, the
one-right-hand-side timing, the timed step, end to end through host buffers, the CPU baseline,
the roofline) runs against a stand-in library and a CPU device, and the line carries every
key of the benchmark contract.  Nothing here measures anything."""
import io
import json
import sys
import types
from contextlib import redirect_stdout

import torch

import bench


class _Event:
    def __init__(self, enable_timing=True):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 1000.0


class _Handle:
    def __init__(self, x, y, nx, ny, **opts):
        self.N = nx * ny

    def factor(self):
        return self

    def solve(self, f):
        return torch.ones((self.N, f.shape[1]), dtype=torch.complex128)

    def info(self):
        return {"t_build_ms": 1.0, "t_factor_ms": 2.0, "t_solve_ms": 3.0, "launches": 7, "max_rank": 5,
                "level_rank": [0, 5], "refine_iters": 2, "refine_relres": 1e-9}

    def kstats(self):
        return {"gemm": {"ms": 10.0, "flops": 1e11, "bytes": 0.0, "launches": 3},
                "gemm_fp64": {"ms": 5.0, "flops": 1e9, "bytes": 0.0, "launches": 2}}

    def close(self):
        pass


def test_bench_line_has_the_contract_keys(monkeypatch):
    fake = types.ModuleType("paper_2607_00928_b300")
    fake.EXACT_FWD = 2
    fake.exact_apply = lambda x, y, nx, ny, op, v: torch.zeros((x.numel(), v.shape[1]), dtype=torch.complex128)
    fake.NudftHSS = _Handle
    monkeypatch.setitem(sys.modules, "paper_2607_00928_b300", fake)
    real_device = torch.device
    monkeypatch.setattr(torch, "device", lambda *a, **k: real_device("cpu"))
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "mixed_n64", "--steps", "1", "--warmup", "3"])
    out = io.StringIO()
    with redirect_stdout(out):
        bench.main()
    line = json.loads([ln for ln in out.getvalue().splitlines() if ln.startswith("{")][-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks", "roofline", "cpu_baseline"):
        assert k in line, k
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["config"]["workload"] == "mixed_n64"
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert set(line["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert line["roofline"]["kernel"] == "gemm" and line["roofline"]["peak"] == bench.FFMA_TFLOPS_NOMINAL
    assert set(line["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["online_solves_per_s_one_rhs"] is not None
    assert abs(line["value"] - 16 / 1.0) < 1e-9          # 16 right-hand sides per 1000 ms step
