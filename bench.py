"""Benchmark of the 2D type-II inverse NUDFT direct solver (HSS face splitting + URV) on B300.

One step = the whole hot path on one synthetic problem: HSS construction (t_c), URV
factorization (t_f) and the solve of every right-hand side (t_s; in MIXED mode including
the FP64 iterative refinement with the exact apply), Algorithm 1 of Li & Liu.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line (rank 0).  value = right-hand sides solved per second over whole steps
(offline stage included), summed over ranks; the paper-style split t_c / t_f / t_s and the
online solve rate are reported alongside.  Multi-GPU runs are independent replicas (the path
has no exchange step).  --impl reference times the FP64 CPU oracle (CGLS with its direct
O(MN) applies) on a bounded sample of the same workload: two iterations, scaled by the measured
iteration count to a 1e-8 residual.  --workload batched_uneven runs the 64-problem batch;
--gemm, --sweep and --one-step are kernel and launch-list profiling modes, not bench lines.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import WORKLOADS, make_workload, noise_like  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FFMA_TFLOPS_NOMINAL = 148 * 128 * 2 * 2.032e9 / 1e12     # FP32 CUDA-core FMA peak at max SM clock
DFMA_TFLOPS_NOMINAL = 1.25                                 # B300 FP64 rate


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# ------------------------------------------------------------------------------------------ oracle arm
CGLS_COUNTS = os.path.join(ROOT, "oracle", "cgls_iterations.json")


def oracle_cgls_sample(w, iters: int = 2):
    """The oracle's CGLS (CG on the normal equations with its direct O(MN) applies of A and A^*)
    on this very workload, one right-hand side, timed over a bounded number of iterations (about
    20-30 s at N = 256^2).  The iteration count to a 1e-8 relative residual is the one measured by
    running the same CGLS to that stop (oracle/measure_cgls.py, stored in
    oracle/cgls_iterations.json); without a stored count it is extrapolated from the contraction
    over the sample.  Dense Householder LS is out of reach at these sizes.  Returns (seconds of the
    timed sample, iterations for 1e-8, estimated seconds per right-hand side, how the count was
    obtained)."""
    import math

    import oracle as orc
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct[:, :1], w.nx, w.ny)                 # data, not timed
    t0 = time.perf_counter()
    c, _ = orc.cgls(x, y, f, w.nx, w.ny, tol=1e-300, maxit=iters)
    dt = time.perf_counter() - t0
    try:
        rec = json.load(open(CGLS_COUNTS))[w.name]
        need, how = int(rec["iterations"]), f"measured: {rec['iterations']} iterations to {rec['rtol']:g}"
    except Exception:
        r = f - orc.forward(x, y, c, w.nx, w.ny)                  # residual, not timed
        rel = float(np.linalg.norm(r) / np.linalg.norm(f))
        rho = rel ** (1.0 / iters) if rel > 0 else 0.0
        need = 500 if rho >= 1 else (iters if rho == 0 else max(iters, int(math.ceil(math.log(1e-8) / math.log(rho)))))
        how = f"extrapolated from the contraction over the sample: {need} iterations"
    # the sample is one adjoint apply plus `iters` iterations of one forward and one adjoint apply
    per_rhs = dt * (need + 0.5) / (iters + 0.5)
    return dt, need, per_rhs, how


def oracle_rate(w):
    dt, need, per_rhs, how = oracle_cgls_sample(w)
    sample = (f"oracle CGLS with direct O(MN) applies (FP64, numpy) on this workload, 1 RHS: 2 iterations took "
              f"{dt:.2f} s; to a 1e-8 relative residual it takes {need} iterations ({how}), i.e. ~{per_rhs:.1f} s "
              f"per RHS")
    return 1.0 / per_rhs, per_rhs, sample


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        th = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(th) if th else os.cpu_count()
    except Exception:
        return os.cpu_count()


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_rate(w)
    runs = [oracle_rate(w) for _ in range(args.steps)]
    rate, per_rhs, sample = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
    sample += f"; median of {args.steps} samples"
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_rhs * w.nrhs * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args),
            "cpu_baseline": {"value": rate, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "2D inverse-NUDFT solves/s (build+factor+solve per step), N=256^2 mixed / FP64"


def config_of(w, args):
    return {"workload": w.name, "nx": w.nx, "ny": w.ny, "M": w.M, "N": w.N, "nrhs": w.nrhs, "levels": w.levels,
            "eps": (args.eps if args.eps else (1e-6 if w.mixed else w.eps)), "precision": "mixed" if w.mixed else "fp64",
            "grid": f"jittered {w.mx}x{w.my}, theta~U{list(w.theta)}", "l2": "working set > L2 (126 MB); no flush",
            "parallelism": f"replicas x{args.gpus}"}


# ------------------------------------------------------------------------------------------ replicas
def aggregate_replicas(ms_local: float, units_per_rank: int, device=None):
    """Max step time over ranks and whole-job throughput (units of all ranks / slowest rank's time).

    Independent replicas: no data-path collective; the only communication is this reduction.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_initialized() else 1
    ms = ms_local
    if world > 1:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3)


# ------------------------------------------------------------------------------------------ our arm
def run_ours(args, w):
    import torch
    import torch.distributed as dist

    import paper_2607_00928_b300 as nh

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    pk, src = peaks()
    pipes = measured_pipes(nh, pk, src)
    x, y, ct = make_workload(w)
    eps = args.eps if args.eps else (1e-6 if w.mixed else w.eps)
    prec = "mixed" if w.mixed else "fp64"
    xt = torch.from_numpy(x).to(dev)
    yt = torch.from_numpy(y).to(dev)
    ctt = torch.from_numpy(ct).to(dev)
    # right-hand side f = A c_true (+ noise) formed with the exact FP64 apply of the library
    f = nh.exact_apply(xt, yt, w.nx, w.ny, nh.EXACT_FWD, ctt)
    if w.noise:
        f = f + torch.from_numpy(noise_like(f.cpu().numpy(), w.noise, w.seed + 7)).to(dev)
    stream = torch.cuda.current_stream()

    def step(extra=None):
        h = nh.NudftHSS(xt, yt, w.nx, w.ny, eps=eps, levels=w.levels, prec=prec, refine_tol=1e-8, refine_max=10,
                        profile=True)
        h.factor()
        c = h.solve(f)
        inf = h.info()
        inf["kstats"] = h.kstats()
        if extra is not None:
            extra(h)
        h.close()
        return c, inf

    # online solve with one right-hand side, on the last warm-up step's handle (outside the timed region)
    s1 = {}

    def time_one_rhs(h):
        f1 = f[:, :1].contiguous()
        for _ in range(2):              # the first call also captures the one-column sweeps
            h.solve(f1)
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            h.solve(f1)                 # each call synchronises its stream before returning
        s1["ms"] = (time.perf_counter() - t0) * 1e3 / reps

    if args.one_step:           # launch lists under a profiler: exactly one step, nothing else
        torch.cuda.synchronize()
        c, inf = step()
        rel = float(torch.max(torch.linalg.norm(c - ctt, dim=0) / torch.linalg.norm(ctt, dim=0)).item())
        print(json.dumps({"mode": "one-step", "config": config_of(w, args), "launches": inf["launches"],
                          "device_bytes": inf.get("device_bytes"),
                          "t_build_ms": inf["t_build_ms"], "t_factor_ms": inf["t_factor_ms"],
                          "t_solve_ms": inf["t_solve_ms"], "rel_err_vs_c_true": rel}), flush=True)
        return
    for i in range(args.warmup):
        c, inf = step(time_one_rhs if i == args.warmup - 1 else None)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        c, inf = step()
        infos.append(inf)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms, value = aggregate_replicas(e0.elapsed_time(e1) / args.steps, w.nrhs, dev)
    if world > 1:
        dist.barrier()
    rel = float(torch.max(torch.linalg.norm(c - ctt, dim=0) / torch.linalg.norm(ctt, dim=0)).item())
    launches = sum(i["launches"] for i in infos)
    t_c = statistics.median(i["t_build_ms"] for i in infos)
    t_f = statistics.median(i["t_factor_ms"] for i in infos)
    t_s = statistics.median(i["t_solve_ms"] for i in infos)

    # ---- end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    fh = f.cpu().pin_memory()
    ch = torch.empty((w.N, w.nrhs), dtype=torch.complex128).pin_memory()
    torch.cuda.synchronize()
    te = []
    for _ in range(max(1, min(args.steps, 2))):
        t0 = time.perf_counter()
        xd = xh.to(dev, non_blocking=True)
        yd = yh.to(dev, non_blocking=True)
        fd = fh.to(dev, non_blocking=True)
        h = nh.NudftHSS(xd, yd, w.nx, w.ny, eps=eps, levels=w.levels, prec=prec, refine_tol=1e-8, refine_max=10)
        h.factor()
        cd = h.solve(fd)
        h.close()
        ch.copy_(cd, non_blocking=True)
        torch.cuda.synchronize()
        te.append(time.perf_counter() - t0)
    t_e2e = statistics.median(te)
    h2d = x.nbytes + y.nbytes + fh.numel() * 16
    d2h = ch.numel() * 16

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, _, sample = oracle_rate(w)
        cpu = {"value": rate, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample}

    kst = {}
    for i in infos:
        for k, v in i["kstats"].items():
            a = kst.setdefault(k, {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
            for f2 in a:
                a[f2] += v[f2]
    roof = roofline(kst, w, pipes)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64" if w.mixed else "f64", "data": "synthetic",
                "config": config_of(w, args),
                "t_build_ms": t_c, "t_factor_ms": t_f, "t_solve_ms": t_s,
                "online_solves_per_s": w.nrhs / (t_s / 1e3) if t_s > 0 else None,
                "online_solves_per_s_one_rhs": (1e3 / s1["ms"]) if s1.get("ms") else None,
                "rel_err_vs_c_true": rel, "max_rank": infos[-1]["max_rank"],
                "level_rank": infos[-1]["level_rank"], "refine_iters": infos[-1]["refine_iters"],
                "device_bytes": infos[-1].get("device_bytes"),
                "refine_relres": infos[-1]["refine_relres"],
                "e2e": {"value": world * w.nrhs / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clocks, "roofline": roof, "cpu_baseline": cpu,
                "peaks": {k: v for k, v in pipes.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


TF32_OVER_BF16 = 1.1 / 2.25     # nominal dense TF32 / BF16 tensor rates of B300


def class_pipe(name: str, mixed: bool, pipes: dict):
    """(bound, peak, unit, source) of the pipe a kernel class runs on.

    gemm_tc, jacobi_tc (the blocked Jacobi step whose Gram and update products run on the tensor
    cores; its flops count those products only): the tcgen05 3xTF32 complex products, against the
    useful complex-FP32 rate of the TF32 tensor pipe (TF32 rate / 3, the TF32 rate taken as the measured BF16 burst rate times the
    nominal TF32/BF16 ratio).  sweep: one URV solve replayed from its graph, against the measured
    HBM copy bandwidth.  FP64 classes (all classes of an FP64 run, the "_fp64" ones of a mixed run)
    against the measured DFMA rate; the other mixed-run classes (CUDA-core GEMM, QR, Jacobi)
    against the measured FFMA rate."""
    if name == "sweep" or name == "sweep_fp64":
        return "hbm", pipes["hbm_gbs"], "GB/s", pipes["hbm_src"]
    if name in ("gemm_tc", "jacobi_tc"):
        # these kernels run inside a seconds-long step: the sustained (power-capped) tensor rate
        return ("tensor", pipes["bf16_sust"] * TF32_OVER_BF16 / 3.0, "TFLOP/s",
                f"3xTF32 useful rate = sustained bf16 {pipes['bf16_sust']:.0f} TFLOP/s ({pipes['bf16_src']}) "
                f"x 1.1/2.25 / 3")
    if name.endswith("_fp64") or not mixed:
        return "alu", pipes["dfma"], "TFLOP/s", pipes["dfma_src"]
    return "alu", pipes["ffma"], "TFLOP/s", pipes["ffma_src"]


def default_pipes(pk=None, src="fallback"):
    pk = pk or {}
    return {"hbm_gbs": pk.get("hbm_gbs", 6400.0), "hbm_src": f"HBM copy, {src}",
            "bf16": pk.get("bf16_tflops", 1800.0), "bf16_src": src,
            "bf16_sust": pk.get("bf16_tflops_sustained", 1400.0),
            "ffma": FFMA_TFLOPS_NOMINAL, "ffma_src": "FP32 FFMA nominal: 148 SM x 128 lanes x 2 x 2.032 GHz",
            "dfma": DFMA_TFLOPS_NOMINAL, "dfma_src": "FP64 DFMA nominal 1.25 TFLOP/s"}


def measured_pipes(nh, pk, src):
    """Roofline denominators: HBM and BF16 from the driver's measured peaks file, FFMA and DFMA
    measured here by the library's FMA probe."""
    p = default_pipes(pk, src)
    try:
        p["ffma"] = nh.peak_fma(nh.MIXED)
        p["ffma_src"] = "FP32 FFMA measured (nudft2_peak_fma)"
        p["dfma"] = nh.peak_fma(nh.FP64)
        p["dfma_src"] = "FP64 DFMA measured (nudft2_peak_fma)"
    except Exception as e:   # keep the nominal figures, say so
        p["ffma_src"] += f" (probe failed: {e})"
    return p


def roofline(kst, w, pipes):
    """Dominant kernel class (most device time) against its pipe's peak, plus every class."""
    if not kst:
        return None
    classes = []
    for name, s in sorted(kst.items(), key=lambda kv: -kv[1]["ms"]):
        if s["ms"] <= 0 or s["launches"] == 0:
            continue
        bound, peak, unit, psrc = class_pipe(name, w.mixed, pipes)
        sec = s["ms"] / 1e3
        achieved = (s["bytes"] / sec / 1e9) if bound == "hbm" else (s["flops"] / sec / 1e12)
        classes.append({"kernel": name, "bound": bound, "ms": s["ms"], "achieved": achieved, "peak": peak,
                        "unit": unit, "frac": achieved / peak, "launches": s["launches"],
                        "avg_launch_ms": s["ms"] / s["launches"], "peak_source": psrc})
    if not classes:
        return None
    d = classes[0]
    return {"kernel": d["kernel"], "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "traffic": TRAFFIC_PER_LAUNCH.get(d["kernel"]),
            "launches": d["launches"], "avg_launch_ms": d["avg_launch_ms"], "peak_source": d["peak_source"],
            "classes": classes}


# DRAM bytes (read + write) per launch of a class's kernel from an ncu capture, where one exists for
# the current kernel (None otherwise).
TRAFFIC_PER_LAUNCH: dict = {}


# ------------------------------------------------------------------------------------------ batched arm
def run_batched(args):
    """Config 4: 64 independent problems of uneven size (synthetic.batched_uneven), 8 right-hand
    sides each, built, factored and solved together (nudft2_hss_run_batched: 8 host threads, one
    stream per problem, each problem run to completion and freed).  Mixed precision at eps 1e-6, refined to 1e-8 with the FP64 residual.
    One step = build + factor + solve of the whole batch; value = right-hand sides per second."""
    import torch

    import paper_2607_00928_b300 as nh
    from synthetic import batched_uneven

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    ps = batched_uneven()
    opts = dict(eps=1e-6, prec="mixed", refine_tol=1e-8, refine_max=10)
    for p in ps:
        p.update(opts)
    fs = [nh.exact_apply(torch.from_numpy(p["x"]).to(dev), torch.from_numpy(p["y"]).to(dev), p["nx"], p["ny"],
                         nh.EXACT_FWD, torch.from_numpy(p["c_true"]).to(dev)) for p in ps]
    units = sum(p["c_true"].shape[1] for p in ps)

    def step():
        return nh.run_batched(ps, fs, threads=8)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = Clocks(local)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        cs = step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.steps * 1e3
    clocks = clk.stop()
    ms = max(e0.elapsed_time(e1) / args.steps, wall)
    err = max(float(torch.max(torch.linalg.norm(c - torch.from_numpy(p["c_true"]).to(dev), dim=0)
                              / torch.linalg.norm(torch.from_numpy(p["c_true"]).to(dev), dim=0))) for c, p in zip(cs, ps))
    # end to end: points and data from pinned host memory, solutions back to the host
    hx = [torch.from_numpy(p["x"]).pin_memory() for p in ps]
    hy = [torch.from_numpy(p["y"]).pin_memory() for p in ps]
    hf = [f.cpu().pin_memory() for f in fs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pd = [dict(p, x=a.to(dev, non_blocking=True), y=b.to(dev, non_blocking=True)) for p, a, b in zip(ps, hx, hy)]
    fd = [f.to(dev, non_blocking=True) for f in hf]
    out = [c.cpu() for c in nh.run_batched(pd, fd, threads=8)]
    t_e2e = time.perf_counter() - t0
    h2d = sum(a.nbytes + b.nbytes + f.numel() * 16 for a, b, f in zip(hx, hy, hf))
    d2h = sum(o.numel() * 16 for o in out)
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": "batched_uneven", "problems": len(ps), "sum_N": sum(p["nx"] * p["ny"] for p in ps),
                       "sum_M": sum(p["x"].size for p in ps), "nrhs_each": 8, "eps": 1e-6, "precision": "mixed",
                       "sizes": "nx, ny uniform in {32,48,64,96,128,192,256}; M/N ~ U[1.5,4]; theta ~ U[-0.25,0.35]",
                       "concurrency": "one stream per problem, 8 host threads, each problem run to completion", "parallelism": "replicas x1"},
            "rel_err_vs_c_true": err,
            "e2e": {"value": units / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------ kernel mode
def run_gemm(args):
    """One complex64 GEMM C = A B (m x k times k x n, NN, beta = 0) through nudft2_la_gemm, the
    library's batched GEMM (tensor cores when the shape qualifies): device time per call with CUDA
    events after args.warmup calls, and the rate with 8 m n k flops per product.  Used for kernel
    profiles; not the solver benchmark."""
    import ctypes

    import torch

    from paper_2607_00928_b300.binding import MIXED, _check, _stream, lib
    parts = [int(v) for v in args.gemm.split(",")]
    m, n, k = parts[:3]
    batch = parts[3] if len(parts) > 3 else 1
    g = torch.Generator(device="cuda").manual_seed(1)
    # (batch, cols, rows) contiguous = column-major rows x cols per item: no layout copies per call
    A = torch.randn((batch, k, m), dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn((batch, n, k), dtype=torch.complex64, device="cuda", generator=g)
    C = torch.zeros((batch, n, m), dtype=torch.complex64, device="cuda")

    def call():
        _check(lib().nudft2_la_gemm(MIXED, 0, 0, m, n, k, 1.0, ctypes.c_void_p(A.data_ptr()), m, m * k,
                                    ctypes.c_void_p(B.data_ptr()), k, k * n, 0.0, ctypes.c_void_p(C.data_ptr()), m,
                                    m * n, batch, _stream()))

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        call()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    print(json.dumps({"metric": "complex64 GEMM rate (8 m n k flops)", "value": 8.0 * m * n * k * batch / ms / 1e9,
                      "unit": "TFLOP/s", "ms": ms, "m": m, "n": n, "k": k, "batch": batch, "steps": args.steps,
                      "warmup": args.warmup}), flush=True)


def run_sweep(args):
    """One call of nudft2_la_qr_apply: blocked Householder QR of a random m x k complex64 matrix
    (merged 256-column blocks), then Q^* C for a random m x s C by the streaming kernels (partial
    V^* C over row slabs, ordered sum, T product, row update).  Prints the wall time per call
    (QR included) and the reflector bytes one application streams; used for kernel profiles of the
    sweep kernels, not as a benchmark line."""
    import torch

    import paper_2607_00928_b300 as nh
    m, k, s = [int(v) for v in args.sweep.split(",")]
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn((m, k), dtype=torch.complex64, device="cuda", generator=g)
    C = torch.randn((m, s), dtype=torch.complex64, device="cuda", generator=g)
    for _ in range(args.warmup):
        nh.la_qr_apply(A, C, conj=True, grouped=True)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out, _ = nh.la_qr_apply(A, C, conj=True, grouped=True)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    kk = min(m, k)
    print(json.dumps({"mode": "sweep", "m": m, "k": k, "s": s, "ms_per_call_with_qr": statistics.median(ts),
                      "reflector_bytes": (m * kk - kk * (kk - 1) / 2) * 8, "steps": args.steps,
                      "warmup": args.warmup}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=os.environ.get("NUDFT_BENCH_WORKLOAD", "mixed_n256"))
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--gemm", default=None, help="m,n,k[,batch]: time one library GEMM instead of the solver")
    ap.add_argument("--sweep", default=None,
                    help="m,k,s: Householder QR of a random m x k complex64 matrix, then Q^* C (m x s) by the "
                         "streaming reflector kernels of the solve sweeps (for kernel profiles)")
    ap.add_argument("--one-step", action="store_true",
                    help="profiling mode: one build + factor + solve of the workload, no warm-up, end-to-end or CPU "
                         "legs; prints the stage times only")
    args = ap.parse_args()
    if args.gemm:
        run_gemm(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.workload == "batched_uneven":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm is timed on the single-problem "
                              "workloads; the batched workload has no CPU arm"}), flush=True)
            return
        run_batched(args)
        return
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
