"""Runs the oracle's CGLS on a benchmark workload (one right-hand side, consistent data) to a
relative residual of 1e-8 and writes the iteration count and the time it took to
oracle/cgls_iterations.json.  The CPU baseline of bench.py times a bounded number of the same
iterations on the host it runs on and multiplies by this measured count.

    python -m oracle.measure_cgls [--workload mixed_n256] [--rtol 1e-8]
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import time

import numpy as np

from . import nudft_oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "cgls_iterations.json")


def main() -> None:
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    from synthetic import WORKLOADS, make_workload
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="mixed_n256")
    ap.add_argument("--rtol", type=float, default=1e-8)
    a = ap.parse_args()
    w = WORKLOADS[a.workload]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct[:, :1], w.nx, w.ny)
    hist = []
    t0 = time.perf_counter()
    c, it = orc.cgls(x, y, f, w.nx, w.ny, tol=1e-300, maxit=500, rtol=a.rtol, history=hist)
    dt = time.perf_counter() - t0
    err = float(np.linalg.norm(c - ct[:, :1]) / np.linalg.norm(ct[:, :1]))
    rec = json.load(open(OUT)) if os.path.exists(OUT) else {}
    rec[a.workload] = {"iterations": it, "rtol": a.rtol, "final_relres": hist[-1], "rel_err_vs_c_true": err,
                       "seconds": dt, "cpu_count": os.cpu_count(), "machine": platform.processor() or platform.machine(),
                       "history": hist}
    json.dump(rec, open(OUT, "w"), indent=1)
    print(json.dumps(rec[a.workload]))


if __name__ == "__main__":
    main()
