"""Parity at the full sizes of the FP64 and mixed-precision configurations, where a dense
oracle solve is out of reach (config 2: A is 32768 x 16384; config 3: 131072 x 65536).

Checked instead:
* the data f: formed by the oracle's direct sum of Eq. 1 (all rows); for config 3 the
  library's exact FP64 apply is also compared with it on every row;
* the solution: consistent data (plus 1e-12 relative noise for config 2) has the LS solution
  c_true up to ~cond(A) * noise, so c must match c_true to the 1e-8 target;
* sampled residuals: r_j = f_j - (A c)_j evaluated by the oracle at sampled points j.
The handles use the same options as bench.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import WORKLOADS, make_workload, noise_like  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


def _relcols(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def _sampled_residual(x, y, c, f, nx, ny, idx):
    Ac = orc.forward(x[idx], y[idx], c, nx, ny)
    return float(np.max(np.abs(f[idx] - Ac)) / np.max(np.abs(f[idx])))


def test_config2_fp64_n128_full_size(nh):
    w = WORKLOADS["fp64_n128"]
    x, y, ct = make_workload(w)
    f0 = orc.forward(x, y, ct, w.nx, w.ny)                     # oracle direct sum, all rows
    f = f0 + noise_like(f0, w.noise, w.seed + 7)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=w.eps, levels=w.levels).factor()
    c = h.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    h.close()
    assert _relcols(c, ct) < 1e-8
    idx = np.random.default_rng(2).choice(w.M, 48, replace=False)
    assert _sampled_residual(x, y, c, f, w.nx, w.ny, idx) < 1e-8


def test_config3_mixed_n256_full_size(nh):
    w = WORKLOADS["mixed_n256"]
    x, y, ct = make_workload(w)
    xt, yt, ctt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(ct).cuda()
    f = orc.forward(x, y, ct, w.nx, w.ny)                      # ~20 s on the host
    ft = torch.from_numpy(f).cuda()
    f_lib = nh.exact_apply(xt, yt, w.nx, w.ny, nh.EXACT_FWD, ctt).cpu().numpy()
    assert np.max(np.abs(f_lib - f)) < 1e-12 * np.max(np.abs(f)) * np.sqrt(w.N)
    idx = np.random.default_rng(3).choice(w.M, 32, replace=False)
    h = nh.NudftHSS(xt, yt, w.nx, w.ny, eps=1e-6, levels=w.levels, prec="mixed", refine_tol=1e-8,
                    refine_max=10).factor()
    c = h.solve(ft).cpu().numpy()
    info = h.info()
    h.close()
    assert 0 <= info["refine_relres"] <= 1e-8
    assert _relcols(c, ct) < 1e-8
    assert _sampled_residual(x, y, c, f, w.nx, w.ny, idx) < 1e-8
