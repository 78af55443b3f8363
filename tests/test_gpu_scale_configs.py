"""Parity at the full sizes of the FP64, mixed-precision and differentiation configurations,
where a dense oracle solve is out of reach (A is 32768 x 16384 or 131072 x 65536).

Checked instead:
* the data f: formed by the oracle's direct sum of Eq. 1 (all rows); for config 3 the
  library's exact FP64 apply is also compared with it on every row;
* the solution: consistent data (plus 1e-12 relative noise for config 2) has the LS solution
  c_true up to ~cond(A) * noise, so c must match c_true to the 1e-8 target;
* sampled residuals: r_j = f_j - (A c)_j evaluated by the oracle at sampled points j.
The handles use the same options as bench.py.  The differentiation workload is checked through
A^* grad_f = g and a directional central difference of the GPU map."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import WORKLOADS, complex_normal, make_workload, noise_like  # noqa: E402

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


def test_grad_config5_scale_properties(nh):
    """n = 128, M = 32768, 16 right-hand sides (the differentiation workload): grad_f solves
    A^* lam = g (checked with the exact adjoint), and the point gradient matches a directional
    central difference of the GPU map along a random direction.  The handles run in mixed
    precision refined to 1e-12 with the FP64 exact applies, so the map and its gradient are the
    FP64 least-squares ones while each build takes seconds (an FP64 build at this size takes
    minutes)."""
    w = WORKLOADS["grad_n128"]
    x, y, c_true = make_workload(w)
    ct = complex_normal((w.N, w.nrhs), 55)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    opts = dict(eps=1e-6, levels=w.levels, prec="mixed", refine_tol=1e-12, refine_max=30)
    h = nh.NudftHSS(xt, yt, w.nx, w.ny, **opts).factor()
    f = h.apply(nh.EXACT_FWD, torch.from_numpy(c_true).cuda())
    c = h.solve(f)
    g = 2 * (c - torch.from_numpy(ct).cuda())
    gf, gx, gy = h.grad(f, c, g)
    back = h.apply(nh.EXACT_ADJ, gf)
    assert float(torch.linalg.norm(back - g) / torch.linalg.norm(g)) < 1e-8
    h.close()
    rng = np.random.default_rng(56)
    dx, dy = rng.standard_normal(w.M), rng.standard_normal(w.M)
    step = 1e-5   # phase changes ~2 pi 128 step: central-difference truncation ~1e-5 relative

    def L(sgn):
        # A is 1-periodic in each coordinate, so wrapping back into [0, 1) leaves the map unchanged
        xs, ys = np.mod(x + sgn * step * dx, 1.0), np.mod(y + sgn * step * dy, 1.0)
        hh = nh.NudftHSS(torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), w.nx, w.ny, **opts).factor()
        cc = hh.solve(f)
        hh.close()
        return float(torch.sum(torch.abs(cc - torch.from_numpy(ct).cuda()) ** 2))

    fd = (L(1) - L(-1)) / (2 * step)
    dd = float(np.dot(gx.cpu().numpy(), dx) + np.dot(gy.cpu().numpy(), dy))
    # both solutions are refined to ~1e-12; the bound covers the O(eps) error of the mixed-mode
    # adjoint (its fixed point lies in the range of the FP32 HSS adjoint) and the truncation error
    assert abs(fd - dd) < 3e-4 * abs(dd)
