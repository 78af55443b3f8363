"""Parity at the full sizes of the FP64, mixed-precision and differentiation configurations,
where a dense oracle solve is out of reach (A is 32768 x 16384 or 131072 x 65536).

Checked instead:
* the data f: formed by the oracle's direct sum of Eq. 1 (all rows); for config 3 the
  library's exact FP64 apply is also compared with it on every row;
* the solution: consistent data (plus 1e-12 relative noise for config 2) has the LS solution
  c_true up to ~cond(A) * noise, so c must match c_true to the 1e-8 target;
* sampled residuals: r_j = f_j - (A c)_j evaluated by the oracle at sampled points j.
The handles use the same options as bench.py.  The differentiation workload is checked against
the oracle's matrix-free least-squares gradient at 64 sampled points and by a central difference
of the map."""
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
    # the oracle's own least-squares solution of the noisy data (CGLS with the direct applies, first
    # column, ~20 s on the host), not only c_true
    c_ls, _ = orc.cgls(x, y, f[:, 0], w.nx, w.ny, tol=1e-13)
    assert _relcols(c[:, :1], c_ls[:, None]) < 1e-8


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


@pytest.fixture(scope="module")
def grad5():
    """The differentiation workload (n = 128, M = 32768, 16 right-hand sides), consistent data
    f = A c_true formed by the oracle, loss L = sum |c - c_target|^2, and the oracle's gradient at
    64 sampled points (matrix-free: CG on the normal equations with the direct applies, ~1 min on
    the host).  For consistent data the least-squares solution is c_true."""
    w = WORKLOADS["grad_n128"]
    x, y, c_true = make_workload(w)
    ctg = complex_normal((w.N, w.nrhs), 55)
    f = orc.forward(x, y, c_true, w.nx, w.ny)
    rows = np.random.default_rng(57).choice(w.M, 64, replace=False)
    g = 2 * (c_true - ctg)
    _, lam, gx, gy = orc.lstsq_grad_rows(x, y, w.nx, w.ny, f, g, rows, c=c_true, tol=1e-13)
    return dict(w=w, x=x, y=y, ctg=ctg, f=f, rows=rows, lam=lam, gx=gx, gy=gy)


def _gpu_grad(nh, d, **opts):
    w = d["w"]
    xt, yt = torch.from_numpy(d["x"]).cuda(), torch.from_numpy(d["y"]).cuda()
    h = nh.NudftHSS(xt, yt, w.nx, w.ny, levels=w.levels, **opts).factor()
    ft = torch.from_numpy(d["f"]).cuda()
    c = h.solve(ft)
    gf, gx, gy = h.grad(ft, c, 2 * (c - torch.from_numpy(d["ctg"]).cuda()))
    h.close()
    return gf.cpu().numpy(), gx.cpu().numpy(), gy.cpu().numpy()


MIXED_13 = dict(eps=1e-6, prec="mixed", refine_tol=1e-13, refine_max=30)


def test_grad_config5_mixed_refined_matches_oracle_and_central_differences(nh, grad5):
    """Mixed precision refined to 1e-13 with the FP64 exact applies: grad_f and the point
    gradient match the oracle's exact least-squares gradient at the sampled points to 1e-8, and
    a central difference (h = 1e-6) of the map along a random direction of all 2M coordinates
    matches the gradient's directional derivative to 1e-6."""
    d = grad5
    w, x, y = d["w"], d["x"], d["y"]
    gf, gx, gy = _gpu_grad(nh, d, **MIXED_13)
    rows = d["rows"]
    assert _relcols(gf, d["lam"]) < 1e-8
    assert float(np.linalg.norm(gx[rows] - d["gx"]) / np.linalg.norm(d["gx"])) < 1e-8
    assert float(np.linalg.norm(gy[rows] - d["gy"]) / np.linalg.norm(d["gy"])) < 1e-8
    rng = np.random.default_rng(56)
    dx, dy = rng.standard_normal(w.M), rng.standard_normal(w.M)
    step = 1e-6   # truncation ~ (2 pi 128 * 4.5e-6)^2 / 6 < 1e-7 relative
    ft = torch.from_numpy(d["f"]).cuda()
    ctg = torch.from_numpy(d["ctg"]).cuda()

    def L(sgn):
        # A is 1-periodic in each coordinate, so wrapping back into [0, 1) leaves the map unchanged
        xs, ys = np.mod(x + sgn * step * dx, 1.0), np.mod(y + sgn * step * dy, 1.0)
        hh = nh.NudftHSS(torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), w.nx, w.ny, levels=w.levels,
                         **MIXED_13).factor()
        cc = hh.solve(ft)
        hh.close()
        return float(torch.sum(torch.abs(cc - ctg) ** 2))

    fd = (L(1) - L(-1)) / (2 * step)
    dd = float(np.dot(gx, dx) + np.dot(gy, dy))
    assert abs(fd - dd) < 1e-6 * abs(dd)


def test_grad_config5_fp64_mode_matches_oracle(nh, grad5):
    """FP64 mode (eps 1e-10, no refinement) at the full size: the gradient of the HSS
    pseudo-inverse matches the oracle's at the sampled points to 1e-7."""
    d = grad5
    gf, gx, gy = _gpu_grad(nh, d, eps=1e-10)
    rows = d["rows"]
    assert _relcols(gf, d["lam"]) < 1e-7
    assert float(np.linalg.norm(gx[rows] - d["gx"]) / np.linalg.norm(d["gx"])) < 1e-7
    assert float(np.linalg.norm(gy[rows] - d["gy"]) / np.linalg.norm(d["gy"])) < 1e-7
