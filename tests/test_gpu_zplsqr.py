"""plsqr: LSQR preconditioned by the HSS direct solver (Sec. 4.1 / Sec. 5 tables), with the
exact FP64 apply of A.  A coarse factorization (eps 1e-4), whose direct solve is only ~1e-4
accurate, must drive the iterations to the least-squares solution in a handful of steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import WORKLOADS, complex_normal, make_workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


def _relcols(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plsqr_coarse_preconditioner_reaches_ls_solution(nh, prec):
    w = WORKLOADS["fp64_n32"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct, w.nx, w.ny)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=1e-4, levels=w.levels,
                    prec=prec, refine_max=1).factor()
    ft = torch.from_numpy(f).cuda()
    c, it, rr = h.plsqr(ft, tol=1e-12, maxit=100)
    c = c.cpu().numpy()
    assert _relcols(c, ct) < 1e-10
    assert rr < 1e-11
    assert 1 <= it <= 30
    # the same factorization as a direct solver is far less accurate
    c_direct = h.apply(nh.PINV, ft).cpu().numpy() if prec == "fp64" else None
    if c_direct is not None:
        assert _relcols(c_direct, ct) > 100 * _relcols(c, ct)
    h.close()


def test_plsqr_inconsistent_data_and_zero_column(nh):
    """Random data (nonzero LS residual) with a fine preconditioner: the result matches the
    oracle's least-squares solution to the 1e-8 target; an all-zero column returns zero."""
    w = WORKLOADS["fp64_n16"]
    x, y, _ = make_workload(w)
    f = complex_normal((w.M, 3), 41)
    f[:, 1] = 0
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=1e-10, levels=w.levels).factor()
    c, it, rr = h.plsqr(torch.from_numpy(f).cuda(), tol=1e-12, maxit=100)
    c = c.cpu().numpy()
    h.close()
    cref, _, _ = orc.lstsq(orc.nudft_matrix(x, y, w.nx, w.ny), f[:, [0, 2]])
    assert _relcols(c[:, [0, 2]], cref) < 1e-8
    assert np.all(c[:, 1] == 0)
    assert it <= 30


def _polar_handle(nh, n, eps, levels):
    from synthetic import polar_grid
    x, y = polar_grid(n)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), n, n, eps=eps, levels=levels).factor()
    return x, y, h


def test_polar_grid_direct_solve(nh):
    """Modified polar grid, n = 16 (cond(A) ~ 2e2): the FP64 direct solve at eps 1e-10 recovers
    c_true of consistent data to within cond(A) times the HSS approximation error (at most
    (1 + C) eps with C from the tree depth; 1e-8 allowed)."""
    n = 16
    x, y, h = _polar_handle(nh, n, 1e-10, 2)
    ct = complex_normal((n * n, 2), 61)
    f = orc.forward(x, y, ct, n, n)
    c = h.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    h.close()
    assert _relcols(c, ct) < 2e2 * 1e-8


def test_polar_grid_plsqr(nh):
    """Modified polar grid, n = 32 (cond(A) ~ 8e2), coarse factorization eps 1e-4 as the
    preconditioner: plsqr reaches c_true of consistent data (the paper's polar-grid use)."""
    n = 32
    x, y, h = _polar_handle(nh, n, 1e-4, 3)
    ct = complex_normal((n * n, 2), 62)
    f = orc.forward(x, y, ct, n, n)
    c, it, rr = h.plsqr(torch.from_numpy(f).cuda(), tol=1e-12, maxit=200)
    h.close()
    assert _relcols(c.cpu().numpy(), ct) < 8e2 * 1e-11
    assert rr < 1e-10
    assert it <= 100
