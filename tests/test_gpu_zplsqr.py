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
