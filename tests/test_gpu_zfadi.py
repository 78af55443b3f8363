"""GPU parity of the fADI + ID construction of the 1D HSS approximations (NUDFT2_FLAG_FADI, the
route Sec. 3.1 cites for Alg. 1 step 1): the same face-splitting HSS, recompression, URV factor
and solve, built on interpolative 1D factors, against the FP64 oracle through the C-ABI.

Tolerances are those of the default route: the forward map within 100 eps of the exact A
(Thm. 3.7 with the 1D factors at eps/10), FP64 solves within 1e-8 of the dense least-squares
solution, MIXED solves refined to 1e-8 of c_true."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import WORKLOADS, complex_normal, jittered_grid, make_workload, noise_like  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


def relerr_cols(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


def to_np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name", ["fp64_n16", "fp64_n32", "fp64_n64"])
def test_fadi_forward_map_error_bound(nh, name):
    w = WORKLOADS[name]
    x, y, _ = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels, fadi=True)
    c = complex_normal((w.N, 4), 77)
    fa = to_np(h.apply(nh.FAST_FWD, torch.from_numpy(c)))
    h.close()
    assert relerr_cols(fa, orc.forward(x, y, c, w.nx, w.ny)) < 100 * w.eps


@pytest.mark.parametrize("name", ["fp64_n16", "fp64_n32"])
def test_fadi_solve_matches_dense_oracle(nh, name):
    w = WORKLOADS[name]
    x, y, ct = make_workload(w)
    f0 = orc.forward(x, y, ct, w.nx, w.ny)
    f = f0 + noise_like(f0, 1e-6, 99)              # inconsistent data: LS solution != c_true
    A = orc.nudft_matrix(x, y, w.nx, w.ny)
    cref, _, _ = orc.lstsq(A, f)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels, fadi=True).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    assert relerr_cols(c, cref) < 1e-8


def test_fadi_ranks_track_the_svd_route(nh):
    """After recompression at eps the 2D ranks do not depend much on how the 1D factors were
    built: the interpolative route keeps at most a few more directions per level."""
    w = WORKLOADS["fp64_n64"]
    x, y, _ = make_workload(w)
    ranks = {}
    for fadi in (False, True):
        h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels, fadi=fadi)
        ranks[fadi] = h.info()["level_rank"]
        h.close()
    for a, b in zip(ranks[False][1:], ranks[True][1:]):
        assert b <= a + max(8, a // 4)


@pytest.mark.parametrize("nx,ny,mx,my,lx,ly,seed", [(16, 64, 32, 64, 2, 4, 7), (24, 12, 48, 14, 2, 2, 123)])
def test_fadi_unbalanced_and_ragged_trees(nh, nx, ny, mx, my, lx, ly, seed):
    x, y = jittered_grid(mx, my, -0.3, 0.3, seed)
    ct = complex_normal((nx * ny, 2), seed + 50)
    f = orc.forward(x, y, ct, nx, ny)
    h = nh.NudftHSS(x, y, nx, ny, eps=1e-10, levels=lx, levels_y=ly, fadi=True).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    cref, _, _ = orc.lstsq(orc.nudft_matrix(x, y, nx, ny), f)
    assert relerr_cols(c, cref) < 1e-8


def test_fadi_mixed_precision_refined(nh):
    w = WORKLOADS["mixed_n64"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct[:, :4], w.nx, w.ny)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=1e-6, levels=w.levels, prec="mixed", refine_tol=1e-10,
                    refine_max=12, fadi=True).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    info = h.info()
    h.close()
    assert info["refine_relres"] <= 1e-10
    assert relerr_cols(c, ct[:, :4]) < 1e-8


def test_fadi_uniform_grid_is_the_inverse_dft(nh):
    """Uniform n x n grid: G~ = I, every off-diagonal block is zero, the solve is A^* f / N."""
    from synthetic import uniform_grid
    n = 32
    x, y = uniform_grid(n, n)
    ct = complex_normal((n * n, 2), 81)
    f = orc.forward(x, y, ct, n, n)
    h = nh.NudftHSS(x, y, n, n, eps=1e-10, levels=3, fadi=True).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    assert relerr_cols(c, ct) < 1e-12
