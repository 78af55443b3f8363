"""GPU parity: every step of the CUDA path against the FP64 oracle, through the C-ABI.

Tolerances (FP64 mode, HSS tolerance eps = 1e-10): kernel entries and the exact apply are
direct FP64 evaluations, checked to 1e-12 relative; the HSS solution is checked to the 1e-8
relative 2-norm error of the target (the HSS approximation error is (1+C) eps by Thm. 3.7 and
the jittered grids here have cond(A) ~ 2-3, so the solve error is ~1e-10).
"""
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


# ------------------------------------------------------------------ kernel entries (Sec. 2.4)
@pytest.mark.parametrize("n,M", [(16, 300), (37, 257), (128, 1000)])
def test_psi_eval_matches_oracle(nh, n, M):
    x, _ = jittered_grid(M, 1, -0.45, 0.45, 100 + n)
    G = to_np(nh.psi_eval(torch.from_numpy(x), n))
    ref = orc.tilde_1d(x, n)
    assert np.max(np.abs(G - ref)) < 1e-12


def test_psi_eval_unperturbed_grid_identity(nh):
    n = 64
    x = np.arange(n) / n
    G = to_np(nh.psi_eval(torch.from_numpy(x), n))
    assert np.max(np.abs(G - np.eye(n))) < 1e-14


# ------------------------------------------------------------------ exact apply (Eq. 1)
@pytest.mark.parametrize("nx,ny,mx,my,s", [(16, 16, 32, 16, 1), (24, 10, 40, 13, 3), (64, 32, 128, 40, 2)])
def test_exact_apply_forward_and_adjoint(nh, nx, ny, mx, my, s):
    x, y = jittered_grid(mx, my, -0.3, 0.3, nx * 7 + ny)
    h = nh.NudftHSS(x, y, nx, ny, levels=1)
    c = complex_normal((nx * ny, s), 5)
    f = to_np(h.apply(nh.EXACT_FWD, torch.from_numpy(c)))
    assert relerr_cols(f, orc.forward(x, y, c, nx, ny)) < 1e-12
    g = complex_normal((x.size, s), 6)
    a = to_np(h.apply(nh.EXACT_ADJ, torch.from_numpy(g)))
    assert relerr_cols(a, orc.adjoint(x, y, g, nx, ny)) < 1e-12
    h.close()


# ------------------------------------------------------------------ HSS approximation (Thm. 3.7)
@pytest.mark.parametrize("name", ["fp64_n16", "fp64_n32", "fp64_n64", "fp64_n128"])
def test_hss_forward_map_error_bound(nh, name):
    """FAST_FWD applies A_fast = G~_hss F; ||A_fast - A|| / ||A|| stays within (1+C) eps, up to
    the n = 128 FP64 workload (three and four tree levels)."""
    w = WORKLOADS[name]
    x, y, _ = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels)
    c = complex_normal((w.N, 4), 77)
    fa = to_np(h.apply(nh.FAST_FWD, torch.from_numpy(c)))
    fe = orc.forward(x, y, c, w.nx, w.ny)
    assert relerr_cols(fa, fe) < 100 * w.eps
    h.close()


# ------------------------------------------------------------------ end-to-end solve
def _dense_ref(w, f):
    x, y, _ = make_workload(w)
    A = orc.nudft_matrix(x, y, w.nx, w.ny)
    c, _, rmin = orc.lstsq(A, f)
    assert rmin > 0
    return c


@pytest.mark.parametrize("name", ["fp64_n16", "fp64_n32"])
def test_solve_fp64_matches_dense_oracle(nh, name):
    w = WORKLOADS[name]
    x, y, ct = make_workload(w)
    f0 = orc.forward(x, y, ct, w.nx, w.ny)
    f = f0 + noise_like(f0, 1e-6, 99)              # inconsistent data: LS solution != c_true
    cref = _dense_ref(w, f)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    assert relerr_cols(c, cref) < 1e-8
    info = h.info()
    assert info["max_rank"] > 0
    h.close()


def test_solve_rectangular_grid_ragged_leaves(nh):
    """nx != ny and leaves with uneven point counts; columns split 3/3 at the leaves."""
    nx, ny = 24, 12
    x, y = jittered_grid(48, 14, -0.35, 0.35, 123)
    c0 = complex_normal((nx * ny, 2), 124)
    f = orc.forward(x, y, c0, nx, ny)
    A = orc.nudft_matrix(x, y, nx, ny)
    cref, _, _ = orc.lstsq(A, f)
    h = nh.NudftHSS(x, y, nx, ny, eps=1e-10, levels=2).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    assert relerr_cols(c, cref) < 1e-8
    h.close()


def test_solve_mixed_precision_refines_to_fp64(nh):
    w = WORKLOADS["fp64_n32"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct, w.nx, w.ny)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=1e-6, levels=w.levels, prec="mixed", refine_tol=1e-10,
                    refine_max=10).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    info = h.info()
    assert info["refine_relres"] <= 1e-10
    assert relerr_cols(c, ct) < 1e-8
    h.close()


def test_solve_before_factor_is_an_ordering_error(nh):
    w = WORKLOADS["fp64_n16"]
    x, y, _ = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, levels=w.levels)
    with pytest.raises(nh.NudftError) as e:
        h.solve(torch.zeros(w.M, dtype=torch.complex128))
    assert e.value.code == 6
    h.close()


def test_points_outside_unit_square_rejected(nh):
    x, y = jittered_grid(32, 16, -0.25, 0.25, 1)
    x = x.copy()
    x[3] = 1.0
    with pytest.raises(nh.NudftError) as e:
        nh.NudftHSS(x, y, 16, 16, levels=2)
    assert e.value.code == 1


# ------------------------------------------------------------------ URV exactness (Sec. 2.3)
@pytest.mark.parametrize("name,levels", [("fp64_n32", 3), ("fp64_n32", 2), ("fp64_n64", 3)])
def test_urv_solves_its_own_hss_matrix_exactly(nh, name, levels):
    """For f' = A_fast c (consistent with the HSS matrix), the URV least-squares solution is c.

    Isolates the URV factorization and sweeps from the approximation error of the HSS
    construction: only rounding remains (the HSS matrix has full column rank here).
    """
    w = WORKLOADS[name]
    x, y, ct = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=levels).factor()
    c = torch.from_numpy(ct).cuda()
    fa = h.apply(nh.FAST_FWD, c)
    c2 = h.solve(fa)
    assert relerr_cols(to_np(c2), ct) < 1e-10
    h.close()


def test_standalone_exact_apply_matches_oracle(nh):
    nx, ny = 20, 12
    x, y = jittered_grid(37, 13, -0.3, 0.3, 444)
    c = complex_normal((nx * ny, 3), 445)
    f = to_np(nh.exact_apply(x, y, nx, ny, nh.EXACT_FWD, torch.from_numpy(c)))
    assert relerr_cols(f, orc.forward(x, y, c, nx, ny)) < 1e-12
    g = complex_normal((x.size, 2), 446)
    a = to_np(nh.exact_apply(x, y, nx, ny, nh.EXACT_ADJ, torch.from_numpy(g)))
    assert relerr_cols(a, orc.adjoint(x, y, g, nx, ny)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_repeated_solves_replay_the_captured_graph(nh, prec):
    """The first solve of a right-hand-side count runs the sweeps and captures them into a CUDA
    graph; later solves replay the graph.  Results must agree with the first solve and with the
    dense oracle, for a second right-hand-side count too."""
    w = WORKLOADS["fp64_n32"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct, w.nx, w.ny)
    eps = 1e-10 if prec == "fp64" else 1e-6
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=eps, levels=w.levels, prec=prec, refine_tol=1e-10, refine_max=10).factor()
    ft = torch.from_numpy(f)
    c1 = to_np(h.solve(ft))
    c2 = to_np(h.solve(ft))
    c3 = to_np(h.solve(ft[:, :1]))
    c4 = to_np(h.solve(ft[:, :1]))
    assert relerr_cols(c1, ct) < 1e-8
    assert relerr_cols(c2, c1) < 1e-13
    assert relerr_cols(c4, c3) < 1e-13
    assert relerr_cols(c3, ct[:, :1]) < 1e-8
    info = h.info()
    assert info["solve_graphs"] == 2 and info["solve_graph_failures"] == 0
    assert info["solve_replays"] >= 2
    h.close()


# ------------------------------------------------------------------ adjoint of the HSS forward map
@pytest.mark.parametrize("name", ["fp64_n16", "fp64_n32"])
def test_hss_adjoint_map_is_the_adjoint(nh, name):
    """FAST_ADJ applies (G~_hss F)^*: <A_fast c, g> = <c, A_fast^* g> to rounding, and A_fast^* g
    stays within the Thm. 3.7 error bound of the exact adjoint A^* g (oracle)."""
    w = WORKLOADS[name]
    x, y, _ = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels)
    c = complex_normal((w.N, 3), 78)
    g = complex_normal((w.M, 3), 79)
    fa = to_np(h.apply(nh.FAST_FWD, torch.from_numpy(c)))
    ga = to_np(h.apply(nh.FAST_ADJ, torch.from_numpy(g)))
    h.close()
    lhs = np.sum(np.conj(g) * fa, axis=0)
    rhs = np.sum(np.conj(ga) * c, axis=0)
    assert np.max(np.abs(lhs - rhs) / (np.linalg.norm(g, axis=0) * np.linalg.norm(fa, axis=0))) < 1e-13
    assert relerr_cols(ga, orc.adjoint(x, y, g, w.nx, w.ny)) < 100 * w.eps


# ------------------------------------------------------------------ degenerate grids
def test_unperturbed_square_grid_identity_kernel(nh):
    """Uniform grid x = i/n, y = j/n, M = N: every point sits on a bin boundary (x = 0 included),
    G~ = I, so every off-diagonal HSS rank is 0 and A^* A = N I: the solve is the inverse DFT,
    c = A^* f / N, exactly up to rounding."""
    from synthetic import uniform_grid
    n = 32
    x, y = uniform_grid(n, n)
    ct = complex_normal((n * n, 2), 81)
    f = orc.forward(x, y, ct, n, n)
    h = nh.NudftHSS(x, y, n, n, eps=1e-10, levels=3).factor()
    assert max(h.info()["level_rank"][1:]) == 0
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    assert relerr_cols(c, orc.adjoint(x, y, f, n, n) / (n * n)) < 1e-13
    assert relerr_cols(c, ct) < 1e-13


def test_oversampled_uniform_grid_on_bin_boundaries(nh):
    """Uniform 2n x n grid: half of the x coordinates sit exactly on column-bin boundaries and
    A^* A = M I; the solve must return c = A^* f / M (= c_true for consistent data)."""
    from synthetic import uniform_grid
    n = 32
    x, y = uniform_grid(2 * n, n)
    ct = complex_normal((n * n, 2), 82)
    f = orc.forward(x, y, ct, n, n) + 0.1 * complex_normal((x.size, 2), 83)   # inconsistent data
    h = nh.NudftHSS(x, y, n, n, eps=1e-10, levels=3).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    assert relerr_cols(c, orc.adjoint(x, y, f, n, n) / x.size) < 1e-10


def test_mixed_refinement_incremental_residual(nh):
    """MIXED refinement: the default (first residual from the exact FP64 apply, later ones updated
    by the FP32 exact apply of the small correction) reaches the same solution as an FP64 residual
    at every step, to the 1e-8 target, with less FP64 apply time."""
    w = WORKLOADS["mixed_n64"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct[:, :4], w.nx, w.ny)
    out = {}
    for full in (False, True):
        h = nh.NudftHSS(x, y, w.nx, w.ny, eps=1e-6, levels=w.levels, prec="mixed", refine_tol=1e-11,
                        refine_max=12, profile=True, fp64_residuals=full).factor()
        c = to_np(h.solve(torch.from_numpy(f)))
        out[full] = (c, h.info(), h.kstats())
        h.close()
    for full in (False, True):
        c, info, _ = out[full]
        assert relerr_cols(c, ct[:, :4]) < 1e-9
        assert info["refine_relres"] <= 1e-11
    fp64_ms = {full: sum(v["ms"] for k, v in out[full][2].items() if k.endswith("_fp64")) for full in (False, True)}
    assert fp64_ms[False] < fp64_ms[True]


# ------------------------------------------------------------------ unbalanced product trees (Def. 3.3 (2), (3))
@pytest.mark.parametrize("nx,ny,mx,my,lx,ly,seed", [
    (16, 16, 32, 16, 1, 2, 1),      # config 1 with 8 x 4 product leaves ("leaf 32")
    (16, 64, 32, 64, 2, 4, 7),      # ny = 4 nx: square 4 x 4 leaves instead of equal-depth 4 x 16
    (64, 16, 128, 16, 4, 2, 8),     # the other way round
    (32, 32, 64, 32, 3, 1, 9),      # x split three times, y once: leaves 4 x 16
])
def test_unbalanced_tree_solve_matches_oracle(nh, nx, ny, mx, my, lx, ly, seed):
    """T^x of depth lx and T^y of depth ly: below min(lx, ly) levels only the deeper tree splits
    (binary product-tree levels).  The HSS forward map stays within the Thm. 3.7 bound of the
    exact A, and the FP64 solve matches the dense oracle's least-squares solution to 1e-8."""
    x, y = jittered_grid(mx, my, -0.25, 0.25, seed)
    ct = complex_normal((nx * ny, 2), seed + 50)
    f = orc.forward(x, y, ct, nx, ny)
    h = nh.NudftHSS(x, y, nx, ny, eps=1e-10, levels=lx, levels_y=ly).factor()
    info = h.info()
    assert info["levels"] == max(lx, ly)
    fa = to_np(h.apply(nh.FAST_FWD, torch.from_numpy(ct)))
    assert relerr_cols(fa, f) < 100 * 1e-10
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    cref, _, _ = orc.lstsq(orc.nudft_matrix(x, y, nx, ny), f)
    assert relerr_cols(c, cref) < 1e-8


def test_unbalanced_tree_mixed_refined(nh):
    """Mixed precision on an unbalanced tree, refined with the FP64 residual to 1e-10."""
    nx, ny = 32, 64
    x, y = jittered_grid(64, 64, -0.3, 0.3, 12)
    ct = complex_normal((nx * ny, 3), 13)
    f = orc.forward(x, y, ct, nx, ny)
    h = nh.NudftHSS(x, y, nx, ny, eps=1e-6, levels=2, levels_y=3, prec="mixed", refine_tol=1e-10,
                    refine_max=12).factor()
    c = to_np(h.solve(torch.from_numpy(f)))
    h.close()
    assert relerr_cols(c, ct) < 1e-8


@pytest.mark.parametrize("prec,s", [("fp64", 20), ("fp64", 1), ("mixed", 16), ("mixed", 5)])
def test_streaming_sweeps_match_gemm_sweeps(nh, monkeypatch, prec, s):
    """The URV solve and its adjoint with the streaming reflector kernels (the default) and with the
    generic blocked-GEMM application (NH_SWEEP_STREAM=0) give the same c to rounding, and both
    match the dense oracle's least-squares solution; s = 20 takes a 16 + 4 column split."""
    w = WORKLOADS["fp64_n32"]
    x, y, _ = make_workload(w)
    c0 = complex_normal((w.N, s), 321)
    f = orc.forward(x, y, c0, w.nx, w.ny)
    f = f + noise_like(f, 1e-6, 322)
    cref = _dense_ref(w, f)
    opts = dict(eps=w.eps, levels=w.levels) if prec == "fp64" else dict(eps=1e-6, levels=w.levels, prec="mixed",
                                                                         refine_tol=1e-10, refine_max=10)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("NH_SWEEP_STREAM", mode)
        h = nh.NudftHSS(x, y, w.nx, w.ny, **opts).factor()
        c = to_np(h.solve(torch.from_numpy(f)))
        g = to_np(h.apply(nh.PINV_ADJ, torch.from_numpy(c0)))
        h.close()
        out[mode] = (c, g)
    assert relerr_cols(out["1"][0], cref) < 1e-8
    assert relerr_cols(out["0"][0], cref) < 1e-8
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert relerr_cols(out["1"][0], out["0"][0]) < max(tol, 1e-9)
    assert relerr_cols(out["1"][1], out["0"][1]) < tol
