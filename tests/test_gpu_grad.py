"""GPU parity of the backward pass of c = A^+ f (adjoint solve and point gradient) against the
FP64 oracle gradient and finite differences of the GPU map (the n = 128 differentiation
workload itself is checked in test_gpu_scale_configs.py).

The gradient of a real loss L(c) in the torch convention (g = dL/dRe c + i dL/dIm c):
  grad_f = lam = (A^+)^* g,  dL/dx_j = sum_q Re[-conj(lam_jq)(A_x c)_jq + conj((A_x mu)_jq) r_jq],
mu = A^+ lam, r = f - A c.  FP64 mode at eps = 1e-10: the HSS pseudo-inverse differs from A^+ by
~1e-10 relative (cond(A) ~ 2-3 on these grids), so the gradients match the oracle to 1e-7.
"""
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


def to_np(t):
    return t.detach().cpu().numpy()


def _case(name, s, seed):
    w = WORKLOADS[name]
    x, y, _ = make_workload(w)
    f = complex_normal((x.size, s), seed)                 # inconsistent data: r != 0
    g = complex_normal((w.N, s), seed + 1)
    return w, x, y, f, g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,levels", [("fp64_n16", 2), ("fp64_n32", 3)])
def test_pinv_adj_matches_oracle(nh, name, levels):
    w, x, y, _, g = _case(name, 3, 7)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=1e-10, levels=levels).factor()
    lam = to_np(h.apply(nh.PINV_ADJ, torch.from_numpy(g).cuda()))
    ref = orc.pinv_adjoint(orc.nudft_matrix(x, y, w.nx, w.ny), g)
    assert _rel(lam, ref) < 1e-8
    h.close()


def test_pinv_adj_is_adjoint_of_pinv(nh):
    """<PINV_ADJ g, f> = <g, PINV f> for the library's own operator (exact for any HSS rank)."""
    w, x, y, f, g = _case("fp64_n32", 2, 9)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=1e-6, levels=3).factor()
    lam = to_np(h.apply(nh.PINV_ADJ, torch.from_numpy(g).cuda()))
    c = to_np(h.solve(torch.from_numpy(f).cuda()))
    lhs, rhs = np.vdot(lam, f), np.vdot(g, c)
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(lam) * np.linalg.norm(f)
    h.close()


@pytest.mark.parametrize("name,levels,prec,tol", [("fp64_n16", 2, "fp64", 1e-7), ("fp64_n32", 3, "fp64", 1e-7),
                                                  ("fp64_n32", 3, "mixed", 1e-5)])
def test_grad_matches_oracle(nh, name, levels, prec, tol):
    w, x, y, f, g = _case(name, 2, 21)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=1e-10 if prec == "fp64" else 1e-6,
                    levels=levels, prec=prec, refine_tol=1e-12, refine_max=20).factor()
    fc = torch.from_numpy(f).cuda()
    c = h.solve(fc)
    gf, gx, gy = h.grad(fc, c, torch.from_numpy(g).cuda())
    c_ref, lam_ref, gx_ref, gy_ref = orc.lstsq_grad(x, y, w.nx, w.ny, f, g)
    assert _rel(to_np(c), c_ref) < tol
    assert _rel(to_np(gf), lam_ref) < tol
    assert _rel(to_np(gx), gx_ref) < tol
    assert _rel(to_np(gy), gy_ref) < tol
    h.close()


def test_autograd_matches_oracle_and_finite_differences(nh):
    """loss = sum |c - c_target|^2 through nh.lstsq; backward against the oracle gradient with
    g = 2 (c - c_target), and against central differences of the GPU map itself."""
    w, x, y, f, _ = _case("fp64_n16", 2, 31)
    ct = complex_normal((w.N, 2), 33)
    opts = dict(eps=1e-10, levels=2)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    yt = torch.from_numpy(y).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    ctt = torch.from_numpy(ct).cuda()
    c = nh.lstsq(ft, xt, yt, w.nx, w.ny, **opts)
    loss = torch.sum(torch.abs(c - ctt) ** 2)
    loss.backward()
    c_np = to_np(c)
    _, lam_ref, gx_ref, gy_ref = orc.lstsq_grad(x, y, w.nx, w.ny, f, 2 * (c_np - ct))
    assert _rel(to_np(ft.grad), lam_ref) < 1e-7
    assert _rel(to_np(xt.grad), gx_ref) < 1e-7
    assert _rel(to_np(yt.grad), gy_ref) < 1e-7

    def L(xv, yv):
        with torch.no_grad():
            cc = nh.lstsq(torch.from_numpy(f).cuda(), torch.from_numpy(xv).cuda(), torch.from_numpy(yv).cuda(),
                          w.nx, w.ny, **opts)
            return float(torch.sum(torch.abs(cc - ctt) ** 2))

    h = 1e-5
    gx = to_np(xt.grad)
    for j in (3, 200, 511):
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (L(np.mod(xp, 1.0), y) - L(np.mod(xm, 1.0), y)) / (2 * h)
        assert abs(fd - gx[j]) < 1e-4 * max(1.0, np.max(np.abs(gx)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpointed_factors_are_recomputed(nh, prec):
    """Per-level checkpointing: handing back the top two levels' factors frees their memory, and
    the next solve / gradient factors them again from the kept levels, giving the same results."""
    w, x, y, f, g = _case("fp64_n32", 2, 91)
    eps = 1e-10 if prec == "fp64" else 1e-6
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=eps, levels=3, prec=prec,
                    refine_tol=1e-12, refine_max=20).factor()
    fc, gc = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    c0 = to_np(h.solve(fc))
    gf0, gx0, gy0 = (to_np(t) for t in h.grad(fc, torch.from_numpy(c0).cuda(), gc))
    bytes0 = h.info()["device_bytes"]
    h.checkpoint(2)
    info = h.info()
    assert info["checkpointed_levels"] == 2 and info["device_bytes"] < bytes0
    c1 = to_np(h.solve(fc))
    assert h.info()["checkpointed_levels"] == 0
    gf1, gx1, gy1 = (to_np(t) for t in h.grad(fc, torch.from_numpy(c1).cuda(), gc))
    h.close()
    assert _rel(c1, c0) < 1e-12
    assert _rel(gf1, gf0) < 1e-12 and _rel(gx1, gx0) < 1e-12 and _rel(gy1, gy0) < 1e-12


def test_autograd_with_checkpointed_levels(nh):
    """lstsq(..., checkpoint_levels=2): the backward pass refactors the handed-back levels and
    returns the gradients of the run without checkpointing."""
    w, x, y, f, _ = _case("fp64_n32", 2, 93)
    ct = torch.from_numpy(complex_normal((w.N, 2), 94)).cuda()
    grads = []
    for ck in (0, 2):
        xt = torch.from_numpy(x).cuda().requires_grad_(True)
        yt = torch.from_numpy(y).cuda().requires_grad_(True)
        ft = torch.from_numpy(f).cuda().requires_grad_(True)
        c = nh.lstsq(ft, xt, yt, w.nx, w.ny, eps=1e-10, levels=3, checkpoint_levels=ck)
        torch.sum(torch.abs(c - ct) ** 2).backward()
        grads.append((to_np(ft.grad), to_np(xt.grad), to_np(yt.grad)))
    for a, b in zip(*grads):
        assert _rel(b, a) < 1e-12
