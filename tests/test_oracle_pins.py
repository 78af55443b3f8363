"""Pins for the CPU oracle: each check ties an oracle function to something other than itself.

* unperturbed grids reduce A to the 2D DFT (checked against numpy's FFT) and A^*A to N I
  (Sec. 1, uniform Cartesian grid remark);
* tiny least-squares problems are solved again by brute force (normal equations, extended
  precision Gaussian elimination);
* the transformed 1D matrix satisfies the Sylvester displacement identity and the
  Cauchy-like closed form of Sec. 2.4, has unit row norms (Sec. 3.3, equal row norms), and
  is the identity on the unperturbed square grid (Psi = 1 at coincidence, Sec. 2.4);
* the face-splitting identity A F^{-1} = (A^x F_x^{-1}) . (A^y F_y^{-1}) (Sec. 3.1).

The mutation tests plant plausible mistakes in copies of oracle routines (sign of the
exponent, transposed column order, dropped reflector factor, DFT normalisation; in the gradient:
residual-term sign, dropped residual term, derivative sign) and assert a pin catches each.

The gradient oracle (pinv_adjoint, lstsq_grad) is pinned by the minimum-norm property of
(A^+)^* g and by central differences of the least-squares map in the point coordinates and in f.
"""
import numpy as np
import pytest

import oracle as orc
from synthetic import WORKLOADS, complex_normal, jittered_grid, make_workload, noise_like, uniform_grid


# ---------------------------------------------------------------- pin helpers (return errors)
def fft_pin_error(forward_fn, nx, ny, seed=7):
    """max |forward(c) - fft2(c)| / max|fft2(c)| on the unperturbed M = N grid."""
    x, y = uniform_grid(nx, ny)
    c = complex_normal(nx * ny, seed)
    f = forward_fn(x, y, c, nx, ny)
    ref = np.fft.fft2(c.reshape(nx, ny)).ravel()     # point (i, j) -> index i*ny + j
    return np.max(np.abs(f - ref)) / np.max(np.abs(ref))


def qr_pin_error(qr_fn, A, compare_lapack=True):
    """max of ||Q R - A||, ||Q^*Q - I|| and the |R_ii| mismatch against LAPACK's QR.

    |R_ii| is unique only for full column rank, so rank-deficient inputs skip that part.
    """
    R, vs, taus = qr_fn(A)
    m, n = A.shape
    Q = orc.apply_q(vs, taus, np.eye(m, dtype=complex))
    e1 = np.max(np.abs(Q @ R - A)) / np.max(np.abs(A))
    e2 = np.max(np.abs(Q.conj().T @ Q - np.eye(m)))
    Rl = np.linalg.qr(A, mode="r")
    p = min(m, n)
    e3 = np.max(np.abs(np.abs(np.diag(R[:p, :p])) - np.abs(np.diag(Rl[:p, :p])))) / np.max(np.abs(A))
    e3 = e3 if compare_lapack else 0.0
    e4 = np.max(np.abs(np.tril(R[:p, :p], -1))) if p > 1 else 0.0
    return max(e1, e2, e3, e4)


# ---------------------------------------------------------------- forward / adjoint
@pytest.mark.parametrize("nx,ny", [(8, 6), (5, 7), (16, 16)])
def test_forward_is_fft2_on_unperturbed_grid(nx, ny):
    assert fft_pin_error(orc.forward, nx, ny) < 1e-13


def test_dense_matrix_matches_direct_sum():
    x, y = jittered_grid(12, 10, -0.3, 0.3, 3)
    nx, ny = 6, 5
    c = complex_normal((nx * ny, 2), 4)
    A = orc.nudft_matrix(x, y, nx, ny)
    assert np.max(np.abs(A @ c - orc.forward(x, y, c, nx, ny))) < 1e-12
    # an entry written out by hand: j=7, (kx, ky)=(3, 2) -> column 2 + 3*ny
    j, kx, ky = 7, 3, 2
    assert abs(A[j, ky + kx * ny] - np.exp(-2j * np.pi * (kx * x[j] + ky * y[j]))) < 1e-13


def test_adjoint_is_conjugate_transpose():
    x, y = jittered_grid(10, 9, -0.3, 0.3, 5)
    nx, ny = 5, 4
    A = orc.nudft_matrix(x, y, nx, ny)
    f = complex_normal((x.size, 3), 6)
    assert np.max(np.abs(orc.adjoint(x, y, f, nx, ny) - A.conj().T @ f)) < 1e-12
    c = complex_normal(nx * ny, 8)
    lhs = np.vdot(orc.forward(x, y, c, nx, ny), f[:, 0])
    rhs = np.vdot(c, orc.adjoint(x, y, f[:, 0], nx, ny))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("nx,ny", [(6, 4), (8, 8)])
def test_unperturbed_normal_matrix_is_N_identity(nx, ny):
    x, y = uniform_grid(nx, ny)
    A = orc.nudft_matrix(x, y, nx, ny)
    assert np.max(np.abs(A.conj().T @ A - nx * ny * np.eye(nx * ny))) < 1e-11


def test_oversampled_grid_lstsq_is_scaled_adjoint():
    nx, ny = 6, 5
    x, y = uniform_grid(2 * nx, 2 * ny)                # M = 4N, columns of a larger DFT
    M = x.size
    A = orc.nudft_matrix(x, y, nx, ny)
    assert np.max(np.abs(A.conj().T @ A - M * np.eye(nx * ny))) < 1e-10
    f = complex_normal(M, 9)
    c, _, _ = orc.lstsq(A, f)
    assert np.max(np.abs(c - orc.adjoint(x, y, f, nx, ny) / M)) < 1e-13


# ---------------------------------------------------------------- least squares
def _normal_eq_bruteforce(A, f):
    """Normal equations A^*A c = A^*f by Gaussian elimination with partial pivoting in long double."""
    A = A.astype(np.clongdouble)
    G = A.conj().T @ A
    b = A.conj().T @ f.astype(np.clongdouble)
    n = G.shape[0]
    M = np.concatenate([G, b[:, None]], axis=1)
    for k in range(n):
        piv = k + int(np.argmax(np.abs(M[k:, k])))
        M[[k, piv]] = M[[piv, k]]
        for i in range(k + 1, n):
            M[i] -= (M[i, k] / M[k, k]) * M[k]
    c = np.zeros(n, dtype=np.clongdouble)
    for i in range(n - 1, -1, -1):
        c[i] = (M[i, n] - np.sum(M[i, i + 1:n] * c[i + 1:])) / M[i, i]
    return c.astype(np.complex128)


def test_lstsq_matches_bruteforce_tiny():
    x, y = jittered_grid(4, 2, -0.3, 0.3, 12)          # M = 8
    nx, ny = 2, 2                                      # N = 4
    A = orc.nudft_matrix(x, y, nx, ny)
    f = complex_normal(8, 13)
    c, res, rmin = orc.lstsq(A, f)
    cb = _normal_eq_bruteforce(A, f)
    assert np.max(np.abs(c - cb)) < 1e-12
    assert rmin > 0
    assert abs(res[0] - np.linalg.norm(A @ c - f)) < 1e-12


def test_lstsq_recovers_consistent_data():
    w = WORKLOADS["fp64_n16"]
    x, y, ct = make_workload(w)
    A = orc.nudft_matrix(x, y, w.nx, w.ny)
    f = orc.forward(x, y, ct, w.nx, w.ny)
    c, res, rmin = orc.lstsq(A, f)
    assert np.max(orc.relerr(c, ct)) < 1e-12
    assert rmin > 1.0          # full column rank with margin (smallest |R_ii| reported)


def test_lstsq_residual_orthogonal_to_range():
    w = WORKLOADS["fp64_n16"]
    x, y, ct = make_workload(w)
    A = orc.nudft_matrix(x, y, w.nx, w.ny)
    f = orc.forward(x, y, ct, w.nx, w.ny) + noise_like(orc.forward(x, y, ct, w.nx, w.ny), 1e-3, 17)
    c, res, _ = orc.lstsq(A, f)
    r = f - A @ c
    assert np.linalg.norm(A.conj().T @ r) < 1e-12 * np.linalg.norm(A) * np.linalg.norm(f)
    assert abs(res[0] - np.linalg.norm(r)) < 1e-10 * np.linalg.norm(f)


@pytest.mark.parametrize("m,n", [(9, 5), (5, 9), (7, 7), (1, 3)])
def test_householder_qr(m, n):
    A = complex_normal((m, n), 21 + m * n)
    assert qr_pin_error(orc.householder_qr, A) < 1e-13


def test_householder_qr_zero_column():
    A = complex_normal((6, 4), 3)
    A[:, 1] = 0.0
    assert qr_pin_error(orc.householder_qr, A, compare_lapack=False) < 1e-13
    R, _, _ = orc.householder_qr(A)
    assert R[1, 1] == 0.0


def test_cgls_matches_dense_lstsq():
    x, y = jittered_grid(16, 8, -0.3, 0.3, 31)
    nx, ny = 8, 8
    A = orc.nudft_matrix(x, y, nx, ny)
    f = complex_normal((x.size, 2), 32)
    c1, _, _ = orc.lstsq(A, f)
    c2, it = orc.cgls(x, y, f, nx, ny, tol=1e-14)
    assert np.max(orc.relerr(c2, c1)) < 1e-11


# ---------------------------------------------------------------- transformed kernel matrix
def test_tilde_sylvester_identity():
    n = 12
    x, _ = jittered_grid(30, 1, -0.4, 0.4, 41)
    G = orc.tilde_1d(x, n)
    gam = np.exp(-2j * np.pi * x)
    xi = np.exp(-2j * np.pi * np.arange(n) / n)
    u = gam ** n - 1.0
    v = xi / n
    lhs = gam[:, None] * G - G * xi[None, :]
    assert np.max(np.abs(lhs - np.outer(u, v))) < 1e-13


def test_tilde_cauchy_closed_form_and_unit_rows():
    n = 10
    x, _ = jittered_grid(25, 1, -0.4, 0.4, 43)
    G = orc.tilde_1d(x, n)
    gam = np.exp(-2j * np.pi * x)
    xi = np.exp(-2j * np.pi * np.arange(n) / n)
    closed = ((gam ** n - 1.0)[:, None] * (xi / n)[None, :]) / (gam[:, None] - xi[None, :])
    assert np.max(np.abs(G - closed)) < 1e-12
    assert np.max(np.abs(np.linalg.norm(G, axis=1) - 1.0)) < 1e-13


def test_tilde_unperturbed_square_grid_is_identity():
    n = 16
    x = np.arange(n) / n
    assert np.max(np.abs(orc.tilde_1d(x, n) - np.eye(n))) < 1e-13


def test_tilde_2d_is_face_splitting_product():
    x, y = jittered_grid(10, 8, -0.3, 0.3, 51)
    nx, ny = 5, 4
    Gx = orc.tilde_1d(x, nx)
    Gy = orc.tilde_1d(y, ny)
    fs = (Gx[:, :, None] * Gy[:, None, :]).reshape(x.size, nx * ny)
    assert np.max(np.abs(orc.tilde_2d(x, y, nx, ny) - fs)) < 1e-12


def test_idft2_matches_numpy_ifft2():
    nx, ny = 8, 6
    Y = complex_normal((nx * ny, 2), 61)
    ref = np.stack([np.fft.ifft2(Y[:, q].reshape(nx, ny)).ravel() for q in range(2)], axis=1)
    assert np.max(np.abs(orc.idft2(Y, nx, ny) - ref)) < 1e-14


def test_solution_through_transformed_basis():
    """c = F^{-1} argmin ||G~ y - f|| equals argmin ||A c - f|| (Sec. 4.1 change of basis)."""
    w = WORKLOADS["fp64_n16"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct, w.nx, w.ny)
    Gt = orc.tilde_2d(x, y, w.nx, w.ny)
    yv, _, _ = orc.lstsq(Gt, f)
    assert np.max(orc.relerr(orc.idft2(yv, w.nx, w.ny), ct)) < 1e-12


# ---------------------------------------------------------------- planted mistakes
def test_pin_catches_wrong_exponent_sign():
    def bad_forward(x, y, c, nx, ny):
        return _forward_sign(x, y, c, nx, ny, +1)        # exp(+2 pi i ...) instead of exp(-...)
    assert fft_pin_error(bad_forward, 8, 6) > 1e-3


def _forward_sign(x, y, c, nx, ny, sgn):
    kx = np.repeat(np.arange(nx), ny)
    ky = np.tile(np.arange(ny), nx)
    A = np.exp(sgn * 2j * np.pi * (np.outer(x, kx) + np.outer(y, ky)))
    return A @ c


def test_pin_catches_transposed_column_order():
    def bad_forward(x, y, c, nx, ny):
        kx = np.tile(np.arange(nx), ny)          # kx + ky*nx ordering instead of ky + kx*ny
        ky = np.repeat(np.arange(ny), nx)
        return np.exp(-2j * np.pi * (np.outer(x, kx) + np.outer(y, ky))) @ c
    assert fft_pin_error(bad_forward, 8, 6) > 1e-3


def test_pin_catches_dropped_reflector_factor():
    def bad_qr(A):
        R, vs, taus = orc.householder_qr(A)
        return R, vs, [t / 2 for t in taus]      # plausible slip: tau = 1/||v||^2
    A = complex_normal((7, 4), 5)
    assert qr_pin_error(bad_qr, A) > 1e-3


def test_pin_catches_wrong_dft_normalisation():
    n = 12
    x, _ = jittered_grid(30, 1, -0.4, 0.4, 41)
    G = orc.nudft_1d(x, n) @ orc.dft_matrix(n).conj()      # forgot the 1/n of F^{-1}
    assert np.max(np.abs(np.linalg.norm(G, axis=1) - 1.0)) > 1.0


# ---------------------------------------------------------------------------- gradient oracle
def _grad_case(seed=11, nx=4, ny=3, M=30, s=2):
    rng = np.random.default_rng(seed)
    x, y = rng.random(M), rng.random(M)
    f = rng.standard_normal((M, s)) + 1j * rng.standard_normal((M, s))   # inconsistent: r != 0
    G = rng.standard_normal((nx * ny, s)) + 1j * rng.standard_normal((nx * ny, s))
    return x, y, f, G, nx, ny


def _loss(x, y, f, G, nx, ny):
    """L = Re <G, c> with c = A^+ f: its gradient in the torch convention is G itself."""
    c, _, _ = orc.lstsq(orc.nudft_matrix(x, y, nx, ny), f)
    return float(np.sum(np.real(np.conj(G) * c)))


def test_pinv_adjoint_min_norm():
    """(A^+)^* g solves A^* lam = g and lies in range(A) (the minimum-norm solution)."""
    x, y, _, G, nx, ny = _grad_case()
    A = orc.nudft_matrix(x, y, nx, ny)
    lam = orc.pinv_adjoint(A, G)
    assert np.max(np.abs(A.conj().T @ lam - G)) < 1e-12 * np.max(np.abs(G)) * A.shape[0]
    Q, _ = np.linalg.qr(A)
    assert np.max(np.abs(lam - Q @ (Q.conj().T @ lam))) < 1e-12 * np.max(np.abs(lam))
    # against the textbook pseudo-inverse
    assert np.allclose(lam, np.linalg.pinv(A).conj().T @ G, atol=1e-12 * np.max(np.abs(lam)))


def test_grad_points_finite_differences():
    """dL/dx_j and dL/dy_j of lstsq_grad against central differences of the least-squares map."""
    x, y, f, G, nx, ny = _grad_case()
    _, _, gx, gy = orc.lstsq_grad(x, y, nx, ny, f, G)
    h = 1e-6
    for j in (0, 7, 29):
        for arr, g in ((x, gx), (y, gy)):
            p, m = arr.copy(), arr.copy()
            p[j] += h
            m[j] -= h
            args_p = (p, y) if arr is x else (x, p)
            args_m = (m, y) if arr is x else (x, m)
            fd = (_loss(*args_p, f, G, nx, ny) - _loss(*args_m, f, G, nx, ny)) / (2 * h)
            assert abs(fd - g[j]) < 1e-6 * max(1.0, abs(fd))


def test_grad_f_finite_differences():
    """lam = dL/dRe f + i dL/dIm f: the loss is linear in f, so differences are exact."""
    x, y, f, G, nx, ny = _grad_case(seed=5)
    _, lam, _, _ = orc.lstsq_grad(x, y, nx, ny, f, G)
    h = 1e-3
    for j, q in ((0, 0), (12, 1), (29, 1)):
        for unit, comp in ((1.0, np.real), (1j, np.imag)):
            fp, fm = f.copy(), f.copy()
            fp[j, q] += h * unit
            fm[j, q] -= h * unit
            fd = (_loss(x, y, fp, G, nx, ny) - _loss(x, y, fm, G, nx, ny)) / (2 * h)
            assert abs(fd - comp(lam[j, q])) < 1e-9 * max(1.0, abs(fd))


def test_grad_points_consistent_data_drops_mu_term():
    """With f = A c_true the residual is zero and only the -<lam, (dA) c> term remains."""
    x, y, _, G, nx, ny = _grad_case(seed=3)
    rng = np.random.default_rng(4)
    ct = rng.standard_normal((nx * ny, 2)) + 1j * rng.standard_normal((nx * ny, 2))
    f = orc.nudft_matrix(x, y, nx, ny) @ ct
    c, lam, gx, _ = orc.lstsq_grad(x, y, nx, ny, f, G)
    A = orc.nudft_matrix(x, y, nx, ny)
    kx = np.repeat(np.arange(nx, dtype=np.float64), ny)
    gx_first = np.sum(np.real(-np.conj(lam) * ((A * (-2j * np.pi * kx)[None, :]) @ c)), axis=1)
    assert np.max(np.abs(gx - gx_first)) < 1e-9 * np.max(np.abs(gx))


# ---------------------------------------------------------------- planted mistakes in the gradient
def _grad_x_variant(x, y, nx, ny, f, G, mu_sign=1.0, deriv_sign=-1.0):
    """lstsq_grad's x-gradient with the two signs exposed, to plant plausible slips."""
    A = orc.nudft_matrix(x, y, nx, ny)
    c, _, _ = orc.lstsq(A, f)
    lam = orc.pinv_adjoint(A, G)
    mu, _, _ = orc.lstsq(A, lam)
    r = f - A @ c
    kx = np.repeat(np.arange(nx, dtype=np.float64), ny)
    Ax = A * (deriv_sign * 2j * np.pi * kx)[None, :]
    return np.sum(np.real(-np.conj(lam) * (Ax @ c) + mu_sign * np.conj(Ax @ mu) * r), axis=1)


def _grad_fd_error(gx_fn):
    x, y, f, G, nx, ny = _grad_case()
    gx = gx_fn(x, y, nx, ny, f, G)
    h, worst = 1e-6, 0.0
    for j in (0, 7, 29):
        p, m = x.copy(), x.copy()
        p[j] += h
        m[j] -= h
        fd = (_loss(p, y, f, G, nx, ny) - _loss(m, y, f, G, nx, ny)) / (2 * h)
        worst = max(worst, abs(fd - gx[j]) / max(1.0, abs(fd)))
    return worst


def test_gradient_pin_accepts_the_oracle_and_catches_planted_slips():
    assert _grad_fd_error(lambda *a: orc.lstsq_grad(*a)[2]) < 1e-6
    assert _grad_fd_error(lambda *a: _grad_x_variant(*a)) < 1e-6                     # the variant itself is right
    assert _grad_fd_error(lambda *a: _grad_x_variant(*a, mu_sign=-1.0)) > 1e-3       # residual term sign
    assert _grad_fd_error(lambda *a: _grad_x_variant(*a, mu_sign=0.0)) > 1e-3        # residual term dropped
    assert _grad_fd_error(lambda *a: _grad_x_variant(*a, deriv_sign=1.0)) > 1e-3     # d/dx of exp(+2 pi i ...)


# ---------------------------------------------------------------- matrix-free gradient
def test_normal_cg_matches_dense_normal_equations():
    x, y = jittered_grid(24, 12, -0.3, 0.3, 501)
    nx, ny = 12, 10
    A = orc.nudft_matrix(x, y, nx, ny)
    b = complex_normal((nx * ny, 2), 502)
    z, it = orc.normal_cg(x, y, b, nx, ny, tol=1e-14)
    ref = np.linalg.solve(A.conj().T @ A, b)
    assert np.max(np.linalg.norm(z - ref, axis=0) / np.linalg.norm(ref, axis=0)) < 1e-12
    assert it < 200


def test_matrix_free_gradient_matches_dense_gradient():
    """lstsq_grad_rows (CG, direct applies, sampled rows) against the dense lstsq_grad, which the
    finite-difference and minimum-norm pins above tie to the definition; inconsistent data, so
    both terms of the formula count."""
    w = WORKLOADS["fp64_n16"]
    x, y, _ = make_workload(w)
    f = complex_normal((w.M, 2), 503)
    G = complex_normal((w.N, 2), 504)
    c_d, lam_d, gx_d, gy_d = orc.lstsq_grad(x, y, w.nx, w.ny, f, G)
    rows = np.array([0, 7, 100, 255, 511])
    c_m, lam_m, gx_m, gy_m = orc.lstsq_grad_rows(x, y, w.nx, w.ny, f, G, rows, tol=1e-14)
    assert np.max(np.abs(c_m - c_d)) < 1e-11 * np.max(np.abs(c_d))
    assert np.max(np.abs(lam_m - lam_d)) < 1e-11 * np.max(np.abs(lam_d))
    assert np.max(np.abs(gx_m - gx_d[rows])) < 1e-10 * np.max(np.abs(gx_d))
    assert np.max(np.abs(gy_m - gy_d[rows])) < 1e-10 * np.max(np.abs(gy_d))


def test_relres_and_relerr_closed_forms():
    """The Sec. 5 error measures on cases with known values: for f = A c0, the relative residual
    is 1 at c = 0 and at c = 2 c0 and vanishes at c = c0; the relative error of (1 + t) c_ref is
    |t| per column, and each column is measured on its own."""
    rng = np.random.default_rng(31)
    nx, ny, M = 6, 5, 45
    x, y = rng.random(M), rng.random(M)
    c0 = rng.standard_normal((nx * ny, 2)) + 1j * rng.standard_normal((nx * ny, 2))
    f = orc.forward(x, y, c0, nx, ny)
    assert np.allclose(orc.relres(x, y, np.zeros_like(c0), f, nx, ny), 1.0, rtol=0, atol=1e-14)
    assert np.allclose(orc.relres(x, y, 2 * c0, f, nx, ny), 1.0, rtol=0, atol=1e-13)
    assert np.max(orc.relres(x, y, c0, f, nx, ny)) < 1e-14
    c = c0 * np.array([1.5, 1 - 0.25j])[None, :]
    assert np.allclose(orc.relerr(c, c0), [0.5, 0.25], rtol=0, atol=1e-15)
    assert np.allclose(orc.relerr(c0[:, 0], c0[:, 0]), [0.0])
