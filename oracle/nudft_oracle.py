"""Plain, slow FP64 CPU oracle for the 2D type-II inverse NUDFT.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA path and never
consumes a value computed there.

What it computes, each by its plain definition (Li & Liu, "A superfast direct solver for the
2D type-II inverse NUDFT based on HSS matrices"):

* ``nudft_matrix``  -- the dense matrix A of Eq. (2): A(j,(kx,ky)) = exp(-2 pi i (kx x_j + ky y_j)),
  columns in lexicographic order ky + kx*ny (Sec. 1, after Eq. 2).
* ``forward`` / ``adjoint`` -- the direct O(MN) sums f = A c (Eq. 1 written as its double sum)
  and A^* f.
* ``householder_qr`` / ``lstsq`` -- the least-squares problem min ||A c - f||_2 (Sec. 1) by a
  hand-written complex Householder QR and back substitution.
* ``cgls`` -- the same least-squares solution by CG on the normal equations with the direct
  apply, for sizes where the dense matrix does not fit.
* ``tilde_1d`` -- the transformed 1D matrix A^x (F^x)^{-1} (Sec. 2.4 and Sec. 3.1, Eq. for
  the entries of the transformed 1D NUDFT matrix) as that matrix product.
* ``idft2`` -- the 2D inverse DFT c = F^{-1} y with F = F^x (x) F^y, F(k,l) = exp(-2 pi i k l / n)
  (Sec. 2.4), by its defining sums.
* ``relres`` / ``relerr`` -- r_s and e_s of Sec. 5.
* ``pinv_adjoint`` / ``lstsq_grad`` -- (A^+)^* g and the gradient of a real loss of the
  least-squares solution with respect to f and to the point coordinates (the derivative of
  the normal equations; the paper itself states no gradient).  Pinned by central finite
  differences of ``lstsq`` and by the minimum-norm characterisation of (A^+)^* g.
* ``normal_cg`` / ``lstsq_grad_rows`` -- the same gradient without the dense matrix (CG on the
  normal equations with the direct applies), at sampled point indices, for sizes where A does
  not fit.  Pinned against ``lstsq_grad`` and against a dense solve of the normal equations.

Pins (tests/test_oracle_pins.py) tie every function to something other than itself: the 2D
FFT on an unperturbed grid, A^*A = N I, brute-force normal equations in extended precision,
the Sylvester displacement identity, the Cauchy-like closed form and unit row norms.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def _expm(t: np.ndarray) -> np.ndarray:
    """exp(-2 pi i t) after reducing t to [-1/2, 1/2): the phase is periodic with period 1."""
    t = t - np.floor(t + 0.5)
    return np.exp(-1j * TWO_PI * t)


def nudft_1d(x: np.ndarray, n: int) -> np.ndarray:
    """A^x(j, k) = exp(-2 pi i k x_j), k = 0..n-1 (the 1D type-II NUDFT matrix, Sec. 3.1)."""
    k = np.arange(n, dtype=np.float64)
    return _expm(np.outer(np.asarray(x, np.float64), k))


def nudft_matrix(x: np.ndarray, y: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Dense A of Eq. (2); column (kx, ky) sits at index ky + kx*ny."""
    kx = np.repeat(np.arange(nx, dtype=np.float64), ny)
    ky = np.tile(np.arange(ny, dtype=np.float64), nx)
    # reduce each product separately before adding: both are exact multiples of the phase period
    px = np.outer(x, kx)
    py = np.outer(y, ky)
    return _expm((px - np.floor(px)) + (py - np.floor(py)))


def _as_cube(c: np.ndarray, nx: int, ny: int) -> np.ndarray:
    c = np.asarray(c, dtype=np.complex128)
    if c.ndim == 1:
        c = c[:, None]
    return c.reshape(nx, ny, c.shape[-1])


def forward(x: np.ndarray, y: np.ndarray, c: np.ndarray, nx: int, ny: int, chunk: int = 8192) -> np.ndarray:
    """f_j = sum_kx sum_ky c[kx,ky] exp(-2 pi i (kx x_j + ky y_j)) (Eq. 1), c is (N,) or (N, s).

    The double sum is taken as written: the inner sum over ky for every (j, kx) is a matrix
    product with the y-factor exp(-2 pi i ky y_j), the outer sum over kx runs elementwise.
    """
    squeeze = np.asarray(c).ndim == 1
    C = _as_cube(c, nx, ny)                    # (nx, ny, s)
    M = len(x)
    s = C.shape[2]
    out = np.empty((M, s), dtype=np.complex128)
    for j0 in range(0, M, chunk):
        j1 = min(M, j0 + chunk)
        Ax = nudft_1d(x[j0:j1], nx)            # (m, nx)
        Ay = nudft_1d(y[j0:j1], ny)            # (m, ny)
        for q in range(s):
            inner = Ay @ C[:, :, q].T          # (m, nx): sum over ky
            out[j0:j1, q] = np.sum(Ax * inner, axis=1)
    return out[:, 0] if squeeze else out


def adjoint(x: np.ndarray, y: np.ndarray, f: np.ndarray, nx: int, ny: int, chunk: int = 8192) -> np.ndarray:
    """(A^* f)[kx, ky] = sum_j conj(A(j,(kx,ky))) f_j, returned as (N,) or (N, s)."""
    f = np.asarray(f, dtype=np.complex128)
    squeeze = f.ndim == 1
    F = f[:, None] if squeeze else f
    M, s = F.shape
    out = np.zeros((nx, ny, s), dtype=np.complex128)
    for j0 in range(0, M, chunk):
        j1 = min(M, j0 + chunk)
        Ax = nudft_1d(x[j0:j1], nx)
        Ay = nudft_1d(y[j0:j1], ny)
        for q in range(s):
            out[:, :, q] += Ax.conj().T @ (F[j0:j1, q:q + 1] * Ay.conj())
    out = out.reshape(nx * ny, s)
    return out[:, 0] if squeeze else out


def householder_qr(A: np.ndarray):
    """Complex Householder QR, column by column, no blocking.

    Returns (R, vs, taus): R is the upper-trapezoidal factor; reflector k is
    H_k = I - tau_k v_k v_k^* acting on rows k..m-1, with v_k[0] = 1 and real tau_k, so each
    H_k is Hermitian and unitary and A = H_0 H_1 ... H_{p-1} R, p = min(m, n).
    v_k = x + phase(x_0) ||x|| e_1 (phase(0) = 1), scaled so that v_k[0] = 1.
    """
    R = np.array(A, dtype=np.complex128, copy=True)
    m, n = R.shape
    p = min(m, n)
    vs, taus = [], []
    for k in range(p):
        x = R[k:, k].copy()
        nrm = np.linalg.norm(x)
        a0 = x[0]
        ph = a0 / abs(a0) if a0 != 0 else 1.0 + 0j
        v = x
        v[0] = a0 + ph * nrm
        if nrm == 0.0:
            v = np.zeros_like(x)
            v[0] = 1.0
        else:
            v = v / v[0]
        tau = 2.0 / np.real(np.vdot(v, v))
        # apply H to the trailing block (and to column k itself)
        w = v.conj() @ R[k:, k:]
        R[k:, k:] -= tau * np.outer(v, w)
        R[k + 1:, k] = 0.0
        vs.append(v)
        taus.append(tau)
    return R, vs, taus


def apply_qh(vs, taus, B: np.ndarray) -> np.ndarray:
    """Q^* B = H_{p-1} ... H_0 B for the reflectors of householder_qr."""
    B = np.array(B, dtype=np.complex128, copy=True)
    for k, (v, tau) in enumerate(zip(vs, taus)):
        w = v.conj() @ B[k:]
        B[k:] -= tau * np.outer(v, w)
    return B


def apply_q(vs, taus, B: np.ndarray) -> np.ndarray:
    """Q B = H_0 ... H_{p-1} B."""
    B = np.array(B, dtype=np.complex128, copy=True)
    for k in range(len(vs) - 1, -1, -1):
        v, tau = vs[k], taus[k]
        w = v.conj() @ B[k:]
        B[k:] -= tau * np.outer(v, w)
    return B


def back_substitute(R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Solve the upper-triangular system R c = g (R square), row by row from the bottom."""
    n = R.shape[0]
    c = np.zeros_like(g, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        c[i] = (g[i] - R[i, i + 1:] @ c[i + 1:]) / R[i, i]
    return c


def lstsq(A: np.ndarray, f: np.ndarray):
    """Least-squares solution of min ||A c - f||_2 (Sec. 1) by Householder QR.

    Returns (c, ls_residual_norms, min_abs_rii).  A must have at least as many rows as columns.
    """
    A = np.asarray(A, dtype=np.complex128)
    f = np.asarray(f, dtype=np.complex128)
    squeeze = f.ndim == 1
    F = f[:, None] if squeeze else f
    m, n = A.shape
    if m < n:
        raise ValueError("least squares needs M >= N")
    R, vs, taus = householder_qr(A)
    G = apply_qh(vs, taus, F)
    c = back_substitute(R[:n, :n], G[:n])
    res = np.linalg.norm(G[n:], axis=0)
    rmin = float(np.min(np.abs(np.diag(R[:n, :n]))))
    return (c[:, 0] if squeeze else c), res, rmin


def forward_substitute_h(R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Solve R^* z = g (R square upper triangular, so R^* is lower triangular), row by row from the top."""
    n = R.shape[0]
    Rh = R.conj().T
    z = np.zeros_like(g, dtype=np.complex128)
    for i in range(n):
        z[i] = (g[i] - Rh[i, :i] @ z[:i]) / Rh[i, i]
    return z


def pinv_adjoint(A: np.ndarray, g: np.ndarray) -> np.ndarray:
    """lam = (A^+)^* g for full column rank A (M >= N): with A = Q [R; 0], A^+ = R^{-1} Q_1^*, so
    lam = Q [R^{-*} g; 0].  Equivalently the minimum-norm solution of A^* lam = g."""
    A = np.asarray(A, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    squeeze = g.ndim == 1
    G = g[:, None] if squeeze else g
    m, n = A.shape
    R, vs, taus = householder_qr(A)
    Z = np.zeros((m, G.shape[1]), dtype=np.complex128)
    Z[:n] = forward_substitute_h(R[:n, :n], G)
    lam = apply_q(vs, taus, Z)
    return lam[:, 0] if squeeze else lam


def lstsq_grad(x, y, nx, ny, f, G):
    """Gradient of a real loss L of the least-squares solution c = A(x, y)^+ f (Sec. 1), for the
    incoming gradient G = dL/dRe c + i dL/dIm c (N x s).  Differentiating the normal equations
    A^* A c = A^* f of a full-column-rank A gives
        dc = -A^+ (dA) c + (A^* A)^{-1} (dA)^* r,   r = f - A c,
    so with lam = (A^+)^* G and mu = (A^* A)^{-1} G = A^+ lam,
        dL = Re[ -<lam, (dA) c> + <(dA) mu, r> ],   <u, v> = sum conj(u) v.
    Row j of A depends on (x_j, y_j) only, with d/dx_j A(j, (kx, ky)) = -2 pi i kx A(j, (kx, ky)).
    Returns (c, lam, grad_x, grad_y); lam is also dL/dRe f + i dL/dIm f."""
    A = nudft_matrix(x, y, nx, ny)
    f = np.asarray(f, dtype=np.complex128).reshape(A.shape[0], -1)
    G = np.asarray(G, dtype=np.complex128).reshape(A.shape[1], -1)
    c, _, _ = lstsq(A, f)
    lam = pinv_adjoint(A, G)
    mu, _, _ = lstsq(A, lam)
    r = f - A @ c
    kx = np.repeat(np.arange(nx, dtype=np.float64), ny)
    ky = np.tile(np.arange(ny, dtype=np.float64), nx)
    Ax = A * (-1j * TWO_PI * kx)[None, :]
    Ay = A * (-1j * TWO_PI * ky)[None, :]
    gx = np.sum(np.real(-np.conj(lam) * (Ax @ c) + np.conj(Ax @ mu) * r), axis=1)
    gy = np.sum(np.real(-np.conj(lam) * (Ay @ c) + np.conj(Ay @ mu) * r), axis=1)
    return c, lam, gx, gy


def cgls(x, y, f, nx, ny, tol=1e-13, maxit=500, rtol=None, history=None):
    """CG on the normal equations A^*A c = A^*f with the direct apply (never forms A^*A).

    Stops when ||A^* r|| <= tol * ||A^* f|| (or, when rtol is given, as soon as
    ||r|| <= rtol * ||f||) for every column.  f is (M,) or (M, s); columns are solved together.
    history, if a list, receives max over columns of ||r|| / ||f|| after each iteration (r is the
    recurrence's residual f - A c).
    """
    f = np.asarray(f, dtype=np.complex128)
    squeeze = f.ndim == 1
    F = f[:, None] if squeeze else f
    s = F.shape[1]
    N = nx * ny
    c = np.zeros((N, s), dtype=np.complex128)
    r = F.copy()
    g = adjoint(x, y, r, nx, ny)
    p = g.copy()
    gg = np.sum(np.abs(g) ** 2, axis=0)
    g0 = np.sqrt(gg)
    f0 = np.linalg.norm(F, axis=0)
    it = 0
    for it in range(1, maxit + 1):
        q = forward(x, y, p, nx, ny)
        qq = np.sum(np.abs(q) ** 2, axis=0)
        alpha = np.where(qq > 0, gg / np.where(qq > 0, qq, 1.0), 0.0)
        c += alpha * p
        r -= alpha * q
        rel = float(np.max(np.linalg.norm(r, axis=0) / np.where(f0 > 0, f0, 1.0)))
        if history is not None:
            history.append(rel)
        if rtol is not None and rel <= rtol:
            break
        g = adjoint(x, y, r, nx, ny)
        gg_new = np.sum(np.abs(g) ** 2, axis=0)
        if np.all(np.sqrt(gg_new) <= tol * g0):
            gg = gg_new
            break
        beta = gg_new / np.where(gg > 0, gg, 1.0)
        p = g + beta * p
        gg = gg_new
    return (c[:, 0] if squeeze else c), it


def normal_cg(x, y, b, nx, ny, tol=1e-13, maxit=500):
    """Solve the normal equations (A^* A) z = b by conjugate gradients with the direct applies
    (A^* A is Hermitian positive definite for full-column-rank A and is never formed).

    Stops when ||b - A^* A z|| <= tol * ||b|| per column.  b is (N,) or (N, s).  Returns (z, its)."""
    b = np.asarray(b, dtype=np.complex128)
    squeeze = b.ndim == 1
    B = b[:, None] if squeeze else b
    z = np.zeros_like(B)
    r = B.copy()
    p = r.copy()
    rr = np.sum(np.abs(r) ** 2, axis=0)
    b0 = np.sqrt(rr)
    it = 0
    for it in range(1, maxit + 1):
        q = adjoint(x, y, forward(x, y, p, nx, ny), nx, ny)
        pq = np.real(np.sum(np.conj(p) * q, axis=0))
        alpha = np.where(pq > 0, rr / np.where(pq > 0, pq, 1.0), 0.0)
        z += alpha * p
        r -= alpha * q
        rr_new = np.sum(np.abs(r) ** 2, axis=0)
        if np.all(np.sqrt(rr_new) <= tol * b0):
            break
        p = r + (rr_new / np.where(rr > 0, rr, 1.0)) * p
        rr = rr_new
    return (z[:, 0] if squeeze else z), it


def lstsq_grad_rows(x, y, nx, ny, f, G, rows, c=None, tol=1e-13):
    """The gradient of lstsq_grad without the dense matrix, at the point indices `rows`.

    c = A^+ f by cgls (unless given), mu = (A^* A)^{-1} G by normal_cg, lam = A mu (so that
    lam = (A^+)^* G, the minimum-norm solution of A^* lam = G), r = f - A c, and
        dL/dx_j = sum_q Re[ -conj(lam_jq) (A_x c)_jq + conj((A_x mu)_jq) r_jq ]
    with (A_x)_jk = -2 pi i kx A_jk, evaluated only at the rows j in `rows` (row j of each product
    needs only the point (x_j, y_j)).  Returns (c, lam, gx[rows], gy[rows]); lam has every row."""
    f = np.asarray(f, dtype=np.complex128).reshape(len(x), -1)
    G = np.asarray(G, dtype=np.complex128).reshape(nx * ny, -1)
    if c is None:
        c, _ = cgls(x, y, f, nx, ny, tol=tol)
    c = np.asarray(c, dtype=np.complex128).reshape(nx * ny, -1)
    mu, _ = normal_cg(x, y, G, nx, ny, tol=tol)
    lam = forward(x, y, mu, nx, ny)
    xr, yr = x[rows], y[rows]
    kx = np.repeat(np.arange(nx, dtype=np.float64), ny)[:, None]
    ky = np.tile(np.arange(ny, dtype=np.float64), nx)[:, None]
    r = f[rows] - forward(xr, yr, c, nx, ny)
    gx = np.sum(np.real(-np.conj(lam[rows]) * forward(xr, yr, -1j * TWO_PI * kx * c, nx, ny)
                        + np.conj(forward(xr, yr, -1j * TWO_PI * kx * mu, nx, ny)) * r), axis=1)
    gy = np.sum(np.real(-np.conj(lam[rows]) * forward(xr, yr, -1j * TWO_PI * ky * c, nx, ny)
                        + np.conj(forward(xr, yr, -1j * TWO_PI * ky * mu, nx, ny)) * r), axis=1)
    return c, lam, gx, gy


def dft_matrix(n: int) -> np.ndarray:
    """F(k, l) = exp(-2 pi i k l / n) (Sec. 2.4)."""
    k = np.arange(n, dtype=np.float64)
    return _expm(np.outer(k, k) / n)


def tilde_1d(x: np.ndarray, n: int) -> np.ndarray:
    """Transformed 1D matrix A^x F^{-1} (Sec. 2.4): its entries are the kernel Psi(gamma_j, xi_k).

    F^{-1} = conj(F)/n; the product is taken as that matrix product.
    """
    return nudft_1d(x, n) @ (dft_matrix(n).conj() / n)


def tilde_2d(x, y, nx, ny) -> np.ndarray:
    """Transformed 2D matrix A F^{-1}, F = F^x (x) F^y (Sec. 3.1), as a dense product."""
    Finv = np.kron(dft_matrix(nx).conj() / nx, dft_matrix(ny).conj() / ny)
    return nudft_matrix(x, y, nx, ny) @ Finv


def idft2(Y: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """c = F^{-1} y for F = F^x (x) F^y, y in lexicographic (kx*ny + ky) order, (N,) or (N, s)."""
    Y = np.asarray(Y, dtype=np.complex128)
    squeeze = Y.ndim == 1
    Yc = _as_cube(Y, nx, ny)
    Fx = dft_matrix(nx).conj() / nx
    Fy = dft_matrix(ny).conj() / ny
    out = np.einsum("ak,klq,bl->abq", Fx, Yc, Fy).reshape(nx * ny, -1)
    return out[:, 0] if squeeze else out


def relres(x, y, c, f, nx, ny) -> np.ndarray:
    """r_s = ||A c - f|| / ||f|| per column (Sec. 5)."""
    r = forward(x, y, c, nx, ny) - f
    return np.linalg.norm(np.atleast_2d(r.T).T, axis=0) / np.linalg.norm(np.atleast_2d(np.asarray(f).T).T, axis=0)


def relerr(c, c_ref) -> np.ndarray:
    """e_s = ||c - c_ref|| / ||c_ref|| per column (Sec. 5)."""
    c = np.atleast_2d(np.asarray(c).T).T
    c_ref = np.atleast_2d(np.asarray(c_ref).T).T
    return np.linalg.norm(c - c_ref, axis=0) / np.linalg.norm(c_ref, axis=0)
