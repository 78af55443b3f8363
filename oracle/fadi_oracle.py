"""Factored ADI (fADI) + interpolative decomposition (ID) construction of the 1D HSS
approximation of the transformed 1D NUDFT matrix, plain FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module.  It shares no code with the CUDA path and never consumes
a value computed there.

What the paper fixes (Li & Liu, Sec. 3.1, "A review of the direct inverse method in 1D case"):

* the transformed 1D matrix G~ = A F^{-1} satisfies the Sylvester equation
  S G~ - G~ D = u v^T with S = diag(s_j), s_j = exp(-2 pi i x_j), D = diag(d_k), d_k =
  exp(-2 pi i k / n), u_j = s_j^n - 1, v_k = d_k / n, so G~(j, k) = u_j v_k / (s_j - d_k)
  (the Cauchy-like form, 1 at s_j = d_k);
* its HSS row and column blocks have numerical rank O(log(1/eps) log n_c) (Thm. 3.2 as quoted);
* the 1D HSS is built by fADI (Benner, Li, Truhar 2009) on that Sylvester equation and the ID
  (Cheng, Gimbutas, Martinsson, Rokhlin 2005).  The details of the cited construction are not
  printed; the readings below fill them in.

Readings (the same ones the CUDA path takes):

* fADI with shift pairs (alpha_i, beta_i) leaves the error X - X_J = r(S) X r(D)^{-1}, r(z) =
  prod (z - alpha_i) / (z - beta_i), so ||X - X_J||_2 <= max_E |r| / min_F |r| ||X||_2 for the
  sets E (row nodes) and F (column nodes).  Shifts: Zolotarev-optimal for the two arcs that hold
  E and F, by a Moebius map of the arcs onto [-gamma, -1] and [1, gamma] and Wachspress's
  elliptic-function shifts p_j = gamma dn((2j-1) K(k') / (2J), k'), k' = sqrt(1 - 1/gamma^2).
  J is the least number of shifts with 1.1 x (sampled max ratio) <= eps1 / 100.
* The row block G~(J_a, K_a^c) of a node a with columns [c0, c1) touches the column c1 (mod n)
  (points may sit just below c1/n): that column is kept exactly, the other columns ("far") are
  at least 1/n away from the node's interval and go through fADI.  The column block G~(J_a^c,
  K_a) touches the points just below c0/n: its column c0 is kept as a unit direction, the other
  columns go through fADI against the arc of outside points.  When the fADI set has no more
  columns than J, every column is kept exactly.
* Energy weighting: the ID runs on B = [exact part, Z diag(g) R_Y^T], where Y is the other fADI
  factor on the column set (far columns: exact; outside points: a uniform proxy of 4 samples per
  1/n on the outside arc, the points themselves are data) and R_Y its QR factor, so that B has
  the singular values of the block (up to the fADI error), so the ID's pivot cut measures the
  block's own singular values, as the truncated SVD would.
* ID: row skeleton S and interpolation matrix T (T(S,:) = I) from the column-pivoted QR of B^*,
  rank = number of pivots above (eps1 / 10) |R_00| (at least 1): the residual rows of a pivoted
  QR add up over the rows of a block, and the nested bases add up over the levels, so the pivot
  cut sits a decade below the target (the 1D HSS then reproduces G~ to a few eps1).  Nested bases: a parent's candidates
  are its children's skeleton rows (columns); B, R, W of the 1D HSS are kernel entries at
  skeletons and the parent's interpolation matrices.
"""
from __future__ import annotations

import mpmath
import numpy as np
import scipy.linalg as sla

from .nudft_oracle import tilde_1d

TWO_PI = 2.0 * np.pi
PROXY_PER_COL = 4
FADI_TARGET = 0.01     # fADI error bound target, relative to eps1
ID_TOL = 0.1           # pivot cut of the ID, relative to eps1


def _em(t):
    """exp(-2 pi i t) after reducing t to [-1/2, 1/2)."""
    t = np.asarray(t, np.float64)
    t = t - np.floor(t + 0.5)
    return np.exp(-1j * TWO_PI * t)


def psi(x, k, n):
    """Psi(x, k) = G~(x, k) = (1/n) sum_l exp(-2 pi i (x - k/n) l), 1 at coincidence (Sec. 3.1)."""
    t = np.subtract.outer(np.asarray(x, np.float64), np.asarray(k, np.float64) / n)
    t = t - np.floor(t + 0.5)
    out = np.ones(t.shape, np.complex128)
    nz = t != 0.0
    tt = t[nz]
    out[nz] = np.exp(-1j * np.pi * (n - 1) * tt) * np.sin(np.pi * n * tt) / (n * np.sin(np.pi * tt))
    return out


# ------------------------------------------------------------------------- arcs and shifts
def cayley_params(E, F):
    """Arcs E = [e1, e2], F = [f1, f2] in units of the circle (x -> exp(-2 pi i x)), with
    e1 <= e2 < f1 <= f2 < e1 + 1.  Returns (g, t1, t2, t3, t4): the centre g of the gap from f2
    to e1 + 1 and the endpoints' images under t = tan(theta/2), theta = 2 pi (x - g) + pi."""
    e1, e2 = E
    f1, f2 = F
    g = 0.5 * (f2 + e1 + 1.0)

    def t(x):
        return np.tan(0.5 * (TWO_PI * (x - g) + np.pi))

    return g, t(e1), t(e2), t(f1), t(f2)


def moebius_gamma(t1, t2, t3, t4):
    """gamma > 1 with the same cross-ratio for (-gamma, -1, 1, gamma) as for (t1, t2, t3, t4)."""
    c = (t3 - t1) * (t4 - t2) / ((t3 - t2) * (t4 - t1))
    return 2.0 * c - 1.0 + 2.0 * np.sqrt(c * (c - 1.0))


def moebius_inverse(w, t2, t3, t4, gamma):
    """t with CR(t; t2, t3, t4) = CR(w; -1, 1, gamma), CR(z; a, b, c) = (z-b)(a-c) / ((z-c)(a-b)):
    the Moebius map sending t2, t3, t4 to -1, 1, gamma, inverted."""
    w = np.asarray(w, np.float64)
    a = -2.0 * (w - gamma)                  # CR(w; -1, 1, gamma) = b / a
    b = (w - 1.0) * (-1.0 - gamma)
    return (t3 * (t2 - t4) * a - b * t4 * (t2 - t3)) / ((t2 - t4) * a - b * (t2 - t3))


def wachspress_p(gamma, J):
    """p_j = gamma dn((2j - 1) K(k') / (2J), k'), k'^2 = 1 - 1/gamma^2, j = 1..J.

    K and dn by mpmath at 30 digits: for gamma above ~3e4 the parameter k'^2 is within 1e-9 of
    1, where scipy's ellipj switches to an approximation good to only about 1 - k'^2."""
    with mpmath.workdps(30):
        m1 = mpmath.mpf(1) / mpmath.mpf(gamma) ** 2         # 1 - k'^2
        K = mpmath.ellipk(1 - m1)
        return np.array([float(mpmath.mpf(gamma) * mpmath.ellipfun("dn", (2 * j - 1) * K / (2 * J), m=1 - m1))
                         for j in range(1, J + 1)])


def zolotarev_ratio(gamma, p, samples=4001):
    """(max over y in [1, gamma] of prod |y - p_j| / (y + p_j))^2 by sampling y geometrically:
    max_E |r| / min_F |r| for r with zeros -p_j on [-gamma, -1] and poles p_j on [1, gamma]."""
    y = gamma ** np.linspace(0.0, 1.0, samples)
    v = np.prod(np.abs(y[:, None] - p[None, :]) / (y[:, None] + p[None, :]), axis=1)
    return float(v.max() ** 2)


def zolotarev_shifts(E, F, J):
    """J shift pairs for the arcs E (zeros alpha) and F (poles beta), in units of the circle.
    Returns (xa, xb, gamma, p)."""
    g, t1, t2, t3, t4 = cayley_params(E, F)
    gamma = moebius_gamma(t1, t2, t3, t4)
    p = wachspress_p(gamma, J)

    def back(w):
        t = moebius_inverse(w, t2, t3, t4, gamma)
        return (2.0 * np.arctan(t) - np.pi) / TWO_PI + g

    return back(-p), back(p), gamma, p


def choose_shifts(E, F, eps1, jmax=64):
    """Least J with 1.1 x ratio <= FADI_TARGET eps1 (J <= jmax)."""
    for J in range(1, jmax + 1):
        xa, xb, gamma, p = zolotarev_shifts(E, F, J)
        r = zolotarev_ratio(gamma, p)
        if 1.1 * r <= FADI_TARGET * eps1:
            break
    return J, xa, xb, r


# ------------------------------------------------------------------------- fADI
def fadi(rn, ru, cn, cv, alpha, beta):
    """Factored ADI for the Cauchy-like X(i, l) = ru_i cv_l / (rn_i - cn_l) (Sylvester equation
    diag(rn) X - X diag(cn) = ru cv^T): X_J = Z diag(g) Y^T with
      z_1 = ru / (rn - beta_1),  z_{i+1} = z_i (rn - alpha_i) / (rn - beta_{i+1}),
      y_1 = cv / (cn - alpha_1), y_{i+1} = y_i (cn - beta_i) / (cn - alpha_{i+1}),
      g_i = beta_i - alpha_i,
    so that X - X_J = r(diag rn) X r(diag cn)^{-1}."""
    J = len(alpha)
    Z = np.zeros((len(rn), J), np.complex128)
    Y = np.zeros((len(cn), J), np.complex128)
    z = ru / (rn - beta[0])
    y = cv / (cn - alpha[0])
    for i in range(J):
        Z[:, i] = z
        Y[:, i] = y
        if i + 1 < J:
            z = z * (rn - alpha[i]) / (rn - beta[i + 1])
            y = y * (cn - beta[i]) / (cn - alpha[i + 1])
    return Z, Y, beta - alpha


def rational(z, alpha, beta):
    """r(z) = prod_i (z - alpha_i) / (z - beta_i)."""
    z = np.asarray(z)
    out = np.ones(z.shape, np.complex128)
    for a, b in zip(alpha, beta):
        out = out * (z - a) / (z - b)
    return out


# ------------------------------------------------------------------------- node plan
def node_plan(side, d, n, eps1, jmax=64):
    """Plan of a node of d columns (node frame: first column 0) of a 1D matrix with n columns.

    side 0 (row block G~(J, K^c)): exact columns ``ex`` (offsets), fADI on the far columns.
    side 1 (column block G~(J^c, K)): exact unit columns ``ex``, fADI on K minus column 0.
    Returns dict(ex, J, xa, xb, C, ratio): the basis row of a candidate is a^T C with
    a = [exact part, z_1..z_J] (z from ``fadi`` with the node-frame shifts)."""
    if side == 0:
        nset = n - d - 1                                   # far columns d+1 .. n-1
        E, F = (0.0, d / n), ((d + 1) / n, (n - 1) / n)
    else:
        nset = d - 1                                       # columns 1 .. d-1
        E, F = (1.0 / n, (d - 1) / n), (d / n, 1.0)
    J = 0
    if nset >= 2:
        J, xa, xb, r = choose_shifts(E, F, eps1, jmax)
    if nset < 2 or J >= nset:
        ex = np.arange(d, n) if side == 0 else np.arange(d)
        return dict(ex=ex, J=0, xa=np.zeros(0), xb=np.zeros(0), C=np.eye(len(ex), dtype=np.complex128),
                    ratio=0.0)
    alpha, beta = _em(xa), _em(xb)
    if side == 0:
        kf = np.arange(d + 1, n)
        dk = _em(kf / n)
        _, Y, g = fadi(np.array([0j]), np.array([0j]), dk, dk / n, alpha, beta)
        R = np.linalg.qr(Y, mode="r")
        C = sla.block_diag(np.eye(1), np.diag(g) @ R.T)
        ex = np.array([d])
    else:
        xP = d / n + (np.arange(PROXY_PER_COL * (n - d)) + 0.5) / (PROXY_PER_COL * n)
        sP = _em(xP)
        uP = _em(n * xP) - 1.0
        _, Y, g = fadi(np.array([0j]), np.array([0j]), sP, uP, alpha, beta)
        Yf = np.concatenate([psi(xP, [0], n), Y], axis=1)
        R = np.linalg.qr(Yf, mode="r")
        C = np.diag(np.concatenate([[1.0 + 0j], g])) @ R.T
        ex = np.array([0])
    return dict(ex=ex, J=J, xa=xa, xb=xb, C=C, ratio=r)


def node_basis(plan, side, cand, c0, n, xs=None):
    """B (len(cand) x (ne + J)) of a node with first column c0.  side 0: cand are point indices
    into xs (rows); side 1: cand are column indices."""
    ex, J = plan["ex"], plan["J"]
    ne = len(ex)
    alpha, beta = _em(plan["xa"]), _em(plan["xb"])
    if side == 0:
        x = np.asarray(xs)[cand]
        a_ex = psi(x, (c0 + ex) % n, n)
        if J:
            xr = x - c0 / n
            s = _em(xr)
            Z, _, _ = fadi(s, _em(n * xr) - 1.0, np.array([0j]), np.array([0j]), alpha, beta)
        else:
            Z = np.zeros((len(x), 0))
    else:
        k = np.asarray(cand)
        kr = (k - c0) % n
        a_ex = (kr[:, None] == ex[None, :]).astype(np.complex128)
        if J:
            dk = _em(kr / n)
            Z, _, _ = fadi(dk, -dk / n, np.array([0j]), np.array([0j]), alpha, beta)
            Z[np.isin(kr, ex), :] = 0.0
        else:
            Z = np.zeros((len(k), 0))
    return np.concatenate([a_ex, Z], axis=1) @ plan["C"]


# ------------------------------------------------------------------------- interpolative decomposition
def row_id(B, tol):
    """Row ID of B (m x q) by the column-pivoted Householder QR of B^* (scipy / LAPACK geqp3):
    B^* P = Q R, rank r = the leading pivots with |R_kk| > tol |R_00| (1 for the zero block),
    skeleton S = P[:r], T = P [I; (R11^{-1} R12)^*] so that T(S, :) = I and B ~= T B(S, :)."""
    m = B.shape[0]
    if m == 0:
        return np.zeros(0, int), np.zeros((0, 0), np.complex128)
    W = B.conj().T
    _, R, P = sla.qr(W, mode="economic", pivoting=True)
    dg = np.abs(np.diag(R))
    T = np.zeros((m, 1), np.complex128)
    if dg[0] == 0.0:               # the zero block: T = the unit vector of the first pivot
        T[P[0], 0] = 1.0
        return P[:1].copy(), T
    r = 0                          # the leading pivots above the cut
    while r < dg.size and dg[r] > tol * dg[0]:
        r += 1
    X = sla.solve_triangular(R[:r, :r], R[:r, r:])
    T = np.zeros((m, r), np.complex128)
    T[P[:r], :] = np.eye(r)
    T[P[r:], :] = X.conj().T
    return P[:r].copy(), T


# ------------------------------------------------------------------------- nested 1D HSS
def tree_1d(n, L):
    """Bisection of the column set (the left child takes floor(d/2)): per level, (c0, c1) lists."""
    levels = [[(0, n)]]
    for _ in range(L):
        nxt = []
        for a, b in levels[-1]:
            h = a + (b - a) // 2
            nxt += [(a, h), (h, b)]
        levels.append(nxt)
    return levels


def hss1d_fadi_id(x, n, L, eps1, jmax=64):
    """1D HSS of G~ (rows sorted by x) by fADI + ID.  Returns dict with the sorted order, the
    tree, per-node row ranges, skeletons and generators: U, V (leaves), R, W (nonroot nodes,
    transfer to the parent), B[(l, i)] = G~(skeleton rows of i, skeleton columns of its sibling)."""
    x = np.asarray(x, np.float64)
    order = np.argsort(x, kind="stable")
    xs = x[order]
    tree = tree_1d(n, L)
    bins = np.floor(xs * n).astype(int) % n
    rows = [[np.nonzero((bins >= a) & (bins < b))[0] for a, b in lv] for lv in tree]
    plans = {}

    def plan(side, d):
        if (side, d) not in plans:
            plans[(side, d)] = node_plan(side, d, n, eps1, jmax)
        return plans[(side, d)]

    Srow, Scol, U, V, Rt, Wt = {}, {}, {}, {}, {}, {}
    for l in range(L, 0, -1):
        for i, (c0, c1) in enumerate(tree[l]):
            d = c1 - c0
            if l == L:
                rc, cc = rows[l][i], np.arange(c0, c1)
            else:
                rc = np.concatenate([Srow[(l + 1, 2 * i)], Srow[(l + 1, 2 * i + 1)]])
                cc = np.concatenate([Scol[(l + 1, 2 * i)], Scol[(l + 1, 2 * i + 1)]])
            Br = node_basis(plan(0, d), 0, rc, c0, n, xs)
            Sr, Tr = row_id(Br, ID_TOL * eps1)
            Bc = node_basis(plan(1, d), 1, cc, c0, n)
            Sc, Tc = row_id(Bc, ID_TOL * eps1)
            Srow[(l, i)], Scol[(l, i)] = rc[Sr], cc[Sc]
            if l == L:
                U[(l, i)], V[(l, i)] = Tr, Tc.conj()
            else:
                ra = len(Srow[(l + 1, 2 * i)])
                va = len(Scol[(l + 1, 2 * i)])
                Rt[(l + 1, 2 * i)], Rt[(l + 1, 2 * i + 1)] = Tr[:ra], Tr[ra:]
                Wt[(l + 1, 2 * i)], Wt[(l + 1, 2 * i + 1)] = Tc.conj()[:va], Tc.conj()[va:]
    B = {}
    for l in range(1, L + 1):
        for i in range(len(tree[l])):
            sib = i ^ 1
            B[(l, i)] = psi(xs[Srow[(l, i)]], Scol[(l, sib)], n)
    return dict(order=order, xs=xs, tree=tree, rows=rows, U=U, V=V, R=Rt, W=Wt, B=B, Srow=Srow, Scol=Scol,
                plans=plans, n=n, L=L)


def hss1d_dense(h):
    """Dense M x n matrix (rows in sorted order) of the 1D HSS: exact diagonal leaf blocks, and
    U_a B_ab V_b^* for every sibling pair with the nested bases U_t = diag(U_a, U_b)[R_a; R_b]."""
    xs, tree, rows, n, L = h["xs"], h["tree"], h["rows"], h["n"], h["L"]
    M = len(xs)
    H = np.zeros((M, n), np.complex128)
    Ub, Vb = dict(h["U"]), dict(h["V"])
    for l in range(L - 1, 0, -1):
        for i in range(len(tree[l])):
            a, b = (l + 1, 2 * i), (l + 1, 2 * i + 1)
            Ub[(l, i)] = np.concatenate([Ub[a] @ h["R"][a], Ub[b] @ h["R"][b]], axis=0)
            Vb[(l, i)] = np.concatenate([Vb[a] @ h["W"][a], Vb[b] @ h["W"][b]], axis=0)
    for i, (c0, c1) in enumerate(tree[L]):
        r = rows[L][i]
        H[np.ix_(r, np.arange(c0, c1))] = psi(xs[r], np.arange(c0, c1), n)
    for l in range(1, L + 1):
        for i, (c0, c1) in enumerate(tree[l]):
            sib = i ^ 1
            s0, s1 = tree[l][sib]
            H[np.ix_(rows[l][i], np.arange(s0, s1))] = Ub[(l, i)] @ h["B"][(l, i)] @ Vb[(l, sib)].conj().T
    return H


def tilde_1d_sorted(h):
    """G~ with rows in the HSS's sorted order (reference for hss1d_dense)."""
    return tilde_1d(h["xs"], h["n"])
