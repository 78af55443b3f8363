"""Pins of the fADI + ID oracle (oracle/fadi_oracle.py) against what the mathematics fixes:
the ADI residual identity X - X_J = r(S) X r(D)^{-1}, the resulting 2-norm bound for normal
coefficient matrices, Wachspress's single-shift optimum (the geometric mean), the Zolotarev-number
bound of Beckermann and Townsend for [-gamma, -1] and [1, gamma], the cross-ratio of the Moebius
map, the ID of an exactly low-rank matrix, and the 1D HSS against the dense transformed matrix."""
import numpy as np
import pytest

from oracle import fadi_oracle as fo
from oracle import tilde_1d


def test_psi_is_the_transformed_1d_matrix():
    rng = np.random.default_rng(1)
    n = 24
    x = np.concatenate([rng.random(40), np.arange(n) / n])
    P = fo.psi(x, np.arange(n), n)
    assert np.abs(P - tilde_1d(x, n)).max() < 1e-13
    # grid points: exactly 1 at coincidence, zero (to rounding of sin(pi n t)) elsewhere
    assert np.all(np.diag(P[40:]) == 1.0)
    assert np.abs(P[40:] - np.eye(n)).max() < 1e-14


def test_moebius_map_sends_the_arc_endpoints_to_the_symmetric_intervals():
    for E, F in [((0.0, 0.1), (0.15, 0.9)), ((0.3, 0.32), (0.33, 1.2)), ((0.0, 0.5), (0.51, 0.99))]:
        g, t1, t2, t3, t4 = fo.cayley_params(E, F)
        assert t1 < t2 < t3 < t4
        gam = fo.moebius_gamma(t1, t2, t3, t4)
        assert gam > 1
        got = fo.moebius_inverse(np.array([-gam, -1.0, 1.0, gam]), t2, t3, t4, gam)
        assert np.allclose(got, [t1, t2, t3, t4], rtol=1e-9, atol=1e-12)


def test_single_shift_is_the_geometric_mean():
    # Wachspress: the best single shift for [1, gamma] is sqrt(gamma); dn(K/2, k') = sqrt(k_c)
    for gam in [1.3, 7.0, 250.0, 3e4]:
        assert fo.wachspress_p(gam, 1)[0] == pytest.approx(np.sqrt(gam), rel=1e-12)


@pytest.mark.parametrize("gam", [1.5, 10.0, 100.0, 1e4])
def test_zolotarev_shifts_meet_the_beckermann_townsend_bound(gam):
    """Z_J([-b,-a],[a,b]) <= 4 exp(-pi^2 J / log(4 b/a)); the elliptic-function shifts attain it
    (up to sampling), and moving any one shift makes the ratio worse."""
    rng = np.random.default_rng(2)
    prev = 1.0
    for J in range(1, 17):
        p = fo.wachspress_p(gam, J)
        r = fo.zolotarev_ratio(gam, p)
        assert r <= 4.0 * np.exp(-np.pi**2 * J / np.log(4.0 * gam)) * (1 + 1e-3)
        assert r < prev
        prev = r
        if J in (3, 8):
            for _ in range(4):
                q = p.copy()
                j = rng.integers(J)
                q[j] *= 1.0 + rng.choice([-1, 1]) * 0.05
                assert fo.zolotarev_ratio(gam, q) > r


def test_shifts_lie_on_their_arcs():
    E, F = (0.0, 0.125), (0.14, 0.97)
    xa, xb, gam, p = fo.zolotarev_shifts(E, F, 12)
    assert np.all((xa >= E[0] - 1e-12) & (xa <= E[1] + 1e-12))
    assert np.all((xb >= F[0] - 1e-12) & (xb <= F[1] + 1e-12))


def _node_cauchy(rng, n, d, m):
    x = rng.random(m) * d / n
    kf = np.arange(d + 1, n)
    s, dk = fo._em(x), fo._em(kf / n)
    u, v = fo._em(n * x) - 1.0, dk / n
    X = u[:, None] * v[None, :] / (s[:, None] - dk[None, :])
    return x, kf, s, dk, u, v, X


def test_fadi_residual_is_the_rational_identity():
    rng = np.random.default_rng(3)
    n, d = 64, 8
    x, kf, s, dk, u, v, X = _node_cauchy(rng, n, d, 120)
    assert np.abs(X - tilde_1d(x, n)[:, kf]).max() < 1e-13      # the Cauchy-like form of Sec. 3.1
    E, F = (0.0, d / n), ((d + 1) / n, (n - 1) / n)
    for J in (1, 4, 9):
        xa, xb, _, _ = fo.zolotarev_shifts(E, F, J)
        al, be = fo._em(xa), fo._em(xb)
        Z, Y, g = fo.fadi(s, u, dk, v, al, be)
        res = X - (Z * g) @ Y.T
        ref = fo.rational(s, al, be)[:, None] * X / fo.rational(dk, al, be)[None, :]
        assert np.abs(res - ref).max() <= 1e-12 * np.abs(X).max()


def test_fadi_error_within_the_rational_bound():
    rng = np.random.default_rng(4)
    n, d = 128, 16
    x, kf, s, dk, u, v, X = _node_cauchy(rng, n, d, 300)
    E, F = (0.0, d / n), ((d + 1) / n, (n - 1) / n)
    nx = np.linalg.norm(X, 2)
    for J in (2, 6, 12):
        xa, xb, gam, p = fo.zolotarev_shifts(E, F, J)
        al, be = fo._em(xa), fo._em(xb)
        Z, Y, g = fo.fadi(s, u, dk, v, al, be)
        disc = np.abs(fo.rational(s, al, be)).max() / np.abs(fo.rational(dk, al, be)).min()
        assert disc <= 1.1 * fo.zolotarev_ratio(gam, p)        # the discrete sets sit inside the arcs
        err = np.linalg.norm(X - (Z * g) @ Y.T, 2)
        assert err <= disc * nx * (1 + 1e-8) + 1e-15


def test_row_id_of_an_exactly_low_rank_matrix():
    rng = np.random.default_rng(5)
    A = (rng.standard_normal((60, 5)) + 1j * rng.standard_normal((60, 5))) @ \
        (rng.standard_normal((5, 9)) + 1j * rng.standard_normal((5, 9)))
    S, T = fo.row_id(A, 1e-10)
    assert len(S) == 5 and T.shape == (60, 5)
    assert np.allclose(T[S], np.eye(5), atol=0, rtol=0)
    assert np.abs(A - T @ A[S]).max() < 1e-11 * np.abs(A).max()


def test_row_id_of_the_zero_block():
    S, T = fo.row_id(np.zeros((7, 4), np.complex128), 1e-10)
    assert len(S) == 1 and T.shape == (7, 1)
    assert T[S[0], 0] == 1.0 and np.count_nonzero(T) == 1


def test_row_side_basis_carries_the_blocks_singular_values():
    """B = [near column, Z diag(g) R_Y^T] has the singular values of G~(J, K^c)."""
    rng = np.random.default_rng(6)
    n, d, m = 128, 8, 400
    x = rng.random(m) * d / n + 3 * d / n        # node with c0 = 3d
    c0 = 3 * d
    plan = fo.node_plan(0, d, n, 1e-12)
    B = fo.node_basis(plan, 0, np.arange(m), c0, n, x)
    Kc = np.r_[0:c0, c0 + d:n]
    sx = np.linalg.svd(tilde_1d(x, n)[:, Kc], compute_uv=False)
    sb = np.linalg.svd(B, compute_uv=False)
    k = min(len(sb), 15)
    assert np.abs(sb[:k] - sx[:k]).max() <= 1e-12 * sx[0]


def test_column_side_id_interpolates_the_outside_points():
    rng = np.random.default_rng(7)
    n, d, eps1 = 256, 32, 1e-10
    c0 = 5 * d
    xo = (c0 + d) / n + rng.random(6000) * (1 - d / n)     # outside [c0/n, (c0+d)/n)
    xo = xo % 1.0
    plan = fo.node_plan(1, d, n, eps1)
    assert plan["J"] > 0 and list(plan["ex"]) == [0]
    K = np.arange(c0, c0 + d)
    B = fo.node_basis(plan, 1, K, c0, n)
    S, T = fo.row_id(B, fo.ID_TOL * eps1)
    V = T.conj()
    G = tilde_1d(xo, n)[:, K]
    err = np.linalg.norm(G - G[:, S] @ V.conj().T, 2) / np.linalg.norm(G, 2)
    assert err < 3 * eps1
    sv = np.linalg.svd(G, compute_uv=False)
    assert len(S) <= int(np.sum(sv > eps1 * sv[0])) + 6


@pytest.mark.parametrize("n,L,M,eps1,seed", [(16, 2, 40, 1e-11, 0), (64, 3, 300, 1e-11, 1),
                                             (128, 4, 1000, 1e-7, 2), (256, 5, 2500, 1e-11, 3)])
def test_hss1d_fadi_id_reproduces_the_transformed_matrix(n, L, M, eps1, seed):
    rng = np.random.default_rng(seed)
    x = rng.random(M)
    h = fo.hss1d_fadi_id(x, n, L, eps1)
    G = fo.tilde_1d_sorted(h)
    H = fo.hss1d_dense(h)
    assert np.linalg.norm(H - G, 2) <= 5 * eps1 * np.linalg.norm(G, 2)
    # ranks: no lower than the SVD's numerical rank of each row block at 100 eps1 (nothing can
    # reach eps1 with fewer), and close to the SVD's rank at eps1
    for l in range(1, L + 1):
        for i, (c0, c1) in enumerate(h["tree"][l]):
            r = h["rows"][l][i]
            if len(r) == 0:
                continue
            Kc = np.r_[0:c0, c1:n]
            sv = np.linalg.svd(G[np.ix_(r, Kc)], compute_uv=False)
            k = len(h["Srow"][(l, i)])
            assert k >= int(np.sum(sv > 100 * eps1 * sv[0]))
            assert k <= int(np.sum(sv > eps1 * sv[0])) + 6


def test_hss1d_on_the_uniform_grid_is_the_identity():
    """Points on the grid k/n: G~ = I, every off-diagonal block is zero."""
    n = 64
    x = np.repeat(np.arange(n) / n, 2)
    h = fo.hss1d_fadi_id(x, n, 3, 1e-12)
    H = fo.hss1d_dense(h)
    assert np.abs(H - fo.tilde_1d_sorted(h)).max() < 1e-13


# ---------------------------------------------------------------- planted mistakes
# Each test plants a plausible slip in the oracle (on the CPU) and checks that one of the pins
# above would fail on it.

def _residual_identity_error(fadi_fn):
    rng = np.random.default_rng(3)
    n, d = 64, 8
    x, kf, s, dk, u, v, X = _node_cauchy(rng, n, d, 120)
    xa, xb, _, _ = fo.zolotarev_shifts((0.0, d / n), ((d + 1) / n, (n - 1) / n), 6)
    al, be = fo._em(xa), fo._em(xb)
    Z, Y, g = fadi_fn(s, u, dk, v, al, be)
    ref = fo.rational(s, al, be)[:, None] * X / fo.rational(dk, al, be)[None, :]
    return np.abs(X - (Z * g) @ Y.T - ref).max() / np.abs(X).max()


def test_pin_catches_a_shifted_shift_index_in_fadi():
    def bad_fadi(rn, ru, cn, cv, alpha, beta):
        J = len(alpha)
        Z = np.zeros((len(rn), J), np.complex128)
        Y = np.zeros((len(cn), J), np.complex128)
        z, y = ru / (rn - beta[0]), cv / (cn - alpha[0])
        for i in range(J):
            Z[:, i], Y[:, i] = z, y
            if i + 1 < J:
                z = z * (rn - alpha[i + 1]) / (rn - beta[i + 1])      # slip: alpha_{i+1} for alpha_i
                y = y * (cn - beta[i]) / (cn - alpha[i + 1])
        return Z, Y, beta - alpha
    assert _residual_identity_error(fo.fadi) < 1e-12
    assert _residual_identity_error(bad_fadi) > 1e-6


def test_pin_catches_a_wrong_sign_of_g():
    def bad_fadi(*a):
        Z, Y, g = fo.fadi(*a)
        return Z, Y, -g                                              # slip: alpha - beta
    assert _residual_identity_error(bad_fadi) > 1e-3


def test_pin_catches_the_complementary_modulus_swapped():
    def bad_p(gam, J):
        import mpmath
        with mpmath.workdps(30):
            m = 1 - mpmath.mpf(1) / mpmath.mpf(gam) ** 2
            K = mpmath.ellipk(1 - m)                                 # slip: K(k) for K(k')
            return np.array([float(gam * mpmath.ellipfun("dn", (2 * j - 1) * K / (2 * J), m=m))
                             for j in range(1, J + 1)])
    gam, J = 100.0, 8
    bound = 4.0 * np.exp(-np.pi**2 * J / np.log(4.0 * gam))
    assert fo.zolotarev_ratio(gam, fo.wachspress_p(gam, J)) <= bound * (1 + 1e-3)
    assert fo.zolotarev_ratio(gam, bad_p(gam, J)) > 2 * bound


def _hss_error():
    rng = np.random.default_rng(1)
    x = rng.random(300)
    h = fo.hss1d_fadi_id(x, 64, 3, 1e-11)
    G = fo.tilde_1d_sorted(h)
    return np.linalg.norm(fo.hss1d_dense(h) - G, 2) / np.linalg.norm(G, 2)


def test_pin_catches_a_dropped_near_column(monkeypatch):
    good = fo.node_plan

    def bad_plan(side, d, n, eps1, jmax=64):
        P = good(side, d, n, eps1, jmax)
        if side == 0 and P["J"]:
            P = dict(P)
            P["C"] = P["C"].copy()
            P["C"][0, 0] = 0.0                                       # slip: the touching column left out
        return P
    assert _hss_error() < 5e-11                                      # the reconstruction pin's bound
    monkeypatch.setattr(fo, "node_plan", bad_plan)
    assert _hss_error() > 5e-11


def test_pin_catches_a_column_basis_without_conjugation(monkeypatch):
    good = fo.row_id
    calls = {"n": 0}

    def bad_row_id(B, tol):
        S, T = good(B, tol)
        calls["n"] += 1
        return S, (T.conj() if calls["n"] % 2 == 0 else T)           # slip: V = T_c instead of conj(T_c)
    monkeypatch.setattr(fo, "row_id", bad_row_id)
    assert _hss_error() > 5e-11                                      # fails the reconstruction pin
