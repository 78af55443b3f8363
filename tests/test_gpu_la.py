"""GPU unit tests of the batched dense kernels behind the HSS stages, against numpy/LAPACK.

* Householder QR (single-CTA panels and cluster-cooperative panels for tall matrices):
  Q R = A, Q^* Q = I, |R_ii| equal to LAPACK's.
* Truncated SVD (pivoted QR -- pivots chosen blockwise on random sketches, or one per step --
  + one-sided Jacobi: blocked Gram steps, scalar rotations in global memory, and
  cluster-resident scalar rotations):
  singular values equal LAPACK's, P^* P = I, and the discarded part of C is below the
  threshold -- the truncation rule of the recompression (Sec. 2.2).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def make_matrix(r, w, kind, seed):
    p = min(r, w)
    U, _ = np.linalg.qr(_rand((r, p), seed))
    V, _ = np.linalg.qr(_rand((w, p), seed + 1))
    if kind == "graded":
        s = np.logspace(0, -14, p)
    elif kind == "repeated":                         # Kronecker-like clusters of equal values
        s = np.repeat(np.logspace(0, -8, max(1, p // 8)), 8)[:p]
        s = np.concatenate([s, np.full(p - s.size, s[-1])]) if s.size < p else s
    elif kind == "wide":                             # 1e0..1e-11, a gap, then a noise floor 1e-16..1e-20
        q = (p * 5) // 6
        s = np.concatenate([np.logspace(0.2, -11, q), np.logspace(-16, -20, p - q)])
    else:                                            # numerically rank deficient: half the spectrum zero
        s = np.concatenate([np.logspace(0, -6, p // 2), np.zeros(p - p // 2)])
    return (U * s) @ V.conj().T


CASES = [(64, 200, "graded"), (300, 120, "graded"), (520, 1500, "graded"), (1577, 3000, "graded"),
         (400, 400, "repeated"), (256, 512, "rankdef"), (1024, 3000, "wide"), (300, 900, "wide")]


@pytest.mark.parametrize("jacobi", ["auto", "block", "scalar", "cluster"])
@pytest.mark.parametrize("r,w,kind", CASES)
def test_tsvd_fp64(nh, monkeypatch, jacobi, r, w, kind):
    if jacobi != "auto":
        monkeypatch.setenv("NH_JACOBI_MODE", jacobi)
    C = make_matrix(r, w, kind, r + w)
    eps = 1e-10
    P, sig = nh.la_tsvd(torch.from_numpy(C).cuda(), eps)
    P = P.cpu().numpy()
    s_ref = np.linalg.svd(C, compute_uv=False)
    k = P.shape[1]
    assert abs(k - int(np.sum(s_ref > eps * s_ref[0]))) <= 1
    assert np.max(np.abs(np.array(sig[:k]) - s_ref[:k])) < 1e-12 * s_ref[0]
    assert np.max(np.abs(P.conj().T @ P - np.eye(k))) < 1e-12
    resid = C - P @ (P.conj().T @ C)
    assert np.linalg.norm(resid, 2) <= 2 * eps * s_ref[0] + 1e-13 * s_ref[0]


@pytest.mark.parametrize("r,w,kind", CASES)
def test_tsvd_fp64_classical_pivoting(nh, monkeypatch, r, w, kind):
    """The truncated SVD with the one-pivot-per-step pivoted QR (NH_QRCP=exact) in place of the
    sketch-pivoted blocks: the same singular values, truncation rank and subspace bound."""
    monkeypatch.setenv("NH_QRCP", "exact")
    C = make_matrix(r, w, kind, r + w)
    eps = 1e-10
    P, sig = nh.la_tsvd(torch.from_numpy(C).cuda(), eps)
    P = P.cpu().numpy()
    s_ref = np.linalg.svd(C, compute_uv=False)
    k = P.shape[1]
    assert abs(k - int(np.sum(s_ref > eps * s_ref[0]))) <= 1
    assert np.max(np.abs(np.array(sig[:k]) - s_ref[:k])) < 1e-12 * s_ref[0]
    assert np.max(np.abs(P.conj().T @ P - np.eye(k))) < 1e-12
    assert np.linalg.norm(C - P @ (P.conj().T @ C), 2) <= 2 * eps * s_ref[0] + 1e-13 * s_ref[0]


@pytest.mark.parametrize("jacobi", ["block", "block_cuda_cores", "scalar"])
@pytest.mark.parametrize("r,w", [(300, 120), (1577, 3000), (2600, 2100)])
def test_tsvd_fp32(nh, monkeypatch, jacobi, r, w):
    """FP32 truncated SVD.  "block": the blocked Jacobi step with its Gram and update products on
    the tensor cores (the default); "block_cuda_cores": the same step on CUDA cores."""
    if jacobi == "block_cuda_cores":
        monkeypatch.setenv("NH_GEMM_TC", "0")
        jacobi = "block"
    monkeypatch.setenv("NH_JACOBI_MODE", jacobi)
    C = make_matrix(r, w, "graded", 5).astype(np.complex64)
    eps = 1e-5
    P, sig = nh.la_tsvd(torch.from_numpy(C).cuda(), eps)
    P = P.cpu().numpy().astype(np.complex128)
    C64 = C.astype(np.complex128)
    s_ref = np.linalg.svd(C64, compute_uv=False)
    k = P.shape[1]
    assert abs(k - int(np.sum(s_ref > eps * s_ref[0]))) <= 2
    # FP32 pivoted QR + Jacobi: every column takes part in ~1e4 rotations or block updates, each
    # rounding at u * sigma_1; 5e-5 * sigma_1 was observed with both sweep kinds
    assert np.max(np.abs(np.array(sig[:k]) - s_ref[:k])) < 2e-4 * s_ref[0]
    # the sweeps stop once every column cosine is below 4 u sqrt(r) (about 1e-5 here), so P is
    # orthonormal to that level; the subspace it spans is checked through an orthonormal basis
    u32 = 2.0 ** -24
    assert np.max(np.abs(P.conj().T @ P - np.eye(k))) < 2 * 4 * u32 * np.sqrt(r)
    Qo, _ = np.linalg.qr(P)
    resid = C64 - Qo @ (Qo.conj().T @ C64)
    assert np.linalg.norm(resid, 2) <= 2 * eps * s_ref[0]


@pytest.mark.parametrize("m,n,grouped", [(100, 60, False), (40, 100, False), (2000, 300, False), (5000, 100, False),
                                         (9000, 40, False), (2000, 600, True), (700, 700, True), (300, 1000, True)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_qr(nh, m, n, grouped, dtype):
    A = _rand((m, n), m + n)
    dt = torch.complex128 if dtype == "fp64" else torch.complex64
    tol = 1e-12 if dtype == "fp64" else 2e-5
    Q, R = nh.la_qr(torch.from_numpy(A).to(dt).cuda(), grouped=grouped)
    Q = Q.cpu().numpy().astype(np.complex128)
    R = R.cpu().numpy().astype(np.complex128)
    A64 = A.astype(dt == torch.complex128 and np.complex128 or np.complex64).astype(np.complex128)
    assert np.max(np.abs(Q @ R - A64)) < tol * np.max(np.abs(A64)) * 10
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(m))) < tol * 10
    p = min(m, n)
    Rl = np.linalg.qr(A64, mode="r")
    assert np.max(np.abs(np.abs(np.diag(R[:p, :p])) - np.abs(np.diag(Rl[:p, :p])))) < tol * 10 * np.max(np.abs(A64)) * np.sqrt(m)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (37, 53, 29), (128, 128, 128), (300, 257, 1000), (1100, 900, 64),
                                   (40, 33, 3000), (515, 700, 0)])
@pytest.mark.parametrize("ops", ["NN", "CN", "NC", "TT"])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_gemm(nh, m, n, k, ops, dtype):
    """Batched GEMM (3 problems, alpha = -1.5, beta = 0.5) against complex128 matmul."""
    dt = torch.complex128 if dtype == "fp64" else torch.complex64
    opa, opb = ops
    sa = (m, k) if opa == "N" else (k, m)
    sb = (k, n) if opb == "N" else (n, k)
    A = torch.from_numpy(_rand((3,) + sa, m + 7 * n + k)).to(dt)
    B = torch.from_numpy(_rand((3,) + sb, m + n + 11 * k)).to(dt)
    C = torch.from_numpy(_rand((3, m, n), 3 * m + n)).to(dt)

    def op(X, o):
        X = X.to(torch.complex128)
        return X if o == "N" else (X.transpose(1, 2) if o == "T" else X.transpose(1, 2).conj())

    ref = -1.5 * (op(A, opa) @ op(B, opb)) + 0.5 * C.to(torch.complex128)
    out = nh.la_gemm(A.cuda(), B.cuda(), opa, opb, alpha=-1.5, beta=0.5, C=C.cuda()).cpu().to(torch.complex128)
    u = 2.0 ** -53 if dtype == "fp64" else 2.0 ** -24
    scale = 1.5 * torch.sqrt(torch.tensor(float(max(k, 1)))) * 4 + 1
    err = (out - ref).abs().max().item()
    assert err < 20 * u * float(scale) * max(1.0, float(ref.abs().max()))


@pytest.mark.skipif(os.environ.get("NH_GEMM_TC") == "0", reason="tensor-core GEMM path turned off (NH_GEMM_TC=0)")
@pytest.mark.parametrize("m,n,k,batch", [(2048, 2048, 300, 2), (1030, 2100, 517, 4), (4100, 700, 64, 2),
                                         (4096, 300, 100, 10), (2050, 260, 5, 12)])
@pytest.mark.parametrize("ops", ["NN", "CN", "NC", "TT"])
def test_gemm_tensor_cores_3xtf32(nh, m, n, k, batch, ops):
    """The tcgen05 3xTF32 complex GEMM (batches of large FP32 products: m, n >= 128 with k >= 256 or
    min(m, n) >= 256) against complex128 matmul: FP32-level accuracy, ragged tile edges, k not a
    multiple of 8 and a single k block, all layout classes."""
    opa, opb = ops
    sa = (m, k) if opa == "N" else (k, m)
    sb = (k, n) if opb == "N" else (n, k)
    A = torch.from_numpy(_rand((batch,) + sa, m + k)).to(torch.complex64)
    B = torch.from_numpy(_rand((batch,) + sb, n + k)).to(torch.complex64)
    C = torch.from_numpy(_rand((batch, m, n), m * n % 97)).to(torch.complex64)

    def op(X, o):
        X = X.to(torch.complex128)
        return X if o == "N" else (X.transpose(1, 2) if o == "T" else X.transpose(1, 2).conj())

    ref = -1.5 * (op(A, opa) @ op(B, opb)) + 0.5 * C.to(torch.complex128)
    out = nh.la_gemm(A.cuda(), B.cuda(), opa, opb, alpha=-1.5, beta=0.5, C=C.cuda()).cpu().to(torch.complex128)
    err = (out - ref).abs().max().item()
    assert err < 20 * 2.0 ** -24 * (1.5 * 4 * np.sqrt(k) + 1) * max(1.0, float(ref.abs().max()))


def test_gemm_autotuner_measures_shape_classes(nh):
    """A mixed-precision build runs its FP32 products through the autotuner: shape classes get
    measured (kernel choice cached per class), and the refined solve still meets the 1e-8 target."""
    import oracle as orc
    from synthetic import WORKLOADS, make_workload
    w = WORKLOADS["mixed_n64"]
    x, y, ct = make_workload(w)
    f = orc.forward(x, y, ct[:, :2], w.nx, w.ny)
    h = nh.NudftHSS(torch.from_numpy(x), torch.from_numpy(y), w.nx, w.ny, eps=1e-6, levels=w.levels, prec="mixed",
                    refine_tol=1e-10, refine_max=10).factor()
    c = h.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    info = h.info()
    h.close()
    assert info["gemm_tuned"] > 0
    assert np.max(np.linalg.norm(c - ct[:, :2], axis=0) / np.linalg.norm(ct[:, :2], axis=0)) < 1e-8


@pytest.mark.parametrize("m,n,s,grouped", [(100, 60, 1, False), (40, 100, 3, False), (2000, 300, 16, False),
                                           (2000, 300, 16, True), (5000, 100, 5, False), (9000, 40, 16, False),
                                           (700, 700, 20, True), (3000, 600, 8, True), (300, 1000, 16, True),
                                           (1537, 517, 2, True)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_qr_apply_streaming(nh, m, n, s, grouped, dtype):
    """The streaming reflector kernels of the solve sweeps (partial V^* C over row slabs, the
    compact-WY T product, the row update), against the explicit Q of the same reflectors:
    Q^* A = R (zero below the diagonal), Q^* C and Q C equal Q_explicit^* C and Q_explicit C, and
    Q (Q^* C) = C.  Covers one and several slabs per block, partial last blocks, panel (32) and
    merged (256) blocks, k < n, and right-hand-side counts that take 1, 4, 8 and 16-wide passes
    and a ragged 16 + 4 split."""
    dt = torch.complex128 if dtype == "fp64" else torch.complex64
    tol = 1e-12 if dtype == "fp64" else 2e-5
    A = torch.from_numpy(_rand((m, n), 3 * m + n)).to(dt)
    C = torch.from_numpy(_rand((m, s), m + 5 * s)).to(dt)
    Qe, R = nh.la_qr(A.cuda(), grouped=grouped)
    Qe = Qe.cpu().numpy().astype(np.complex128)
    R = R.cpu().numpy().astype(np.complex128)
    QhA, R2 = nh.la_qr_apply(A.cuda(), A.cuda(), conj=True, grouped=grouped)
    QhA = QhA.cpu().numpy().astype(np.complex128)
    scale = float(np.max(np.abs(A.numpy())))
    assert np.max(np.abs(QhA - R)) < tol * 10 * scale * np.sqrt(m)
    assert np.max(np.abs(R2.cpu().numpy() - R)) < tol * scale   # the same factorization both times
    C64 = C.numpy().astype(np.complex128)
    QhC, _ = nh.la_qr_apply(A.cuda(), C.cuda(), conj=True, grouped=grouped)
    QC, _ = nh.la_qr_apply(A.cuda(), C.cuda(), conj=False, grouped=grouped)
    QhC = QhC.cpu().numpy().astype(np.complex128)
    QC = QC.cpu().numpy().astype(np.complex128)
    cs = float(np.max(np.abs(C64)))
    assert np.max(np.abs(QhC - Qe.conj().T @ C64)) < tol * 10 * cs * np.sqrt(m)
    assert np.max(np.abs(QC - Qe @ C64)) < tol * 10 * cs * np.sqrt(m)
    back, _ = nh.la_qr_apply(A.cuda(), torch.from_numpy(QhC).to(dt).cuda(), conj=False, grouped=grouped)
    assert np.max(np.abs(back.cpu().numpy().astype(np.complex128) - C64)) < tol * 10 * cs * np.sqrt(m)
