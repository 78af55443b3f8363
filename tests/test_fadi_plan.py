"""The host-side fADI plan of the CUDA library (nudft2_fadi_plan: shifts from its own elliptic
functions and Moebius map, the mixing matrix from its own Householder QR) against the oracle's
(scipy's elliptic functions, numpy's QR).  No device work."""
import numpy as np
import pytest

from oracle import fadi_oracle as fo


@pytest.fixture(scope="module")
def plan():
    from paper_2607_00928_b300 import build
    build.build()
    from paper_2607_00928_b300.binding import fadi_plan
    return fadi_plan


@pytest.mark.parametrize("side,d,n,eps1", [(0, 8, 64, 1e-11), (1, 32, 256, 1e-11), (0, 128, 256, 1e-7),
                                           (1, 64, 128, 1e-7), (0, 4, 16, 1e-11), (1, 8, 64, 1e-11),
                                           (0, 16, 512, 1e-15), (1, 256, 512, 1e-15), (0, 7, 50, 1e-9)])
def test_library_plan_matches_the_oracle(plan, side, d, n, eps1):
    got = plan(side, d, n, eps1)
    ref = fo.node_plan(side, d, n, eps1)
    assert got["J"] == ref["J"]
    assert got["ex"] == list(ref["ex"])
    if ref["J"]:
        assert np.abs(np.array(got["xa"]) - ref["xa"]).max() < 1e-11
        assert np.abs(np.array(got["xb"]) - ref["xb"]).max() < 1e-11
        assert got["ratio"] == pytest.approx(ref["ratio"], rel=1e-6)
    C = np.array(got["C"]).T          # columns -> matrix
    # the R factor of a QR is unique up to a unitary diagonal, so compare C C^H
    G1, G2 = C @ C.conj().T, ref["C"] @ ref["C"].conj().T
    assert np.abs(G1 - G2).max() <= 1e-9 * np.abs(G2).max()


def test_library_plan_rejects_bad_nodes(plan):
    from paper_2607_00928_b300.binding import NudftError
    with pytest.raises(NudftError):
        plan(0, 0, 16, 1e-10)
    with pytest.raises(NudftError):
        plan(1, 16, 16, 1e-10)
    with pytest.raises(NudftError):
        plan(2, 4, 16, 1e-10)


def test_library_plan_weights_carry_the_blocks_singular_values(plan):
    """With the library's shifts and mixing matrix, the oracle's basis of a row block has the
    block's singular values (the property the ID's pivot cut relies on)."""
    from oracle import tilde_1d
    n, d, m, c0 = 128, 16, 500, 48
    got = plan(0, d, n, 1e-12)
    P = dict(ex=np.array(got["ex"]), J=got["J"], xa=np.array(got["xa"]), xb=np.array(got["xb"]),
             C=np.array(got["C"]).T)
    x = c0 / n + np.random.default_rng(9).random(m) * d / n
    B = fo.node_basis(P, 0, np.arange(m), c0, n, x)
    Kc = np.r_[0:c0, c0 + d:n]
    sx = np.linalg.svd(tilde_1d(x, n)[:, Kc], compute_uv=False)
    sb = np.linalg.svd(B, compute_uv=False)
    k = min(len(sb), 20)
    assert np.abs(sb[:k] - sx[:k]).max() <= 1e-12 * sx[0]
