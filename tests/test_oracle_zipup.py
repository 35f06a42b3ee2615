"""Pins of the zip-up oracle (Sec. 2.2, Alg. 2 and its right-to-left mirror)."""
import numpy as np
import pytest

from oracle.mpo import mpo_diff_norm, mpo_norm, naive_product, to_dense
from oracle.zipup import compress, project_bonds, zipup_left_to_right, zipup_right_to_left
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo


def _reverse(X):
    """The same operator on the site-reversed chain: sites in reverse order, bonds swapped."""
    return [np.ascontiguousarray(x.transpose(3, 1, 2, 0)) for x in X[::-1]]


@pytest.mark.parametrize("zip_fn", [zipup_left_to_right, zipup_right_to_left])
def test_zipup_without_truncation_is_the_exact_product(zip_fn):
    A = gaussian_mpo(6, 2, 3, 1, 0, 0.6)
    B = gaussian_mpo(6, 2, 2, 1, 1, 0.6)
    C = zip_fn(A, B, chi_max=64)
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(C) - D) <= 1e-12 * np.linalg.norm(D)
    # a one-pass zip-up bounds a bond by the sites it has contracted: min(chi_A chi_B, 4^l) from the
    # left, min(chi_A chi_B, 4^(L-l)) from the right
    want = [4, 6, 6, 6, 6] if zip_fn is zipup_left_to_right else [6, 6, 6, 6, 4]
    assert [c.shape[3] for c in C[:-1]] == want


def test_zipup_mirror_equals_left_to_right_on_the_reversed_chain():
    A = kron_sum_mpo(7, 5, 3, 0)
    B = kron_sum_mpo(7, 5, 3, 1)
    for update in ("svd", "rsvd"):
        Crl = zipup_right_to_left(A, B, chi_max=6, update=update, oversample=3, seed=4)
        Clr = zipup_left_to_right(_reverse(A), _reverse(B), chi_max=6, update=update, oversample=3, seed=4)
        if update == "svd":   # the sketches are drawn per site index, so only the exact SVD mirrors
            assert mpo_diff_norm(_reverse(Clr), Crl) <= 1e-11 * mpo_norm(Crl)
        assert [c.shape[3] for c in Crl[:-1]] == [min(6, 4 ** (6 - l)) for l in range(6)]


def test_zipup_right_to_left_leaves_c_right_canonical():
    A = kron_sum_mpo(7, 5, 2, 0)
    B = kron_sum_mpo(7, 5, 2, 1)
    C = zipup_right_to_left(A, B, chi_max=6)
    for c in C[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(c.shape[0]), atol=1e-12)


def test_zipup_rsvd_with_a_sketch_covering_the_rank_is_exact_svd():
    A = kron_sum_mpo(6, 4, 5, 0)
    B = kron_sum_mpo(6, 4, 5, 1)
    C1 = zipup_right_to_left(A, B, chi_max=6, update="svd")
    C2 = zipup_right_to_left(A, B, chi_max=6, update="rsvd", oversample=40, seed=1)
    assert mpo_diff_norm(C1, C2) <= 1e-11 * mpo_norm(C1)


def test_zipup_residual_bounded_below_by_the_optimal_truncation():
    """L = 2: one bond, so the best rank-k operator is the truncated SVD of the dense
    product across it (Eckart-Young); a zip-up to the same bond cannot beat it, and
    with k at the full rank both are exact."""
    A = gaussian_mpo(2, 2, 3, 7, 0, 0.6)
    B = gaussian_mpo(2, 2, 3, 7, 1, 0.6)
    D = (to_dense(A) @ to_dense(B)).reshape(2, 2, 2, 2)          # (x1, x2, y1, y2)
    M = D.transpose(0, 2, 1, 3).reshape(4, 4)                   # (x1 y1) x (x2 y2)
    s = np.linalg.svd(M, compute_uv=False)
    N = naive_product(A, B)
    for k in (1, 2, 3, 4):
        C = zipup_right_to_left(A, B, chi_max=k)
        res = mpo_diff_norm(N, C)
        opt = np.sqrt(np.sum(s[k:] ** 2))
        assert res >= opt * (1 - 1e-12) - 1e-14
        if k == 4:
            assert res <= 1e-12 * np.linalg.norm(M)


def test_compress_without_truncation_is_exact_and_right_canonical():
    X = naive_product(kron_sum_mpo(6, 3, 2, 0), kron_sum_mpo(6, 3, 2, 1))
    C = compress(X, chi_max=64)
    D = to_dense(X)
    assert np.linalg.norm(to_dense(C) - D) <= 1e-12 * np.linalg.norm(D)
    for c in C[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(c.shape[0]), atol=1e-12)
    # the exact ranks of a sum of 9 Kronecker products, bounded by 4^l at the ends
    assert [c.shape[3] for c in C[:-1]] == [4, 9, 9, 9, 4]


def test_compress_of_two_sites_is_the_eckart_young_truncation():
    """L = 2: compress keeps the best rank-k operator across the bond exactly."""
    X = gaussian_mpo(2, 2, 4, 3, 0, 0.5)
    D = to_dense(X).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    U, s, Vt = np.linalg.svd(D)
    for k in (1, 2, 3):
        C = compress(X, chi_max=k)
        E = to_dense(C).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
        assert np.linalg.norm(E - (U[:, :k] * s[:k]) @ Vt[:k]) <= 1e-12 * s[0]


def test_compress_error_is_the_sum_of_the_discarded_weights():
    """Right to left with a left-orthonormal remainder of the chain and right-orthonormal
    kept cores, the pieces each step discards are mutually orthogonal, so
    ||X - compress(X)||^2 = sum over the steps of the discarded weight squared."""
    X = naive_product(kron_sum_mpo(7, 4, 6, 0), kron_sum_mpo(7, 4, 6, 1))
    for chi in (3, 6, 10):
        C, disc = compress(X, chi_max=chi, return_discarded=True)
        err = mpo_diff_norm(X, C)
        want = np.sqrt(np.sum(np.square(disc)))
        assert want > 0
        assert abs(err - want) <= 1e-9 * mpo_norm(X) + 1e-9 * want


def test_fit_from_the_zipup_guess():
    """Sec. 2.3.5: with chi_max above the rank the zip-up guess is already the exact
    product, so the first sweep keeps all of ||AB||^2; with truncation the fit from the
    zip-up guess reaches the optimum the random guess reaches."""
    from oracle.fit import FitOracle
    A = kron_sum_mpo(6, 3, 8, 0)
    B = kron_sum_mpo(6, 3, 8, 1)
    f = FitOracle(A, B, 9, 0.0, init="zipup", conv_tol=0.0)
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(f.result()) - D) <= 1e-12 * np.linalg.norm(D)
    f.sweep(1)
    assert abs(f.st.history[-1].norm2 - np.sum(D ** 2)) <= 1e-12 * np.sum(D ** 2)
    # generic (Gaussian) cores: both guesses lead to the same optimum. (On sums of Kronecker
    # products with degenerate weights the zip-up guess can start the fit next to a worse
    # stationary point, which it leaves only slowly: a property of the guess, not checked here.)
    A = gaussian_mpo(10, 2, 4, 3, 0)
    B = gaussian_mpo(10, 2, 4, 3, 1)
    n2 = []
    for init in ("zipup", "random"):
        f = FitOracle(A, B, 8, 0.0, init=init, update="svd", conv_tol=0.0)
        f.sweep(10, stop_on_converge=False)
        n2.append(f.st.history[-1].norm2)
    assert abs(n2[0] - n2[1]) <= 1e-8 * n2[1]


def _pad_bonds(X, width, seed):
    """The same operator with every inner bond widened to `width` by random isometries
    (bond rank unchanged)."""
    rng = np.random.default_rng(seed)
    X = [x.copy() for x in X]
    for l in range(len(X) - 1):
        r = X[l].shape[3]
        V, _ = np.linalg.qr(rng.standard_normal((width, r)))      # width x r, orthonormal columns
        X[l] = np.einsum("asty,zy->astz", X[l], V)
        X[l + 1] = np.einsum("zy,yuvb->zuvb", V, X[l + 1])
    return X


def test_bond_projection_is_exact_when_k_covers_the_bond_rank():
    """Sec. 3.2's range finder: a chi x (d d' chi) matrix of rank r <= k is captured
    exactly by k Gaussian test vectors; here the bonds are 12 wide but of rank 4,
    so rank-6 projectors keep the operator (and shrink the bonds to 6)."""
    X = _pad_bonds(kron_sum_mpo(7, 4, 3, 0), 12, 1)
    assert max(x.shape[3] for x in X) == 12
    P = project_bonds(X, 6, seed=2)
    assert mpo_diff_norm(X, P) <= 1e-12 * mpo_norm(X)
    assert max(p.shape[3] for p in P) == 6
    for c in P[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(c.shape[0]), atol=1e-12)


def test_bond_projection_error_of_two_sites():
    """L = 2: the projected operator is M Q Q^T across the bond, whose error is at
    least the Eckart-Young tail and equals || M (I - Q Q^T) || computed densely."""
    X = gaussian_mpo(2, 2, 8, 4, 0, 0.5)
    D = to_dense(X).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    s = np.linalg.svd(D, compute_uv=False)
    for k in (1, 2, 3):
        P = project_bonds(X, k, seed=9)
        E = to_dense(P).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
        err = np.linalg.norm(D - E)
        assert err >= np.sqrt(np.sum(s[k:] ** 2)) * (1 - 1e-12)
        Q = P[1].reshape(P[1].shape[0], -1).T                      # (s t) x k, orthonormal
        assert abs(err - np.linalg.norm(D - D @ Q @ Q.T)) <= 1e-12 * s[0]


def test_fit_with_projected_inputs():
    """ab_rank above every bond of A and B leaves the fit as it was; a smaller rank fits
    the product of the projected chains."""
    from oracle.fit import FitOracle
    A = kron_sum_mpo(8, 6, 5, 0)
    B = kron_sum_mpo(8, 6, 5, 1)
    f0 = FitOracle(A, B, 12, 0.0, conv_tol=0.0)
    f1 = FitOracle(A, B, 12, 0.0, conv_tol=0.0, ab_rank=16)
    f0.sweep(3, stop_on_converge=False)
    f1.sweep(3, stop_on_converge=False)
    assert abs(f0.st.history[-1].norm2 - f1.st.history[-1].norm2) <= 1e-12 * f0.st.history[-1].norm2
    # a smaller rank fits the product of the projected chains
    from oracle.mpo import canonicalize_input
    f2 = FitOracle(A, B, 12, 0.0, conv_tol=0.0, ab_rank=3, seed=4)
    f2.sweep(3, stop_on_converge=False)
    Ap = project_bonds(canonicalize_input(A), 3, 4, 0)
    Bp = project_bonds(canonicalize_input(B), 3, 4, 1)
    assert max(x.shape[3] for x in Ap) == 3
    f3 = FitOracle(Ap, Bp, 12, 0.0, conv_tol=0.0, seed=4, prepare_inputs=False)
    f3.sweep(3, stop_on_converge=False)
    assert mpo_diff_norm(f2.result(), f3.result()) <= 1e-12 * mpo_norm(f3.result())
