"""Pins of the zip-up oracle (Sec. 2.2, Alg. 2 and its right-to-left mirror)."""
import numpy as np
import pytest

from oracle.mpo import mpo_diff_norm, mpo_norm, naive_product, to_dense
from oracle.zipup import zipup_left_to_right, zipup_right_to_left
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
