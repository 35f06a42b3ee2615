"""Pins of the oracle's gradients (oracle/grad.py) against facts outside its
formulas: dense brute force, exact linearity and quadratic structure in one
core, Euler's relation for homogeneous functions, the minimum at C = A B, and
central finite differences."""
import numpy as np
import pytest

from oracle.grad import f1_and_grads, f2_and_grads, inner, inner_grads, norm2_ab, norm2_ab_grads
from oracle.mpo import naive_product, to_dense
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo


def _small(L=4, chi=3, seed=0):
    A = gaussian_mpo(L, 2, chi, seed, 0, 0.6)
    B = gaussian_mpo(L, 2, chi, seed, 1, 0.6)
    W = gaussian_mpo(L, 2, chi + 1, seed, 2, 0.6)
    return A, B, W


def _replace(X, l, core):
    Y = list(X)
    Y[l] = core
    return Y


def test_values_match_dense_brute_force():
    A, B, W = _small()
    P = to_dense(A) @ to_dense(B)
    assert np.isclose(inner(W, A, B), np.sum(to_dense(W) * P), rtol=1e-12)
    assert np.isclose(norm2_ab(A, B), np.sum(P * P), rtol=1e-12)
    f1, _, _ = f1_and_grads(W, A, B)
    assert np.isclose(f1, np.sum((to_dense(W) - P) ** 2), rtol=1e-12)


def test_inner_gradient_is_exact_for_a_linear_function():
    """<W, AB> is linear in each core: f(A_l + E) - f(A_l) = <grad, E> exactly,
    both sides from dense matrices and the oracle's gradient."""
    A, B, W = _small(seed=1)
    gA, gB = inner_grads(W, A, B)
    Dw = to_dense(W)
    rng = np.random.default_rng(7)
    for l in range(len(A)):
        E = rng.standard_normal(A[l].shape)
        lhs = np.sum(Dw * (to_dense(_replace(A, l, A[l] + E)) @ to_dense(B))) - np.sum(Dw * (to_dense(A) @ to_dense(B)))
        assert np.isclose(lhs, np.sum(gA[l] * E), rtol=1e-10, atol=1e-12)
        F = rng.standard_normal(B[l].shape)
        lhs = np.sum(Dw * (to_dense(A) @ to_dense(_replace(B, l, B[l] + F)))) - np.sum(Dw * (to_dense(A) @ to_dense(B)))
        assert np.isclose(lhs, np.sum(gB[l] * F), rtol=1e-10, atol=1e-12)


def test_norm_gradient_from_a_quadratic_in_one_core():
    """||AB||^2 is quadratic in A_l: q(1) - q(-1) = 2 <grad, E> exactly (dense)."""
    A, B, _ = _small(seed=2)
    gA, gB = norm2_ab_grads(A, B)
    rng = np.random.default_rng(8)
    for l in range(len(A)):
        E = rng.standard_normal(A[l].shape)
        q = lambda t: np.sum((to_dense(_replace(A, l, A[l] + t * E)) @ to_dense(B)) ** 2)  # noqa: E731
        assert np.isclose(q(1.0) - q(-1.0), 2.0 * np.sum(gA[l] * E), rtol=1e-10)
        F = rng.standard_normal(B[l].shape)
        q = lambda t: np.sum((to_dense(A) @ to_dense(_replace(B, l, B[l] + t * F))) ** 2)  # noqa: E731
        assert np.isclose(q(1.0) - q(-1.0), 2.0 * np.sum(gB[l] * F), rtol=1e-10)


def test_euler_relations():
    """f2 is homogeneous of degree 1 and ||AB||^2 of degree 2 in every core."""
    A = kron_sum_mpo(6, 4, 3, 0)
    B = kron_sum_mpo(6, 4, 3, 1)
    W = gaussian_mpo(6, 2, 5, 3, 2, 0.5)
    f2 = inner(W, A, B)
    gA, gB = inner_grads(W, A, B)
    n2 = norm2_ab(A, B)
    hA, hB = norm2_ab_grads(A, B)
    for l in range(6):
        assert np.isclose(np.sum(gA[l] * A[l]), f2, rtol=1e-11)
        assert np.isclose(np.sum(gB[l] * B[l]), f2, rtol=1e-11)
        assert np.isclose(np.sum(hA[l] * A[l]), 2 * n2, rtol=1e-11)
        assert np.isclose(np.sum(hB[l] * B[l]), 2 * n2, rtol=1e-11)


def test_residual_gradient_vanishes_at_the_exact_product():
    A = kron_sum_mpo(5, 3, 4, 0)
    B = kron_sum_mpo(5, 3, 4, 1)
    C = naive_product(A, B)
    f1, gA, gB = f1_and_grads(C, A, B)
    scale = norm2_ab(A, B)
    assert abs(f1) <= 1e-12 * scale
    for g, x in zip(gA + gB, A + B):
        assert np.linalg.norm(g) <= 1e-11 * scale / np.linalg.norm(x)


@pytest.mark.parametrize("which", ["A", "B"])
def test_central_finite_differences(which):
    """FP64 central differences (step 1e-6) of the oracle's f1 on L = 6."""
    A = gaussian_mpo(6, 2, 4, 5, 0, 0.7)
    B = gaussian_mpo(6, 2, 4, 5, 1, 0.7)
    C = gaussian_mpo(6, 2, 6, 5, 2, 0.7)
    _, gA, gB = f1_and_grads(C, A, B)
    rng = np.random.default_rng(9)
    h = 1e-6
    for l in (0, 3, 5):
        X, g = (A, gA) if which == "A" else (B, gB)
        E = rng.standard_normal(X[l].shape)
        E /= np.linalg.norm(E)
        def f(t):
            Y = _replace(X, l, X[l] + t * E)
            return f1_and_grads(C, Y, B)[0] if which == "A" else f1_and_grads(C, A, Y)[0]
        fd = (f(h) - f(-h)) / (2 * h)
        assert np.isclose(fd, np.sum(g[l] * E), rtol=1e-6, atol=1e-9)
