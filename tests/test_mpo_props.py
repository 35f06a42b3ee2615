"""Pins of the PyTorch checkers in tests/mpo_props.py (used by the full-size GPU
test) against dense matrices and the oracle, on CPU."""
import numpy as np
import pytest

from oracle.grad import inner
from oracle.mpo import to_dense
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo

torch = pytest.importorskip("torch")
from mpo_props import diff_norm, inner_ab, norm2  # noqa: E402


def _t(X):
    return [torch.from_numpy(np.ascontiguousarray(x)) for x in X]


def test_norm2_matches_dense():
    C = gaussian_mpo(5, 2, 3, 4, 0, 0.7)
    D = to_dense(C)
    assert np.isclose(norm2(_t(C)), np.sum(D * D), rtol=1e-12)


def test_inner_ab_matches_dense_and_oracle():
    A = kron_sum_mpo(5, 3, 2, 0)
    B = gaussian_mpo(5, 2, 2, 2, 1, 0.6)
    C = gaussian_mpo(5, 2, 4, 2, 2, 0.6)
    dense = np.sum(to_dense(C) * (to_dense(A) @ to_dense(B)))
    got = inner_ab(_t(C), _t(A), _t(B))
    assert np.isclose(got, dense, rtol=1e-11)
    assert np.isclose(got, inner(C, A, B), rtol=1e-11)
    # a transposed operand (B A) or a swapped leg gives a different number
    assert not np.isclose(inner_ab(_t(C), _t(B), _t(A)), dense, rtol=1e-6)


def test_diff_norm_matches_dense_and_oracle():
    from oracle.mpo import mpo_diff_norm
    X = gaussian_mpo(6, 2, 3, 4, 3, 0.7)
    Y = gaussian_mpo(6, 2, 3, 3, 4, 0.7)
    dense = np.linalg.norm(to_dense(X) - to_dense(Y))
    got = diff_norm(_t(X), _t(Y))
    assert np.isclose(got, dense, rtol=1e-11)
    assert np.isclose(got, mpo_diff_norm(X, Y), rtol=1e-11)
    # a near-identical pair: the result is the size of the perturbation, with no
    # cancellation floor at sqrt(eps) ||X||
    Z = [x.copy() for x in X]
    Z[3] = Z[3] + 1e-9 * gaussian_mpo(6, 2, 3, 4, 5, 0.7)[3]
    dz = np.linalg.norm(to_dense(X) - to_dense(Z))
    assert np.isclose(diff_norm(_t(X), _t(Z)), dz, rtol=1e-5)
    assert diff_norm(_t(X), _t(X)) <= 1e-14 * np.linalg.norm(to_dense(X))


def test_bench_rel_frobenius_matches_oracle():
    """bench.py's accuracy figure ||X - Y||_F / ||Y||_F (torch, QR sweep) against the oracle's
    stable difference norm and against dense matrices."""
    import importlib
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    bench = importlib.import_module("bench")
    from oracle.mpo import mpo_diff_norm, mpo_norm
    X = gaussian_mpo(6, 2, 3, 21, 0, 0.7)
    Y = [x.copy() for x in X]
    Y[2] = Y[2] + 1e-7 * gaussian_mpo(6, 2, 3, 21, 1, 0.7)[2]
    got = bench.rel_frobenius(_t(X), _t(Y))
    ref = mpo_diff_norm(X, Y) / mpo_norm(Y)
    dense = np.linalg.norm(to_dense(X) - to_dense(Y)) / np.linalg.norm(to_dense(Y))
    assert np.isclose(got, ref, rtol=1e-6) and np.isclose(got, dense, rtol=1e-5)
    assert bench.rel_frobenius(_t(X), _t(X)) <= 1e-14
