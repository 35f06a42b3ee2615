"""Pins of the oracle's segment-parallel fit (Sec. 4, Alg. 6, inverse gauge)."""
import numpy as np
import pytest

from oracle.fit import fit
from oracle.mpo import is_left_orthogonal, is_right_orthogonal, mpo_diff_norm, mpo_norm, naive_product, to_dense
from oracle.parallel import ParallelFitOracle, partition
from paper_2606_23274_gb300.synth import mpo_pair


def test_partition_covers_chain_with_edge_extra():
    for L, n, e in ((20, 4, 0), (20, 4, 3), (64, 8, 3), (30, 2, 0), (9, 3, 1)):
        segs = partition(L, n, e)
        assert segs[0][0] == 1 and segs[-1][1] == L
        assert all(b + 1 == c for (_, b), (c, _) in zip(segs, segs[1:]))
        assert all(b - a + 1 >= 2 for a, b in segs)
    s = partition(64, 8, 3)
    assert s[0][1] - s[0][0] > s[1][1] - s[1][0]          # edge segments are longer


@pytest.mark.parametrize("n_seg", [2, 3, 4])
def test_parallel_fit_reproduces_exact_product(n_seg):
    A, B = mpo_pair("gauss_L8_chi8", 0)
    D = to_dense(A) @ to_dense(B)
    p = ParallelFitOracle(A, B, 64, 0.0, n_seg)
    for _ in range(2):
        p.full_sweep_set()
    assert np.linalg.norm(to_dense(p.result()) - D) <= 1e-12 * np.linalg.norm(D)


def test_initial_inverse_form_is_vidal():
    A, B = mpo_pair("kron_L10_chi16", 2)
    p = ParallelFitOracle(A, B, 10, 0.0, 3)
    st = p.st
    for l in range(1, p.L):
        assert is_left_orthogonal(st.Psi[l - 1] * st.Y[l][None, None, None, :], 1e-10)
        assert is_right_orthogonal(st.Y[l][:, None, None, None] * st.Psi[l], 1e-10)


def test_parallel_fit_converges_with_residual_identity():
    A, B = mpo_pair("kron_L12_chi32", 1)
    N = naive_product(A, B)
    nAB2 = mpo_norm(N) ** 2
    p = ParallelFitOracle(A, B, 12, 0.0, 3)
    out = [p.full_sweep_set() for _ in range(8)]
    assert out[-1][1] < 1e-8                                 # ||C||^2 has converged
    C = p.result()
    # the converged C is a fixed point of the local projections: Pythagoras holds
    assert abs(mpo_diff_norm(N, C) ** 2 - (nAB2 - out[-1][0])) <= 1e-8 * nAB2


def test_single_segment_equals_serial_inverse_fit():
    A, B = mpo_pair("kron_L10_chi16", 3)
    p = ParallelFitOracle(A, B, 8, 0.0, 1)
    C_init = p.result()                                      # the guess in its inverse canonical form
    p.full_sweep_set()                                       # one set = forward + backward
    Cs, _ = fit(A, B, 8, 0.0, 2, gauge="inverse", init="given", init_C=C_init, stop_on_converge=False)
    assert mpo_diff_norm(p.result(), Cs) <= 1e-10 * mpo_norm(Cs)
