"""Pins of the oracle's helpers that the fit, the zip-up and the projection build on, each
against something other than the helper itself: exact rational arithmetic, dense matrices,
closed forms and invariants."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import philox
from oracle.fit import fix_signs, init_bonds, random_right_canonical
from oracle.mpo import (is_right_orthogonal, left_orthogonalize, mpo_sum, qr_pos, to_dense,
                        trim_right)
from oracle.zipup import project_stream, zipup_stream
from paper_2606_23274_gb300.synth import gaussian_mpo


def _gram_schmidt_exact(M):
    """Classical Gram-Schmidt in exact rationals on a small integer matrix: the QR factorisation
    with a positive R diagonal, which is unique for full column rank."""
    m, n = M.shape
    cols = [[Fraction(int(x)) for x in M[:, j]] for j in range(n)]
    Q2, R = [], [[Fraction(0)] * n for _ in range(n)]   # Q2: unnormalised orthogonal columns
    for j in range(n):
        v = cols[j][:]
        for i, q in enumerate(Q2):
            qq = sum(a * a for a in q)
            c = sum(a * b for a, b in zip(q, cols[j])) / qq
            R[i][j] = c                                  # in units of the unnormalised q_i
            v = [a - c * b for a, b in zip(v, q)]
        Q2.append(v)
    norms = [float(sum(a * a for a in q)) ** 0.5 for q in Q2]
    Q = np.array([[float(q[r]) / norms[j] for j, q in enumerate(Q2)] for r in range(m)])
    Rf = np.array([[float(R[i][j]) * norms[i] if i < j else (norms[i] if i == j else 0.0)
                    for j in range(n)] for i in range(n)])
    return Q, Rf


def test_qr_pos_is_the_unique_qr_with_positive_diagonal():
    rng = np.random.default_rng(0)
    M = rng.integers(-5, 6, size=(7, 4)).astype(float)
    Q, R = qr_pos(M)
    Qe, Re = _gram_schmidt_exact(M)
    assert np.all(np.diag(R) >= 0)
    assert np.allclose(np.triu(R), R)
    assert np.abs(Q - Qe).max() <= 1e-13 and np.abs(R - Re).max() <= 1e-12
    # a column of M's sign flipped flips the same column of Q and row of R, nothing else
    M2 = M.copy()
    M2[:, 1] *= -1
    Q2, R2 = qr_pos(M2)
    assert np.allclose(Q2[:, 1], -Q[:, 1]) and np.allclose(np.abs(R2), np.abs(R))


def test_trim_right_keeps_the_operator_and_bounds_the_bonds():
    rng = np.random.default_rng(1)
    d = 2
    # bonds above the rank bound on the right: chi_{L-1} = 9 > d d' = 4, chi_{L-2} = 20 > 4 * 4
    X = [rng.standard_normal(s) for s in [(1, d, d, 3), (3, d, d, 20), (20, d, d, 9), (9, d, d, 1)]]
    Y = trim_right(X)
    assert np.allclose(to_dense(Y), to_dense(X), atol=1e-12 * np.abs(to_dense(X)).max())
    b = [Y[0].shape[0]] + [y.shape[3] for y in Y]
    assert b == [1, 3, 16, 4, 1]                      # min(chi, d d' chi_right) from the right
    # the trimmed cores right of the first untouched bond are right-orthogonal
    assert is_right_orthogonal(Y[3]) and is_right_orthogonal(Y[2])
    # nothing to trim: the chain comes back unchanged
    Z = [rng.standard_normal(s) for s in [(1, d, d, 2), (2, d, d, 4), (4, d, d, 1)]]
    assert all(np.array_equal(a, b) for a, b in zip(trim_right(Z), Z))


def test_trim_right_stops_at_the_first_site_within_its_bound():
    rng = np.random.default_rng(2)
    d = 2
    # the last bond needs no trim, so the sweep stops at once, although chi_1 = 9 > 4 would trim
    X = [rng.standard_normal(s) for s in [(1, d, d, 9), (9, d, d, 3), (3, d, d, 1)]]
    Y = trim_right(X)
    assert [y.shape for y in Y] == [x.shape for x in X]


def test_fix_signs_convention_and_invariance():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((9, 6))
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    U2, Vt2 = fix_signs(-U, -Vt)                      # any sign pattern lands on the same pair
    U3, Vt3 = fix_signs(U, Vt)
    assert np.allclose(U2, U3) and np.allclose(Vt2, Vt3)
    j = np.arange(U3.shape[1])
    assert np.all(U3[np.argmax(np.abs(U3), axis=0), j] > 0)
    assert np.allclose((U3 * S) @ Vt3, M)


@pytest.mark.parametrize("dout,din,chi", [([2] * 6, [2] * 6, 5), ([2, 3, 1, 2], [3, 1, 2, 2], 100),
                                          ([2] * 3, [2] * 3, 64)])
def test_init_bonds_closed_form(dout, din, chi):
    L = len(dout)
    b = init_bonds(dout, din, chi)
    assert b[0] == 1 and b[-1] == 1 and len(b) == L + 1
    for l in range(1, L):
        left = int(np.prod([dout[j] * din[j] for j in range(l)]))
        right = int(np.prod([dout[j] * din[j] for j in range(l, L)]))
        assert b[l] == min(chi, left, right)


def test_random_guess_is_right_canonical_with_the_stated_bonds():
    dout, din, chi = [2] * 7, [2] * 7, 12
    C = random_right_canonical(dout, din, chi, seed=5)
    assert [C[0].shape[0]] + [c.shape[3] for c in C] == init_bonds(dout, din, chi)
    assert all(is_right_orthogonal(c) for c in C[1:])
    # core 1 is the Philox Gaussian itself (stream init_stream(1)), unnormalised
    g = philox.normals(5, philox.init_stream(1), C[0].size).reshape(C[0].shape)
    assert np.array_equal(C[0], g)


def test_mpo_sum_is_the_sum_of_the_dense_operators():
    X = gaussian_mpo(4, 2, 3, 0, 0)
    Y = gaussian_mpo(4, 2, 2, 0, 1)
    for beta in (1.0, -1.0, 0.25):
        assert np.allclose(to_dense(mpo_sum(X, Y, beta)), to_dense(X) + beta * to_dense(Y), atol=1e-12)
    one_x, one_y = [X[0][:, :, :, :1]], [Y[0][:, :, :, :1]]
    assert np.allclose(to_dense(mpo_sum(one_x, one_y, 2.0)), to_dense(one_x) + 2.0 * to_dense(one_y))


def test_philox_stream_families_do_not_overlap():
    """The fit's sketches, the guess, the zip-up sketches and the two projection families use
    disjoint Philox streams: the top bits name the family, the low bits the sweep and the site."""
    L = 300
    fam = {
        "fit": {philox.omega_stream(s, l) for s in range(40) for l in range(1, L)},
        "guess": {philox.init_stream(l) for l in range(1, L)},
        "zipup": {zipup_stream(l) for l in range(1, L)},
        "proj_a": {project_stream(0, l) for l in range(1, L)},
        "proj_b": {project_stream(1, l) for l in range(1, L)},
    }
    names = list(fam)
    for i, a in enumerate(names):
        assert len(fam[a]) == (40 * (L - 1) if a == "fit" else L - 1)   # no collision inside a family
        for b in names[i + 1:]:
            assert not fam[a] & fam[b], (a, b)


def test_left_orthogonalize_keeps_the_operator():
    X = gaussian_mpo(5, 2, 3, 0, 4)
    Y = left_orthogonalize(X)
    assert np.allclose(to_dense(Y), to_dense(X), atol=1e-12 * np.abs(to_dense(X)).max())
