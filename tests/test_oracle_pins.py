"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published known-answer vectors, dense brute force on tiny chains, closed forms of
the Kronecker-sum inputs, and invariants of canonical forms and of the fit."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import philox
from oracle.fit import FitOracle, fit, keep_rank, left_env, local_tensor, randomized_svd, right_env
from oracle.mpo import (bonds, canonicalize_input, is_left_orthogonal, is_right_orthogonal,
                        left_orthogonalize, mpo_diff_norm, mpo_norm, naive_product,
                        right_orthogonalize, to_dense)
from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo, mpo_pair, uniform_mpo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox / Omega
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]


def test_gaussian_stream_moments():
    z = philox.normals(seed=7, stream=philox.omega_stream(3, 5), count=400_000)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05            # Gaussian kurtosis
    assert abs(np.mean(z > 1.0) - 0.15865525393145707) < 0.003   # 1 - Phi(1)
    # streams and offsets are independent coordinates of one counter space
    a = philox.normals(1, 2, 10, start=5)
    b = philox.normals(1, 2, 15)[5:]
    assert np.array_equal(a, b)
    assert not np.allclose(philox.normals(1, 2, 10), philox.normals(1, 3, 10))


# ---------------------------------------------------------------- dense / naive
def _dense_bruteforce(X):
    """Element-wise definition: D[x, y] = product over sites of X_l[:, x_l, y_l, :]."""
    L = len(X)
    dims_o = [x.shape[1] for x in X]
    dims_i = [x.shape[2] for x in X]
    D = np.zeros((math.prod(dims_o), math.prod(dims_i)))
    for xs in itertools.product(*[range(d) for d in dims_o]):
        r = 0
        for d, x in zip(dims_o, xs):
            r = r * d + x
        for ys in itertools.product(*[range(d) for d in dims_i]):
            c = 0
            for d, y in zip(dims_i, ys):
                c = c * d + y
            v = np.eye(1)
            for l in range(L):
                v = v @ X[l][:, xs[l], ys[l], :]
            D[r, c] = v[0, 0]
    return D


def test_dense_matches_elementwise_definition():
    X = gaussian_mpo(3, 2, 3, seed=11)
    assert np.allclose(to_dense(X), _dense_bruteforce(X), atol=1e-13)


def test_naive_product_is_exact_dense_product():
    A, B = mpo_pair("gauss_L8_chi8", 3, L=5)
    C = naive_product(A, B)
    assert bonds(C) == [1] + [64] * 4 + [1]
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(C) - D) <= 1e-13 * np.linalg.norm(D)


def test_kron_sum_closed_form_norm():
    """||AB||^2 = sum_{j,k,j',k'} w_j w_k w_j' w_k' prod_l <a_jl b_kl, a_j'l b_k'l>."""
    L, K = 6, 3
    A = kron_sum_mpo(L, K, seed=4, which=0)
    B = kron_sum_mpo(L, K, seed=4, which=1)
    w = 0.8 ** np.arange(K)

    def factors(X):             # read the d x d factors back out of the diagonal-bond layout
        f = np.zeros((L, K, 2, 2))
        for k in range(K):
            f[0, k] = X[0][0, :, :, k] / w[k]
            f[L - 1, k] = X[L - 1][k, :, :, 0]
            for l in range(1, L - 1):
                f[l, k] = X[l][k, :, :, k]
        return f

    fa, fb = factors(A), factors(B)
    total = 0.0
    for j, k, jp, kp in itertools.product(range(K), repeat=4):
        p = w[j] * w[k] * w[jp] * w[kp]
        for l in range(L):
            p *= np.sum((fa[l, j] @ fb[l, k]) * (fa[l, jp] @ fb[l, kp]))
        total += p
    assert abs(mpo_norm(naive_product(A, B)) ** 2 - total) <= 1e-12 * total
    D = to_dense(A) @ to_dense(B)
    assert abs(np.linalg.norm(D) ** 2 - total) <= 1e-12 * total


def test_canonical_forms_preserve_operator_and_trim_bonds():
    X = kron_sum_mpo(7, 20, seed=2)
    D = to_dense(X)
    Lx, Rx, Cx = left_orthogonalize(X), right_orthogonalize(X), canonicalize_input(X)
    for Y in (Lx, Rx, Cx):
        assert np.linalg.norm(to_dense(Y) - D) <= 1e-12 * np.linalg.norm(D)
    assert all(is_left_orthogonal(x) for x in Lx[:-1])
    assert all(is_right_orthogonal(x) for x in Rx[1:])
    assert all(is_left_orthogonal(x) for x in Cx[:-1])
    assert bonds(Cx) == [1, 4, 16, 20, 20, 16, 4, 1]     # min(K, 4^l, 4^(L-l))


def test_diff_norm_matches_dense():
    X = gaussian_mpo(6, 2, 5, seed=1)
    Y = gaussian_mpo(6, 2, 4, seed=2)
    ref = np.linalg.norm(to_dense(X) - to_dense(Y))
    assert abs(mpo_diff_norm(X, Y) - ref) <= 1e-12 * ref
    assert mpo_diff_norm(X, X) <= 1e-14 * mpo_norm(X)


# ---------------------------------------------------------------- truncation rule
def test_keep_rank_rule():
    S = np.array([4.0, 2.0, 1.0, 0.5, 0.25])
    nM = float(np.linalg.norm(S))
    assert keep_rank(S, nM, 0.0, 10, 3, 1e-13) == 3                 # chi cap only
    assert keep_rank(S, nM, 0.0, 10, 99, 1e-13) == 5
    # tail after k=3 is sqrt(0.25+0.0625)=0.559; after k=2 it is 1.146
    thr_tau = lambda t: t * 10 / nM
    assert keep_rank(S, nM, thr_tau(0.6), 10, 99, 1e-13) == 3
    assert keep_rank(S, nM, thr_tau(1.2), 10, 99, 1e-13) == 2
    assert keep_rank(S, nM, thr_tau(100.0), 10, 99, 1e-13) == 1    # k >= 1
    assert keep_rank(S, nM, 0.0, 10, 99, 0.2) == 3                   # s_j <= 0.2 s_1 dropped
    assert keep_rank(np.zeros(3), 0.0, 0.0, 10, 5, 1e-13) == 1


# ---------------------------------------------------------------- randomized SVD
def test_rsvd_exact_when_sketch_spans_range():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((40, 6)) @ rng.standard_normal((6, 30))   # rank 6
    U, S, Vt = randomized_svd(M, 9, seed=3, stream=philox.omega_stream(0, 1))
    assert np.linalg.norm(U @ np.diag(S) @ Vt - M) <= 1e-12 * np.linalg.norm(M)
    S_ref = np.linalg.svd(M, compute_uv=False)
    assert np.allclose(S[:6], S_ref[:6], rtol=1e-12)
    assert np.all(S[6:] <= 1e-12 * S[0])


def test_rsvd_error_at_least_tail():
    """Sec. 3.1: the exact tail sqrt(sum_{j>k} s_j^2) is a lower bound of the RSVD error."""
    rng = np.random.default_rng(1)
    M = rng.standard_normal((60, 50)) * (0.7 ** np.arange(50))[None, :]
    k = 8
    U, S, Vt = randomized_svd(M, k, seed=5, stream=11)
    err = np.linalg.norm(M - U @ np.diag(S) @ Vt)
    tail = np.sqrt(np.sum(np.linalg.svd(M, compute_uv=False)[k:] ** 2))
    assert err >= tail * (1 - 1e-12)


# ---------------------------------------------------------------- environments / local tensor
def _interleave_dense(X):
    """Dense operator as a tensor with axes (x1,y1,x2,y2,...)."""
    L = len(X)
    D = to_dense(X)
    do = [x.shape[1] for x in X]
    di = [x.shape[2] for x in X]
    T = D.reshape(do + di)
    perm = [a for l in range(L) for a in (l, L + l)]
    return T.transpose(perm)


def _chain(cores):
    """Contract consecutive cores into E[left_bond, (x y)..., right_bond]."""
    E = cores[0]
    for c in cores[1:]:
        E = np.tensordot(E, c, axes=([E.ndim - 1], [0]))
    return E


def test_local_tensor_is_projection_of_dense_product():
    """Fig. derivatives: with C left-orthogonal left of the window and right-orthogonal
    right of it, Theta equals the dense product projected on the environment bases."""
    L, win = 5, 2
    A, B = mpo_pair("gauss_L8_chi8", 5, L=L)
    f = FitOracle(A, B, chi_max=6, tol=0.0)
    f._update(1, True, 0)                                  # forward step at window 1
    st = f.st
    st.Lenv[1] = left_env(st.Lenv[0], st.A[0], st.B[0], f._c_left(1))
    Theta = local_tensor(st.Lenv[1], st.A[1], st.B[1], st.A[2], st.B[2], st.Renv[4])
    assert is_left_orthogonal(f._c_left(1))
    assert all(is_right_orthogonal(f._c_right(l)) for l in (4, 5))
    T = _interleave_dense(naive_product(A, B))            # (x1,y1,...,x5,y5)
    El = _chain([f._c_left(1)])[0]                         # (x1, y1, c1)
    Er = _chain([f._c_right(4), f._c_right(5)])[..., 0]    # (c3, x4, y4, x5, y5)
    ref = np.einsum("abc,abdefgxyuv,hxyuv->cdefgh", El, T, Er)
    assert np.linalg.norm(Theta - ref) <= 1e-12 * np.linalg.norm(ref)


def test_envs_are_partial_inner_products():
    """L_l contracted with R_{l+1} gives <C, AB> for every cut l."""
    L = 6
    A, B = mpo_pair("gauss_L8_chi8", 2, L=L)
    C = gaussian_mpo(L, 2, 3, seed=9)
    Le = [np.ones((1, 1, 1))]
    for l in range(L):
        Le.append(left_env(Le[-1], A[l], B[l], C[l]))
    Re = [np.ones((1, 1, 1))]
    for l in range(L - 1, -1, -1):
        Re.insert(0, right_env(Re[0], A[l], B[l], C[l]))
    ref = float(np.sum(to_dense(C) * (to_dense(A) @ to_dense(B))))
    for cut in range(L + 1):
        val = float(np.einsum("abc,abc->", Le[cut], Re[cut]))
        assert abs(val - ref) <= 1e-12 * abs(ref)


# ---------------------------------------------------------------- the fit
@pytest.mark.parametrize("gauge", ["site", "inverse"])
def test_fit_reproduces_exact_product(gauge):
    A, B = mpo_pair("gauss_L8_chi8", 0)
    D = to_dense(A) @ to_dense(B)
    for sweeps in (1, 2):
        C, f = fit(A, B, 64, 0.0, sweeps, gauge=gauge, stop_on_converge=False)
        assert np.linalg.norm(to_dense(C) - D) <= 1e-12 * np.linalg.norm(D)
    assert f.bonds() == [1, 4, 16, 64, 64, 64, 16, 4, 1]


def test_fit_gauges_agree_and_residual_identity():
    A, B = mpo_pair("kron_L10_chi16", 1)
    Cs, fs = fit(A, B, 12, 0.0, 5, gauge="site", stop_on_converge=False)
    Ci, fi = fit(A, B, 12, 0.0, 5, gauge="inverse", stop_on_converge=False)
    nC = mpo_norm(Cs)
    assert mpo_diff_norm(Cs, Ci) <= 1e-12 * nC
    N = naive_product(A, B)
    nAB2 = mpo_norm(N) ** 2
    res2 = [nAB2 - h.norm2 for h in fs.st.history]
    # Pythagoras at the optimum of the last update: ||AB - C||^2 = ||AB||^2 - ||C||^2
    assert abs(mpo_diff_norm(N, Cs) ** 2 - res2[-1]) <= 1e-9 * nAB2
    assert abs(fs.st.history[-1].norm2 - nC ** 2) <= 1e-12 * nC ** 2
    # monotone residual over sweeps (Sec. 5.2)
    assert all(b <= a * (1 + 1e-12) + 1e-15 * nAB2 for a, b in zip(res2, res2[1:]))


def test_fit_isometries_during_sweep():
    A, B = mpo_pair("kron_L10_chi16", 2)
    C, f = fit(A, B, 10, 0.0, 3, gauge="site", stop_on_converge=False)   # ends after a forward sweep
    assert all(is_left_orthogonal(c) for c in C[:-1])
    f.sweep(1)                                                             # backward sweep
    C = f.result()
    assert all(is_right_orthogonal(c) for c in C[1:])


def test_inverse_gauge_psi_y_isometries():
    """Alg. 4 bookkeeping: after a forward sweep every Psi_l Y_l is left-orthogonal, after a
    backward sweep every Y_{l-1} Psi_l is right-orthogonal; once C is the exact product
    (a true Vidal-type form, Sec. 2.3.1) both hold at once."""
    A, B = mpo_pair("kron_L10_chi16", 3)
    f = FitOracle(A, B, 10, 0.0, gauge="inverse")
    st = f.st
    for sweep in range(3):
        f.sweep(1, stop_on_converge=False)
        for l in range(1, f.L):
            if sweep % 2 == 0:
                assert is_left_orthogonal(st.Psi[l - 1] * st.Y[l][None, None, None, :], 1e-10)
            else:
                assert is_right_orthogonal(st.Y[l][:, None, None, None] * st.Psi[l], 1e-10)
    A, B = mpo_pair("gauss_L8_chi8", 6)
    f = FitOracle(A, B, 64, 0.0, gauge="inverse")
    f.sweep(2, stop_on_converge=False)
    st = f.st
    for l in range(1, f.L):
        assert is_left_orthogonal(st.Psi[l - 1] * st.Y[l][None, None, None, :], 1e-8)
        assert is_right_orthogonal(st.Y[l][:, None, None, None] * st.Psi[l], 1e-8)


def test_rsvd_fit_equals_exact_when_sketch_covers_rank():
    """k_s >= rank(M) at every window (exact product, rank <= 64): the randomized
    update reproduces the exact one (Sec. 3.1 with Q Q^T M = M)."""
    A, B = mpo_pair("gauss_L8_chi8", 4)
    Ce, _ = fit(A, B, 64, 0.0, 2, stop_on_converge=False)
    Cr, _ = fit(A, B, 64, 0.0, 2, update="rsvd", oversample=2, stop_on_converge=False)
    D = to_dense(A) @ to_dense(B)
    assert np.linalg.norm(to_dense(Cr) - D) <= 1e-11 * np.linalg.norm(D)
    assert mpo_diff_norm(Ce, Cr) <= 1e-11 * np.linalg.norm(D)


def test_uniform_workload_fit_converges():
    A, B = mpo_pair("uniform_L12_chi12", 0)
    C, f = fit(A, B, 12, 0.0, 6, stop_on_converge=False)
    d = [h.delta for h in f.st.history]
    assert d[-1] < 1e-3


def test_mpo_inner_matches_dense():
    from oracle.mpo import mpo_inner
    X = gaussian_mpo(5, 2, 3, 11, 0, 0.7)
    Y = gaussian_mpo(5, 2, 4, 11, 1, 0.6)
    assert np.isclose(mpo_inner(X, Y), np.sum(to_dense(X) * to_dense(Y)), rtol=1e-12)
    # <X, X> is the squared norm, and a transposed leg order gives another number
    assert np.isclose(mpo_inner(X, X), mpo_norm(X) ** 2, rtol=1e-12)
    Xt = [np.ascontiguousarray(x.transpose(0, 2, 1, 3)) for x in X]
    assert not np.isclose(mpo_inner(Xt, Y), mpo_inner(X, Y), rtol=1e-6)


def test_bond_spectra_match_dense_matricisations():
    """The singular values across bond l are those of the dense operator
    reshaped to (x_1 y_1 .. x_l y_l) x (x_{l+1} y_{l+1} .. x_L y_L) (C13 order)."""
    from oracle.mpo import bond_spectra
    L, d = 5, 2
    X = gaussian_mpo(L, d, 3, 12, 0, 0.7)
    D = to_dense(X).reshape([d] * L + [d] * L)              # (x_1..x_L, y_1..y_L)
    perm = [i for l in range(L) for i in (l, L + l)]          # (x_1, y_1, x_2, y_2, ...)
    T = D.transpose(perm)
    got = bond_spectra(X)
    assert len(got) == L - 1
    for l in range(1, L):
        M = T.reshape(d ** (2 * l), -1)
        ref = np.linalg.svd(M, compute_uv=False)
        r = len(got[l - 1])
        assert np.allclose(got[l - 1], ref[:r], rtol=1e-10, atol=1e-13 * ref[0])
        assert np.all(ref[r:] <= 1e-12 * ref[0])               # the bond holds the whole rank


def test_gap_report_marks_a_degenerate_cut():
    """A two-site operator with singular values (3, 2, 2, 1) across its bond, fitted to bond 2:
    the cut falls inside the degenerate pair, so the gap is 1 and the bond is unpinned; to bond
    3 the gap is 2 and the bond is pinned."""
    from oracle.fit import FitOracle
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    s = np.array([3.0, 2.0, 2.0, 1.0])
    X = [(U * s).reshape(1, 2, 2, 4), V.T.reshape(4, 2, 2, 1)]
    I = [np.eye(2).reshape(1, 2, 2, 1), np.eye(2).reshape(1, 2, 2, 1)]
    for chi, gap, pinned in ((2, 1.0, []), (3, 2.0, [1])):
        f = FitOracle(X, I, chi, 0.0, conv_tol=0.0)
        f.sweep(1)
        assert f.gaps()[0] == pytest.approx(gap, rel=1e-12)
        assert f.pinned_bonds() == pinned
