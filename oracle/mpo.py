"""Plain FP64 MPO operations: exact product, dense expansion, canonical forms,
difference norm.

ORACLE: test infrastructure only. Imported by tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference leg; never by the product path.

Core convention (Sec. 2, MPO definition): ``X[l]`` has shape
``(chi_{l-1}, d_l, d'_l, chi_l)``, ``d`` the output (row) leg and ``d'`` the
input (column) leg; ``chi_0 = chi_L = 1``. ``C = A B`` contracts A's input leg
with B's output leg (Sec. 2, the MPO-MPO contraction).
"""
from __future__ import annotations

import numpy as np


def qr_pos(M: np.ndarray):
    """Thin QR with the diagonal of R made non-negative (unique for full rank)."""
    Q, R = np.linalg.qr(M, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def naive_product(A, B):
    """Alg. 1 without the final compression (Sec. 2.1): per-site contraction
    C_l[(ia,ib), s, t, (ja,jb)] = sum_u A_l[ia,s,u,ja] B_l[ib,u,t,jb];
    the combined bond index is ia*chi_B + ib. Exact, bond chi_A*chi_B."""
    out = []
    for Al, Bl in zip(A, B):
        a0, d, dp, a1 = Al.shape
        b0, dp2, t, b1 = Bl.shape
        assert dp == dp2
        Cl = np.einsum("isuj,kutl->ikstjl", Al, Bl)
        out.append(Cl.reshape(a0 * b0, d, t, a1 * b1))
    return out


def to_dense(X) -> np.ndarray:
    """Dense matrix of an MPO: row index (x_1..x_L), column (y_1..y_L), x_1
    most significant (big-endian)."""
    T = X[0][0]                                       # (d, d', chi_1)
    rows, cols = T.shape[0], T.shape[1]
    T = T.reshape(rows, cols, -1)
    for Xl in X[1:]:
        _, d, dp, chr_ = Xl.shape
        T = np.einsum("rcb,bxyk->rxcyk", T, Xl)
        rows, cols = rows * d, cols * dp
        T = T.reshape(rows, cols, chr_)
    return T[:, :, 0]


def left_orthogonalize(X):
    """QR sweep l = 1..L-1 (Sec. 2.3.1 site-canonical form): every core but the
    last becomes left-orthogonal, the bond shrinks to min(rows, cols)."""
    X = [x.copy() for x in X]
    for l in range(len(X) - 1):
        a0, d, dp, a1 = X[l].shape
        Q, R = qr_pos(X[l].reshape(a0 * d * dp, a1))
        k = Q.shape[1]
        X[l] = Q.reshape(a0, d, dp, k)
        X[l + 1] = np.einsum("ka,axyb->kxyb", R, X[l + 1])
    return X


def right_orthogonalize(X):
    """RQ sweep l = L..2 (Sec. 2.3.1): every core but the first becomes
    right-orthogonal, computed as the QR of the transposed core."""
    X = [x.copy() for x in X]
    for l in range(len(X) - 1, 0, -1):
        a0, d, dp, a1 = X[l].shape
        Q, R = qr_pos(X[l].reshape(a0, d * dp * a1).T)   # X^T = Q R  =>  X = R^T Q^T
        k = Q.shape[1]
        X[l] = Q.T.reshape(k, d, dp, a1)
        X[l - 1] = np.einsum("axyb,kb->axyk", X[l - 1], R)
    return X


def trim_right(X):
    """RQ steps from the right end (Sec. 2.3.1), each as right_orthogonalize
    takes it, only while they trim: the sweep ends at the first site whose
    left bond is already within its bound d d' chi_right. The operator is
    unchanged."""
    X = [x.copy() for x in X]
    for l in range(len(X) - 1, 0, -1):
        a0, d, dp, a1 = X[l].shape
        if a0 <= d * dp * a1:
            break
        Q, R = qr_pos(X[l].reshape(a0, d * dp * a1).T)
        k = Q.shape[1]
        X[l] = Q.T.reshape(k, d, dp, a1)
        X[l - 1] = np.einsum("axyb,kb->axyk", X[l - 1], R)
    return X


def canonicalize_input(X):
    """Input preparation of Alg. 5 (left_orthogonalize): bonds first trimmed to
    their rank bound from the right (trim_right), then the QR sweep the
    algorithm names. The operator is unchanged; the left gauge it leaves is the
    one a Gaussian sketch over the input bonds (the randomized zip-up) sees."""
    return left_orthogonalize(trim_right(X))


def is_left_orthogonal(Xl, tol=1e-12) -> bool:
    a0, d, dp, a1 = Xl.shape
    M = Xl.reshape(a0 * d * dp, a1)
    return np.allclose(M.T @ M, np.eye(a1), atol=tol)


def is_right_orthogonal(Xl, tol=1e-12) -> bool:
    a0, d, dp, a1 = Xl.shape
    M = Xl.reshape(a0, d * dp * a1)
    return np.allclose(M @ M.T, np.eye(a0), atol=tol)


def bonds(X):
    return [X[0].shape[0]] + [x.shape[3] for x in X]


def mpo_norm(X) -> float:
    """Frobenius norm: left-orthogonalize, then the norm of the last core."""
    Y = left_orthogonalize(X)
    return float(np.linalg.norm(Y[-1]))


def mpo_sum(X, Y, beta: float = 1.0):
    """MPO of X + beta*Y with block (direct-sum) bonds."""
    L = len(X)
    if L == 1:
        return [X[0] + beta * Y[0]]
    out = []
    for l in range(L):
        x, y = X[l], Y[l]
        if l == 0:
            out.append(np.concatenate([x, beta * y], axis=3))
        elif l == L - 1:
            out.append(np.concatenate([x, y], axis=0))
        else:
            a0, d, dp, a1 = x.shape
            b0, _, _, b1 = y.shape
            Z = np.zeros((a0 + b0, d, dp, a1 + b1))
            Z[:a0, :, :, :a1] = x
            Z[a0:, :, :, a1:] = y
            out.append(Z)
    return out


def mpo_diff_norm(X, Y) -> float:
    """||X - Y||_F computed stably: the direct-sum MPO X (+) (-Y) is
    left-orthogonalized by Householder QR and the norm read off the last core
    (a backward-stable reading of the paper's error metric, Sec. 5.2)."""
    return mpo_norm(mpo_sum(X, Y, -1.0))


def mpo_inner(X, Y) -> float:
    """<X, Y>_F by a left-to-right transfer contraction."""
    E = np.ones((1, 1))
    for x, y in zip(X, Y):
        E = np.einsum("ab,aijc,bijd->cd", E, x, y)
    return float(E[0, 0])


def bond_spectra(X):
    """Singular values across every inner bond (exact, via canonical forms)."""
    Y = right_orthogonalize(X)
    out = []
    for l in range(len(Y) - 1):
        a0, d, dp, a1 = Y[l].shape
        U, S, Vt = np.linalg.svd(Y[l].reshape(a0 * d * dp, a1), full_matrices=False)
        out.append(S)
        k = S.shape[0]
        Y[l] = U.reshape(a0, d, dp, k)
        Y[l + 1] = np.einsum("k,ka,axyb->kxyb", S, Vt, Y[l + 1])
    return out
